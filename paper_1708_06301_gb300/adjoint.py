"""torch.autograd.Function over the adjoint entry points of the C ABI (argument marshalling only).

WarpKalman maps theta = (w0, w1, w2, t0, t1, t2, q, s_r) (float64, CPU) and fixed device maps
(previous D and P, measurement D_z and r_z) to the Kalman-updated maps (D, P) of one time step
(prediction Sec. 2.2, Eq. 3, 5, 6; update Sec. 2.4, Eq. 10-12), with the rotation given as a
rotation vector (R = exp([w]x)) and the measurement variance scaled by s_r. Its backward calls
tsgm_adjoint_backward, which recomputes everything but the z-buffer winners on the GPU.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tsgm as _t


class WarpKalman(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, prev_D, prev_P, D_z, r_z, K, baseline, tctx):
        th = theta.detach().cpu().numpy().astype(np.float64)
        D = torch.empty_like(prev_D)
        P = torch.empty_like(prev_P)
        tctx.adjoint_forward(prev_D, prev_P, th[:6], K, baseline, th[6], th[7], D_z, r_z, D, P)
        gen = getattr(tctx, "_adj_gen", 0) + 1
        tctx._adj_gen = gen
        fctx.save_for_backward(theta, prev_D, prev_P, D_z, r_z)
        fctx.tctx, fctx.K, fctx.baseline, fctx.gen = tctx, K, baseline, gen
        return D, P

    @staticmethod
    def backward(fctx, grad_D, grad_P):
        theta, prev_D, prev_P, D_z, r_z = fctx.saved_tensors
        th = theta.detach().cpu().numpy().astype(np.float64)
        tctx = fctx.tctx
        if grad_D is None:
            grad_D = torch.zeros_like(prev_D)
        if grad_P is None:
            grad_P = torch.zeros_like(prev_P)
        if getattr(tctx, "_adj_gen", 0) != fctx.gen:
            # another forward ran on this context since: restore this one's z-buffer winners
            D = torch.empty_like(prev_D)
            P = torch.empty_like(prev_P)
            tctx.adjoint_forward(prev_D, prev_P, th[:6], fctx.K, fctx.baseline, th[6], th[7], D_z,
                                 r_z, D, P)
            tctx._adj_gen = fctx.gen
        g = tctx.adjoint_backward(prev_D, prev_P, th[:6], fctx.K, fctx.baseline, th[6], th[7], D_z,
                                  r_z, grad_D.contiguous(), grad_P.contiguous())
        return (torch.from_numpy(g).to(theta.dtype), None, None, None, None, None, None, None)


def warp_kalman(theta, prev_D, prev_P, D_z, r_z, K, baseline, tctx):
    """(D, P) of one prediction + update step, differentiable in theta (see WarpKalman)."""
    return WarpKalman.apply(theta, prev_D, prev_P, D_z, r_z, K, baseline, tctx)
