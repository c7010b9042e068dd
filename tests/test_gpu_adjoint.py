"""GPU adjoint of prediction + Kalman update: forward parity with the oracle, gradients against
binary64 central finite differences (h = 1e-4) and the oracle's analytic gradient, the
autograd.Function wrapper, and a small pose/noise fit on a synthetic scene with ground truth."""
import numpy as np
import pytest

import oracle
from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, f32, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B = f32(0.54)


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def config3_inputs(seed, W=1242, H=375):
    """Random previous maps (D 1-127 px, P 0.1-4 px^2), random 6-DoF pose (|t| <= 1.5 m,
    each rotation angle within 3 deg), random measurements with 10% invalid pixels."""
    D, P = synth.random_maps(seed, W, H, d_range=(1, 127), p_range=(0.1, 4.0))
    Dz, rz = synth.random_maps(seed + 1, W, H, d_range=(1, 127), p_range=(0.5, 4.0), invalid_frac=0.1)
    rs = synth.Stream(seed, 0xAD)
    w = np.array([np.radians(rs.uniform(-3, 3)) for _ in range(3)])
    _, t = synth.random_pose(seed + 2, max_t=1.5)
    pose6 = np.concatenate([w, t.astype(np.float64)])
    rng = np.random.default_rng(seed)
    gD = rng.normal(size=(H, W)).astype(np.float32)
    gP = rng.normal(size=(H, W)).astype(np.float32)
    K = synth.Camera(W, H, 721.0, 0.54).K
    return D, P, Dz, rz, pose6, gD, gP, K


@pytest.mark.parametrize("seed,q,s_r", [(11, 0.25, 1.0), (12, 0.6, 1.7)])
def test_adjoint_forward_parity_and_gradients(tsgm, seed, q, s_r):
    D, P, Dz, rz, pose6, gD, gP, K = config3_inputs(seed)
    H, W = D.shape
    with tsgm.Context(tsgm.default_params(W, H)) as ctx:
        dD, dP, dDz, drz = dev(D), dev(P), dev(Dz), dev(rz)
        oD, oP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.adjoint_forward(dD, dP, pose6, K, B, q, s_r, dDz, drz, oD, oP)
        keys = empty((H, W), np.uint64)
        ctx.inspect("zkeys", keys, W * H)
        g = ctx.adjoint_backward(dD, dP, pose6, K, B, q, s_r, dDz, drz, dev(gD), dev(gP))
        Dg, Pg, kg = host(oD, np.float32), host(oP, np.float32), host(keys, np.uint64)
    # forward parity with the oracle's binary32 pipeline (R rounded once from binary64)
    R32 = oracle.rodrigues(pose6[:3]).astype(np.float32)
    _, H32 = oracle.build_H(R32, pose6[3:].astype(np.float32), float(K[0, 0]), float(B))
    Dp, Pp, win = oracle.warp_predict(D, P, H32, K[0, 2], K[1, 2], q)
    rz_scaled = np.where(rz >= 0, (np.float32(s_r) * rz).astype(np.float32), rz)
    Do, Po = oracle.kalman(Dp, Pp, Dz, rz_scaled)
    src = np.where(kg == np.uint64(0xFFFFFFFFFFFFFFFF), -1, (kg & np.uint64(0xFFFFFFFF)).astype(np.int64))
    assert np.array_equal(src, win)
    assert np.array_equal(Dg < 0, Do < 0)
    v = Do >= 0
    assert np.max(np.abs(Dg[v] - Do[v])) <= 1e-4
    assert np.max(np.abs(Pg[v] - Po[v]) / Po[v]) <= 1e-5
    # gradients: binary64 finite differences with the same winners, and the analytic reference
    g_fd = oracle.adjoint_fd(D, P, win, pose6, K, B, q, s_r, Dz, rz, gD, gP, h=1e-4)
    g_an = oracle.adjoint_grad_f64(D, P, win, pose6, K, B, q, s_r, Dz, rz, gD, gP)
    scale = np.abs(g_fd).max()
    for ref in (g_fd, g_an):
        big = np.abs(ref) > 1e-6 * scale
        assert np.all(np.abs(g[big] - ref[big]) <= 1e-3 * np.abs(ref[big])), (g, ref)
        assert np.all(np.abs(g[~big] - ref[~big]) <= 1e-6 * scale)
    assert g[3] == 0 and g[4] == 0


def test_autograd_function_matches_direct_calls(tsgm):
    from paper_1708_06301_gb300.adjoint import warp_kalman
    D, P, Dz, rz, pose6, gD, gP, K = config3_inputs(21, W=320, H=96)
    H, W = D.shape
    with tsgm.Context(tsgm.default_params(W, H, d_max=63)) as ctx:
        theta = torch.tensor(np.concatenate([pose6, [0.3, 1.2]]), dtype=torch.float64,
                             requires_grad=True)
        dD, dP, dDz, drz = dev(D), dev(P), dev(Dz), dev(rz)
        Dt, Pt = warp_kalman(theta, dD, dP, dDz, drz, K, B, ctx)
        loss = (Dt * dev(gD)).sum(dtype=torch.float64) + (Pt * dev(gP)).sum(dtype=torch.float64)
        loss.backward()
        g_direct = ctx.adjoint_backward(dD, dP, pose6, K, B, 0.3, 1.2, dDz, drz, dev(gD), dev(gP))
    assert np.allclose(theta.grad.numpy(), g_direct, rtol=1e-9, atol=1e-9)


def test_fit_pose_and_noise_on_synthetic_scene(tsgm):
    """Refine t_z and fit q, s_r by gradient descent on sum((D - gt)^2) over a rendered forward
    motion: the loss drops and t_z moves towards the true translation."""
    from paper_1708_06301_gb300.adjoint import warp_kalman
    seq = synth.small_pair(1)
    W, H = seq.cam.W, seq.cam.H
    gt0, gt1 = seq.gt_disp[0], seq.gt_disp[1]
    rng = np.random.default_rng(0)
    Dz = (gt1 + rng.normal(scale=0.4, size=gt1.shape)).astype(np.float32)
    rz = np.full_like(Dz, 0.2)
    P0 = np.full_like(gt0, 0.5)
    true_tz = float(seq.t[1][2])
    theta = torch.tensor([0, 0, 0, 0, 0, true_tz + 0.15, 0.5, 2.0], dtype=torch.float64,
                         requires_grad=True)
    target = dev(gt1)
    losses = []
    opt = torch.optim.Adam([theta], lr=0.01)
    with tsgm.Context(tsgm.default_params(W, H, d_max=63, census_w=5, census_h=5, n_paths=4)) as ctx:
        dD, dP, dDz, drz = dev(gt0), dev(P0), dev(Dz), dev(rz)
        for _ in range(60):
            opt.zero_grad()
            Dt, _ = warp_kalman(theta, dD, dP, dDz, drz, seq.K, f32(seq.cam.b), ctx)
            m = Dt >= 0
            loss = ((Dt - target)[m].double() ** 2).mean()
            loss.backward()
            with torch.no_grad():
                theta.grad[:5] = 0  # refine t_z, q and s_r only
            opt.step()
            with torch.no_grad():
                theta[6:].clamp_(min=1e-3)
            losses.append(float(loss.detach()))
    assert losses[-1] < 0.8 * losses[0]
    assert abs(float(theta[5]) - true_tz) < 0.5 * 0.15
