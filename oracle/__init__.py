"""CPU oracle of the ego-motion-reduced SGM hot path (arXiv 1708.06301), for tests only.

TEST INFRASTRUCTURE: only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package. The product path (the CUDA library and its binding) never
imports, links or runs it, and this package imports nothing from the product package.

The arithmetic lives in `tsgm_oracle.cpp` (plain C++17, built with `-O2 -ffp-contract=off`);
this module compiles it, marshals numpy arrays through ctypes, and composes the per-stage
functions into the per-frame pipeline of the paper (Sec. 2: prediction, matching, update).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsgm_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, no SIMD intrinsics, no FP contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                        "-shared", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_OUT)
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _same_shape(shape, **arrays):
    """The C functions trust the sizes they are given: every array a call reads or writes must
    have the shape the call takes its sizes from, or it would be read past its end."""
    for name, a in arrays.items():
        if np.shape(a) != tuple(shape):
            raise ValueError(f"{name} has shape {np.shape(a)}, expected {tuple(shape)}")


def _ragged(lo, hi, off, **volumes):
    """A ragged volume is indexed through off: it must be the exclusive scan of the window
    lengths of lo, hi (inside [0, 2^15)), and every volume must hold off[n] cells."""
    _same_shape(np.shape(lo), hi=hi)
    if np.any(np.asarray(lo) < 0) or np.any(np.asarray(hi) < np.asarray(lo)):
        raise ValueError("windows need 0 <= lo <= hi")
    if not np.array_equal(np.asarray(off).reshape(-1), offsets(lo, hi)):
        raise ValueError("off is not the exclusive scan of the window lengths")
    cells = int(np.asarray(off).reshape(-1)[-1])
    for name, a in volumes.items():
        if np.size(a) != cells:
            raise ValueError(f"{name} has {np.size(a)} cells, expected {cells}")


# ----------------------------------------------------------------------------------------------
# Parameters (defaults are the readings listed in the design notes)
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    width: int
    height: int
    d_max: int = 63            # D = d_max + 1 labels
    census_w: int = 5
    census_h: int = 5
    n_paths: int = 4
    P1: int = 8
    P2: int = 32
    sigma_mult: float = 3.0    # Sec. 2.3, +-3 sigma window
    q: float = 0.25            # Sec. 2.2, constant ego-motion variance (value not given)
    S_max: float = 10.0        # Sec. 2.3, Eq. 9 threshold per path
    r_min: float = 0.5
    lr_tol: int = 1
    fill_gaps: bool = False    # Sec. 2.2, Eq. 7-8 on the prediction
    gamma_f: float = 1.0       # Eq. 8 similarity threshold (value not given)
    edge_reject: bool = False  # Sec. 2.2, reject predicted pixels near disparity discontinuities
    edge_thr: float = 1.0      # discontinuity threshold of the edge rejection (value not given)
    pred_lr_check: bool = False  # Sec. 2.2 / Fig. 3(d), left-right check of the prediction
    pred_lr_tol: float = 1.0     # its similarity threshold (value not given)
    sad_check: bool = False      # Sec. 2.4, SAD check of the updated map on the two images
    sad_w: int = 5               # patch (odd sizes; not given)
    sad_h: int = 5
    sad_thr: float = 30.0        # mean absolute difference per patch pixel (value not given)
    full_range: bool = False     # search [0, D-1] everywhere (prediction and update as usual)

    @property
    def D(self) -> int:
        return self.d_max + 1

    @property
    def Bc(self) -> int:
        return self.census_w * self.census_h - 1

    @property
    def s_thr(self) -> float:
        return float(np.float32(self.S_max) * np.float32(self.n_paths))


# ----------------------------------------------------------------------------------------------
# Per-stage wrappers
# ----------------------------------------------------------------------------------------------

def build_H(R, t, f: float, b: float):
    """Eq. 4 in binary64; returns (H64, H32) row-major 4x4."""
    lib = _load()
    R64 = _c(np.asarray(R, dtype=np.float64).reshape(9), np.float64)   # reshape checks the sizes
    t64 = _c(np.asarray(t, dtype=np.float64).reshape(3), np.float64)
    H = np.zeros(16, dtype=np.float64)
    lib.oracle_build_H(_p(R64), _p(t64), ctypes.c_double(f), ctypes.c_double(b), _p(H))
    return H.reshape(4, 4), H.astype(np.float32).reshape(4, 4)


def warp_predict(Dprev, Pprev, H32, cx: float, cy: float, q: float):
    lib = _load()
    Hh, W = Dprev.shape
    _same_shape((Hh, W), Pprev=Pprev)
    Dprev = _c(Dprev, np.float32)
    Pprev = _c(Pprev, np.float32)
    Hm = _c(H32, np.float32).reshape(16)
    Dp = np.empty((Hh, W), np.float32)
    Pp = np.empty((Hh, W), np.float32)
    win = np.empty((Hh, W), np.int32)
    lib.oracle_warp_predict(W, Hh, _p(Dprev), _p(Pprev), _p(Hm), ctypes.c_float(cx),
                            ctypes.c_float(cy), ctypes.c_float(q), _p(Dp), _p(Pp), _p(win))
    return Dp, Pp, win


def fill_gaps(Dp, Pp, gamma_f: float):
    """Eq. 7-8: horizontal then vertical one-pixel gap filling of a prediction (copies)."""
    lib = _load()
    Hh, W = Dp.shape
    _same_shape((Hh, W), Pp=Pp)
    D = np.array(Dp, dtype=np.float32, copy=True)
    P = np.array(Pp, dtype=np.float32, copy=True)
    lib.oracle_fill_gaps(W, Hh, ctypes.c_float(gamma_f), _p(D), _p(P))
    return D, P


def edge_reject(Dp, Pp, edge_thr: float):
    """Sec. 2.2 disparity refinement: reject predicted pixels next to a disparity discontinuity
    (8-neighbourhood, |d - d_n| >= edge_thr with a valid neighbour; copies)."""
    lib = _load()
    Hh, W = Dp.shape
    _same_shape((Hh, W), Pp=Pp)
    D = np.array(Dp, dtype=np.float32, copy=True)
    P = np.array(Pp, dtype=np.float32, copy=True)
    lib.oracle_edge_reject(W, Hh, ctypes.c_float(edge_thr), _p(D), _p(P))
    return D, P


def pred_lr_check(Dp, Pp, tol: float):
    """Sec. 2.2 / Fig. 3(d): left-right consistency check of the prediction against the right
    view's prediction formed from it (nearest surface per right pixel); copies."""
    lib = _load()
    Hh, W = Dp.shape
    _same_shape((Hh, W), Pp=Pp)
    D = np.array(Dp, dtype=np.float32, copy=True)
    P = np.array(Pp, dtype=np.float32, copy=True)
    lib.oracle_pred_lr_check(W, Hh, ctypes.c_float(tol), _p(D), _p(P))
    return D, P


def sad_check(left, right, D, P, sw: int, sh: int, sad_thr: float):
    """Sec. 2.4: reject pixels of the updated map whose left/right patch SAD exceeds sad_thr per
    patch pixel; copies."""
    lib = _load()
    Hh, W = D.shape
    _same_shape((Hh, W), P=P, left=left, right=right)
    D = np.array(D, dtype=np.float32, copy=True)
    P = np.array(P, dtype=np.float32, copy=True)
    lib.oracle_sad_check(W, Hh, int(sw), int(sh), ctypes.c_float(sad_thr),
                         _p(_c(left, np.uint8)), _p(_c(right, np.uint8)), _p(D), _p(P))
    return D, P


def windows(Dp, Pp, D: int, sigma_mult: float):
    lib = _load()
    Hh, W = Dp.shape
    _same_shape((Hh, W), Pp=Pp)
    Dp = _c(Dp, np.float32)
    Pp = _c(Pp, np.float32)
    lo = np.empty((Hh, W), np.int16)
    hi = np.empty((Hh, W), np.int16)
    off = np.empty(W * Hh + 1, np.uint32)
    lib.oracle_windows.restype = ctypes.c_int64
    n = lib.oracle_windows(W, Hh, D, ctypes.c_float(sigma_mult), _p(Dp), _p(Pp), _p(lo), _p(hi),
                           _p(off))
    return lo, hi, off, int(n)


def offsets(lo, hi):
    """Exclusive prefix sum of the window lengths (row-major), length n+1."""
    w = (np.asarray(hi, np.int64) - np.asarray(lo, np.int64) + 1).reshape(-1)
    off = np.zeros(w.size + 1, np.uint64)
    np.cumsum(w, out=off[1:])
    return off.astype(np.uint32)


def census(img, cw: int, ch: int):
    lib = _load()
    Hh, W = img.shape
    img = _c(img, np.uint8)
    codes = np.empty((Hh, W), np.uint64)
    lib.oracle_census(W, Hh, cw, ch, _p(img), _p(codes))
    return codes


def cost(cl, cr, lo, hi, off, Bc: int):
    lib = _load()
    Hh, W = cl.shape
    _same_shape((Hh, W), cr=cr, lo=lo)
    _ragged(lo, hi, off)
    C = np.empty(int(off[-1]), np.uint8)
    lib.oracle_cost(W, Hh, Bc, _p(_c(cl, np.uint64)), _p(_c(cr, np.uint64)), _p(_c(lo, np.int16)),
                    _p(_c(hi, np.int16)), _p(_c(off, np.uint32)), _p(C))
    return C


def sgm_path(C, lo, hi, off, direction: int, P1: int, P2: int):
    lib = _load()
    Hh, W = lo.shape
    _ragged(lo, hi, off, C=C)
    L = np.empty(int(off[-1]), np.uint16)
    lib.oracle_sgm_path(W, Hh, direction, P1, P2, _p(_c(C, np.uint8)), _p(_c(lo, np.int16)),
                        _p(_c(hi, np.int16)), _p(_c(off, np.uint32)), _p(L))
    return L


def sgm(C, lo, hi, off, n_paths: int, P1: int, P2: int):
    lib = _load()
    Hh, W = lo.shape
    _ragged(lo, hi, off, C=C)
    S = np.empty(int(off[-1]), np.uint16)
    lib.oracle_sgm(W, Hh, n_paths, P1, P2, _p(_c(C, np.uint8)), _p(_c(lo, np.int16)),
                   _p(_c(hi, np.int16)), _p(_c(off, np.uint32)), _p(S))
    return S


def select(S, lo, hi, off, s_thr: float, r_min: float):
    lib = _load()
    Hh, W = lo.shape
    _ragged(lo, hi, off, S=S)
    dstar = np.empty((Hh, W), np.int32)
    Dz = np.empty((Hh, W), np.float32)
    rz = np.empty((Hh, W), np.float32)
    lib.oracle_select(W, Hh, _p(_c(S, np.uint16)), _p(_c(lo, np.int16)), _p(_c(hi, np.int16)),
                      _p(_c(off, np.uint32)), ctypes.c_float(s_thr), ctypes.c_float(r_min),
                      _p(dstar), _p(Dz), _p(rz))
    return dstar, Dz, rz


def lr_check(S, lo, hi, off, dstar, D: int, tol: int, Dz, rz):
    """Returns (dright, valid, Dz_masked, rz_masked); inputs Dz, rz are not modified."""
    lib = _load()
    Hh, W = lo.shape
    _ragged(lo, hi, off, S=S)
    _same_shape((Hh, W), dstar=dstar, Dz=Dz, rz=rz)
    dright = np.empty((Hh, W), np.int32)
    valid = np.empty((Hh, W), np.uint8)
    Dz = np.array(Dz, dtype=np.float32, copy=True)
    rz = np.array(rz, dtype=np.float32, copy=True)
    lib.oracle_lr_check(W, Hh, D, _p(_c(S, np.uint16)), _p(_c(lo, np.int16)), _p(_c(hi, np.int16)),
                        _p(_c(off, np.uint32)), _p(_c(dstar, np.int32)), tol, _p(dright),
                        _p(valid), _p(Dz), _p(rz))
    return dright, valid, Dz, rz


def kalman(Dp, Pp, Dz, rz):
    lib = _load()
    shape = np.shape(Dp)
    _same_shape(shape, Pp=Pp, Dz=Dz, rz=rz)
    n = int(np.prod(shape))
    D = np.empty(shape, np.float32)
    P = np.empty(shape, np.float32)
    lib.oracle_kalman(n, _p(_c(Dp, np.float32)), _p(_c(Pp, np.float32)), _p(_c(Dz, np.float32)),
                      _p(_c(rz, np.float32)), _p(D), _p(P))
    return D, P


# ----------------------------------------------------------------------------------------------
# Composite stages (Sec. 2: steps 2-4 of the per-frame algorithm)
# ----------------------------------------------------------------------------------------------

def match(left, right, lo, hi, prm: Params, keep: bool = False):
    """Stereo matching in the given windows: census, ragged cost, SGM, WTA + sub-pixel + r,
    left-right check. Returns (Dz, rz) or, with keep=True, a dict of every intermediate."""
    off = offsets(lo, hi)
    cl = census(left, prm.census_w, prm.census_h)
    cr = census(right, prm.census_w, prm.census_h)
    C = cost(cl, cr, lo, hi, off, prm.Bc)
    S = sgm(C, lo, hi, off, prm.n_paths, prm.P1, prm.P2)
    dstar, Dz0, rz0 = select(S, lo, hi, off, prm.s_thr, prm.r_min)
    dright, valid, Dz, rz = lr_check(S, lo, hi, off, dstar, prm.D, prm.lr_tol, Dz0, rz0)
    if not keep:
        return Dz, rz
    return dict(off=off, cl=cl, cr=cr, C=C, S=S, dstar=dstar, Dz_raw=Dz0, rz_raw=rz0,
                dright=dright, valid=valid, Dz=Dz, rz=rz)


def _finite_nonneg(a):
    """The validity test of a disparity or variance: finite and >= 0 (NaN, inf, -1 invalid)."""
    a = np.asarray(a, np.float32)
    return (a >= 0) & (a <= np.finfo(np.float32).max)


def K_fbc(K):
    K = np.asarray(K, dtype=np.float64).reshape(3, 3)
    return float(K[0, 0]), float(K[0, 2]), float(K[1, 2])


class Tracker:
    """Per-frame loop of Sec. 2 on the CPU: predict (warp + variance), reduce the search space,
    match, update. The first frame has no prediction and searches the whole range."""

    def __init__(self, prm: Params):
        self.prm = prm
        self.D = None
        self.P = None

    def frame(self, left, right, R, t, K, baseline: float, keep: bool = False):
        prm = self.prm
        Hh, W = prm.height, prm.width
        out = {}
        # calibration and pose enter as binary32, like the C interface of the path
        baseline = float(np.float32(baseline))
        K = np.asarray(K, dtype=np.float32)
        if self.D is None:
            Dp = np.full((Hh, W), -1.0, np.float32)
            Pp = np.full((Hh, W), -1.0, np.float32)
        else:
            f, cx, cy = K_fbc(K)
            _, H32 = build_H(np.asarray(R, np.float32), np.asarray(t, np.float32), f, baseline)
            Dp, Pp, win = warp_predict(self.D, self.P, H32, np.float32(cx), np.float32(cy), prm.q)
            out["winner"] = win
            out["H32"] = H32
            out["Dpred_raw"], out["Ppred_raw"] = Dp, Pp
            if prm.edge_reject:
                Dp, Pp = edge_reject(Dp, Pp, prm.edge_thr)
            if prm.fill_gaps:
                Dp, Pp = fill_gaps(Dp, Pp, prm.gamma_f)
            if prm.pred_lr_check:
                Dp, Pp = pred_lr_check(Dp, Pp, prm.pred_lr_tol)
        if prm.full_range:
            lo = np.zeros((Hh, W), np.int16)
            hi = np.full((Hh, W), prm.D - 1, np.int16)
            n_cells = W * Hh * prm.D
        else:
            lo, hi, off, n_cells = windows(Dp, Pp, prm.D, prm.sigma_mult)
        m = match(left, right, lo, hi, prm, keep=True)
        D, P = kalman(Dp, Pp, m["Dz"], m["rz"])
        if prm.sad_check:
            out["D_unchecked"], out["P_unchecked"] = D, P
            D, P = sad_check(left, right, D, P, prm.sad_w, prm.sad_h, prm.sad_thr)
        # Sec. 2.4, disparity consistency check: where the matched disparity was rejected, the
        # true minimum may lie outside the reduced window, so the next frame searches the whole
        # range there. The updated map still carries the prediction (Sec. 3: it combines the
        # matched and the predicted map), but the state passed to the next frame keeps no value.
        meas = _finite_nonneg(m["Dz"]) & _finite_nonneg(m["rz"])
        self.D = np.where(meas, D, np.float32(-1.0)).astype(np.float32)
        self.P = np.where(meas, P, np.float32(-1.0)).astype(np.float32)
        if keep:
            out.update(m)
            out.update(Dpred=Dp, Ppred=Pp, lo=lo, hi=hi, n_cells=n_cells, D=D, P=P,
                       D_state=self.D, P_state=self.P)
            return out
        return D, P


# ----------------------------------------------------------------------------------------------
# Adjoint references (float stages: prediction Eq. 3, 5, 6 then Kalman Eq. 10-12), binary64
# ----------------------------------------------------------------------------------------------

def rodrigues(w):
    """R = exp([w]x) for a rotation vector w (binary64)."""
    w = np.asarray(w, np.float64).reshape(3)
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.eye(3)
    k = w / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)


def warp_kalman_f64(prevD, prevP, winner, pose6, K, b, q, s_r, Dz, rz):
    """Prediction and update in binary64 with the z-buffer winners held fixed (`winner`: source
    index per target or -1). Returns (D, P) as float64 maps."""
    pose6 = np.asarray(pose6, np.float64)
    f, cx, cy = K_fbc(K)
    H64, _ = build_H(rodrigues(pose6[:3]), pose6[3:], f, float(b))
    Hh, W = prevD.shape
    win = np.asarray(winner).reshape(-1)
    has = win >= 0
    s = win[has]
    d = prevD.reshape(-1)[s].astype(np.float64)
    p = prevP.reshape(-1)[s].astype(np.float64)
    u = (s % W).astype(np.float64) - float(np.float32(cx))
    v = (s // W).astype(np.float64) - float(np.float32(cy))
    w = H64 @ np.stack([u, v, d, np.ones_like(d)])
    dp = w[2] / w[3]                       # Eq. 3: divide by the fourth component
    pp = (dp / d) ** 2 * p + q             # Eq. 5-6
    n = W * Hh
    Dp = np.full(n, -1.0)
    Pp = np.full(n, -1.0)
    Dp[has] = dp
    Pp[has] = pp
    dz = Dz.reshape(-1).astype(np.float64)
    rr = rz.reshape(-1).astype(np.float64)
    mv = (dz >= 0) & (rr >= 0) & np.isfinite(dz) & np.isfinite(rr)
    r = s_r * rr
    D = np.full(n, -1.0)
    P = np.full(n, -1.0)
    both = has & mv
    Kg = Pp[both] / (Pp[both] + r[both])   # Eq. 10
    D[both] = Dp[both] + Kg * (dz[both] - Dp[both])  # Eq. 11
    P[both] = (1 - Kg) * Pp[both]          # Eq. 12
    mo = mv & ~has
    D[mo], P[mo] = dz[mo], r[mo]
    po = has & ~mv
    D[po], P[po] = Dp[po], Pp[po]
    return D.reshape(Hh, W), P.reshape(Hh, W)


def adjoint_fd(prevD, prevP, winner, pose6, K, b, q, s_r, Dz, rz, gD, gP, h=1e-4):
    """Central finite differences (binary64) of L = sum(gD * D + gP * P) with respect to
    (w0, w1, w2, t0, t1, t2, q, s_r)."""
    th = np.concatenate([np.asarray(pose6, np.float64), [q, s_r]])
    gD = gD.astype(np.float64)
    gP = gP.astype(np.float64)

    def loss(x):
        D, P = warp_kalman_f64(prevD, prevP, winner, x[:6], K, b, x[6], x[7], Dz, rz)
        return float(np.sum(gD * D) + np.sum(gP * P))

    g = np.zeros(8)
    for i in range(8):
        e = np.zeros(8)
        e[i] = h
        g[i] = (loss(th + e) - loss(th - e)) / (2 * h)
    return g


def adjoint_grad_f64(prevD, prevP, winner, pose6, K, b, q, s_r, Dz, rz, gD, gP):
    """Analytic gradient of L = sum(gD * D + gP * P) in binary64, written from the forward
    definitions above; dR/dw by central differences of `rodrigues` (step 1e-6)."""
    pose6 = np.asarray(pose6, np.float64)
    f, cx, cy = K_fbc(K)
    R = rodrigues(pose6[:3])
    t = pose6[3:]
    Hh, W = prevD.shape
    win = np.asarray(winner).reshape(-1)
    has = win >= 0
    s = win[has]
    d = prevD.reshape(-1)[s].astype(np.float64)
    p = prevP.reshape(-1)[s].astype(np.float64)
    u = (s % W).astype(np.float64) - float(np.float32(cx))
    v = (s // W).astype(np.float64) - float(np.float32(cy))
    # fourth row of H = Gamma T Gamma^{-1}: (R20/f, R21/f, t2/(f b), R22)
    w3 = R[2, 0] * u / f + R[2, 1] * v / f + t[2] * d / (f * b) + R[2, 2]
    dp = d / w3
    pp = (dp / d) ** 2 * p + q
    dz = Dz.reshape(-1)[has].astype(np.float64)
    rr = rz.reshape(-1)[has].astype(np.float64)
    mv = (dz >= 0) & (rr >= 0)
    gd = gD.reshape(-1)[has].astype(np.float64)
    gp = gP.reshape(-1)[has].astype(np.float64)
    r = s_r * rr
    den = pp + r
    dD_ddp = np.where(mv, r / den, 1.0)
    dD_dpp = np.where(mv, (dz - dp) * r / den ** 2, 0.0)
    dP_dpp = np.where(mv, (r / den) ** 2, 1.0)
    dD_dr = np.where(mv, -(dz - dp) * pp / den ** 2, 0.0)
    dP_dr = np.where(mv, (pp / den) ** 2, 0.0)
    dL_dpp = gd * dD_dpp + gp * dP_dpp
    dL_ddp = gd * dD_ddp + dL_dpp * 2 * p * dp / d ** 2
    dL_dw3 = dL_ddp * (-d / w3 ** 2)
    g_R2 = np.array([np.sum(dL_dw3 * u / f), np.sum(dL_dw3 * v / f), np.sum(dL_dw3)])
    g_t2 = np.sum(dL_dw3 * d / (f * b))
    g_q = np.sum(dL_dpp)
    g_sr = np.sum((gd * dD_dr + gp * dP_dr) * rr)
    # measurement-only targets: P = s_r r_z
    dzall = Dz.reshape(-1).astype(np.float64)
    rall = rz.reshape(-1).astype(np.float64)
    mo = (~has) & (dzall >= 0) & (rall >= 0)
    g_sr += np.sum(gP.reshape(-1)[mo].astype(np.float64) * rall[mo])
    g = np.zeros(8)
    hstep = 1e-6
    for i in range(3):
        e = np.zeros(3)
        e[i] = hstep
        dR = (rodrigues(pose6[:3] + e) - rodrigues(pose6[:3] - e)) / (2 * hstep)
        g[i] = float(np.dot(g_R2, dR[2]))
    g[5] = g_t2
    g[6] = g_q
    g[7] = g_sr
    return g
