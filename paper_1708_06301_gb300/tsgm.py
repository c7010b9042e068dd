"""Python binding of the tsgm C ABI (`include/tsgm.h`): argument marshalling only.

Every step of the path runs in the CUDA library `_build/libtsgm.so`; this module loads it with
ctypes and passes device pointers (torch tensors' `data_ptr()` or plain integers), host arrays
for poses and calibration, and the current torch CUDA stream. The kernels trust the sizes a
context was created with, so every tensor or host array is checked against them (element count
and element size) before the call; raw integer pointers are passed on unchecked. There is no
fallback: if the library is missing, loading fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtsgm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "tsgm.h")

OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_CUDA, ERR_TIMEOUT, ERR_STATE, ERR_UNIMPLEMENTED = range(7)
FLAG_KEEP_INTERNALS = 1
FLAG_FULL_RANGE = 2
FLAG_FILL_GAPS = 4
FLAG_EDGE_REJECT = 8
FLAG_PRED_LR_CHECK = 16
FLAG_SAD_CHECK = 32
N_STAGES = 8
STAGES = ["warp", "windows", "census", "cost", "sgm", "select", "kalman", "offsets"]
BUF = dict(census_l=0, census_r=1, offsets=2, cost=3, S=4, dstar=5, dright=6, lr_valid=7,
           zkeys=8, windows_lo=9, windows_hi=10, pred_d=11, pred_p=12, counts=13)


class TsgmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tsgm status {status}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("d_max", ctypes.c_int32),
                ("census_w", ctypes.c_int32), ("census_h", ctypes.c_int32),
                ("n_paths", ctypes.c_int32), ("P1", ctypes.c_int32), ("P2", ctypes.c_int32),
                ("sigma_mult", ctypes.c_float), ("q", ctypes.c_float), ("S_max", ctypes.c_float),
                ("r_min", ctypes.c_float), ("lr_tol", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("gamma_f", ctypes.c_float),
                ("edge_thr", ctypes.c_float),
                ("pred_lr_tol", ctypes.c_float),
                ("sad_w", ctypes.c_int32), ("sad_h", ctypes.c_int32),
                ("sad_thr", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_vp = ctypes.c_void_p
_fp = ctypes.POINTER(ctypes.c_float)
_SIGS = {
    "tsgm_default_params": (None, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32]),
    "tsgm_create": (ctypes.c_int, [ctypes.POINTER(Params), _vp, ctypes.POINTER(_vp)]),
    "tsgm_destroy": (None, [_vp]),
    "tsgm_last_error": (ctypes.c_char_p, [_vp]),
    "tsgm_set_stream": (ctypes.c_int, [_vp, _vp]),
    "tsgm_build_H": (ctypes.c_int, [_fp, _fp, _fp, ctypes.c_float, _fp]),
    "tsgm_warp_predict": (ctypes.c_int, [_vp, _vp, _vp, _fp, _fp, _fp, ctypes.c_float, _vp, _vp]),
    "tsgm_windows": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_match": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsgm_kalman_update": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsgm_frame": (ctypes.c_int, [_vp, _vp, _vp, _fp, _fp, _fp, ctypes.c_float, _vp, _vp]),
    "tsgm_frame_host": (ctypes.c_int, [_vp, _vp, _vp, _fp, _fp, _fp, ctypes.c_float, _vp, _vp]),
    "tsgm_reset": (ctypes.c_int, [_vp]),
    "tsgm_state_export": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int32)]),
    "tsgm_state_import": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32]),
    "tsgm_census": (ctypes.c_int, [_vp, _vp, _vp]),
    "tsgm_fill_gaps": (ctypes.c_int, [_vp, _vp, _vp]),
    "tsgm_edge_reject": (ctypes.c_int, [_vp, _vp, _vp]),
    "tsgm_pred_lr_check": (ctypes.c_int, [_vp, _vp, _vp]),
    "tsgm_frame_host_async": (ctypes.c_int, [_vp, _vp, _vp, _fp, _fp, _fp, ctypes.c_float, _vp, _vp]),
    "tsgm_wait": (ctypes.c_int, [_vp]),
    "tsgm_warp_predict_noalloc": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _fp, _fp,
                                                 _fp, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp,
                                                 ctypes.c_char_p, ctypes.c_size_t]),
    "tsgm_sad_check": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "tsgm_inspect": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_uint64]),
    "tsgm_cells": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_profile": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "tsgm_launches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_batch_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_int32,
                                         _vp, ctypes.POINTER(_vp)]),
    "tsgm_batch_destroy": (None, [_vp]),
    "tsgm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "tsgm_batch_match": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsgm_batch_autotune": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_int32)]),
    "tsgm_batch_cells": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_int32)]),
    "tsgm_batch_launches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_batch_frame": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tsgm_batch_reset": (ctypes.c_int, [_vp]),
    "tsgm_batch_stream_status": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32)]),
    "tsgm_batch_pool": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_batch_profile": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                          ctypes.POINTER(ctypes.c_float),
                                          ctypes.POINTER(ctypes.c_float)]),
    "tsgm_server_create": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.POINTER(_vp)]),
    "tsgm_server_destroy": (None, [_vp]),
    "tsgm_server_submit": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _fp, _fp, _fp,
                                          ctypes.c_float, _vp, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_server_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "tsgm_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint64),
                                         ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "tsgm_adjoint_forward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _fp,
                                            ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp,
                                            _vp, _vp, _vp]),
    "tsgm_adjoint_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(ctypes.c_double), _fp,
                                             ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp,
                                             _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "tsgm_stage_times": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]),
}


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"tsgm CUDA library not found at {path}; build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def header_symbols(path: str = HEADER):
    """Function names declared in the public header."""
    text = open(path).read()
    return sorted(set(re.findall(r"\b(tsgm_[A-Za-z_0-9]+)\s*\(", text)))


def default_params(width: int, height: int, **kw) -> Params:
    p = Params()
    load().tsgm_default_params(ctypes.byref(p), int(width), int(height))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if hasattr(x, "is_contiguous") and not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _dptr(x, n: int, esize: int, what: str) -> int:
    """Device pointer of a buffer that a call reads or writes as n elements of esize bytes. The
    kernels trust the sizes the context was created with, so a CUDA tensor must be at least that
    large, with elements of that size. A raw integer pointer, or None where the call allows it,
    is passed on unchecked."""
    p = _ptr(x)
    if hasattr(x, "numel") and hasattr(x, "element_size"):
        if x.element_size() != esize:
            raise ValueError(f"{what}: expected elements of {esize} bytes, got {x.element_size()}")
        if x.numel() < n:
            raise ValueError(f"{what}: expected at least {n} elements, got {x.numel()}")
    return p


def _hptr(a, n: int, esize: int, what: str) -> int:
    """Address of a host buffer (a numpy array or a CPU tensor, pinned for the asynchronous
    calls) of at least n contiguous elements of esize bytes."""
    if hasattr(a, "data_ptr"):
        if getattr(a, "is_cuda", False):
            raise ValueError(f"{what}: expected a host buffer, got a CUDA tensor")
        if not a.is_contiguous():
            raise ValueError(f"{what}: expected a contiguous tensor")
        size, item, ptr = a.numel(), a.element_size(), a.data_ptr()
    elif isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: expected a contiguous array")
        size, item, ptr = a.size, a.itemsize, a.ctypes.data
    else:
        raise TypeError(f"{what}: cannot take a host address of {type(a)}")
    if item != esize:
        raise ValueError(f"{what}: expected elements of {esize} bytes, got {item}")
    if size < n:
        raise ValueError(f"{what}: expected at least {n} elements, got {size}")
    return ptr


# element bytes of the internal buffers that tsgm_inspect copies out
_BUF_BYTES = dict(census_l=8, census_r=8, offsets=4, cost=1, S=2, dstar=2, dright=2, lr_valid=1,
                  zkeys=8, windows_lo=2, windows_hi=2, pred_d=4, pred_p=4, counts=4)


def _host_f32(a, n: int):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32).reshape(-1))
    if arr.size != n:
        raise ValueError(f"expected {n} floats, got {arr.size}")
    return arr, arr.ctypes.data_as(_fp)


def build_H(R, t, K, baseline: float) -> np.ndarray:
    lib = load()
    Ra, Rp = _host_f32(R, 9)
    ta, tp = _host_f32(t, 3)
    Ka, Kp = _host_f32(K, 9)
    out = np.zeros(16, np.float32)
    st = lib.tsgm_build_H(Rp, tp, Kp, ctypes.c_float(baseline), out.ctypes.data_as(_fp))
    if st != OK:
        raise TsgmError(st, "tsgm_build_H: invalid pose or calibration")
    return out.reshape(4, 4)


def _current_stream() -> int:
    """Handle of torch's current CUDA stream (0 is the legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


class Context:
    """One tsgm context: scratch for one image size plus the per-stream previous state."""

    def __init__(self, params: Params, stream: int | None = None):
        self.lib = load()
        self.params = params
        self.W, self.H = params.width, params.height
        self.n = self.W * self.H
        h = _vp()
        s = _current_stream() if stream is None else int(stream)
        st = self.lib.tsgm_create(ctypes.byref(params), _vp(s or None), ctypes.byref(h))
        if st != OK:
            raise TsgmError(st, "tsgm_create failed (see stderr for the parameter check)")
        self.h = h

    # -- plumbing -------------------------------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != OK:
            msg = self.lib.tsgm_last_error(self.h)
            raise TsgmError(st, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsgm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_stream(self, stream: int | None):
        self._check(self.lib.tsgm_set_stream(self.h, _vp(stream or None)), "tsgm_set_stream")

    # -- the path ---------------------------------------------------------------------------------
    def warp_predict(self, prev_D, prev_P, R, t, K, baseline, pred_D, pred_P):
        Ra, Rp = _host_f32(R, 9)
        ta, tp = _host_f32(t, 3)
        Ka, Kp = _host_f32(K, 9)
        n = self.n
        self._check(self.lib.tsgm_warp_predict(self.h, _dptr(prev_D, n, 4, "prev_D"),
                                               _dptr(prev_P, n, 4, "prev_P"), Rp, tp, Kp,
                                               ctypes.c_float(baseline), _dptr(pred_D, n, 4, "pred_D"),
                                               _dptr(pred_P, n, 4, "pred_P")), "tsgm_warp_predict")

    def windows(self, pred_D, pred_P, d_lo, d_hi, want_cells: bool = False):
        cells = ctypes.c_uint64(0)
        n = self.n
        self._check(self.lib.tsgm_windows(self.h, _dptr(pred_D, n, 4, "pred_D"),
                                          _dptr(pred_P, n, 4, "pred_P"), _dptr(d_lo, n, 2, "d_lo"),
                                          _dptr(d_hi, n, 2, "d_hi"),
                                          ctypes.byref(cells) if want_cells else None),
                    "tsgm_windows")
        return int(cells.value) if want_cells else None

    def match(self, left, right, d_lo, d_hi, D_z, r_z):
        n = self.n
        self._check(self.lib.tsgm_match(self.h, _dptr(left, n, 1, "left"), _dptr(right, n, 1, "right"),
                                        _dptr(d_lo, n, 2, "d_lo"), _dptr(d_hi, n, 2, "d_hi"),
                                        _dptr(D_z, n, 4, "D_z"), _dptr(r_z, n, 4, "r_z")),
                    "tsgm_match")

    def kalman_update(self, pred_D, pred_P, D_z, r_z, D, P):
        n = self.n
        self._check(self.lib.tsgm_kalman_update(self.h, _dptr(pred_D, n, 4, "pred_D"),
                                                _dptr(pred_P, n, 4, "pred_P"), _dptr(D_z, n, 4, "D_z"),
                                                _dptr(r_z, n, 4, "r_z"), _dptr(D, n, 4, "D"),
                                                _dptr(P, n, 4, "P")), "tsgm_kalman_update")

    def frame(self, left, right, R, t, K, baseline, D, P):
        Ra, Rp = _host_f32(R, 9)
        ta, tp = _host_f32(t, 3)
        Ka, Kp = _host_f32(K, 9)
        n = self.n
        self._check(self.lib.tsgm_frame(self.h, _dptr(left, n, 1, "left"), _dptr(right, n, 1, "right"),
                                        Rp, tp, Kp, ctypes.c_float(baseline), _dptr(D, n, 4, "D"),
                                        _dptr(P, n, 4, "P")), "tsgm_frame")

    def frame_host(self, left: np.ndarray, right: np.ndarray, R, t, K, baseline, D: np.ndarray,
                   P: np.ndarray):
        """Host buffers (numpy or pinned torch CPU tensors) in and out; synchronises."""
        Ra, Rp = _host_f32(R, 9)
        ta, tp = _host_f32(t, 3)
        Ka, Kp = _host_f32(K, 9)
        n = self.n
        self._check(self.lib.tsgm_frame_host(self.h, _hptr(left, n, 1, "left"), _hptr(right, n, 1, "right"),
                                             Rp, tp, Kp, ctypes.c_float(baseline),
                                             _hptr(D, n, 4, "D"), _hptr(P, n, 4, "P")),
                    "tsgm_frame_host")

    def frame_host_async(self, left, right, R, t, K, baseline, D, P):
        """Pinned host buffers in and out; returns at once (see tsgm_frame_host_async). The image
        and map buffers must stay alive and untouched until wait(); R, t, K are read during the
        call."""
        Ra, Rp = _host_f32(R, 9)
        ta, tp = _host_f32(t, 3)
        Ka, Kp = _host_f32(K, 9)
        n = self.n
        self._check(self.lib.tsgm_frame_host_async(self.h, _hptr(left, n, 1, "left"),
                                                   _hptr(right, n, 1, "right"), Rp, tp, Kp,
                                                   ctypes.c_float(baseline), _hptr(D, n, 4, "D"),
                                                   _hptr(P, n, 4, "P")),
                    "tsgm_frame_host_async")

    def wait(self):
        self._check(self.lib.tsgm_wait(self.h), "tsgm_wait")

    def reset(self):
        self._check(self.lib.tsgm_reset(self.h), "tsgm_reset")

    def state_export(self):
        D = np.empty((self.H, self.W), np.float32)
        P = np.empty((self.H, self.W), np.float32)
        has = ctypes.c_int32(0)
        self._check(self.lib.tsgm_state_export(self.h, D.ctypes.data, P.ctypes.data, ctypes.byref(has)),
                    "tsgm_state_export")
        return D, P, bool(has.value)

    def state_import(self, D, P, has_prev: bool = True):
        D = np.ascontiguousarray(D, np.float32)
        P = np.ascontiguousarray(P, np.float32)
        self._check(self.lib.tsgm_state_import(self.h, _hptr(D, self.n, 4, "D"),
                                               _hptr(P, self.n, 4, "P"), int(has_prev)),
                    "tsgm_state_import")

    def fill_gaps(self, pred_D, pred_P):
        self._check(self.lib.tsgm_fill_gaps(self.h, _dptr(pred_D, self.n, 4, "pred_D"),
                                            _dptr(pred_P, self.n, 4, "pred_P")), "tsgm_fill_gaps")

    def edge_reject(self, pred_D, pred_P):
        self._check(self.lib.tsgm_edge_reject(self.h, _dptr(pred_D, self.n, 4, "pred_D"),
                                              _dptr(pred_P, self.n, 4, "pred_P")),
                    "tsgm_edge_reject")

    def pred_lr_check(self, pred_D, pred_P):
        self._check(self.lib.tsgm_pred_lr_check(self.h, _dptr(pred_D, self.n, 4, "pred_D"),
                                                _dptr(pred_P, self.n, 4, "pred_P")),
                    "tsgm_pred_lr_check")

    def sad_check(self, left, right, D, P):
        n = self.n
        self._check(self.lib.tsgm_sad_check(self.h, _dptr(left, n, 1, "left"), _dptr(right, n, 1, "right"),
                                            _dptr(D, n, 4, "D"), _dptr(P, n, 4, "P")),
                    "tsgm_sad_check")

    def census(self, img, codes):
        self._check(self.lib.tsgm_census(self.h, _dptr(img, self.n, 1, "img"),
                                         _dptr(codes, self.n, 8, "codes")), "tsgm_census")

    def inspect(self, which: str, dst, count: int):
        need = int(count) * _BUF_BYTES[which]
        if hasattr(dst, "numel") and dst.numel() * dst.element_size() < need:
            raise ValueError(f"inspect {which}: dst holds {dst.numel() * dst.element_size()} bytes, "
                             f"{need} needed")
        self._check(self.lib.tsgm_inspect(self.h, BUF[which], _ptr(dst), int(count)), "tsgm_inspect")

    def cells(self) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.lib.tsgm_cells(self.h, ctypes.byref(v)), "tsgm_cells")
        return int(v.value)

    def adjoint_forward(self, prev_D, prev_P, pose6, K, baseline, q, r_scale, D_z, r_z, D, P):
        p6 = (ctypes.c_double * 6)(*[float(v) for v in np.asarray(pose6, np.float64).reshape(6)])
        Ka, Kp = _host_f32(K, 9)
        n = self.n
        self._check(self.lib.tsgm_adjoint_forward(self.h, _dptr(prev_D, n, 4, "prev_D"),
                                                  _dptr(prev_P, n, 4, "prev_P"), p6, Kp,
                                                  ctypes.c_float(baseline), ctypes.c_float(q),
                                                  ctypes.c_float(r_scale), _dptr(D_z, n, 4, "D_z"),
                                                  _dptr(r_z, n, 4, "r_z"), _dptr(D, n, 4, "D"),
                                                  _dptr(P, n, 4, "P")), "tsgm_adjoint_forward")

    def adjoint_backward(self, prev_D, prev_P, pose6, K, baseline, q, r_scale, D_z, r_z, grad_D,
                         grad_P) -> np.ndarray:
        p6 = (ctypes.c_double * 6)(*[float(v) for v in np.asarray(pose6, np.float64).reshape(6)])
        Ka, Kp = _host_f32(K, 9)
        g = (ctypes.c_double * 8)()
        n = self.n
        self._check(self.lib.tsgm_adjoint_backward(self.h, _dptr(prev_D, n, 4, "prev_D"),
                                                   _dptr(prev_P, n, 4, "prev_P"), p6, Kp,
                                                   ctypes.c_float(baseline), ctypes.c_float(q),
                                                   ctypes.c_float(r_scale), _dptr(D_z, n, 4, "D_z"),
                                                   _dptr(r_z, n, 4, "r_z"), _dptr(grad_D, n, 4, "grad_D"),
                                                   _dptr(grad_P, n, 4, "grad_P"), g),
                    "tsgm_adjoint_backward")
        return np.array(list(g), dtype=np.float64)

    def launches(self) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.lib.tsgm_launches(self.h, ctypes.byref(v)), "tsgm_launches")
        return int(v.value)

    def profile(self, enable: bool):
        self._check(self.lib.tsgm_profile(self.h, int(bool(enable))), "tsgm_profile")

    def stage_times(self):
        ms = (ctypes.c_double * N_STAGES)()
        cnt = (ctypes.c_int64 * N_STAGES)()
        self._check(self.lib.tsgm_stage_times(self.h, ms, cnt), "tsgm_stage_times")
        return {STAGES[s]: (ms[s], cnt[s]) for s in range(N_STAGES)}


class Batch:
    """Batched matching over streams of different sizes (tsgm_batch_* of the C ABI)."""

    def __init__(self, params_list, max_labels: int = 0, stream: int | None = None):
        self.lib = load()
        self.params = list(params_list)
        self.n = len(self.params)
        arr = (Params * self.n)(*self.params)
        h = _vp()
        s = _current_stream() if stream is None else int(stream)
        st = self.lib.tsgm_batch_create(arr, self.n, int(max_labels), _vp(s or None), ctypes.byref(h))
        if st != OK:
            raise TsgmError(st, "tsgm_batch_create failed")
        self.h = h

    def _check(self, st, what):
        if st != OK:
            msg = self.lib.tsgm_batch_last_error(self.h)
            raise TsgmError(st, f"{what}: {msg.decode() if msg else ''}")

    def _arr(self, xs, esize: int, what: str):
        """Per-stream device pointers, each buffer checked against its stream's image size."""
        xs = list(xs)
        if len(xs) != self.n:
            raise ValueError(f"{what}: expected {self.n} buffers, got {len(xs)}")
        ptrs = [_dptr(x, int(p.width) * int(p.height), esize, f"{what}[{i}]")
                for i, (x, p) in enumerate(zip(xs, self.params))]
        return (ctypes.c_void_p * len(ptrs))(*ptrs)

    def _arrs(self, lefts, rights, los, his, Dzs, rzs):
        return (self._arr(lefts, 1, "lefts"), self._arr(rights, 1, "rights"), self._arr(los, 2, "los"),
                self._arr(his, 2, "his"), self._arr(Dzs, 4, "Dzs"), self._arr(rzs, 4, "rzs"))

    def match(self, lefts, rights, los, his, Dzs, rzs):
        self._check(self.lib.tsgm_batch_match(self.h, *self._arrs(lefts, rights, los, his, Dzs, rzs)),
                    "tsgm_batch_match")

    def frame(self, lefts, rights, Rs, ts, Ks, baselines, Ds, Ps):
        """One time step of every stream (tsgm_batch_frame). lefts[i] = rights[i] = None: stream i
        sits the step out. Rs (n x 3 x 3), ts (n x 3) may be None when no stream has a previous
        frame; Ks (n x 3 x 3), baselines (n) float32."""
        lefts, rights = list(lefts), list(rights)
        if len(lefts) != self.n or len(rights) != self.n:
            raise ValueError(f"expected {self.n} image pairs")
        act = [l is not None for l in lefts]
        if any((r is not None) != a for r, a in zip(rights, act)):
            raise ValueError("left and right must both be given or both be None")

        def arr(xs, esize, what):
            xs = list(xs)
            if len(xs) != self.n:
                raise ValueError(f"{what}: expected {self.n} buffers, got {len(xs)}")
            ptrs = [_dptr(x, int(p.width) * int(p.height), esize, f"{what}[{i}]") if a else None
                    for i, (x, p, a) in enumerate(zip(xs, self.params, act))]
            return (ctypes.c_void_p * self.n)(*ptrs)

        def host(x, shape):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, np.float32).reshape(shape))
            return a

        R = host(Rs, (self.n, 9))
        t = host(ts, (self.n, 3))
        K = host(Ks, (self.n, 9))
        b = host(baselines, (self.n,))
        fp = lambda a: None if a is None else a.ctypes.data_as(_vp)
        self._check(self.lib.tsgm_batch_frame(self.h, arr(lefts, 1, "lefts"), arr(rights, 1, "rights"),
                                              fp(R), fp(t), fp(K), fp(b), arr(Ds, 4, "Ds"),
                                              arr(Ps, 4, "Ps")), "tsgm_batch_frame")

    def reset(self):
        self._check(self.lib.tsgm_batch_reset(self.h), "tsgm_batch_reset")

    RAN, SAT_OUT, REFUSED = 0, 1, 2

    def stream_status(self):
        """Per stream, what the last step did with it: RAN, SAT_OUT or REFUSED (no pool cells)."""
        st = (ctypes.c_int32 * self.n)()
        self._check(self.lib.tsgm_batch_stream_status(self.h, st), "tsgm_batch_stream_status")
        return [int(x) for x in st]

    def pool(self):
        """(cells of the volume pool, cells of the largest stream at full range)."""
        c, m = ctypes.c_uint64(0), ctypes.c_uint64(0)
        self._check(self.lib.tsgm_batch_pool(self.h, ctypes.byref(c), ctypes.byref(m)),
                    "tsgm_batch_pool")
        return int(c.value), int(m.value)

    def autotune(self, lefts, rights, los, his, Dzs, rzs, reps: int = 3):
        ms = ctypes.c_double(0)
        shape = ctypes.c_int32(0)
        self._check(self.lib.tsgm_batch_autotune(self.h, *self._arrs(lefts, rights, los, his, Dzs, rzs),
                                                 int(reps), ctypes.byref(ms),
                                                 ctypes.byref(shape)), "tsgm_batch_autotune")
        return float(ms.value), int(shape.value)

    def cells(self):
        c = ctypes.c_uint64(0)
        o = ctypes.c_int32(0)
        self._check(self.lib.tsgm_batch_cells(self.h, ctypes.byref(c), ctypes.byref(o)),
                    "tsgm_batch_cells")
        return int(c.value), int(o.value)

    def launches(self) -> int:
        v = ctypes.c_uint64(0)
        self._check(self.lib.tsgm_batch_launches(self.h, ctypes.byref(v)), "tsgm_batch_launches")
        return int(v.value)

    def profile(self, lefts, rights, los, his, Dzs, rzs):
        """(aggregation ms, whole step ms) of one step with direct launches."""
        a, z = ctypes.c_float(0), ctypes.c_float(0)
        self._check(self.lib.tsgm_batch_profile(self.h, *self._arrs(lefts, rights, los, his, Dzs, rzs),
                                                ctypes.byref(a), ctypes.byref(z)),
                    "tsgm_batch_profile")
        return float(a.value), float(z.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsgm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Server:
    """Serving loop of the C ABI (tsgm_server_*): submit frames per camera stream, wait for them."""

    def __init__(self, params_list, hbm_budget_bytes: int):
        self.lib = load()
        self.params = list(params_list)
        arr = (Params * len(self.params))(*self.params)
        h = _vp()
        st = self.lib.tsgm_server_create(arr, len(self.params), int(hbm_budget_bytes), ctypes.byref(h))
        if st != OK:
            raise TsgmError(st, "tsgm_server_create failed")
        self.h = h
        self._keep = {}

    def submit(self, stream: int, left: np.ndarray, right: np.ndarray, R, t, K, baseline,
               D_out: np.ndarray, P_out: np.ndarray) -> int:
        """Queue a frame; D_out/P_out (float32 numpy, the stream's size) receive the result."""
        left = np.ascontiguousarray(left, np.uint8)
        right = np.ascontiguousarray(right, np.uint8)
        Ra, Rp = _host_f32(R, 9)
        ta, tp = _host_f32(t, 3)
        Ka, Kp = _host_f32(K, 9)
        tk = ctypes.c_uint64(0)
        if not 0 <= int(stream) < len(self.params):
            raise ValueError(f"stream {stream} out of range")
        n = int(self.params[int(stream)].width) * int(self.params[int(stream)].height)
        st = self.lib.tsgm_server_submit(self.h, int(stream), _hptr(left, n, 1, "left"),
                                         _hptr(right, n, 1, "right"), Rp, tp, Kp,
                                         ctypes.c_float(baseline), _hptr(D_out, n, 4, "D_out"),
                                         _hptr(P_out, n, 4, "P_out"), ctypes.byref(tk))
        if st != OK:
            raise TsgmError(st, "tsgm_server_submit failed")
        self._keep[int(tk.value)] = (D_out, P_out)
        return int(tk.value)

    def wait(self, ticket: int) -> float:
        lat = ctypes.c_double(0)
        st = self.lib.tsgm_server_wait(self.h, int(ticket), ctypes.byref(lat))
        self._keep.pop(int(ticket), None)
        if st != OK:
            raise TsgmError(st, "tsgm_server_wait: frame failed")
        return float(lat.value)

    def stats(self):
        p50, p99 = ctypes.c_double(0), ctypes.c_double(0)
        done, fl = ctypes.c_uint64(0), ctypes.c_uint64(0)
        slots = ctypes.c_int32(0)
        self.lib.tsgm_server_stats(self.h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(done),
                                   ctypes.byref(slots), ctypes.byref(fl))
        return dict(p50_ms=p50.value, p99_ms=p99.value, completed=int(done.value),
                    slots=int(slots.value), max_in_flight=int(fl.value))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsgm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
