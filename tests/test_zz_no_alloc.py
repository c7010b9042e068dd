"""The allocation-free prediction entry point, called through the C ABI with ctypes.

It serves callers that cannot allocate device memory (for example when another framework's
caching allocator owns the GPU memory, or in a loop that must not block in cudaMalloc). Its
output must equal the context-based tsgm_warp_predict on the same inputs, on two calls in a row
(the second call must not see the first one's z-buffer). This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, host, f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_fp = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm
    lib = tsgm.load()
    fn = lib.tsgm_warp_predict_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, _fp, _fp, _fp,
                   ctypes.c_float, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    return lib


def _host(a):
    a = np.ascontiguousarray(np.asarray(a, np.float32).reshape(-1))
    return a, a.ctypes.data_as(_fp)


def call_noalloc(lib, D, P, R, t, K, b, q, outD, outP):
    H, W = D.shape
    Ra, Rp = _host(R)
    ta, tp = _host(t)
    Ka, Kp = _host(K)
    err = ctypes.create_string_buffer(256)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.tsgm_warp_predict_noalloc(D.data_ptr(), P.data_ptr(), W, H, Rp, tp, Kp,
                                       ctypes.c_float(b), ctypes.c_float(q), outD.data_ptr(),
                                       outP.data_ptr(), stream or None, err, 256)
    return st, err.value.decode()


def test_noalloc_matches_context_entry_point_twice(lib):
    from paper_1708_06301_gb300 import tsgm
    W, H = 1242, 375
    K = synth.Camera(W, H, 721.0, 0.54).K
    b = f32(0.54)
    ctx = tsgm.Context(tsgm.default_params(W, H))
    for call, seed in enumerate((3, 4)):  # two calls in a row, different inputs
        D, P = synth.random_maps(seed, W, H, invalid_frac=0.1)
        R, t = synth.random_pose(seed + 50)
        dD, dP = dev(D), dev(P)
        outD, outP = empty((H, W), np.float32), empty((H, W), np.float32)
        st, msg = call_noalloc(lib, dD, dP, R, t, K, b, 0.25, outD, outP)
        assert st == 0, msg
        refD, refP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dD, dP, R, t, K, b, refD, refP)
        gD, gP = host(outD, np.float32), host(outP, np.float32)
        eD, eP = host(refD, np.float32), host(refP, np.float32)
        assert np.array_equal(gD < 0, eD < 0), f"call {call}"
        v = eD >= 0
        assert v.mean() > 0.3
        assert np.max(np.abs(gD[v] - eD[v])) <= 1e-4
        assert np.max(np.abs(gP[v] - eP[v]) / eP[v]) <= 1e-5
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    """An image larger than the fixed scratch is refused before anything is launched."""
    from paper_1708_06301_gb300 import tsgm
    W, H = 2049, 1024  # 2,098,176 pixels > TSGM_NOALLOC_MAX_PIXELS = 2,097,152
    # four distinct buffers (never read: the call is refused first), so that the size is what
    # is refused and not an aliasing of outputs and inputs
    x = [torch.empty(8, dtype=torch.float32, device="cuda") for _ in range(4)]
    Ra, Rp = _host(np.eye(3))
    ta, tp = _host(np.zeros(3))
    Ka, Kp = _host(synth.Camera(W, H, 721.0, 0.54).K)
    err = ctypes.create_string_buffer(256)
    st = lib.tsgm_warp_predict_noalloc(x[0].data_ptr(), x[1].data_ptr(), W, H, Rp, tp, Kp,
                                       ctypes.c_float(0.54), ctypes.c_float(0.25), x[2].data_ptr(),
                                       x[3].data_ptr(), None, err, 256)
    assert st == tsgm.ERR_INVALID_ARG
    assert "exceeds" in err.value.decode()


def test_noalloc_refuses_aliased_outputs_and_bad_q(lib):
    """Outputs that alias inputs would race inside the gather, and an infinite q would make every
    predicted variance infinite: both are refused before anything is enqueued."""
    from paper_1708_06301_gb300 import tsgm
    W, H = 64, 32
    K = synth.Camera(W, H, 721.0, 0.54).K
    D, P = synth.random_maps(7, W, H)
    dD, dP = dev(D), dev(P)
    o = empty((H, W), np.float32)
    for outD, outP in ((dD, o), (o, dP), (dP, o), (o, dD)):
        st, msg = call_noalloc(lib, dD, dP, np.eye(3), np.zeros(3), K, 0.54, 0.25, outD, outP)
        assert st == tsgm.ERR_INVALID_ARG and "alias" in msg
    o2 = empty((H, W), np.float32)
    for q in (float("inf"), float("nan"), -1.0):
        st, msg = call_noalloc(lib, dD, dP, np.eye(3), np.zeros(3), K, 0.54, q, o, o2)
        assert st == tsgm.ERR_INVALID_ARG and "q must be" in msg


def test_noalloc_at_exactly_its_maximum_size(lib):
    """An image of exactly TSGM_NOALLOC_MAX_PIXELS pixels (2048 x 1024), where an off-by-one in
    the bound or in the reset of the key array would show, equals the context entry point."""
    from paper_1708_06301_gb300 import tsgm
    W, H = 2048, 1024
    K = synth.Camera(W, H, 721.0, 0.54).K
    b = f32(0.54)
    ctx = tsgm.Context(tsgm.default_params(W, H))
    for seed in (11, 12):  # a moved pose, then the identity (every key of the array in use)
        D, P = synth.random_maps(seed, W, H, d_range=(1.0, 20.0), invalid_frac=0.05)
        R, t = (synth.random_pose(seed) if seed == 11 else (np.eye(3), np.zeros(3)))
        dD, dP = dev(D), dev(P)
        outD, outP = empty((H, W), np.float32), empty((H, W), np.float32)
        st, msg = call_noalloc(lib, dD, dP, R, t, K, b, 0.25, outD, outP)
        assert st == 0, msg
        refD, refP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dD, dP, R, t, K, b, refD, refP)
        gD, gP = host(outD, np.float32), host(outP, np.float32)
        eD, eP = host(refD, np.float32), host(refP, np.float32)
        assert np.array_equal(gD < 0, eD < 0)
        v = eD >= 0
        assert v.mean() > 0.3
        assert np.max(np.abs(gD[v] - eD[v])) <= 1e-4
        assert np.max(np.abs(gP[v] - eP[v]) / eP[v]) <= 1e-5
    ctx.close()
