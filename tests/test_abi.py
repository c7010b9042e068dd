"""The C ABI library on the CPU: it loads, exports every function the header declares, and its
host-side pieces (parameter checks, the homography) behave; no GPU calls."""
import ast
import os

import numpy as np
import pytest

import oracle
from paper_1708_06301_gb300 import build as tbuild
from paper_1708_06301_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tsgm():
    tbuild.build()
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def test_exports_every_declared_symbol(tsgm):
    lib = tsgm.load()
    syms = tsgm.header_symbols()
    assert len(syms) >= 19
    for s in syms:
        assert hasattr(lib, s), s
    for s in ("tsgm_create", "tsgm_warp_predict", "tsgm_windows", "tsgm_match",
              "tsgm_kalman_update", "tsgm_frame"):
        assert s in syms


def test_default_params(tsgm):
    p = tsgm.default_params(1242, 375)
    assert (p.d_max, p.census_w, p.census_h, p.n_paths, p.P1, p.P2) == (127, 9, 7, 8, 8, 32)
    assert (p.sigma_mult, p.q, p.S_max, p.r_min, p.lr_tol) == (3.0, 0.25, 10.0, 0.5, 1)
    assert (p.flags, p.gamma_f, p.edge_thr, p.pred_lr_tol) == (0, 1.0, 1.0, 1.0)
    assert (p.sad_w, p.sad_h, p.sad_thr) == (5, 5, 30.0)


def test_binding_covers_the_header(tsgm):
    """Every function the header declares has a ctypes signature in the binding."""
    missing = [s for s in tsgm.header_symbols() if s not in tsgm._SIGS]
    assert not missing, missing


@pytest.mark.parametrize("bad", [dict(n_paths=5), dict(d_max=256), dict(census_w=4),
                                 dict(census_w=11, census_h=7), dict(P1=40, P2=30),
                                 dict(P2=200), dict(width=0), dict(q=-1.0), dict(sad_w=4),
                                 dict(sad_h=0), dict(sad_w=33), dict(sad_thr=-0.5),
                                 dict(pred_lr_tol=float("inf")), dict(edge_thr=float("nan"))])
def test_create_rejects_bad_params_before_touching_the_gpu(tsgm, bad):
    p = tsgm.default_params(64, 32)
    for k, v in bad.items():
        setattr(p, k, v)
    with pytest.raises(tsgm.TsgmError) as e:
        tsgm.Context(p, stream=0)
    assert e.value.status == tsgm.ERR_INVALID_ARG


@pytest.mark.parametrize("seed", range(20))
def test_build_H_matches_oracle_bits(tsgm, seed):
    """Host-side homography (binary64, rounded once): identical to the oracle's."""
    R, t = synth.random_pose(300 + seed)
    K = synth.Camera(1242, 375, 721.0, 0.54).K
    b = np.float32(0.54)
    H = tsgm.build_H(R, t, K, b)
    _, Ho = oracle.build_H(R, t, float(K[0, 0]), float(b))
    assert np.array_equal(H, Ho)


def test_build_H_rejects_bad_calibration(tsgm):
    K = synth.Camera(64, 32, 721.0, 0.54).K
    with pytest.raises(tsgm.TsgmError):
        tsgm.build_H(np.eye(3), np.zeros(3), K, 0.0)
    K2 = K.copy()
    K2[0, 0] = -1
    with pytest.raises(tsgm.TsgmError):
        tsgm.build_H(np.eye(3), np.zeros(3), K2, 0.54)


def _imports(path):
    tree = ast.parse(open(path).read())
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.module:
            names.add(node.module.split(".")[0])
    return names


def test_product_and_oracle_are_independent():
    pkg = os.path.join(ROOT, "paper_1708_06301_gb300")
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            assert "oracle" not in _imports(os.path.join(pkg, f)), f
    for f in os.listdir(os.path.join(pkg, "csrc")):
        assert "oracle" not in open(os.path.join(pkg, "csrc", f)).read().lower().replace(
            "the oracle", ""), f
    od = os.path.join(ROOT, "oracle")
    for f in os.listdir(od):
        if f.endswith(".py"):
            assert "paper_1708_06301_gb300" not in _imports(os.path.join(od, f)), f
        if f.endswith((".cpp", ".h")):
            assert "tsgm.h" not in open(os.path.join(od, f)).read()


def test_missing_library_fails_loudly(tsgm):
    """No fallback: without the built CUDA library the binding raises and says how to build it."""
    saved = tsgm._lib
    tsgm._lib = None
    try:
        with pytest.raises(ImportError, match="build"):
            tsgm.load(os.path.join(ROOT, "paper_1708_06301_gb300", "_build", "no_such_libtsgm.so"))
    finally:
        tsgm._lib = saved


class _FakeCudaTensor:
    """Stands in for a CUDA tensor on a machine without a GPU: only what the binding reads."""

    is_cuda = True

    def __init__(self, numel, esize, contiguous=True):
        self._n, self._e, self._c = numel, esize, contiguous

    def numel(self):
        return self._n

    def element_size(self):
        return self._e

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x7F0000000000


def test_binding_checks_device_buffer_sizes(tsgm):
    """Kernels trust the context's sizes: the binding refuses a device buffer that is smaller than
    the call needs or has another element size, before anything reaches the GPU."""
    assert tsgm._dptr(_FakeCudaTensor(12, 4), 12, 4, "D") == 0x7F0000000000
    assert tsgm._dptr(_FakeCudaTensor(20, 4), 12, 4, "D") == 0x7F0000000000
    assert tsgm._dptr(None, 12, 4, "D") == 0
    assert tsgm._dptr(1234, 12, 4, "D") == 1234          # a raw pointer: the caller vouches
    with pytest.raises(ValueError, match="at least 12"):
        tsgm._dptr(_FakeCudaTensor(11, 4), 12, 4, "D")
    with pytest.raises(ValueError, match="4 bytes"):
        tsgm._dptr(_FakeCudaTensor(12, 8), 12, 4, "D")
    with pytest.raises(ValueError, match="contiguous"):
        tsgm._dptr(_FakeCudaTensor(12, 4, contiguous=False), 12, 4, "D")


def test_binding_checks_host_buffer_sizes(tsgm):
    a = np.zeros((3, 4), np.float32)
    assert tsgm._hptr(a, 12, 4, "D") == a.ctypes.data
    with pytest.raises(ValueError, match="at least 13"):
        tsgm._hptr(a, 13, 4, "D")
    with pytest.raises(ValueError, match="4 bytes"):
        tsgm._hptr(a.astype(np.float64), 12, 4, "D")
    with pytest.raises(ValueError, match="contiguous"):
        tsgm._hptr(np.zeros((4, 6), np.float32)[:, ::2], 12, 4, "D")
    with pytest.raises(ValueError, match="host buffer"):
        tsgm._hptr(_FakeCudaTensor(12, 4), 12, 4, "D")
    import torch
    t = torch.zeros((3, 4), dtype=torch.float32)
    assert tsgm._hptr(t, 12, 4, "D") == t.data_ptr()


def test_batch_checks_each_stream_against_its_size(tsgm):
    b = object.__new__(tsgm.Batch)
    b.params = [tsgm.default_params(8, 4), tsgm.default_params(16, 2)]
    b.n = 2
    imgs = [_FakeCudaTensor(32, 1), _FakeCudaTensor(32, 1)]
    assert len(b._arr(imgs, 1, "lefts")) == 2
    with pytest.raises(ValueError, match=r"lefts\[1\]"):
        b._arr([_FakeCudaTensor(32, 1), _FakeCudaTensor(31, 1)], 1, "lefts")
    with pytest.raises(ValueError, match="expected 2 buffers"):
        b._arr(imgs[:1], 1, "lefts")
