"""GPU path vs the CPU oracle, stage by stage and end to end, through the C ABI.

Integer results (census codes, costs, aggregated costs, windows, offsets, z-buffer winners,
d*, right-view disparities, the LR mask) must be bit-exact. Float results must agree within
1e-4 px (disparities) and 1e-5 relative (variances); both sides compute them in binary32 with
the same operation order, so in practice they are identical as well.
"""
import numpy as np
import pytest

import oracle
from paper_1708_06301_gb300 import synth

from gpu_util import compact, dev, empty, f32, host, padded_offsets

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_D = 1e-4
TOL_P_REL = 1e-5


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def make_ctx(tsgm, W, H, d_max=63, cw=5, ch=5, n_paths=4, flags=1, **kw):
    prm = tsgm.default_params(W, H, d_max=d_max, census_w=cw, census_h=ch, n_paths=n_paths,
                              flags=flags, **kw)
    return tsgm.Context(prm)


def oparams(W, H, d_max=63, cw=5, ch=5, n_paths=4, **kw):
    return oracle.Params(W, H, d_max=d_max, census_w=cw, census_h=ch, n_paths=n_paths, **kw)


def assert_maps(Dg, Pg, Do, Po):
    assert np.array_equal(Dg < 0, Do < 0)
    v = Do >= 0
    if v.any():
        assert np.max(np.abs(Dg[v] - Do[v])) <= TOL_D
        assert np.max(np.abs(Pg[v] - Po[v]) / np.maximum(np.abs(Po[v]), 1e-12)) <= TOL_P_REL
    assert np.all(Dg[~v] == -1) and np.all(Pg[~v] == -1)


# ----------------------------------------------------------------------------------------------
# census
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("W,H,cw,ch", [(1242, 375, 9, 7), (97, 45, 5, 5), (33, 1, 5, 5),
                                       (1, 17, 9, 7), (40, 9, 3, 3), (71, 23, 15, 3)])
def test_census_bitexact(tsgm, W, H, cw, ch):
    a, b = synth.random_images(100 + W, W, H)
    with make_ctx(tsgm, W, H, cw=cw, ch=ch) as ctx:
        out = empty((H, W), np.uint64)
        ctx.census(dev(a), out)
        assert np.array_equal(host(out, np.uint64), oracle.census(a, cw, ch))


# ----------------------------------------------------------------------------------------------
# prediction
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_warp_bitexact_random_pose(tsgm, seed):
    W, H = 1242, 375
    D, P = synth.random_maps(seed, W, H, invalid_frac=0.1)
    R, t = synth.random_pose(seed + 10)
    K = synth.Camera(W, H, 721.0, 0.54).K
    b = f32(0.54)
    with make_ctx(tsgm, W, H, d_max=127) as ctx:
        pD, pP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dev(D), dev(P), R, t, K, b, pD, pP)
        keys = empty((H, W), np.uint64)
        ctx.inspect("zkeys", keys, W * H)
        kg = host(keys, np.uint64)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    _, H32 = oracle.build_H(R, t, float(K[0, 0]), float(b))
    Do, Po, win = oracle.warp_predict(D, P, H32, K[0, 2], K[1, 2], 0.25)
    src = np.where(kg == np.uint64(0xFFFFFFFFFFFFFFFF), -1, (kg & np.uint64(0xFFFFFFFF)).astype(np.int64))
    assert np.array_equal(src, win)  # z-buffer winners
    assert np.array_equal(Dg, Do)
    assert np.array_equal(Pg, Po)
    assert (win >= 0).mean() > 0.3  # random maps scatter widely: about 35-50% of targets hit


def test_warp_identity_pose(tsgm):
    W, H = 320, 96
    D, P = synth.random_maps(5, W, H, invalid_frac=0.2)
    K = synth.Camera(W, H, 721.0, 0.54).K
    with make_ctx(tsgm, W, H) as ctx:
        pD, pP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dev(D), dev(P), np.eye(3), np.zeros(3), K, f32(0.54), pD, pP)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    v = D > 0
    assert np.array_equal(Dg[v], D[v]) and np.all(Dg[~v] == -1)
    assert np.array_equal(Pg[v], (P[v] + f32(0.25)).astype(np.float32))


@pytest.mark.parametrize("W,H,D", [(1242, 375, 128), (33, 7, 64), (5, 1, 1)])
def test_windows_bitexact(tsgm, W, H, D):
    Dp, Pp = synth.random_maps(7, W, H, d_range=(-5, D + 5), p_range=(0, 9), invalid_frac=0.2)
    Pp[0, 0] = np.nan
    Pp[-1, -1] = np.inf
    with make_ctx(tsgm, W, H, d_max=D - 1) as ctx:
        lo, hi = empty((H, W), np.int16), empty((H, W), np.int16)
        n = ctx.windows(dev(Dp), dev(Pp), lo, hi, want_cells=True)
        off = empty((W * H + 1,), np.uint32)
        ctx.inspect("offsets", off, W * H + 1)
        log, hig, offg = host(lo, np.int16), host(hi, np.int16), host(off, np.uint32)
    loo, hio, offo, no = oracle.windows(Dp, Pp, D, 3.0)
    assert np.array_equal(log, loo) and np.array_equal(hig, hio)
    assert n == no  # true cell count: sum of the window lengths
    assert np.array_equal(offg, padded_offsets(loo, hio))  # block starts of the GPU layout


# ----------------------------------------------------------------------------------------------
# matching stages on random windows (narrow, wide and full-range mixed)
# ----------------------------------------------------------------------------------------------

# W, H, D, census, paths, windows
#   ("rand", w_min, w_max, full_frac): independent random windows (neighbours rarely overlap)
#   ("mixed", narrow, wide, wide_frac, full_frac): windows around a smooth surface (overlapping)
#   ("border", narrow, cols): narrow windows around a smooth surface, full range in the first and
#                             last `cols` columns
CASES = [
    (97, 45, 64, (5, 5), 4, ("rand", 1, 24, 0.2)),
    (131, 37, 128, (9, 7), 8, ("rand", 1, 40, 0.25)),
    (64, 32, 256, (9, 7), 8, ("rand", 20, 80, 0.1)),
    (200, 3, 64, (5, 5), 8, ("rand", 1, 64, 0.5)),
    (3, 70, 32, (5, 5), 8, ("rand", 1, 32, 0.3)),
    (1, 1, 16, (5, 5), 8, ("rand", 1, 16, 1.0)),
    (50, 20, 1, (5, 5), 8, ("rand", 1, 1, 0.0)),
    (211, 29, 128, (9, 7), 8, ("mixed", (1, 16), (17, 40), 0.02, 0.03)),
    (173, 31, 64, (5, 5), 4, ("mixed", (4, 24), (25, 40), 0.0, 0.02)),
    (97, 41, 256, (9, 7), 8, ("mixed", (1, 16), (17, 60), 0.02, 0.02)),
    (160, 24, 128, (9, 7), 8, ("mixed", (3, 12), (17, 32), 0.0, 0.0)),
    # full range in the border columns: those columns' lines take the full-range walker
    (150, 40, 128, (9, 7), 8, ("border", (3, 12), 6)),
    (77, 50, 64, (5, 5), 8, ("mixed", (4, 24), (17, 64), 0.05, 0.05)),
    # every window the full range: pairs of lines take the full-range walker (LPL 2, 4 and 8,
    # D not a multiple of 8)
    (61, 23, 128, (9, 7), 8, ("rand", 1, 1, 1.0)),
    (45, 17, 64, (5, 5), 4, ("rand", 1, 1, 1.0)),
    (33, 9, 37, (5, 5), 8, ("rand", 1, 1, 1.0)),
    (40, 12, 200, (9, 7), 8, ("rand", 1, 1, 1.0)),
    # long horizontal lines walked in segments from guessed starts (2 or 4 per line): with the
    # 3x3 census the costs are small against P1, P2, so a guessed start often does not agree
    # with the true state within the re-walk and the correction goes on to the segment's end and
    # into the next segment (several passes)
    (600, 8, 64, (3, 3), 8, ("rand", 1, 1, 1.0)),
    (700, 12, 128, (3, 3), 4, ("mixed", (1, 16), (17, 40), 0.02, 0.03)),
    (300, 20, 128, (9, 7), 8, ("mixed", (3, 12), (17, 32), 0.0, 0.0)),
    (1300, 6, 256, (5, 5), 4, ("rand", 1, 1, 1.0)),
    (1242, 16, 128, (9, 7), 8, ("border", (3, 12), 35)),
    # vertical and diagonal lines in segments too, with slow agreement (3x3 census): several
    # correction passes, where a segment walking again reads the end state of a predecessor
    # that walks again in the same pass
    (48, 600, 64, (3, 3), 8, ("rand", 1, 1, 1.0)),
    (520, 520, 64, (3, 3), 8, ("mixed", (1, 16), (17, 40), 0.05, 0.05)),
]


def case_windows(W, H, D, spec):
    if spec[0] == "rand":
        _, wmin, wmax, ff = spec
        return synth.random_windows(W + H, W, H, D, wmin, min(wmax, D), full_frac=ff)
    if spec[0] == "border":
        _, narrow, cols = spec
        lo, hi = synth.mixed_windows(W * 3 + H, W, H, D, narrow, (17, 32), 0.0, 0.0)
        lo, hi = lo.copy(), hi.copy()
        for sl in (slice(0, cols), slice(W - cols, W)):
            lo[:, sl] = 0
            hi[:, sl] = D - 1
        return lo, hi
    _, narrow, wide, wf, ff = spec
    return synth.mixed_windows(W * 3 + H, W, H, D, narrow, wide, wf, ff)


@pytest.mark.parametrize("case", CASES)
def test_match_stages_bitexact(tsgm, case):
    W, H, D, (cw, ch), npaths, spec = case
    seq_l, seq_r = synth.random_images(W * 7 + H, W, H)
    # make the right image a shifted copy so that matching has structure
    right = np.roll(seq_l, -min(5, D - 1), axis=1)
    right[:, -5:] = seq_r[:, -5:]
    lo, hi = case_windows(W, H, D, spec)
    with make_ctx(tsgm, W, H, d_max=D - 1, cw=cw, ch=ch, n_paths=npaths) as ctx:
        Dz, rz = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.match(dev(seq_l), dev(right), dev(lo), dev(hi), Dz, rz)
        n = ctx.cells()
        off = empty((W * H + 1,), np.uint32)
        ctx.inspect("offsets", off, W * H + 1)
        offg = host(off, np.uint32)
        storage = int(offg[-1])
        C = empty((storage,), np.uint8)
        S = empty((storage,), np.uint16)
        ctx.inspect("cost", C, storage)
        ctx.inspect("S", S, storage)
        ds, dr, va = empty((H, W), np.int16), empty((H, W), np.int16), empty((H, W), np.uint8)
        ctx.inspect("dstar", ds, W * H)
        ctx.inspect("dright", dr, W * H)
        ctx.inspect("lr_valid", va, W * H)
        counts = empty((2,), np.uint32)
        ctx.inspect("counts", counts, 2)
        counts = host(counts, np.uint32)
        g = dict(C=compact(host(C, np.uint8), offg, lo, hi), S=compact(host(S, np.uint16), offg, lo, hi),
                 ds=host(ds, np.int16),
                 dr=host(dr, np.int16), va=host(va, np.uint8), Dz=host(Dz, np.float32),
                 rz=host(rz, np.float32))
    prm = oparams(W, H, d_max=D - 1, cw=cw, ch=ch, n_paths=npaths)
    o = oracle.match(seq_l, right, lo, hi, prm, keep=True)
    assert n == int(o["off"][-1]) == int(counts[0])
    assert int(counts[1]) == int(((hi.astype(np.int64) - lo + 1) > 32).sum())
    assert np.array_equal(offg, padded_offsets(lo, hi))
    assert np.array_equal(g["C"], o["C"])
    assert np.array_equal(g["S"], o["S"])
    assert np.array_equal(g["ds"].astype(np.int32), o["dstar"])
    assert np.array_equal(g["dr"].astype(np.int32), o["dright"])
    assert np.array_equal(g["va"], o["valid"])
    assert_maps(g["Dz"], g["rz"], o["Dz"], o["rz"])


# First frames: every window is [0, D - 1], and the aggregation and the selection run their
# full-range kernels (one warp per line or pixel); D ragged against the lanes' labels (41, 101,
# 201), exact (64, 128, 256), a single label, lines shorter than a warp and long horizontal lines.
FULL_CASES = [
    # W, H, D, census, paths[, P1, P2]; with census bits + P2 >= 128 the selection sums the path
    # costs without the bytewise pairing
    (97, 45, 41, (5, 5), 4),
    (131, 37, 101, (9, 7), 8, 10, 90),
    (150, 21, 128, (9, 7), 4, 20, 120),
    (70, 19, 256, (9, 7), 8, 8, 66),
    (64, 33, 64, (5, 5), 8),
    (131, 37, 101, (9, 7), 8),
    (300, 20, 128, (9, 7), 8),
    (1242, 16, 128, (3, 3), 8),
    (40, 12, 201, (9, 7), 8),
    (1300, 6, 256, (5, 5), 4),
    (5, 3, 1, (3, 3), 8),
    (1, 9, 16, (5, 5), 8),
    (13, 1, 33, (5, 5), 8),
    (3, 2, 128, (3, 3), 8),
]


@pytest.mark.parametrize("case", FULL_CASES)
def test_first_frame_full_range_bitexact(tsgm, case):
    W, H, D, (cw, ch), npaths = case[:5]
    pen = dict(P1=case[5], P2=case[6]) if len(case) > 5 else {}
    seq_l, seq_r = synth.random_images(W * 5 + H + D, W, H)
    right = np.roll(seq_l, -min(5, D - 1), axis=1)
    right[:, -5:] = seq_r[:, -5:]
    K = np.array([[0.9 * W, 0, W / 2], [0, 0.9 * W, H / 2], [0, 0, 1]], np.float32)
    with make_ctx(tsgm, W, H, d_max=D - 1, cw=cw, ch=ch, n_paths=npaths, **pen) as ctx:
        Dg, Pg = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.frame(dev(seq_l), dev(right), None, None, K, f32(0.5), Dg, Pg)
        off = empty((W * H + 1,), np.uint32)
        ctx.inspect("offsets", off, W * H + 1)
        offg = host(off, np.uint32)
        storage = int(offg[-1])
        C = empty((storage,), np.uint8)
        S = empty((storage,), np.uint16)
        ctx.inspect("cost", C, storage)
        ctx.inspect("S", S, storage)
        ds, dr, va = empty((H, W), np.int16), empty((H, W), np.int16), empty((H, W), np.uint8)
        ctx.inspect("dstar", ds, W * H)
        ctx.inspect("dright", dr, W * H)
        ctx.inspect("lr_valid", va, W * H)
        lo = np.zeros((H, W), np.int16)
        hi = np.full((H, W), D - 1, np.int16)
        g = dict(C=compact(host(C, np.uint8), offg, lo, hi), S=compact(host(S, np.uint16), offg, lo, hi),
                 ds=host(ds, np.int16), dr=host(dr, np.int16), va=host(va, np.uint8),
                 D=host(Dg, np.float32), P=host(Pg, np.float32))
    o = oracle.match(seq_l, right, lo, hi,
                     oparams(W, H, d_max=D - 1, cw=cw, ch=ch, n_paths=npaths, **pen), keep=True)
    assert storage == W * H * ((D + 3) // 4 * 4)
    assert np.array_equal(g["C"], o["C"])
    assert np.array_equal(g["S"], o["S"])
    assert np.array_equal(g["ds"].astype(np.int32), o["dstar"])
    assert np.array_equal(g["dr"].astype(np.int32), o["dright"])
    assert np.array_equal(g["va"], o["valid"])
    # no prediction on a first frame: the Kalman update passes the measurement through
    assert_maps(g["D"], g["P"], o["Dz"], o["rz"])


def test_kalman_elementwise(tsgm):
    W, H = 257, 3
    n = W * H
    Dp, Pp = synth.random_maps(31, W, H, invalid_frac=0.3)
    Dz, rz = synth.random_maps(32, W, H, p_range=(0.5, 5), invalid_frac=0.3)
    with make_ctx(tsgm, W, H) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.kalman_update(dev(Dp), dev(Pp), dev(Dz), dev(rz), D, P)
        Dg, Pg = host(D, np.float32), host(P, np.float32)
    Do, Po = oracle.kalman(Dp, Pp, Dz, rz)
    assert_maps(Dg, Pg, Do, Po)
    assert n == Do.size


# ----------------------------------------------------------------------------------------------
# whole frames
# ----------------------------------------------------------------------------------------------

def run_sequence(tsgm, seq, n_frames, d_max, cw, ch, npaths, flags=1):
    W, H = seq.cam.W, seq.cam.H
    b = f32(seq.cam.b)
    out = []
    with make_ctx(tsgm, W, H, d_max=d_max, cw=cw, ch=ch, n_paths=npaths, flags=flags) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        for k in range(n_frames):
            ctx.frame(dev(seq.left[k]), dev(seq.right[k]), seq.R[k], seq.t[k], seq.K, b, D, P)
            lo, hi = empty((H, W), np.int16), empty((H, W), np.int16)
            ctx.inspect("windows_lo", lo, W * H)
            ctx.inspect("windows_hi", hi, W * H)
            out.append(dict(D=host(D, np.float32), P=host(P, np.float32), lo=host(lo, np.int16),
                            hi=host(hi, np.int16)))
    return out


def test_frames_small_pair(tsgm):
    seq = synth.small_pair(1)
    g = run_sequence(tsgm, seq, 2, 63, 5, 5, 4)
    tr = oracle.Tracker(oparams(320, 96))
    for k in range(2):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


@pytest.mark.slow
def test_frames_kitti_like_full_size(tsgm):
    """The benchmark's workload at full size (1242x375, D = 128, census 9x7, 8 paths), first
    three frames, every pixel compared."""
    seq = synth.kitti_like(2, n_frames=3)
    g = run_sequence(tsgm, seq, 3, 127, 9, 7, 8)
    tr = oracle.Tracker(oparams(1242, 375, d_max=127, cw=9, ch=7, n_paths=8))
    for k in range(3):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


def test_frame_host_equals_device(tsgm):
    seq = synth.small_pair(1)
    W, H = 320, 96
    b = f32(seq.cam.b)
    g = run_sequence(tsgm, seq, 2, 63, 5, 5, 4)
    with make_ctx(tsgm, W, H) as ctx:
        D = np.empty((H, W), np.float32)
        P = np.empty((H, W), np.float32)
        for k in range(2):
            ctx.frame_host(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, b, D, P)
            assert np.array_equal(D, g[k]["D"]) and np.array_equal(P, g[k]["P"])


def test_frame_host_async_equals_device(tsgm):
    """Frames enqueued with pinned host buffers and no wait in between (copies on the transfer
    streams, two staging slots in turn), then one wait: every frame's maps equal the device
    path's; a blocking call afterwards still works on the same context."""
    import torch
    seq = synth.make_sequence(7, 320, 96, 721.0, 0.54, n_frames=5, n_boxes=4, step_range=(0.4, 0.6),
                              yaw_deg=1.0, noise_sigma=1.0)
    W, H, n = 320, 96, 5
    b = f32(seq.cam.b)
    g = run_sequence(tsgm, seq, n, 63, 5, 5, 4)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    L = [pin(seq.left[k]) for k in range(n)]
    R = [pin(seq.right[k]) for k in range(n)]
    D = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(n)]
    P = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(n)]
    with make_ctx(tsgm, W, H) as ctx:
        for k in range(n):
            ctx.frame_host_async(L[k], R[k], seq.R[k], seq.t[k], seq.K, b, D[k], P[k])
        ctx.wait()
        for k in range(n):
            assert np.array_equal(D[k].numpy(), g[k]["D"]) and np.array_equal(P[k].numpy(), g[k]["P"])
        ctx.reset()
        Dh = np.empty((H, W), np.float32)
        Ph = np.empty((H, W), np.float32)
        ctx.frame_host(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, b, Dh, Ph)
        assert np.array_equal(Dh, g[0]["D"]) and np.array_equal(Ph, g[0]["P"])


def test_state_export_import_resume(tsgm):
    seq = synth.small_pair(1)
    W, H = 320, 96
    b = f32(seq.cam.b)
    g = run_sequence(tsgm, seq, 2, 63, 5, 5, 4)
    with make_ctx(tsgm, W, H) as a:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        a.frame(dev(seq.left[0]), dev(seq.right[0]), None, None, seq.K, b, D, P)
        sD, sP, has = a.state_export()
    assert has
    with make_ctx(tsgm, W, H) as c:
        c.state_import(sD, sP, True)
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        c.frame(dev(seq.left[1]), dev(seq.right[1]), seq.R[1], seq.t[1], seq.K, b, D, P)
        assert np.array_equal(host(D, np.float32), g[1]["D"])


def test_full_range_flag_equals_full_windows(tsgm):
    """TSGM_FLAG_FULL_RANGE: frame 2 matched over [0, D-1] everywhere equals tsgm_match with
    full windows, then the Kalman update with the prediction."""
    seq = synth.small_pair(1)
    W, H = 320, 96
    g = run_sequence(tsgm, seq, 2, 63, 5, 5, 4, flags=1 | 2)
    assert np.all(g[1]["lo"] == 0) and np.all(g[1]["hi"] == 63)
    prm = oparams(W, H)
    tr = oracle.Tracker(prm)
    o0 = tr.frame(seq.left[0], seq.right[0], seq.R[0], seq.t[0], seq.K, f32(seq.cam.b), keep=True)
    _, H32 = oracle.build_H(seq.R[1], seq.t[1], float(seq.K[0, 0]), float(f32(seq.cam.b)))
    Dp, Pp, _ = oracle.warp_predict(o0["D"], o0["P"], H32, seq.K[0, 2], seq.K[1, 2], prm.q)
    lo = np.zeros((H, W), np.int16)
    hi = np.full((H, W), 63, np.int16)
    Dz, rz = oracle.match(seq.left[1], seq.right[1], lo, hi, prm)
    Do, Po = oracle.kalman(Dp, Pp, Dz, rz)
    assert_maps(g[1]["D"], g[1]["P"], Do, Po)


def test_errors_are_status_codes(tsgm):
    with pytest.raises(tsgm.TsgmError):
        tsgm.Context(tsgm.default_params(64, 32, n_paths=5))
    with pytest.raises(tsgm.TsgmError):
        tsgm.Context(tsgm.default_params(64, 32, d_max=300))
    for bad in (dict(sad_w=4), dict(sad_h=33), dict(sad_thr=-1.0), dict(pred_lr_tol=float("nan"))):
        with pytest.raises(tsgm.TsgmError):
            tsgm.Context(tsgm.default_params(64, 32, **bad))
    with make_ctx(tsgm, 64, 32) as ctx:
        with pytest.raises(tsgm.TsgmError) as e:
            ctx.match(0, 0, 0, 0, 0, 0)
        assert e.value.status == tsgm.ERR_INVALID_ARG
        D = empty((32, 64), np.float32)
        # the first frame needs no pose
        ctx.frame(dev(np.zeros((32, 64), np.uint8)), dev(np.zeros((32, 64), np.uint8)),
                  None, None, synth.Camera(64, 32, 721.0, 0.54).K, f32(0.54), D, empty((32, 64), np.float32))
        # later frames do
        with pytest.raises(tsgm.TsgmError) as e:
            ctx.frame(dev(np.zeros((32, 64), np.uint8)), dev(np.zeros((32, 64), np.uint8)),
                      None, None, synth.Camera(64, 32, 721.0, 0.54).K, f32(0.54), D, empty((32, 64), np.float32))
        assert e.value.status == tsgm.ERR_INVALID_ARG
        # a zero baseline cannot build H
        with pytest.raises(tsgm.TsgmError) as e:
            ctx.frame(dev(np.zeros((32, 64), np.uint8)), dev(np.zeros((32, 64), np.uint8)),
                      np.eye(3), np.zeros(3), synth.Camera(64, 32, 721.0, 0.54).K, f32(0.0), D,
                      empty((32, 64), np.float32))
        assert e.value.status == tsgm.ERR_INVALID_ARG


# ----------------------------------------------------------------------------------------------
# gap filling of the prediction (Sec. 2.2, Eq. 7-8)
# ----------------------------------------------------------------------------------------------

def test_fill_gaps_bitexact(tsgm):
    """Forward motion opens one-pixel gaps in a warped map; the GPU fill equals the oracle's."""
    W, H = 1242, 375
    D, P = synth.random_maps(41, W, H, d_range=(20, 40), invalid_frac=0.05)
    K = synth.Camera(W, H, 721.0, 0.54).K
    b = f32(0.54)
    R, t = np.eye(3, dtype=np.float32), np.array([0, 0, -1.0], np.float32)
    with make_ctx(tsgm, W, H, d_max=127, gamma_f=1.5) as ctx:
        pD, pP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dev(D), dev(P), R, t, K, b, pD, pP)
        Dw, Pw = host(pD, np.float32), host(pP, np.float32)
        ctx.fill_gaps(pD, pP)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    Do, Po = oracle.fill_gaps(Dw, Pw, 1.5)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)
    assert (Do >= 0).sum() > (Dw >= 0).sum()  # something was filled


@pytest.mark.parametrize("slow_case", [False, pytest.param(True, marks=pytest.mark.slow)])
def test_frames_with_gap_filling(tsgm, slow_case):
    if slow_case:
        seq, n, dm, cw, ch, npaths = synth.kitti_like(2, n_frames=3), 3, 127, 9, 7, 8
    else:
        seq, n, dm, cw, ch, npaths = synth.small_pair(1), 2, 63, 5, 5, 4
    W, H = seq.cam.W, seq.cam.H
    g = run_sequence(tsgm, seq, n, dm, cw, ch, npaths, flags=1 | 4)
    tr = oracle.Tracker(oparams(W, H, d_max=dm, cw=cw, ch=ch, n_paths=npaths, fill_gaps=True))
    for k in range(n):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


@pytest.mark.parametrize("thr", [1.0, 2.5])
def test_edge_reject_bitexact(tsgm, thr):
    """Edge rejection of a warped prediction (objects at several depths and holes): the GPU pass
    equals the oracle's, and it rejects something."""
    W, H = 1242, 375
    seq = synth.kitti_like(2, n_frames=2)
    D = seq.gt_disp[0].astype(np.float32)
    P = np.full_like(D, 0.5)
    D[::97, ::13] = -1.0                             # a few holes
    K = synth.Camera(W, H, 721.0, 0.54).K
    with make_ctx(tsgm, W, H, d_max=127, edge_thr=thr) as ctx:
        pD, pP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dev(D), dev(P), seq.R[1], seq.t[1], K, f32(0.54), pD, pP)
        Dw, Pw = host(pD, np.float32), host(pP, np.float32)
        ctx.edge_reject(pD, pP)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    Do, Po = oracle.edge_reject(Dw, Pw, thr)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)
    assert (Do < 0).sum() > (Dw < 0).sum()


def test_frames_with_edge_rejection_and_gap_filling(tsgm):
    seq, n = synth.small_pair(1), 2
    W, H = seq.cam.W, seq.cam.H
    g = run_sequence(tsgm, seq, n, 63, 5, 5, 4, flags=1 | 4 | 8)
    tr = oracle.Tracker(oparams(W, H, d_max=63, fill_gaps=True, edge_reject=True))
    for k in range(n):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


@pytest.mark.parametrize("tol", [0.5, 1.0])
def test_pred_lr_check_bitexact(tsgm, tol):
    """The prediction's left-right check (Sec. 2.2, Fig. 3(d)) of a warped, gap-filled
    prediction: the GPU pass equals the oracle's and removes the band seen by the left camera
    only, plus the occluded background."""
    W, H = 1242, 375
    seq = synth.kitti_like(2, n_frames=2)
    D = seq.gt_disp[0].astype(np.float32)
    P = np.full_like(D, 0.5)
    D[::97, ::13] = -1.0
    K = synth.Camera(W, H, 721.0, 0.54).K
    with make_ctx(tsgm, W, H, d_max=127, pred_lr_tol=tol) as ctx:
        pD, pP = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.warp_predict(dev(D), dev(P), seq.R[1], seq.t[1], K, f32(0.54), pD, pP)
        ctx.fill_gaps(pD, pP)
        Dw, Pw = host(pD, np.float32), host(pP, np.float32)
        ctx.pred_lr_check(pD, pP)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    Do, Po = oracle.pred_lr_check(Dw, Pw, tol)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)
    assert (Do < 0).sum() > (Dw < 0).sum()
    # every pixel kept lands inside the right image
    ys, xs = np.nonzero(Do >= 0)
    assert np.all(xs >= np.floor(Do[ys, xs] + np.float32(0.5)))


def test_pred_lr_check_small_and_large_disparities(tsgm):
    """Rows narrower than the disparities (landing columns far outside the image), huge values,
    holes and invalid variances, on a 7 x 3 image."""
    rng = np.random.default_rng(11)
    W, H = 7, 3
    D = rng.uniform(0, 12, (H, W)).astype(np.float32)
    D[0, 3] = 3.0e38
    D[1, 1] = -1.0
    P = np.full_like(D, 1.0)
    P[2, 5] = -1.0
    with make_ctx(tsgm, W, H, d_max=63, pred_lr_tol=2.0) as ctx:
        pD, pP = dev(D), dev(P)
        ctx.pred_lr_check(pD, pP)
        Dg, Pg = host(pD, np.float32), host(pP, np.float32)
    Do, Po = oracle.pred_lr_check(D, P, 2.0)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)


@pytest.mark.parametrize("sw,sh,thr", [(5, 5, 20.0), (3, 7, 8.0), (1, 1, 0.0), (9, 3, 12.5)])
def test_sad_check_bitexact(tsgm, sw, sh, thr):
    """SAD check (Sec. 2.4) of a map near the true disparities with noise, outliers and holes,
    on a rendered pair: the GPU pass equals the oracle's."""
    seq = synth.kitti_like(2, n_frames=1)
    W, H = seq.cam.W, seq.cam.H
    rng = np.random.default_rng(sw * 100 + sh)
    D = (seq.gt_disp[0] + rng.normal(0, 0.7, (H, W))).astype(np.float32)
    out = rng.random((H, W)) < 0.05
    D[out] = rng.uniform(0, 127, out.sum()).astype(np.float32)
    D[rng.random((H, W)) < 0.02] = -1.0
    D[D < 0] = -1.0
    P = np.where(D >= 0, 0.7, -1.0).astype(np.float32)
    with make_ctx(tsgm, W, H, d_max=127, sad_w=sw, sad_h=sh, sad_thr=thr) as ctx:
        gD, gP = dev(D), dev(P)
        ctx.sad_check(dev(seq.left[0]), dev(seq.right[0]), gD, gP)
        Dg, Pg = host(gD, np.float32), host(gP, np.float32)
    Do, Po = oracle.sad_check(seq.left[0], seq.right[0], D, P, sw, sh, thr)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)
    if thr > 0:
        assert 0 < (Do < 0).sum() - (D < 0).sum() < 0.5 * D.size


def test_frames_with_prediction_checks(tsgm):
    """Whole frames with gap filling, the prediction's left-right check and the SAD check of the
    updated map (flags 4 | 16 | 32): windows and maps equal the oracle tracker's."""
    seq = synth.make_sequence(5, 320, 96, 721.0, 0.54, n_frames=3, n_boxes=4, step_range=(0.4, 0.6),
                              yaw_deg=1.0, noise_sigma=1.0)
    n = 3
    W, H = seq.cam.W, seq.cam.H
    g = run_sequence(tsgm, seq, n, 63, 5, 5, 4, flags=1 | 4 | 16 | 32)
    tr = oracle.Tracker(oparams(W, H, d_max=63, fill_gaps=True, pred_lr_check=True, sad_check=True))
    for k in range(n):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


@pytest.mark.parametrize("extra", [0, 1])
def test_selection_split_boundary(tsgm, extra):
    """The wide windows (> 16 labels) are selected apart from their rows while they are at most a
    quarter of the image, and by their rows beyond: exactly a quarter and one more both equal the
    oracle (the two selection kernels take the same decision)."""
    W, H, D = 96, 40, 64
    n = W * H
    lo, hi = synth.mixed_windows(21, W, H, D, (2, 12), (17, 64), 0.0, 0.0)
    lo = lo.copy()
    hi = hi.copy()
    rng = np.random.default_rng(4)
    idx = rng.permutation(n)[: n // 4 + extra]
    wl, wh = lo.reshape(-1), hi.reshape(-1)
    wl[idx] = 0
    wh[idx] = rng.integers(17, D, idx.size)               # 18 .. D labels: every one wide
    assert int(((hi.astype(np.int64) - lo + 1) > 16).sum()) == n // 4 + extra
    left, right = synth.random_images(77, W, H)
    right = np.roll(left, -3, axis=1)
    with make_ctx(tsgm, W, H, d_max=D - 1, n_paths=8) as ctx:
        Dz, rz = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.match(dev(left), dev(right), dev(lo), dev(hi), Dz, rz)
        ds, dr, va = empty((H, W), np.int16), empty((H, W), np.int16), empty((H, W), np.uint8)
        ctx.inspect("dstar", ds, n)
        ctx.inspect("dright", dr, n)
        ctx.inspect("lr_valid", va, n)
        g = dict(ds=host(ds, np.int16), dr=host(dr, np.int16), va=host(va, np.uint8),
                 Dz=host(Dz, np.float32), rz=host(rz, np.float32))
    o = oracle.match(left, right, lo, hi, oparams(W, H, d_max=D - 1, n_paths=8), keep=True)
    assert np.array_equal(g["ds"].astype(np.int32), o["dstar"])
    assert np.array_equal(g["dr"].astype(np.int32), o["dright"])
    assert np.array_equal(g["va"], o["valid"])
    assert_maps(g["Dz"], g["rz"], o["Dz"], o["rz"])


@pytest.mark.parametrize("W,H", [(1, 9), (13, 1), (3, 2)])
def test_consistency_checks_degenerate_shapes(tsgm, W, H):
    """One-pixel-wide and one-row images, and patches larger than the image (every coordinate
    clamps): both checks equal the oracle."""
    rng = np.random.default_rng(W * 31 + H)
    D = rng.uniform(0, 6, (H, W)).astype(np.float32)
    D[rng.random((H, W)) < 0.2] = -1.0
    P = np.where(D >= 0, 1.0, -1.0).astype(np.float32)
    L = rng.integers(0, 256, (H, W), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W), dtype=np.uint8)
    with make_ctx(tsgm, W, H, d_max=15, pred_lr_tol=0.5, sad_w=31, sad_h=5, sad_thr=60.0) as ctx:
        gD, gP = dev(D), dev(P)
        ctx.pred_lr_check(gD, gP)
        Dg, Pg = host(gD, np.float32), host(gP, np.float32)
        sD, sP = dev(D), dev(P)
        ctx.sad_check(dev(L), dev(R), sD, sP)
        Sg, SPg = host(sD, np.float32), host(sP, np.float32)
    Do, Po = oracle.pred_lr_check(D, P, 0.5)
    assert np.array_equal(Dg, Do) and np.array_equal(Pg, Po)
    So, SPo = oracle.sad_check(L, R, D, P, 31, 5, 60.0)
    assert np.array_equal(Sg, So) and np.array_equal(SPg, SPo)


def test_frames_full_size_every_refinement(tsgm):
    """The benchmark's workload at full size with every refinement on (edge rejection, gap
    filling, the prediction's left-right check, the SAD check of the updated map; flags
    4 | 8 | 16 | 32): windows and maps of three frames equal the oracle tracker's."""
    seq = synth.kitti_like(2, n_frames=3)
    g = run_sequence(tsgm, seq, 3, 127, 9, 7, 8, flags=1 | 4 | 8 | 16 | 32)
    tr = oracle.Tracker(oparams(1242, 375, d_max=127, cw=9, ch=7, n_paths=8, fill_gaps=True,
                                edge_reject=True, pred_lr_check=True, sad_check=True))
    for k in range(3):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, f32(seq.cam.b), keep=True)
        assert np.array_equal(g[k]["lo"], o["lo"]) and np.array_equal(g[k]["hi"], o["hi"])
        assert_maps(g[k]["D"], g[k]["P"], o["D"], o["P"])


def test_selection_split_with_256_labels(tsgm):
    """Wide windows of up to 256 labels (two chunks of 128 per lane set) selected apart from their
    rows (a few percent of the pixels wide): equal to the oracle."""
    W, H, D = 160, 48, 256
    lo, hi = synth.mixed_windows(33, W, H, D, (2, 14), (17, 256), 0.06, 0.04)
    n = W * H
    assert 0 < int(((hi.astype(np.int64) - lo + 1) > 16).sum()) <= n // 4
    left, _ = synth.random_images(91, W, H)
    right = np.roll(left, -9, axis=1)
    with make_ctx(tsgm, W, H, d_max=D - 1, n_paths=8) as ctx:
        Dz, rz = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.match(dev(left), dev(right), dev(lo), dev(hi), Dz, rz)
        ds, dr, va = empty((H, W), np.int16), empty((H, W), np.int16), empty((H, W), np.uint8)
        ctx.inspect("dstar", ds, n)
        ctx.inspect("dright", dr, n)
        ctx.inspect("lr_valid", va, n)
        g = dict(ds=host(ds, np.int16), dr=host(dr, np.int16), va=host(va, np.uint8),
                 Dz=host(Dz, np.float32), rz=host(rz, np.float32))
    o = oracle.match(left, right, lo, hi, oparams(W, H, d_max=D - 1, n_paths=8), keep=True)
    assert np.array_equal(g["ds"].astype(np.int32), o["dstar"])
    assert np.array_equal(g["dr"].astype(np.int32), o["dright"])
    assert np.array_equal(g["va"], o["valid"])
    assert_maps(g["Dz"], g["rz"], o["Dz"], o["rz"])
