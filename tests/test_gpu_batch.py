"""Batched matching over streams of mixed sizes and disparity ranges: every stream's result must
equal the single-image path (itself bit-exact against the oracle) on the same inputs, across
graph replays with new inputs, after autotuning, and streams too large for their storage must be
skipped, not overrun."""
import numpy as np
import pytest

import oracle
from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(97, 45, 64), (131, 37, 128), (64, 32, 256), (200, 3, 64), (40, 70, 32),
          (1242, 375, 128), (33, 1, 16)]


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def inputs(seed):
    out = []
    for k, (W, H, D) in enumerate(SHAPES):
        a, b = synth.random_images(seed * 100 + k, W, H)
        right = np.roll(a, -min(3, D - 1), axis=1)
        right[:, -3:] = b[:, -3:]
        if W >= 1000:  # windows around a smooth surface, mostly narrow (8 lanes per path line)
            lo, hi = synth.mixed_windows(seed * 100 + k + 50, W, H, D, (1, 16), (17, 40), 0.02,
                                         0.02)
        else:
            lo, hi = synth.random_windows(seed * 100 + k + 50, W, H, D, 4, min(24, D),
                                          full_frac=0.1)
        out.append((a, right, lo, hi))
    return out


def run_batch(tsgm, batch, data):
    dl = [dev(x[0]) for x in data]
    dr = [dev(x[1]) for x in data]
    lo = [dev(x[2]) for x in data]
    hi = [dev(x[3]) for x in data]
    Dz = [empty((H, W), np.float32) for (W, H, _) in SHAPES]
    rz = [empty((H, W), np.float32) for (W, H, _) in SHAPES]
    batch.match(dl, dr, lo, hi, Dz, rz)
    return [host(d, np.float32) for d in Dz], [host(r, np.float32) for r in rz], (dl, dr, lo, hi, Dz, rz)


def single(tsgm, W, H, D, x):
    with tsgm.Context(tsgm.default_params(W, H, d_max=D - 1)) as ctx:
        Dz, rz = empty((H, W), np.float32), empty((H, W), np.float32)
        ctx.match(dev(x[0]), dev(x[1]), dev(x[2]), dev(x[3]), Dz, rz)
        return host(Dz, np.float32), host(rz, np.float32)


def params(tsgm):
    return [tsgm.default_params(W, H, d_max=D - 1) for (W, H, D) in SHAPES]


def test_batch_equals_single_streams_over_replays_and_autotune(tsgm):
    with tsgm.Batch(params(tsgm)) as batch:
        for seed in (1, 2):  # the second call replays the graph with new pointers and data
            data = inputs(seed)
            Dzs, rzs, _ = run_batch(tsgm, batch, data)
            for k, (W, H, D) in enumerate(SHAPES):
                Ds, rs = single(tsgm, W, H, D, data[k])
                assert np.array_equal(Dzs[k], Ds), (seed, k)
                assert np.array_equal(rzs[k], rs), (seed, k)
        data = inputs(3)
        dl = [dev(x[0]) for x in data]
        dr = [dev(x[1]) for x in data]
        lo = [dev(x[2]) for x in data]
        hi = [dev(x[3]) for x in data]
        Dz = [empty((H, W), np.float32) for (W, H, _) in SHAPES]
        rz = [empty((H, W), np.float32) for (W, H, _) in SHAPES]
        ms, shape = batch.autotune(dl, dr, lo, hi, Dz, rz, reps=2)
        assert ms > 0 and shape >= 0
        batch.match(dl, dr, lo, hi, Dz, rz)
        for k, (W, H, D) in enumerate(SHAPES):
            Ds, rs = single(tsgm, W, H, D, data[k])
            assert np.array_equal(host(Dz[k], np.float32), Ds), k
        cells, over = batch.cells()
        assert over == 0
        assert cells == sum(int((x[3].astype(np.int64) - x[2] + 1).sum()) for x in data)


def test_batch_small_streams_against_oracle(tsgm):
    data = inputs(4)
    with tsgm.Batch(params(tsgm)) as batch:
        Dzs, rzs, _ = run_batch(tsgm, batch, data)
    for k in (0, 3, 4):
        W, H, D = SHAPES[k]
        prm = oracle.Params(W, H, d_max=D - 1, census_w=9, census_h=7, n_paths=8)
        Do, ro = oracle.match(data[k][0], data[k][1], data[k][2], data[k][3], prm)
        assert np.array_equal(Dzs[k] < 0, Do < 0)
        v = Do >= 0
        assert np.max(np.abs(Dzs[k][v] - Do[v]), initial=0) <= 1e-4
        assert np.array_equal(rzs[k][v], ro[v])


def test_batch_refuses_streams_the_pool_cannot_hold(tsgm):
    """Storage for 2 labels per pixel (a pool of sum W x H x 4 cells), windows of up to 24: the
    streams reserve their padded cells in stream order and those that do not fit the cells left
    are refused (-1 outputs); the others still equal the single-image path. A refused stream is
    served first at the next step."""
    data = inputs(5)
    need = [((int((((x[3].astype(np.int64) - x[2] + 1) + 3) & ~3).sum()) + 255) & ~255)
            for x in data]
    with tsgm.Batch(params(tsgm), max_labels=2) as batch:
        pool, _ = batch.pool()
        assert pool == sum(((W * H * 4) + 255) & ~255 for (W, H, _) in SHAPES)
        expect, used = [], 0
        for k in range(len(SHAPES)):
            fit = need[k] <= pool - used
            expect.append(tsgm.Batch.RAN if fit else tsgm.Batch.REFUSED)
            used += need[k] if fit else 0
        assert tsgm.Batch.REFUSED in expect and tsgm.Batch.RAN in expect
        Dzs, rzs, _ = run_batch(tsgm, batch, data)
        st = batch.stream_status()
        cells, over = batch.cells()
        assert st == expect
        assert over == expect.count(tsgm.Batch.REFUSED)
        # the next step serves the refused streams first
        run_batch(tsgm, batch, data)
        st2 = batch.stream_status()
    for k, (W, H, D) in enumerate(SHAPES):
        if st[k] == tsgm.Batch.REFUSED:
            assert np.all(Dzs[k] == -1) and np.all(rzs[k] == -1)
        else:
            Ds, rs = single(tsgm, W, H, D, data[k])
            assert np.array_equal(Dzs[k], Ds), k
            assert np.array_equal(rzs[k], rs), k
    first = [k for k in range(len(SHAPES)) if st[k] == tsgm.Batch.REFUSED]
    used = 0
    for k in first + [k for k in range(len(SHAPES)) if k not in first]:
        fit = need[k] <= pool - used
        assert st2[k] == (tsgm.Batch.RAN if fit else tsgm.Batch.REFUSED), k
        used += need[k] if fit else 0


@pytest.mark.slow
def test_batch_full_size_workload_against_oracle_and_single_streams(tsgm):
    """The batched workload as timed (32 streams of 640x480 D=64, 1242x375 D=128 and 1920x1080
    D=256 with 4-24-label windows, storage for 24 labels, autotuned launch shape): every stream
    equals the single-image path, and one stream of each size equals the oracle."""
    import bench
    seqs = bench.render_mix(1)
    streams = [bench.batched_stream(seqs, i) for i in range(bench.BATCH_STREAMS)]
    prm = [tsgm.default_params(W, H, d_max=D - 1) for (W, H, D, *_r) in streams]
    data = [(a, b, lo, hi) for (_W, _H, _D, a, b, lo, hi) in streams]
    with tsgm.Batch(prm, max_labels=bench.BATCH_MAX_LABELS) as batch:
        dl = [dev(x[0]) for x in data]
        dr = [dev(x[1]) for x in data]
        lo = [dev(x[2]) for x in data]
        hi = [dev(x[3]) for x in data]
        Dz = [empty((H, W), np.float32) for (W, H, *_r) in streams]
        rz = [empty((H, W), np.float32) for (W, H, *_r) in streams]
        batch.autotune(dl, dr, lo, hi, Dz, rz, reps=1)
        batch.match(dl, dr, lo, hi, Dz, rz)
        Dzs = [host(d, np.float32) for d in Dz]
        rzs = [host(r, np.float32) for r in rz]
        _, over = batch.cells()
    assert over == 0
    for k, (W, H, D, *_r) in enumerate(streams):
        Ds, rs = single(tsgm, W, H, D, data[k])
        assert np.array_equal(Dzs[k], Ds), k
        assert np.array_equal(rzs[k], rs), k
    for k in range(3):
        W, H, D, a, b, lo_k, hi_k = streams[k]
        Do, ro = oracle.match(a, b, lo_k, hi_k, oracle.Params(W, H, d_max=D - 1, census_w=9,
                                                               census_h=7, n_paths=8))
        assert np.array_equal(Dzs[k] < 0, Do < 0), k
        v = Do >= 0
        assert np.max(np.abs(Dzs[k][v] - Do[v]), initial=0) <= 1e-4, k
        assert np.array_equal(rzs[k][v], ro[v]), k
