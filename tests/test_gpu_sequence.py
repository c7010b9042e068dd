"""The timed workload, every frame, against the oracle.

The benchmark runs the 10-frame 1242x375 sequence (census 9x7, 8 paths, D = 128) with the gap
filling of the prediction (Sec. 2.2, Eq. 7-8) and nothing kept for inspection, and beside it the
same frames with the whole disparity range searched (prediction and Kalman update as usual). Here
both run with exactly those flags and every frame is compared with the oracle: the windows
bit-exact, D within 1e-4 px and P within 1e-5 relative. The later frames are where the windows are
narrowest (Sec. 3: the search space shrinks frame after frame), so all ten are checked.

The oracle's sequences take about a minute on the CPU; they run in a spawn process pool while the
GPU runs its own.
"""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, f32, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_D = 1e-4
TOL_P_REL = 1e-5
N_FRAMES = 10


def _oracle_sequence(mode: str, n_frames: int):
    """The oracle's per-frame loop (Sec. 2) on the kitti-shaped sequence: 'reduced' = windows of
    +-3 sigma around the gap-filled prediction; 'full' = the prediction without gap filling and
    windows spanning [0, D-1], then the Kalman update with that prediction."""
    import oracle
    seq = synth.kitti_like(2, n_frames=n_frames)
    W, H = seq.cam.W, seq.cam.H
    b = float(np.float32(seq.cam.b))
    prm = oracle.Params(W, H, d_max=127, census_w=9, census_h=7, n_paths=8,
                        fill_gaps=(mode == "reduced"), full_range=(mode == "full"))
    tr = oracle.Tracker(prm)
    out = []
    for k in range(n_frames):
        o = tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, b, keep=True)
        out.append(dict(D=o["D"], P=o["P"], lo=o["lo"], hi=o["hi"]))
    return out


@pytest.fixture(scope="module")
def oracle_runs():
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(2)
    res = {m: pool.apply_async(_oracle_sequence, (m, N_FRAMES)) for m in ("reduced", "full")}
    pool.close()
    yield res
    pool.terminate()


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def _gpu_sequence(tsgm, flags: int, n_frames: int):
    seq = synth.kitti_like(2, n_frames=n_frames)
    W, H = seq.cam.W, seq.cam.H
    b = f32(seq.cam.b)
    out = []
    with tsgm.Context(tsgm.default_params(W, H, flags=flags)) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        left = [dev(x) for x in seq.left]
        right = [dev(x) for x in seq.right]
        for k in range(n_frames):
            ctx.frame(left[k], right[k], seq.R[k], seq.t[k], seq.K, b, D, P)
            lo, hi = empty((H, W), np.int16), empty((H, W), np.int16)
            ctx.inspect("windows_lo", lo, W * H)
            ctx.inspect("windows_hi", hi, W * H)
            out.append(dict(D=host(D, np.float32), P=host(P, np.float32), lo=host(lo, np.int16),
                            hi=host(hi, np.int16)))
    return seq, out


def _compare(g, o, k):
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"]), f"frame {k + 1}"
    Dg, Pg, Do, Po = g["D"], g["P"], o["D"], o["P"]
    assert np.array_equal(Dg < 0, Do < 0), f"frame {k + 1}: validity"
    v = Do >= 0
    assert np.max(np.abs(Dg[v] - Do[v])) <= TOL_D, f"frame {k + 1}: D"
    assert np.max(np.abs(Pg[v] - Po[v]) / np.maximum(np.abs(Po[v]), 1e-12)) <= TOL_P_REL, \
        f"frame {k + 1}: P"
    assert np.all(Dg[~v] == -1) and np.all(Pg[~v] == -1)


@pytest.mark.slow
def test_timed_sequence_reduced_every_frame(tsgm, oracle_runs):
    """The headline configuration: gap filling on, internals not kept (as timed)."""
    _, g = _gpu_sequence(tsgm, tsgm.FLAG_FILL_GAPS, N_FRAMES)
    o = oracle_runs["reduced"].get(timeout=1800)
    for k in range(N_FRAMES):
        _compare(g[k], o[k], k)
    # the later frames really are reduced: well under half of the range is searched
    for k in range(1, N_FRAMES):
        w = g[k]["hi"].astype(np.int64) - g[k]["lo"] + 1
        assert w.sum() < 0.5 * w.size * 128


@pytest.mark.slow
def test_timed_sequence_full_range_every_frame(tsgm, oracle_runs):
    """The full-range comparison line: the same frames searched over [0, D-1]."""
    _, g = _gpu_sequence(tsgm, tsgm.FLAG_FULL_RANGE, N_FRAMES)
    o = oracle_runs["full"].get(timeout=1800)
    for k in range(N_FRAMES):
        assert np.all(g[k]["lo"] == 0) and np.all(g[k]["hi"] == 127)
        _compare(g[k], o[k], k)


@pytest.mark.slow
def test_timed_sequence_on_a_stream_of_its_own_equals_the_default_stream(tsgm):
    """On a non-default CUDA stream tsgm_frame launches each step as a CUDA graph (captured,
    then updated in place frame after frame); on the legacy default stream it launches the
    kernels one by one. Both give the same maps, bit for bit, on every frame, also after a reset
    (a first frame again: another graph) and with stage timing switched on mid-sequence (back to
    direct launches)."""
    seq = synth.kitti_like(2, n_frames=N_FRAMES)
    W, H = seq.cam.W, seq.cam.H
    b = f32(seq.cam.b)
    left = [dev(x) for x in seq.left]
    right = [dev(x) for x in seq.right]

    def run(stream, profile_from=None):
        out = []
        with tsgm.Context(tsgm.default_params(W, H, flags=tsgm.FLAG_FILL_GAPS),
                          stream=stream) as ctx:
            D, P = empty((H, W), np.float32), empty((H, W), np.float32)
            for rep in range(2):
                ctx.reset()
                for k in range(N_FRAMES):
                    if profile_from is not None and rep == 1 and k == profile_from:
                        ctx.profile(True)
                    ctx.frame(left[k], right[k], seq.R[k], seq.t[k], seq.K, b, D, P)
                    out.append((host(D, np.float32), host(P, np.float32)))
        return out

    ref = run(0)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        got = run(s.cuda_stream, profile_from=6)
    for k, ((Dg, Pg), (Dr, Pr)) in enumerate(zip(got, ref)):
        assert np.array_equal(Dg, Dr), k
        assert np.array_equal(Pg, Pr), k
