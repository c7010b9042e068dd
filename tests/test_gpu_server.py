"""Serving loop: frames of several camera streams submitted interleaved (many waiting at once)
must give exactly the results each stream gets alone through a plain context; ticks of the
batched time step must run several streams' frames together when the HBM budget allows, and
with the smallest budget (the volume pool holds one full-range stream) frames refused by the
pool must run in a later tick, never be dropped."""
import numpy as np
import pytest

from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, host, f32

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def camera_streams():
    """Five streams of two image sizes, four frames each (forward motion and yaw)."""
    specs = [(160, 64, 31), (160, 64, 32), (224, 72, 33), (160, 64, 34), (224, 72, 35)]
    seqs = [synth.make_sequence(seed, W, H, 400.0, 0.54, n_frames=4, n_boxes=3,
                                step_range=(0.3, 0.6), yaw_deg=1.0, noise_sigma=1.0)
            for (W, H, seed) in specs]
    return seqs


def params_for(tsgm, seq):
    return tsgm.default_params(seq.cam.W, seq.cam.H, d_max=63, census_w=5, census_h=5, n_paths=8)


def alone(tsgm, seq):
    W, H = seq.cam.W, seq.cam.H
    out = []
    with tsgm.Context(params_for(tsgm, seq)) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        for k in range(len(seq.left)):
            ctx.frame(dev(seq.left[k]), dev(seq.right[k]), seq.R[k] if k else None,
                      seq.t[k] if k else None, seq.K, f32(seq.cam.b), D, P)
            out.append((host(D, np.float32), host(P, np.float32)))
    return out


@pytest.mark.parametrize("budget", [1 << 40, 1])
def test_results_alone_equal_results_in_the_mix(tsgm, budget):
    seqs = camera_streams()
    ref = [alone(tsgm, s) for s in seqs]
    rng = np.random.default_rng(7)
    with tsgm.Server([params_for(tsgm, s) for s in seqs], hbm_budget_bytes=budget) as srv:
        nxt = [0] * len(seqs)
        outs = {}
        tickets = []
        # interleave submissions across streams in a random order (each stream in frame order)
        order = [i for i in range(len(seqs)) for _ in range(4)]
        rng.shuffle(order)
        for i in order:
            k = nxt[i]
            nxt[i] += 1
            s = seqs[i]
            D = np.empty((s.cam.H, s.cam.W), np.float32)
            P = np.empty_like(D)
            tk = srv.submit(i, s.left[k], s.right[k], s.R[k] if k else None, s.t[k] if k else None,
                            s.K, f32(s.cam.b), D, P)
            outs[(i, k)] = (D, P)
            tickets.append(tk)
        lat = [srv.wait(tk) for tk in tickets]
        st = srv.stats()
    assert st["completed"] == len(order)
    assert all(x > 0 for x in lat) and st["p99_ms"] >= st["p50_ms"] > 0
    if budget > 1:  # the pool holds every stream at full range; ticks run several frames
        assert st["slots"] == len(seqs) and st["max_in_flight"] >= 2
    else:  # the smallest pool: the largest stream at full range
        assert 1 <= st["slots"] < len(seqs)
    for (i, k), (D, P) in outs.items():
        assert np.array_equal(D, ref[i][k][0]), (i, k)
        assert np.array_equal(P, ref[i][k][1]), (i, k)


def frames_alone(tsgm, seq, ks):
    """The stream's frames ks (in order, each with its own pose) through a plain context."""
    W, H = seq.cam.W, seq.cam.H
    out = {}
    with tsgm.Context(params_for(tsgm, seq)) as ctx:
        D, P = empty((H, W), np.float32), empty((H, W), np.float32)
        for i, k in enumerate(ks):
            ctx.frame(dev(seq.left[k]), dev(seq.right[k]), seq.R[k] if i else None,
                      seq.t[k] if i else None, seq.K, f32(seq.cam.b), D, P)
            out[k] = (host(D, np.float32), host(P, np.float32))
    return out


def test_a_failing_frame_leaves_the_other_streams_untouched(tsgm):
    """Frames that cannot run are refused on their own while the others go on: a zero baseline
    (no disparity-space homography, Eq. 1-4) and a later frame without a pose. Each such ticket
    reports INVALID_ARG; its stream keeps the state of its last good frame (its next frame is the
    one a context gives when the refused frame is left out); every other stream's results equal
    its results alone."""
    seqs = camera_streams()
    ref = [alone(tsgm, s) for s in seqs]
    bad = {(1, 2): "zero baseline", (3, 1): "no pose"}
    rng = np.random.default_rng(11)
    with tsgm.Server([params_for(tsgm, s) for s in seqs], hbm_budget_bytes=1 << 40) as srv:
        nxt = [0] * len(seqs)
        order = [i for i in range(len(seqs)) for _ in range(4)]
        rng.shuffle(order)
        outs, tickets = {}, {}
        for i in order:
            k = nxt[i]
            nxt[i] += 1
            s = seqs[i]
            D = np.empty((s.cam.H, s.cam.W), np.float32)
            P = np.empty_like(D)
            R, t, b = (s.R[k], s.t[k], f32(s.cam.b)) if k else (None, None, f32(s.cam.b))
            if bad.get((i, k)) == "zero baseline":
                b = f32(0.0)
            elif bad.get((i, k)) == "no pose":
                R = t = None
            tickets[(i, k)] = srv.submit(i, s.left[k], s.right[k], R, t, s.K, b, D, P)
            outs[(i, k)] = (D, P)
        for key, tk in tickets.items():
            if key in bad:
                with pytest.raises(tsgm.TsgmError) as e:
                    srv.wait(tk)
                assert e.value.status == tsgm.ERR_INVALID_ARG, bad[key]
            else:
                srv.wait(tk)
        assert srv.stats()["completed"] == len(order)
    for i in (0, 2, 4):
        for k in range(4):
            assert np.array_equal(outs[(i, k)][0], ref[i][k][0]), (i, k)
            assert np.array_equal(outs[(i, k)][1], ref[i][k][1]), (i, k)
    for i, ks in ((1, [0, 1, 3]), (3, [0, 2, 3])):
        skipped = frames_alone(tsgm, seqs[i], ks)
        for k in ks:
            assert np.array_equal(outs[(i, k)][0], skipped[k][0]), (i, k)
            assert np.array_equal(outs[(i, k)][1], skipped[k][1]), (i, k)
