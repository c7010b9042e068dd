"""Batched time step (tsgm_batch_frame): every stream of a batch must get, frame after frame, exactly
what a plain tsgm_frame context gives it on the same frames. The previous state of every stream
lives in the batch, so equality over several frames covers the prediction (warp with z-buffer,
gap filling), the windows, the matching and the Kalman update of every stream, all in one graph.

The big case is the multi-camera mix timed by the benchmark: 32 streams (640x480 D=64,
1242x375 D=128, 1920x1080 D=256 in turn), three frames each, streams of one size made distinct by
rolling their images (and moving cx with them). The small cases check a stream sitting a step
out, a refused call that leaves every state as it was, the full-range flag, reset, and the
parameter checks.
"""
import numpy as np
import pytest

from paper_1708_06301_gb300 import synth

from gpu_util import dev, empty, f32, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NS = 32
N_FRAMES = 3


@pytest.fixture(scope="module")
def tsgm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_06301_gb300 import tsgm as t
    t.load()
    return t


def mix_streams(n_streams, n_frames):
    seqs = synth.camera_mix(n_frames)
    out = []
    for i in range(n_streams):
        W, H, D = synth.mix_shape(i)
        sq = seqs[(W, H)]
        left, right, K = synth.shifted_view(sq, 7 * (i // 3))
        out.append(dict(W=W, H=H, D=D, left=left, right=right, K=K, b=f32(sq.cam.b), R=sq.R,
                        t=sq.t))
    return out


def alone(tsgm, s, flags, ks=None, poses=None):
    """Frames ks of stream s through a plain context; poses[j] = (R, t) into frame ks[j]."""
    ks = list(range(len(s["left"]))) if ks is None else ks
    out = []
    with tsgm.Context(tsgm.default_params(s["W"], s["H"], d_max=s["D"] - 1, flags=flags)) as ctx:
        D, P = empty((s["H"], s["W"]), np.float32), empty((s["H"], s["W"]), np.float32)
        for j, k in enumerate(ks):
            R, t = poses[j] if poses and poses[j] else (s["R"][k], s["t"][k])
            ctx.frame(dev(s["left"][k]), dev(s["right"][k]), R if j else None, t if j else None,
                      s["K"], s["b"], D, P)
            out.append((host(D, np.float32), host(P, np.float32)))
    return out


def batch_params(tsgm, streams, flags):
    return [tsgm.default_params(s["W"], s["H"], d_max=s["D"] - 1, flags=flags) for s in streams]


def batch_frame(bt, streams, k, active=None, poses=None, baselines=None):
    """Frame k of every active stream; returns the device outputs (None for streams sitting out)."""
    n = len(streams)
    active = [True] * n if active is None else active
    L = [dev(s["left"][k]) if a else None for s, a in zip(streams, active)]
    Rr = [dev(s["right"][k]) if a else None for s, a in zip(streams, active)]
    Rs = np.stack([poses[i][0] if poses and poses[i] else s["R"][k] for i, s in enumerate(streams)])
    ts = np.stack([poses[i][1] if poses and poses[i] else s["t"][k] for i, s in enumerate(streams)])
    Ks = np.stack([s["K"] for s in streams])
    bs = np.array([s["b"] for s in streams], np.float32) if baselines is None else baselines
    Ds = [empty((s["H"], s["W"]), np.float32) if a else None for s, a in zip(streams, active)]
    Ps = [empty((s["H"], s["W"]), np.float32) if a else None for s, a in zip(streams, active)]
    bt.frame(L, Rr, Rs, ts, Ks, bs, Ds, Ps)
    return Ds, Ps


@pytest.mark.slow
def test_32_stream_mix_equals_single_contexts_for_3_frames(tsgm):
    streams = mix_streams(NS, N_FRAMES)
    got = [[] for _ in range(NS)]
    with tsgm.Batch(batch_params(tsgm, streams, tsgm.FLAG_FILL_GAPS)) as bt:
        l0 = bt.launches()
        for k in range(N_FRAMES):
            Ds, Ps = batch_frame(bt, streams, k)
            for i in range(NS):
                got[i].append((host(Ds[i], np.float32), host(Ps[i], np.float32)))
        # one graph per step: prediction (scatter, gather, two gap-filling passes), windows,
        # pool reservation, offsets, census, cost, aggregation, selection, update
        assert (bt.launches() - l0) == 12 * N_FRAMES
    for i, s in enumerate(streams):
        ref = alone(tsgm, s, tsgm.FLAG_FILL_GAPS)
        for k in range(N_FRAMES):
            assert np.array_equal(got[i][k][0], ref[k][0]), (i, k, "D")
            assert np.array_equal(got[i][k][1], ref[k][1]), (i, k, "P")
        # the later frames search reduced windows: most pixels are matched and valid
        assert np.mean(got[i][-1][0] >= 0) > 0.5, i


def small_streams(n_frames=4, specs=((160, 64, 41), (224, 72, 42), (160, 64, 43), (96, 40, 44))):
    out = []
    for (W, H, seed) in specs:
        sq = synth.make_sequence(seed, W, H, 400.0, 0.54, n_frames=n_frames, n_boxes=3,
                                 step_range=(0.3, 0.6), yaw_deg=1.0, noise_sigma=1.0)
        out.append(dict(W=W, H=H, D=64, left=sq.left, right=sq.right, K=sq.K.astype(np.float32),
                        b=f32(sq.cam.b), R=sq.R, t=sq.t, seq=sq))
    return out


def test_sitting_out_and_a_refused_call_keep_the_state(tsgm):
    """Stream 1 sits frame 2 out (its frame 3 then warps from frame 1); at frame 3 a call with a
    zero baseline for stream 2 is refused as a whole (INVALID_ARG) and changes no state, so the
    repeated call with valid arguments gives what a context gives."""
    streams = small_streams(4)
    flags = tsgm.FLAG_FILL_GAPS
    outs = {}
    with tsgm.Batch(batch_params(tsgm, streams, flags)) as bt:
        for k in range(3):
            active = [not (i == 1 and k == 2) for i in range(len(streams))]
            Ds, Ps = batch_frame(bt, streams, k, active=active)
            for i, a in enumerate(active):
                if a:
                    outs[(i, k)] = (host(Ds[i], np.float32), host(Ps[i], np.float32))
        poses = [None, streams[1]["seq"].pose_between(1, 3), None, None]
        bad = np.array([s["b"] for s in streams], np.float32)
        bad[2] = 0.0
        with pytest.raises(tsgm.TsgmError) as e:
            batch_frame(bt, streams, 3, poses=poses, baselines=bad)
        assert e.value.status == tsgm.ERR_INVALID_ARG
        Ds, Ps = batch_frame(bt, streams, 3, poses=poses)
        for i in range(len(streams)):
            outs[(i, 3)] = (host(Ds[i], np.float32), host(Ps[i], np.float32))
    for i, s in enumerate(streams):
        if i == 1:
            ks = [0, 1, 3]
            ref = alone(tsgm, s, flags, ks, [None, (s["R"][1], s["t"][1]), poses[1]])
        else:
            ks = [0, 1, 2, 3]
            ref = alone(tsgm, s, flags)
        for j, k in enumerate(ks):
            assert np.array_equal(outs[(i, k)][0], ref[j][0]), (i, k)
            assert np.array_equal(outs[(i, k)][1], ref[j][1]), (i, k)


def test_frames_refused_by_the_pool_run_in_a_later_step(tsgm):
    """A pool that holds one stream at full range (max_labels = 16 of 64 labels, four streams of
    one size): the first frames are full range, so each step runs some streams and refuses the
    others, which keep their state and get the same frame again at the next step (longest
    refused first). Every stream's outputs, frame by frame, equal its context's."""
    streams = small_streams(4, [(160, 64, 51), (160, 64, 52), (160, 64, 53), (160, 64, 54)])
    flags = tsgm.FLAG_FILL_GAPS
    n = len(streams)
    with tsgm.Batch(batch_params(tsgm, streams, flags), max_labels=16) as bt:
        pool, largest = bt.pool()
        assert pool == largest == 160 * 64 * 64
        nxt = [0] * n
        outs = [[] for _ in range(n)]
        refused = 0
        for _ in range(40):
            if min(nxt) >= 4:
                break
            active = [k < 4 for k in nxt]
            poses = [(s["R"][k], s["t"][k]) if k < 4 else None for s, k in zip(streams, nxt)]
            L = [dev(s["left"][k]) if a else None for s, k, a in zip(streams, nxt, active)]
            Rr = [dev(s["right"][k]) if a else None for s, k, a in zip(streams, nxt, active)]
            Ds = [empty((s["H"], s["W"]), np.float32) if a else None for s, a in zip(streams, active)]
            Ps = [empty((s["H"], s["W"]), np.float32) if a else None for s, a in zip(streams, active)]
            eye = (np.eye(3, dtype=np.float32), np.zeros(3, np.float32))
            bt.frame(L, Rr, np.stack([(p or eye)[0] for p in poses]),
                     np.stack([(p or eye)[1] for p in poses]), np.stack([s["K"] for s in streams]),
                     np.array([s["b"] for s in streams], np.float32), Ds, Ps)
            st = bt.stream_status()
            for i in range(n):
                if st[i] == tsgm.Batch.RAN:
                    outs[i].append((host(Ds[i], np.float32), host(Ps[i], np.float32)))
                    nxt[i] += 1
                elif st[i] == tsgm.Batch.REFUSED:
                    refused += 1
        assert min(nxt) == 4 and refused > 0
    for i, s in enumerate(streams):
        ref = alone(tsgm, s, flags)
        for k in range(4):
            assert np.array_equal(outs[i][k][0], ref[k][0]), (i, k)
            assert np.array_equal(outs[i][k][1], ref[k][1]), (i, k)


def test_full_range_and_reset(tsgm):
    """With the full-range flag every stream equals its full-range context; after reset the next
    frame is a first frame for every stream."""
    streams = small_streams(3)
    flags = tsgm.FLAG_FULL_RANGE
    with tsgm.Batch(batch_params(tsgm, streams, flags)) as bt:
        got = []
        for k in range(3):
            Ds, Ps = batch_frame(bt, streams, k)
            got.append([(host(d, np.float32), host(p, np.float32)) for d, p in zip(Ds, Ps)])
        bt.reset()
        Ds, Ps = batch_frame(bt, streams, 2)
        after = [(host(d, np.float32), host(p, np.float32)) for d, p in zip(Ds, Ps)]
    for i, s in enumerate(streams):
        ref = alone(tsgm, s, flags)
        for k in range(3):
            assert np.array_equal(got[k][i][0], ref[k][0]), (i, k)
            assert np.array_equal(got[k][i][1], ref[k][1]), (i, k)
        first = alone(tsgm, s, flags, [2])
        assert np.array_equal(after[i][0], first[0][0]), i
        assert np.array_equal(after[i][1], first[0][1]), i


def test_parameter_checks(tsgm):
    streams = small_streams(2)
    prm = batch_params(tsgm, streams, tsgm.FLAG_FILL_GAPS)
    prm[1] = tsgm.default_params(streams[1]["W"], streams[1]["H"], d_max=63, flags=0)
    with tsgm.Batch(prm) as bt:  # matching alone is still fine; the time step is refused
        with pytest.raises(tsgm.TsgmError) as e:
            batch_frame(bt, streams, 0)
        assert e.value.status == tsgm.ERR_INVALID_ARG
    with tsgm.Batch(batch_params(tsgm, streams, tsgm.FLAG_SAD_CHECK)) as bt:
        with pytest.raises(tsgm.TsgmError) as e:
            batch_frame(bt, streams, 0)
        assert e.value.status == tsgm.ERR_UNIMPLEMENTED
    with tsgm.Batch(batch_params(tsgm, streams, 0)) as bt:
        batch_frame(bt, streams, 0)
        with pytest.raises(tsgm.TsgmError) as e:  # a second frame needs poses
            bt.frame([dev(s["left"][1]) for s in streams], [dev(s["right"][1]) for s in streams],
                     None, None, np.stack([s["K"] for s in streams]),
                     np.array([s["b"] for s in streams], np.float32),
                     [empty((s["H"], s["W"]), np.float32) for s in streams],
                     [empty((s["H"], s["W"]), np.float32) for s in streams])
        assert e.value.status == tsgm.ERR_INVALID_ARG
