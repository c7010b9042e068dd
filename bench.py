"""Benchmark of the ego-motion-reduced SGM path on one GB300 (or N independent replicas).

Workload: the driving-shaped synthetic sequence, 10 frames of 1242x375 uint8 stereo (ground
plane + 20 boxes at 5-60 m, image noise sigma 2, forward 0.5-1.5 m and yaw +-2 deg per frame),
census 9x7, 8 paths, D = 128: frame 1 searches the whole range, frames 2-10 the +-3 sigma
windows around the warped prediction. One step = the whole 10-frame sequence through
tsgm_frame (prediction, windows, census, ragged cost, SGM, selection + LR check, Kalman).

Prints one JSON line: frames/s of the reduced-window pipeline (value), SGM Gcells/s, the same
figures for full-range SGM on the same frames, bad-3px of both against the rendered ground
truth, the search-space fraction, the roofline of the dominant kernel (SGM aggregation, CUDA
events on the context stream over the timed region), the CPU oracle on a bounded sample, an
end-to-end number through the host-buffer entry points (tsgm_frame_host_async per frame with a
wait per step, and the blocking tsgm_frame_host beside it), and SM clocks sampled during the
timed region.

`--impl reference` times the CPU oracle instead (the paper has no reference implementation).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "reduced-range SGM Gcells/s and fps vs full-range on same GB300; % HBM roofline"
WORKLOAD = ("kitti-shaped synthetic sequence: 10 frames 1242x375 uint8 stereo, f=721, b=0.54, "
            "ground + 20 boxes, noise sigma 2, census 9x7, 8 paths, P1=8, P2=32, D=128; frame 1 "
            "full range, frames 2-10 +-3 sigma windows around the warped prediction with its "
            "one-pixel gaps filled (Eq. 7-8, gamma_f = 1 px)")
N_FRAMES = 10
L2_FLUSH_BYTES = 256 << 20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in a background process."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    import torch.distributed as dist
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def reduce_max(values, ws, device=None):
    """Max over ranks of a list of floats (identity at world size 1)."""
    if ws == 1:
        return list(values)
    import torch
    import torch.distributed as dist
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


# ----------------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ----------------------------------------------------------------------------------------------

def oracle_frames(seq, frames):
    """Time the CPU oracle (single thread) on the given frame indices, run in order by one
    tracker that restarts (no prediction) whenever frame 0 comes up."""
    import oracle
    oracle.build()
    prm = oracle.Params(1242, 375, d_max=127, census_w=9, census_h=7, n_paths=8, fill_gaps=True)
    tr = oracle.Tracker(prm)
    b = np.float32(seq.cam.b)
    times = []
    for k in frames:
        if k == 0:
            tr = oracle.Tracker(prm)
        t0 = time.perf_counter()
        tr.frame(seq.left[k], seq.right[k], seq.R[k], seq.t[k], seq.K, b)
        times.append(time.perf_counter() - t0)
    return times


def _oracle_worker(frames_data, reps):
    """One host thread's share of the threaded CPU baseline: the whole sequence `reps` times with
    its own tracker (frames of different sequences are independent)."""
    import oracle
    left, right, Rs, ts, K, b = frames_data
    prm = oracle.Params(1242, 375, d_max=127, census_w=9, census_h=7, n_paths=8, fill_gaps=True)
    t0 = time.perf_counter()
    for _ in range(reps):
        tr = oracle.Tracker(prm)
        for k in range(len(left)):
            tr.frame(left[k], right[k], Rs[k], ts[k], K, b)
    return len(left) * reps, time.perf_counter() - t0


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_threaded(seq, threads: int):
    """The oracle (itself single-threaded, as it stands) run as `threads` independent copies of
    the 10-frame sequence in a spawn process pool, one per host core: aggregate frames/s."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    data = (list(seq.left), list(seq.right), list(seq.R), list(seq.t), seq.K,
            np.float32(seq.cam.b))
    ctx = mp.get_context("spawn")
    with ctx.Pool(threads) as pool:
        pool.starmap(_oracle_worker, [(data, 0)] * threads)  # start-up outside the clock
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_worker, [(data, 1)] * threads)
        wall = time.perf_counter() - t0
    return sum(r[0] for r in res) / wall


def run_reference(args, ws, rank):
    """The oracle on the host cores: step s processes frame s mod 10 of the sequence (so ten
    steps have the same full-range/reduced mix as one GPU step)."""
    if rank != 0:
        return
    from paper_1708_06301_gb300 import synth
    seq = synth.kitti_like(2, n_frames=N_FRAMES)
    order = [i % N_FRAMES for i in range(args.warmup + args.steps)]
    times = oracle_frames(seq, order)[args.warmup:]
    total = sum(times)
    fps = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u8/u16 (costs), f32 (warp, Kalman)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "one frame of the sequence (frame s mod 10)"},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} frames cycling through the 10-frame sequence "
                                   "(frame 1 full range), single thread"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------

def mix_shape(i: int):
    """Stream i of the multi-stream workloads: 640x480 D=64, 1242x375 D=128, 1920x1080 D=256."""
    from paper_1708_06301_gb300 import synth
    return synth.mix_shape(i)


def render_mix(n_frames: int):
    """One rendered driving-shaped sequence per image size (focal length scaled with the width)."""
    from paper_1708_06301_gb300 import synth
    return synth.camera_mix(n_frames)


def bench_adjoint(dev, steps: int):
    """Adjoint of prediction + Kalman at 1242x375 (random maps D 1-127, P 0.1-4, random 6-DoF pose
    with |t| <= 1.5 m and angles within 3 deg): device time of forward and backward."""
    import torch
    from paper_1708_06301_gb300 import synth, tsgm
    W, H = 1242, 375
    D, P = synth.random_maps(5, W, H, d_range=(1, 127), p_range=(0.1, 4.0))
    Dz, rz = synth.random_maps(6, W, H, d_range=(1, 127), p_range=(0.5, 4.0), invalid_frac=0.1)
    _, t = synth.random_pose(7, max_t=1.5)
    pose6 = np.concatenate([np.radians([1.5, -2.0, 0.7]), t.astype(np.float64)])
    K = synth.Camera(W, H, 721.0, 0.54).K
    b = np.float32(0.54)
    dD, dP, dDz, drz = (torch.from_numpy(x).to(dev) for x in (D, P, Dz, rz))
    gD = torch.randn((H, W), device=dev)
    gP = torch.randn((H, W), device=dev)
    oD, oP = torch.empty_like(dD), torch.empty_like(dP)
    with tsgm.Context(tsgm.default_params(W, H), stream=torch.cuda.current_stream(dev).cuda_stream) as c:
        for _ in range(3):
            c.adjoint_forward(dD, dP, pose6, K, b, 0.25, 1.0, dDz, drz, oD, oP)
            c.adjoint_backward(dD, dP, pose6, K, b, 0.25, 1.0, dDz, drz, gD, gP)
        fwd, bwd = [], []
        st = torch.cuda.current_stream(dev)
        for _ in range(steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            c.adjoint_forward(dD, dP, pose6, K, b, 0.25, 1.0, dDz, drz, oD, oP)
            e1.record(st)
            c.adjoint_backward(dD, dP, pose6, K, b, 0.25, 1.0, dDz, drz, gD, gP)
            e2.record(st)
            torch.cuda.synchronize()
            fwd.append(e0.elapsed_time(e1))
            bwd.append(e1.elapsed_time(e2))
    return {"workload": "1242x375 random maps, random 6-DoF pose, gradients w.r.t. pose, q, r-scale",
            "forward_ms": float(np.median(fwd)),
            "backward_ms_incl_host_reduction": float(np.median(bwd))}


BATCH_STREAMS = 32
BATCH_MAX_LABELS = 24


def batched_stream(seqs, i: int):
    """Inputs of stream i of the batched workload: its size (W, H, D), the rendered left and right
    images, and per-pixel windows of 4-24 labels (uniform, seeded) around the rounded ground
    truth, clipped into [0, D - 1]."""
    from paper_1708_06301_gb300 import synth
    W, H, D = mix_shape(i)
    sq = seqs[(W, H)]
    gt = np.clip(np.floor(sq.gt_disp[0] + 0.5), 0, D - 1).astype(np.int64).reshape(-1)
    n = W * H
    w = 4 + np.floor(synth.uniform01(200 + i, np.arange(n)) * 21).astype(np.int64)
    lo = np.clip(gt - w // 2, 0, D - w)
    hi = lo + w - 1
    return (W, H, D, sq.left[0], sq.right[0], lo.astype(np.int16).reshape(H, W),
            hi.astype(np.int16).reshape(H, W))


def bench_batched(dev, steps: int, warmup: int):
    """32 streams (i mod 3 -> 640x480 D=64, 1242x375 D=128, 1920x1080 D=256), per-pixel windows of
    4-24 labels around the ground truth, one graph replay per step."""
    import torch
    from paper_1708_06301_gb300 import tsgm
    seqs = render_mix(1)
    NS = BATCH_STREAMS
    params, L, R, LO, HI, DZ, RZ = [], [], [], [], [], [], []
    px = 0
    for i in range(NS):
        W, H, D, left_i, right_i, lo_i, hi_i = batched_stream(seqs, i)
        params.append(tsgm.default_params(W, H, d_max=D - 1))
        L.append(torch.from_numpy(left_i).to(dev))
        R.append(torch.from_numpy(right_i).to(dev))
        LO.append(torch.from_numpy(lo_i).to(dev))
        HI.append(torch.from_numpy(hi_i).to(dev))
        DZ.append(torch.empty((H, W), dtype=torch.float32, device=dev))
        RZ.append(torch.empty((H, W), dtype=torch.float32, device=dev))
        px += W * H
    st = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    with tsgm.Batch(params, max_labels=BATCH_MAX_LABELS, stream=st.cuda_stream) as bt:
        tune_ms, shape = bt.autotune(L, R, LO, HI, DZ, RZ, reps=2)
        for _ in range(warmup):
            bt.match(L, R, LO, HI, DZ, RZ)
        torch.cuda.synchronize()
        cells, over = bt.cells()
        ms, sgm_ms, prof_step = [], [], []
        l0 = bt.launches()
        for s_ in range(steps):
            flush.fill_(float(s_))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            bt.match(L, R, LO, HI, DZ, RZ)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        launches = bt.launches() - l0
        for s_ in range(steps):  # aggregation kernel alone: direct launches with events around it
            flush.fill_(float(s_))
            torch.cuda.synchronize()
            a_ms, z_ms = bt.profile(L, R, LO, HI, DZ, RZ)
            sgm_ms.append(a_ms)
            prof_step.append(z_ms)
    step_s = float(np.mean(ms)) / 1000.0
    sgm_s = float(np.mean(sgm_ms)) / 1000.0
    peak, kind = peaks()
    agg_bytes = algorithmic_sgm_bytes(cells, px)
    # matching step (no prediction or update): 4 B/cell; per pixel images 2, census re-read 32,
    # windows 4, offsets 4, D_z + r 8 out
    step_bytes = 4 * cells + 50 * px
    return {"workload": "32 streams: 11x 640x480 D=64, 11x 1242x375 D=128, 10x 1920x1080 D=256; "
                        "windows 4-24 labels around ground truth; inputs larger than L2",
            "px_per_step": px, "cells_per_step": cells, "overflowed_streams": over,
            "ms_per_step": step_s * 1000.0, "gcells_per_s": cells / step_s / 1e9,
            "frames_per_s": NS / step_s, "autotuned_shape": shape, "autotune_ms": tune_ms,
            "kernels_per_step": launches / max(steps, 1),
            "ms_per_step_direct_launches": float(np.mean(prof_step)),
            "roofline_sgm": {"bound": "hbm", "achieved": agg_bytes / sgm_s / 1e9, "peak": peak,
                             "unit": "GB/s", "frac": agg_bytes / sgm_s / 1e9 / peak,
                             "peak_kind": kind, "avg_launch_us": sgm_s * 1e6,
                             "algorithmic_bytes_per_launch": agg_bytes},
            "step_hbm_frac": step_bytes / step_s / 1e9 / peak}


BATCH_FRAMES = 4


def bench_batched_frame(dev, steps: int, warmup: int):
    """The whole time step of 32 camera streams (same size mix; streams of one size see the scene
    from principal points 7 px apart) in one graph replay per step: prediction with gap filling,
    windows, matching and update of every stream. The frames go back and forth through a
    4-frame sequence (0 1 2 3 2 1 0 1 ...) with the true relative pose of each move; the first
    step (no previous state) runs in the warm-up."""
    import torch
    from paper_1708_06301_gb300 import synth, tsgm
    seqs = render_mix(BATCH_FRAMES)
    NS = BATCH_STREAMS
    params, Ls, Rs_img, Ks, bs, Ds, Ps = [], [], [], [], [], [], []
    views = []
    px = 0
    for i in range(NS):
        W, H, D = mix_shape(i)
        sq = seqs[(W, H)]
        left, right, K = synth.shifted_view(sq, 7 * (i // 3))
        views.append(sq)
        params.append(tsgm.default_params(W, H, d_max=D - 1, flags=tsgm.FLAG_FILL_GAPS))
        Ls.append([torch.from_numpy(x).to(dev) for x in left])
        Rs_img.append([torch.from_numpy(x).to(dev) for x in right])
        Ks.append(K)
        bs.append(np.float32(sq.cam.b))
        Ds.append(torch.empty((H, W), dtype=torch.float32, device=dev))
        Ps.append(torch.empty((H, W), dtype=torch.float32, device=dev))
        px += W * H
    Ks = np.stack(Ks)
    bs = np.array(bs, np.float32)
    cyc = list(range(BATCH_FRAMES)) + list(range(BATCH_FRAMES - 2, 0, -1))
    order = [cyc[s_ % len(cyc)] for s_ in range(1 + warmup + steps)]
    poses = {}
    for a, b in zip(order[:-1], order[1:]):
        if (a, b) not in poses:
            per = [views[i].pose_between(a, b) for i in range(NS)]
            poses[(a, b)] = (np.stack([x[0] for x in per]), np.stack([x[1] for x in per]))
    st = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ms, cells = [], []
    with tsgm.Batch(params, stream=st.cuda_stream) as bt:
        def step(j):
            f = order[j]
            R, t = poses[(order[j - 1], f)] if j else (None, None)
            bt.frame([x[f] for x in Ls], [x[f] for x in Rs_img], R, t, Ks, bs, Ds, Ps)
        for j in range(1 + warmup):
            step(j)
        torch.cuda.synchronize()
        l0 = bt.launches()
        for j in range(1 + warmup, 1 + warmup + steps):
            flush.fill_(float(j))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            step(j)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            cells.append(bt.cells()[0])
        launches = bt.launches() - l0
    step_s = float(np.mean(ms)) / 1000.0
    mean_cells = float(np.mean(cells))
    peak, kind = peaks()
    step_bytes = algorithmic_step_bytes(int(mean_cells), px)
    return {"workload": "32 streams: 11x 640x480 D=64, 11x 1242x375 D=128, 10x 1920x1080 D=256; "
                        "rendered 4-frame driving sequences played back and forth; whole time step "
                        "(prediction, gap filling, windows, matching, Kalman update); inputs larger "
                        "than L2",
            "px_per_step": px, "mean_cells_per_step": mean_cells,
            "searched_fraction": mean_cells / sum(p.width * p.height * (p.d_max + 1) for p in params),
            "ms_per_step": step_s * 1000.0, "frames_per_s": NS / step_s,
            "kernels_per_step": launches / max(steps, 1),
            "step_hbm_frac": step_bytes / step_s / 1e9 / peak, "peak_kind": kind,
            "algorithmic_bytes_per_step": step_bytes}


def bench_serving(duration_s: float, budget_gb: float):
    """64 camera streams (same size mix), each sending frames as a Poisson process at 10-30 Hz.
    Every stream's first frame (full range: no previous state) is served before the clock starts;
    then frames arrive for `duration_s` seconds and are measured: served frames/s = frames done /
    time from the first arrival to the last result, latency from submission to result."""
    import queue
    from paper_1708_06301_gb300 import synth, tsgm
    F = 6
    seqs = render_mix(F)
    NS = 64
    params = []
    for i in range(NS):
        W, H, D = mix_shape(i)
        params.append(tsgm.default_params(W, H, d_max=D - 1, flags=tsgm.FLAG_FILL_GAPS))
    rs = synth.Stream(11, 0x5E7)
    events = []
    for i in range(NS):
        rate = rs.uniform(10.0, 30.0)
        tcur = rs.uniform(0.0, 1.0 / rate)
        k = 1
        while tcur < duration_s:
            events.append((tcur, i, k))
            k += 1
            tcur += -np.log(max(rs.uniform(), 1e-12)) / rate
    events.sort()
    done_q = queue.Queue()
    lat = []

    def waiter(srv):
        while True:
            item = done_q.get()
            if item is None:
                return
            lat.append(srv.wait(item[0]))

    def frame_of(k):  # frames go back and forth through the F rendered ones
        cyc = list(range(F)) + list(range(F - 2, 0, -1))
        return cyc[k % len(cyc)]

    def submit(srv, i, k):
        W, H, D = mix_shape(i)
        sq = seqs[(W, H)]
        f = frame_of(k)
        Rm, tv = (None, None) if k == 0 else sq.pose_between(frame_of(k - 1), f)
        Dout = np.empty((H, W), np.float32)
        Pout = np.empty((H, W), np.float32)
        return srv.submit(i, sq.left[f], sq.right[f], Rm, tv, sq.K, np.float32(sq.cam.b), Dout,
                          Pout), Dout, Pout

    with tsgm.Server(params, hbm_budget_bytes=int(budget_gb * (1 << 30))) as srv:
        first = [submit(srv, i, 0) for i in range(NS)]
        for tk, _, _ in first:
            srv.wait(tk)
        th = threading.Thread(target=waiter, args=(srv,), daemon=True)
        th.start()
        t0 = time.perf_counter()
        for (ta, i, k) in events:
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            done_q.put(submit(srv, i, k))
        done_q.put(None)
        th.join()
        t_end = time.perf_counter() - t0
        st = srv.stats()
    lat_ms = np.array(lat)
    return {"workload": "64 camera streams (22x 640x480 D=64, 22x 1242x375 D=128, 20x 1920x1080 "
                        "D=256), Poisson frame arrivals at 10-30 Hz per stream, frames going back "
                        "and forth through 6 rendered ones with the true relative poses",
            "duration_s": duration_s, "frames": len(events), "frames_per_s": len(events) / t_end,
            "offered_frames_per_s": len(events) / duration_s,
            "served_over_offered": (len(events) / t_end) / (len(events) / duration_s),
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "warmup": "every stream's first (full-range) frame served before the clock starts",
            "slots_full_range": st["slots"], "max_frames_per_tick": st["max_in_flight"],
            "hbm_budget_gb": budget_gb}


# DRAM bytes (read + write) of one frame's aggregation, mean over the ten frames of one step of the
# sequence from ncu's dram__bytes_read.sum + dram__bytes_write.sum
# (profiles/k_sgm_kitti_1242x375_reduced.md): the full-range frame, one launch of k_sgm_full, 676
# MB; nine reduced frames, two launches each (the lane-group form that does the work and the
# other, which returns at once), 11-22 MB.
SGM_DRAM_BYTES_PER_LAUNCH = 80998682
SGM_DRAM_NOTE = None


def algorithmic_sgm_bytes(cells: int, px: int, census_bytes: int = 8) -> int:
    """Bytes the path aggregation must move once (the method's minimum, not this kernel's
    layout): the directions cannot all be walked in one pass, so a 16-bit partial sum crosses
    from a forward to a backward sweep, 2 B written + 2 B read per window cell; per pixel the
    census codes of both images are read in both sweeps (2 x 2 x census_bytes) and the window
    bounds and ragged offsets once (4 + 4 B): 4 B/cell + 40 B/px with the 9x7 census."""
    return 4 * cells + (2 * 2 * census_bytes + 8) * px


def algorithmic_step_bytes(cells: int, px: int, census_bytes: int = 8) -> int:
    """Bytes of a whole time step (prediction, windows, matching, update): 4 B/cell as above;
    per pixel: images 2, census re-read 2 x 2 x census_bytes, windows 4, offsets 4, D_z + r 8
    out; warp: D, P in 8, z-buffer key read-modify-write 16, predicted D, P out 8; Kalman: 16 in,
    8 out (106 B/px with the 9x7 census)."""
    return 4 * cells + (2 + 4 * census_bytes + 4 + 4 + 8 + 8 + 16 + 8 + 16 + 8) * px


def run_ours(args, ws, rank, local):
    import torch
    from paper_1708_06301_gb300 import build as tbuild
    from paper_1708_06301_gb300 import synth, tsgm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    # one non-default stream for everything: the library's kernels, the events, the L2 flush
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        run_ours_on_stream(args, ws, rank, local, dev, stream)


def run_only(args, dev):
    """One of the extra measurements alone, printed as one JSON line."""
    k = max(3, args.steps // 2)
    fn = {"adjoint": lambda: bench_adjoint(dev, 10),
          "batched": lambda: bench_batched(dev, k, 2),
          "batched_frame": lambda: bench_batched_frame(dev, k, 3),
          "serving": lambda: bench_serving(args.serving_seconds, 64.0)}[args.only]
    print(json.dumps({"only": args.only, args.only: fn()}), flush=True)


def run_ours_on_stream(args, ws, rank, local, dev, stream):
    import torch
    from paper_1708_06301_gb300 import synth, tsgm

    if args.only:
        if rank == 0:
            run_only(args, dev)
        return

    seq = synth.kitti_like(2, n_frames=N_FRAMES)
    W, H = seq.cam.W, seq.cam.H
    n = W * H
    b = np.float32(seq.cam.b)
    K = seq.K
    left = [torch.from_numpy(x).to(dev) for x in seq.left]
    right = [torch.from_numpy(x).to(dev) for x in seq.right]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def make(flags):
        return tsgm.Context(tsgm.default_params(W, H, flags=flags), stream=stream.cuda_stream)

    ctx = make(tsgm.FLAG_FILL_GAPS)
    ctx_full = make(tsgm.FLAG_FULL_RANGE)
    ctx_plain = make(0)  # the prediction without gap filling, for comparison
    # the prediction with its edges rejected (Sec. 2.2) before the gap filling, for comparison
    ctx_edge = make(tsgm.FLAG_FILL_GAPS | tsgm.FLAG_EDGE_REJECT)
    # the prediction's left-right check (Sec. 2.2, Fig. 3(d)) and the SAD check of the updated
    # map (Sec. 2.4) on top of the gap filling, for comparison
    ctx_chk = make(tsgm.FLAG_FILL_GAPS | tsgm.FLAG_PRED_LR_CHECK | tsgm.FLAG_SAD_CHECK)
    Dout = torch.empty((H, W), dtype=torch.float32, device=dev)
    Pout = torch.empty_like(Dout)

    def step(c):
        c.reset()
        for k in range(N_FRAMES):
            c.frame(left[k], right[k], seq.R[k], seq.t[k], K, b, Dout, Pout)

    # untimed pass: cell counts and accuracy per frame
    def characterise(c):
        c.reset()
        cells, bad = [], []
        for k in range(N_FRAMES):
            c.frame(left[k], right[k], seq.R[k], seq.t[k], K, b, Dout, Pout)
            cells.append(c.cells())
            D = Dout.cpu().numpy()
            gt = seq.gt_disp[k]
            bad.append(float(np.mean((D < 0) | (np.abs(D - gt) > 3))))
        return cells, bad

    if args.quick:
        # only the reduced-window steps (for profiler captures): no oracle, no extra passes
        for _ in range(args.warmup + args.steps):
            step(ctx)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"quick": True, "steps": args.steps, "warmup": args.warmup,
                              "launches": ctx.launches()}), flush=True)
        return
    cells_red, bad_red = characterise(ctx)
    cells_full, bad_full = characterise(ctx_full)
    cells_plain, bad_plain = characterise(ctx_plain)
    cells_edge, bad_edge = characterise(ctx_edge)
    cells_chk, bad_chk = characterise(ctx_chk)

    def timed(c, K_steps, W_steps, profile):
        for _ in range(W_steps):
            step(c)
        torch.cuda.synchronize()
        if profile:
            c.profile(True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K_steps)]
        l0 = c.launches()
        barrier(ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in range(K_steps):
            flush.fill_(float(s))  # L2 flush outside the timed events
            ev[s][0].record(stream)
            step(c)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
        barrier(ws)
        wall = time.perf_counter() - t0
        ms = [a.elapsed_time(e) for a, e in ev]
        stages = c.stage_times() if profile else None
        if profile:
            c.profile(False)
        return sum(ms), wall, c.launches() - l0, stages

    sampler = ClockSampler(local)
    sampler.start()
    t_red, wall_red, launches, _ = timed(ctx, args.steps, args.warmup, profile=False)
    clocks = sampler.stop()
    k_full = max(1, args.steps // 2)
    t_full, _, _, _ = timed(ctx_full, k_full, max(3, args.warmup // 2), profile=False)
    # stage times (CUDA events around every stage on the context's streams) from separate passes
    # over the same steps: the events themselves are not in the timed headline
    k_prof = max(3, args.steps // 2)
    _, _, _, stages = timed(ctx, k_prof, 2, profile=True)
    _, _, _, stages_full = timed(ctx_full, k_full, 2, profile=True)
    t_plain, _, _, _ = timed(ctx_plain, k_full, 3, profile=False)
    t_edge, _, _, _ = timed(ctx_edge, k_full, 3, profile=False)
    t_chk, _, _, _ = timed(ctx_chk, k_full, 3, profile=False)

    # end to end through the host-buffer entry point (pinned host memory)
    hl = [torch.from_numpy(x).pin_memory() for x in seq.left]
    hr = [torch.from_numpy(x).pin_memory() for x in seq.right]
    hD = torch.empty((H, W), dtype=torch.float32).pin_memory()
    hP = torch.empty_like(hD).pin_memory()

    def step_host():
        # the streaming form: frames enqueued with their copies, one wait per step
        ctx.reset()
        for k in range(N_FRAMES):
            ctx.frame_host_async(hl[k], hr[k], seq.R[k], seq.t[k], K, b, hD, hP)
        ctx.wait()

    def step_host_blocking():
        ctx.reset()
        for k in range(N_FRAMES):
            ctx.frame_host(hl[k], hr[k], seq.R[k], seq.t[k], K, b, hD, hP)

    def time_host(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for s in range(args.steps):
            flush.fill_(float(s))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            ms.append(1000 * (time.perf_counter() - t0))
        return ms

    e2e_ms = time_host(step_host)
    e2e_blocking_ms = time_host(step_host_blocking)

    tmax = reduce_max([t_red, t_full, sum(e2e_ms)], ws, device=dev)
    t_red_max, t_full_max, e2e_max = tmax
    if rank != 0:
        return

    frames = N_FRAMES * args.steps * ws
    fps = frames / (t_red_max / 1000.0)
    fps_full = N_FRAMES * k_full * ws / (t_full_max / 1000.0)
    # SGM stages a5-a9 (census, cost, aggregation, selection + LR) per frame
    sgm_stages = ("census", "cost", "sgm", "select")
    ms_sgm_red = sum(stages[s][0] for s in sgm_stages) / k_prof
    ms_sgm_full = sum(stages_full[s][0] for s in sgm_stages) / k_full
    gcells_red = sum(cells_red) / (ms_sgm_red / 1000.0) / 1e9
    gcells_full = sum(cells_full) / (ms_sgm_full / 1000.0) / 1e9

    # roofline of the dominant kernel (SGM aggregation): average launch over the profiled pass of
    # the same steps (CUDA events on the stream it is launched on)
    agg_ms, agg_cnt = stages["sgm"]
    agg_avg_s = agg_ms / agg_cnt / 1000.0
    bytes_per_launch = algorithmic_sgm_bytes(int(np.mean(cells_red)), n)
    achieved = bytes_per_launch / agg_avg_s / 1e9
    peak, peak_kind = peaks()

    extra = {}
    if not args.skip_forms:
        extra["adjoint"] = bench_adjoint(dev, 10)
        extra["batched"] = bench_batched(dev, max(3, args.steps // 2), 2)
        extra["batched_frame"] = bench_batched_frame(dev, max(3, args.steps // 2), 3)
        extra["serving"] = bench_serving(args.serving_seconds, 64.0)
    cpu_s = sum(oracle_frames(seq, list(range(N_FRAMES))))
    n_threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cpu_fps_threaded = oracle_threaded(seq, n_threads)
    cpu_name = cpu_model()
    line = {
        "metric": METRIC,
        "value": fps,
        "unit": "frames/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_red_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8/u16 (costs), f32 (warp, Kalman)",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": N_FRAMES,
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "sgm_gcells_per_s": gcells_red,
        "full_range": {"fps": fps_full, "sgm_gcells_per_s": gcells_full,
                       "ms_per_step": t_full_max / k_full,
                       "ms_sgm_stages_per_step": ms_sgm_full},
        "speedup_vs_full_range": fps / fps_full,
        "without_gap_fill": {"fps": N_FRAMES * k_full / (t_plain / 1000.0),
                             "search_space_frac": [c / (n * 128) for c in cells_plain],
                             "bad3px_updated": bad_plain},
        "with_edge_rejection": {"fps": N_FRAMES * k_full / (t_edge / 1000.0),
                                "search_space_frac": [c / (n * 128) for c in cells_edge],
                                "bad3px_updated": bad_edge},
        "with_consistency_checks": {"fps": N_FRAMES * k_full / (t_chk / 1000.0),
                                    "search_space_frac": [c / (n * 128) for c in cells_chk],
                                    "bad3px_updated": bad_chk},
        "search_space_frac": [c / (n * 128) for c in cells_red],
        "bad3px": {"reduced_updated": bad_red, "full_range_updated": bad_full},
        "stage_ms_per_step": {k: v[0] / k_prof for k, v in stages.items() if v[1]},
        "roofline": {"bound": "hbm", "kernel": "k_sgm (path aggregation)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": SGM_DRAM_BYTES_PER_LAUNCH,
                     "traffic_note": SGM_DRAM_NOTE if SGM_DRAM_BYTES_PER_LAUNCH is None else None,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_us": agg_avg_s * 1e6,
                     "timed_in": "a profiled pass of the same steps beside the headline's"},
        "cpu_baseline": {"value": N_FRAMES / cpu_s, "unit": "frames/s", "cores": 1,
                         "kind": "oracle", "cpu": cpu_name,
                         "sample": "one step: the 10-frame sequence (1 full-range, 9 reduced), "
                                   "single thread",
                         "threaded": {"value": cpu_fps_threaded, "unit": "frames/s",
                                      "cores": n_threads, "cpu": cpu_name,
                                      "sample": f"{n_threads} independent copies of the 10-frame "
                                                "sequence at once, one process per core (the "
                                                "oracle itself is single-threaded)"}},
        "e2e": {"value": frames / (e2e_max / 1000.0), "unit": "frames/s",
                "h2d_bytes_per_step": N_FRAMES * 2 * n,
                "d2h_bytes_per_step": N_FRAMES * 2 * 4 * n,
                "call": "tsgm_frame_host_async per frame, tsgm_wait per step (pinned host buffers)",
                "blocking_value": frames / (sum(e2e_blocking_ms) / 1000.0),
                "blocking_call": "tsgm_frame_host per frame (copies in, step, copies out, wait)"},
        "gpu_launches": launches,
        **extra,
        "wall_s_timed_region": wall_red,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true",
                    help="run only the reduced-window steps (for profiler captures)")
    ap.add_argument("--skip-forms", action="store_true",
                    help="skip the adjoint, batched and serving measurements")
    ap.add_argument("--serving-seconds", type=float, default=5.0)
    ap.add_argument("--only", choices=["adjoint", "batched", "batched_frame", "serving"],
                    help="run one of the multi-stream or adjoint measurements alone (one JSON "
                         "line with that measurement; for profiler captures)")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if ws > 1:
            init_dist(ws, "gloo")
        run_reference(args, ws, rank)
        return
    if args.warmup < 3:
        args.warmup = 3
    if ws > 1:
        init_dist(ws, "nccl")
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
