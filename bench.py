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
end-to-end number through tsgm_frame_host with host buffers, and SM clocks sampled during the
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
            "full range, frames 2-10 +-3 sigma windows")
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
    prm = oracle.Params(1242, 375, d_max=127, census_w=9, census_h=7, n_paths=8)
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

def algorithmic_sgm_bytes(cells: int, px: int) -> int:
    """Bytes the aggregation kernel must move once: the ragged cost C read (1 B/cell), the
    aggregated S written (2 B/cell), window bounds and offsets read (8 B/px)."""
    return 3 * cells + 8 * px


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


def run_ours_on_stream(args, ws, rank, local, dev, stream):
    import torch
    from paper_1708_06301_gb300 import synth, tsgm

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

    ctx = make(0)
    ctx_full = make(tsgm.FLAG_FULL_RANGE)
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
    t_red, wall_red, launches, stages = timed(ctx, args.steps, args.warmup, profile=True)
    clocks = sampler.stop()
    t_full, _, _, stages_full = timed(ctx_full, max(1, args.steps // 2), max(3, args.warmup // 2),
                                      profile=True)
    k_full = max(1, args.steps // 2)

    # end to end through the host-buffer entry point (pinned host memory)
    hl = [torch.from_numpy(x).pin_memory() for x in seq.left]
    hr = [torch.from_numpy(x).pin_memory() for x in seq.right]
    hD = torch.empty((H, W), dtype=torch.float32).pin_memory()
    hP = torch.empty_like(hD).pin_memory()

    def step_host():
        ctx.reset()
        for k in range(N_FRAMES):
            ctx.frame_host(hl[k], hr[k], seq.R[k], seq.t[k], K, b, hD, hP)

    for _ in range(args.warmup):
        step_host()
    torch.cuda.synchronize()
    e2e_ms = []
    for s in range(args.steps):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_host()
        e2e_ms.append(1000 * (time.perf_counter() - t0))

    tmax = reduce_max([t_red, t_full, sum(e2e_ms)], ws, device=dev)
    t_red_max, t_full_max, e2e_max = tmax
    if rank != 0:
        return

    frames = N_FRAMES * args.steps * ws
    fps = frames / (t_red_max / 1000.0)
    fps_full = N_FRAMES * k_full * ws / (t_full_max / 1000.0)
    # SGM stages a5-a9 (census, cost, aggregation, selection + LR) per frame
    sgm_stages = ("census", "cost", "sgm", "select")
    ms_sgm_red = sum(stages[s][0] for s in sgm_stages) / args.steps
    ms_sgm_full = sum(stages_full[s][0] for s in sgm_stages) / k_full
    gcells_red = sum(cells_red) / (ms_sgm_red / 1000.0) / 1e9
    gcells_full = sum(cells_full) / (ms_sgm_full / 1000.0) / 1e9

    # roofline of the dominant kernel (SGM aggregation), average launch over the timed region
    agg_ms, agg_cnt = stages["sgm"]
    agg_avg_s = agg_ms / agg_cnt / 1000.0
    bytes_per_launch = algorithmic_sgm_bytes(int(np.mean(cells_red)), n)
    achieved = bytes_per_launch / agg_avg_s / 1e9
    peak, peak_kind = peaks()

    cpu_s = sum(oracle_frames(seq, list(range(N_FRAMES))))
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
        "search_space_frac": [c / (n * 128) for c in cells_red],
        "bad3px": {"reduced_updated": bad_red, "full_range_updated": bad_full},
        "stage_ms_per_step": {k: v[0] / args.steps for k, v in stages.items() if v[1]},
        "roofline": {"bound": "hbm", "kernel": "k_sgm (path aggregation)", "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": bytes_per_launch,
                     "avg_launch_us": agg_avg_s * 1e6},
        "cpu_baseline": {"value": N_FRAMES / cpu_s, "unit": "frames/s", "cores": 1,
                         "kind": "oracle",
                         "sample": "one step: the 10-frame sequence (1 full-range, 9 reduced), "
                                   "single thread"},
        "e2e": {"value": frames / (e2e_max / 1000.0), "unit": "frames/s",
                "h2d_bytes_per_step": N_FRAMES * 2 * n,
                "d2h_bytes_per_step": N_FRAMES * 2 * 4 * n},
        "gpu_launches": launches,
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
