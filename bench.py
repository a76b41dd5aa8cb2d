#!/usr/bin/env python3
"""Throughput of the integral-histogram path on synthetic tracker frames.

One step is one pass of the whole path over one full-motion-video frame
(1920x1080 RGB): the feature pre-pass (R, G, B, intensity, three
gradient-orientation planes), the 91-bin integral histogram (Eq. 2.15), the
four moment planes of the intensity channel (Eq. 3.4), 100,000 rectangle
histograms (Eq. 2.16) and 4,096 spatially weighted intensity histograms
(Eq. 3.1, Epanechnikov window), followed by releasing the frame.

Prints one JSON line.  `value` is integral-histogram output cells (bins x H x
W int32 cells, whole job) per second of device time with inputs resident in
HBM; L2 is flushed (256 MiB write) between timed steps.  `e2e` is the same
metric with the frame and queries copied from pinned host memory and the
query results copied back inside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun (N > 1) every rank builds its own frame (different seed); the
ranks never exchange data (weak scaling); rank 0 prints.  `--impl reference`
times the CPU oracle on a bounded sample of the same step instead.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "integral-hist cells/s & % HBM peak; batched/served vs per-frame, same GB300"
UNIT = "cells/s"
H, W = 1080, 1920
N_RECTS = 100_000
N_WINDOWS = 4096
WEIGHTED_CH = 3  # intensity
FLUSH_BYTES = 256 << 20
WORKLOAD = ("FMV tracker frame 1920x1080 RGB -> 7 feature channels (R,G,B,I: 16 bins; "
            "3 orientation planes s=1,2,4: 9 bins) = 91-bin int32 integral histogram, "
            "intensity moment planes (4 x 16 bins int64), 100,000 rect queries, "
            "4,096 weighted windows (side 32..256)")


def rank_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def rank_seed(base: int, rank: int) -> int:
    """Each rank draws an independent frame: the work units are frames."""
    return int(base) + 7919 * int(rank)


def reduce_max(value: float) -> float:
    """Max of `value` over the ranks of the default process group (or itself)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_inputs(seed: int):
    from paper_1711_01656_gb300 import synth
    rgb = synth.blob_rgb(H, W, seed)
    rects = synth.rects_uniform_corners(H, W, N_RECTS, seed + 100)
    wins = synth.rects_side_range(H, W, N_WINDOWS, 32, 256, seed + 200)
    return rgb, rects, wins


def total_bins():
    from paper_1711_01656_gb300 import synth
    return sum(b for b, _ in synth.FMV_CHANNELS)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self, t0: float, t1: float):
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        inside = [r for t, r in self.rows if t0 <= t <= t1 + 0.15]
        used = inside if inside else [r for _, r in self.rows[-3:]]
        if not used:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = sorted(v for v in (num(r[1]) for r in used) if v is not None)
        mx = [v for v in (num(r[2]) for r in used) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in used for k in range(4)
                          if len(r) > 5 + k and r[5 + k].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


# ----------------------------------------------------------------- roofline

def algorithmic_bytes(kernel: str, B: int, Bw: int, n_rects: int, n_wins: int) -> float:
    """Bytes a kernel must move per launch at minimum (inputs read once,
    outputs written once) for this workload."""
    hw = H * W
    if kernel == "tiles/count":
        return 7 * hw + 4.0 * B * hw          # 7 channel planes in, B int32 planes out
    if kernel == "tiles/moments":
        return hw + 4 * 8.0 * Bw * hw        # intensity in, 4 x Bw int64 planes out
    if kernel == "features":
        return 3 * hw + 4 * hw
    if kernel == "query_rects":
        return n_rects * (16 + 4 * B * 4 + 4 * B)
    if kernel == "query_weighted":
        return n_wins * (16 + 4 * Bw * (4 + 4 * 8) + 4 * Bw)
    if kernel == "tile_sums/count":
        return 6 * hw
    if kernel == "tile_sums/weighted":
        return hw
    return float("nan")


def source_digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1711_01656_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_1711_01656_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def dram_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None if absent or taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("source_digest") != source_digest():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------- CPU oracle

def oracle_step_sample(rgb, rects, wins, frac: float = 1.0):
    """The CPU oracle on a bounded sample of one step, scaled to a full step:
    the feature planes, the 91-bin integral histogram (Algorithm 5) and the
    four intensity moment planes (Eq. 3.4) of the first `frac` of the frame's
    rows, times H / rows; a subset of the rectangles (enumeration) and of the
    weighted windows (direct FP64 sum, Eq. 3.1), each scaled to the full count.
    Returns (seconds for one full step, description of the sample)."""
    import oracle
    from paper_1711_01656_gb300 import synth
    chans = synth.FMV_CHANNELS
    hs = max(8, min(H, int(round(frac * H))))
    nr = max(10, min(len(rects), int(1000 * frac)))
    nw = max(10, min(len(wins), int(len(wins) * frac)))
    band = rgb[:, :hs].copy()
    t0 = time.perf_counter()
    feats = oracle.features(band)
    oracle.frame_integral_histogram(feats, chans)
    for wk in oracle.MOMENT_WEIGHTS:
        oracle.weighted_integral_histogram(feats[WEIGHTED_CH], 16, wk)
    t1 = time.perf_counter()
    full = oracle.features(rgb) if hs < H else feats
    t2 = time.perf_counter()
    oracle.frame_rect_hist(full, chans, rects[:nr])
    t3 = time.perf_counter()
    oracle.weighted_hist(full[WEIGHTED_CH], 16, wins[:nw])
    t4 = time.perf_counter()
    total = (t1 - t0) * H / hs + (t3 - t2) * len(rects) / nr + (t4 - t3) * len(wins) / nw
    desc = ("1 host thread; features + 91-bin Alg. 5 tensor + 4 intensity moment planes on %d of %d rows "
            "(x%.2f), %d of %d rects by enumeration (x%d), %d of %d weighted windows by direct sum (x%.1f)"
            % (hs, H, H / hs, nr, len(rects), len(rects) // nr, nw, len(wins), len(wins) / nw))
    return total, desc


def run_reference(args):
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    from paper_1711_01656_gb300 import synth
    import oracle
    oracle.build()
    rgb, rects, wins = make_inputs(synth.config_seed(2))
    B = total_bins()
    # size each step's sample so that warmup + steps take about two minutes
    t_probe0 = time.perf_counter()
    oracle_step_sample(rgb, rects, wins, 0.05)
    probe = time.perf_counter() - t_probe0
    frac = max(0.01, min(1.0, 0.05 * (120.0 / max(1, args.steps + args.warmup)) / max(probe, 1e-3)))
    for _ in range(args.warmup):
        oracle_step_sample(rgb, rects, wins, frac)
    times = []
    desc = ""
    for _ in range(args.steps):
        t, desc = oracle_step_sample(rgb, rects, wins, frac)
        times.append(t)
    tot = sum(times)
    value = B * H * W * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "global_batch": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- engine

def run_engine(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1711_01656_gb300 import ih, synth

    seed = rank_seed(synth.config_seed(2), rank)
    rgb, rects, wins = make_inputs(seed)
    chans = synth.FMV_CHANNELS
    B = total_bins()
    Bw = 16
    stream = torch.cuda.current_stream()

    ctx = ih.ih_create(local, flags=ih.IH_CFG_PROFILE)
    d_rgb = torch.from_numpy(rgb).to(dev)
    d_rects = torch.from_numpy(rects).to(dev)
    d_wins = torch.from_numpy(wins).to(dev)
    out_r = torch.empty((N_RECTS, B), dtype=torch.int32, device=dev)
    out_w = torch.empty((N_WINDOWS, Bw), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(pix):
        h, = ih.ih_build(ctx, ih.Frame(pix, chans, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=WEIGHTED_CH,
                                       layout=ih.IH_LAYOUT_SLAB))
        ih.ih_query_rects(ctx, h, d_rects, out_r)
        ih.ih_query_weighted(ctx, h, d_wins, out_w)
        ih.ih_release(ctx, h)

    def timed(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.fill_(i & 0xFF)
            ev[i][0].record()
            fn()
            ev[i][1].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # device-resident path
    for _ in range(args.warmup):
        step(d_rgb)
    ih.ih_sync(ctx)
    ih.ih_profile_read(ctx, reset=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    launches0 = ih.ih_launch_count(ctx)
    t_wall0 = time.time()
    dev_s = timed(lambda: step(d_rgb), args.steps)
    t_wall1 = time.time()
    barrier()
    launches = ih.ih_launch_count(ctx) - launches0
    clocks.stop()
    ih.ih_sync(ctx)
    prof = ih.ih_profile_read(ctx, reset=True)

    # end-to-end: host buffers, copies inside the timed region
    h_rgb = torch.from_numpy(rgb).pin_memory()
    h_rects = torch.from_numpy(rects).pin_memory()
    h_wins = torch.from_numpy(wins).pin_memory()
    h_out_r = torch.empty(out_r.shape, dtype=out_r.dtype).pin_memory()
    h_out_w = torch.empty(out_w.shape, dtype=out_w.dtype).pin_memory()
    x_rgb = torch.empty_like(d_rgb)

    def e2e_step():
        x_rgb.copy_(h_rgb, non_blocking=True)
        d_rects.copy_(h_rects, non_blocking=True)
        d_wins.copy_(h_wins, non_blocking=True)
        step(x_rgb)
        h_out_r.copy_(out_r, non_blocking=True)
        h_out_w.copy_(out_w, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    e2e_s = timed(e2e_step, args.steps)
    barrier()
    ih.ih_sync(ctx)
    ih.ih_profile_read(ctx, reset=True)

    dev_max = reduce_max(dev_s)
    e2e_max = reduce_max(e2e_s)
    cells_step = B * H * W
    value = cells_step * args.steps * world / dev_max
    e2e_value = cells_step * args.steps * world / e2e_max

    # roofline of the dominant kernel
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (nl, tot_ms) = dom
    per_launch_s = tot_ms / nl / 1e3
    abytes = algorithmic_bytes(name, B, Bw, N_RECTS, N_WINDOWS)
    achieved = abytes / per_launch_s / 1e9
    peak, peak_src = measured_peak()
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src, "traffic": dram_traffic(name),
            "algorithmic_bytes_per_launch": abytes, "avg_launch_ms": per_launch_s * 1e3}
    kernels = {k: {"launches": v[0], "total_ms": round(v[1], 4),
                   "share": round(v[1] / sum(x[1] for x in prof.values()), 4),
                   "gbs": round(algorithmic_bytes(k, B, Bw, N_RECTS, N_WINDOWS) / (v[1] / v[0] / 1e3) / 1e9, 1)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    line = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            t_cpu, desc = oracle_step_sample(rgb, rects, wins, 1.0)
            cpu = {"value": cells_step / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dev_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "global_batch": world, "frames_per_gpu": 1,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas: one frame per GPU, no collective",
                       "layout": "slab (bins innermost, groups of <= 8 bins)"},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(h_rgb.numel() + h_rects.numel() * 4 + h_wins.numel() * 4),
                    "d2h_bytes_per_step": int(h_out_r.numel() * 4 + h_out_w.numel() * 4)},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(t_wall0, t_wall1),
            "kernels": kernels,
        }
        print(json.dumps(line))
    ih.ih_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "engine":
        ap.error("--warmup must be >= 3")
    return run_reference(args) if args.impl == "reference" else run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
