#!/usr/bin/env python3
"""Throughput of the integral-histogram path on synthetic tracker frames.

One step is one pass of the whole path over one frame: ih_build (the
integral histogram of every channel, Eq. 2.15, and the four moment planes
of the weighted channel, Eq. 3.4), one ih_query call (rectangle histograms,
Eq. 2.16, and spatially weighted histograms with the Epanechnikov window,
Eq. 3.1) and ih_release.

The headline workload is the wide-area frame: 8192 x 8192 gray, 32 bins,
int64 moment planes (77 GB written per step), 1,000,000 rectangles of side
16..256 and 100,000 windows of side 32..256.  The `fmv` section measures the
full-motion-video step the same way: one 1920 x 1080 RGB frame through the
feature pre-pass (R, G, B, intensity, three orientation planes: 91 bins),
intensity moment planes, 100,000 rectangles and 4,096 windows.

Prints one JSON line.  `value` is integral-histogram output cells (bins x H x
W int32 cells, whole job) per second of device time with inputs resident in
HBM; L2 is flushed (256 MiB write) between timed steps.  `e2e` is the same
metric with the frame and queries copied from pinned host memory and the
query results copied back inside the timed region.  `cpu_baseline` is the
oracle on all host cores (and on one thread) over a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl engine|reference]

Under torchrun (N > 1) every rank builds its own frame (different seed); the
ranks never exchange data (weak scaling); rank 0 prints.  `--impl reference`
times the CPU oracle on bounded samples of the headline step instead.
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
# --layout: (ih_layout value, description for the JSON line)
LAYOUTS = {
    "record": (2, "record (bins innermost; per-pixel records of up to 16 words in planes)"),
    "slab": (1, "slab (bins innermost, groups of <= 8 bins of one channel)"),
    "bin-major": (0, "bin-major (b x h x pitch, Fig. 5.1)"),
}
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


WAMI_H = WAMI_W = 8192
WAMI_BINS = 32
WAMI_RECTS = 1_000_000
WAMI_WINDOWS = 100_000


def make_wami_inputs(seed: int, side: int = WAMI_H):
    """The wide-area frame: one 8192 x 8192 blob plane, 1,000,000 rectangles
    of side 16..256 inside it and 100,000 windows of side 32..256 (a smaller
    square side, for profiling captures, scales the query counts with the
    area)."""
    from paper_1711_01656_gb300 import synth
    frac = side * side / float(WAMI_H * WAMI_W)
    img = synth.blob_plane(side, side, seed)
    rects = synth.rects_side_range(side, side, max(1, int(WAMI_RECTS * frac)), 16, min(256, side), seed + 100)
    wins = synth.rects_side_range(side, side, max(1, int(WAMI_WINDOWS * frac)), 32, min(256, side), seed + 200)
    return img, rects, wins


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


# ----------------------------------------------------------------- workloads

class Spec:
    """One workload of the path: a frame, its channels and its queries.

    A step is ih_build (counts and the weighted channel's moment planes),
    one ih_query call (every rectangle and every weighted window) and
    ih_release, on one frame."""

    def __init__(self, kind: str, seed: int, layout: int, side: int = 0):
        from paper_1711_01656_gb300 import synth
        self.kind, self.seed, self.layout = kind, seed, layout
        if kind == "fmv":
            self.frame, self.rects, self.wins = make_inputs(seed)
            self.chans = list(synth.FMV_CHANNELS)
            self.rgb_input, self.wch = True, WEIGHTED_CH
            self.H, self.W = H, W
            self.planes = 7          # channel planes the tile kernels read
            self.workload = WORKLOAD
        elif kind == "wami":
            side = side or WAMI_H
            img, self.rects, self.wins = make_wami_inputs(seed, side)
            self.frame = img[None]
            self.chans = [(WAMI_BINS, 0)]
            self.rgb_input, self.wch = False, 0
            self.H = self.W = side
            self.planes = 1
            self.workload = WAMI_WORKLOAD if side == WAMI_H else (
                "profiling case of the WAMI step: %dx%d gray, 32 bins, int64 moments, %d rects, %d windows"
                % (side, side, len(self.rects), len(self.wins)))
        else:
            raise ValueError(kind)
        self.B = sum(b for b, _ in self.chans)
        self.Bw = self.chans[self.wch][0]
        self.cells = self.B * self.H * self.W   # count cells per step (the metric's unit)

    def ih_frame(self, ih, pixels):
        return ih.Frame(pixels, self.chans, input=ih.IH_INPUT_RGB_FEATURES if self.rgb_input else ih.IH_INPUT_PLANES,
                        weighted_channel=self.wch, layout=self.layout)


WAMI_WORKLOAD = ("WAMI frame 8192x8192 gray (50 blobs + N(0,8)) -> 32-bin int32 integral histogram "
                 "(2.15 G cells) with the 4 int64 moment planes (Eq. 3.4, 68.7 GB), 1,000,000 rect queries "
                 "(side 16..256), 100,000 Epanechnikov weighted windows (side 32..256)")


# ----------------------------------------------------------------- roofline

def algorithmic_bytes(kernel: str, B: int, Bw: int, n_rects: int, n_wins: int, hw: int = H * W,
                      planes: int = 7) -> float:
    """Bytes a kernel must move per launch at minimum (inputs read once,
    outputs written once): `planes` uint8 channel planes of hw pixels, B
    int32 count planes, Bw x 4 int64 moment planes, the queries."""
    if kernel == "tiles/count":
        return planes * hw + 4.0 * B * hw      # channel planes in, B int32 planes out
    if kernel == "tiles/moments":
        return hw + 4 * 8.0 * Bw * hw        # weighted channel in, 4 x Bw int64 planes out
    if kernel == "tiles/count+moments":      # both kinds of tiles in one launch
        return (algorithmic_bytes("tiles/count", B, Bw, n_rects, n_wins, hw, planes) +
                algorithmic_bytes("tiles/moments", B, Bw, n_rects, n_wins, hw, planes))
    if kernel == "features":
        return 3 * hw + 4 * hw
    if kernel == "query_rects":
        return n_rects * (16 + 4 * B * 4 + 4 * B)
    if kernel == "query_weighted":
        return n_wins * (16 + 4 * Bw * (4 + 4 * 8) + 4 * Bw)
    if kernel == "queries":                  # both query kinds in one launch
        return (algorithmic_bytes("query_rects", B, Bw, n_rects, n_wins, hw, planes) +
                algorithmic_bytes("query_weighted", B, Bw, n_rects, n_wins, hw, planes))
    if kernel == "tile_sums":                # all windows of the frame in one launch
        return planes * hw
    return float("nan")


def spec_bytes(spec, kernel: str) -> float:
    return algorithmic_bytes(kernel, spec.B, spec.Bw, len(spec.rects), len(spec.wins), spec.H * spec.W, spec.planes)


def source_digest() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1711_01656_gb300", "csrc"))):
        h.update(open(os.path.join(ROOT, "paper_1711_01656_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def dram_traffic(kernel: str, workload: str = "fmv"):
    """Per-launch DRAM bytes of `kernel` on `workload` from the committed ncu
    summary, or None if absent or taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(p))
    except (OSError, ValueError):
        return None
    if d.get("source_digest") != source_digest():
        return None
    k = d.get("workloads", {}).get(workload, {}).get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ----------------------------------------------------------------- CPU oracle

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(spec, rows: int, threads: int):
    """The CPU oracle on a bounded sample of one step: the first `rows` rows
    of the frame (the feature pre-pass for an RGB frame, the count tensor by
    Algorithm 5 and the weighted channel's four moment planes by Eq. 3.4) and
    the same fraction rows/H of the queries (rectangles by enumeration,
    windows by the FP64 direct sum of Eq. 3.1), on `threads` host threads:
    the tensors split over bins, the queries over chunks (the oracle's C calls
    release the GIL).  The sample is the step scaled by rows/H.
    Returns (seconds, count cells of the sample, description)."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    rows = max(1, min(spec.H, int(rows)))
    frac = rows / spec.H
    nr = max(1, int(round(len(spec.rects) * frac)))
    nw = max(1, int(round(len(spec.wins) * frac)))
    band = np.ascontiguousarray(spec.frame[:, :rows])
    rects, wins = spec.rects[:nr], spec.wins[:nw]
    ex = cf.ThreadPoolExecutor(max_workers=threads) if threads > 1 else None

    def split(fn, q):
        if ex is None:
            return fn(q)
        return np.concatenate(list(ex.map(fn, np.array_split(q, threads))), axis=0)

    t0 = time.perf_counter()
    planes = oracle.features(band) if spec.rgb_input else band
    oracle.frame_integral_histogram(planes, spec.chans, threads=threads)
    for wk in oracle.MOMENT_WEIGHTS:
        oracle.weighted_integral_histogram(planes[spec.wch], spec.Bw, wk, threads=threads)
    full = spec.frame if not spec.rgb_input else None
    t1 = time.perf_counter()
    if spec.rgb_input:  # the queries read the whole frame's feature planes (made outside the timing)
        full = oracle.features(spec.frame)
    t2 = time.perf_counter()
    split(lambda q: oracle.frame_rect_hist(full, spec.chans, q), rects)
    split(lambda q: oracle.weighted_hist(full[spec.wch], spec.Bw, q), wins)
    t3 = time.perf_counter()
    if ex is not None:
        ex.shutdown()
    secs = (t1 - t0) + (t3 - t2)
    desc = ("%d host thread%s; %d of %d rows (%s%d-bin Alg. 5 tensor + 4 moment planes of %d bins), "
            "%d of %d rects by enumeration, %d of %d weighted windows by direct FP64 sum; "
            "the step scaled by %.5f"
            % (threads, "s" if threads > 1 else "", rows, spec.H, "features + " if spec.rgb_input else "",
               spec.B, spec.Bw, nr, len(spec.rects), nw, len(spec.wins), frac))
    return secs, spec.B * rows * spec.W, desc


def size_sample(spec, threads: int, target_s: float) -> int:
    """Rows of a sample that takes about target_s seconds on `threads`."""
    probe = max(4, spec.H // 512)
    t, _, _ = oracle_sample(spec, probe, threads)
    return max(probe, min(spec.H, int(probe * target_s / max(t, 1e-4))))


def cpu_baseline(spec, target_s: float = 10.0):
    """The oracle on all host cores and on one thread, each on a sample of
    about target_s seconds of the step (rate in count cells/s)."""
    cores = host_cores()
    rows = size_sample(spec, cores, target_s)
    t, cells, desc = oracle_sample(spec, rows, cores)
    rows1 = size_sample(spec, 1, target_s)
    t1, cells1, desc1 = oracle_sample(spec, rows1, 1)
    return {"value": cells / t, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "sample_s": round(t, 3),
            "single_thread": {"value": cells1 / t1, "unit": UNIT, "cores": 1, "sample": desc1,
                              "sample_s": round(t1, 3)}}


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the
    headline step (sized so that warm-up + steps take about two minutes),
    timed as it ran; `value` is its rate in count cells/s."""
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1711_01656_gb300 import synth
    oracle.build()
    spec = Spec("wami", synth.config_seed(3), LAYOUTS[args.layout][0])
    cores = host_cores()
    per_step = min(5.0, 120.0 / max(1, args.steps + args.warmup))
    rows = size_sample(spec, cores, per_step)
    for _ in range(args.warmup):
        oracle_sample(spec, rows, cores)
    tot, cells, desc = 0.0, 0, ""
    for _ in range(args.steps):
        t, c, desc = oracle_sample(spec, rows, cores)
        tot += t
        cells += c
    value = cells / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "ms_per_step_is": "the sampled step as timed (rows %d of %d); a full step would take about %.1f s"
                              % (rows, spec.H, tot / args.steps * spec.H / rows),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": {"workload": spec.workload, "global_batch": 1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- engine

def measure_step(ih, dev, spec, steps: int, warmup: int, world: int, flush, barrier, sample_clocks=True):
    """Times `steps` steps of `spec` on this GPU after `warmup` untimed ones.

    Device-resident leg: inputs in HBM, L2 flushed before each step, CUDA
    events around each step on the launching stream.  The warm-up steps time
    every kernel (the kernel table); the timed steps carry event pairs only
    around the dominant kernel, whose live average launch time gives the
    roofline.  End-to-end leg: the frame and the queries are copied from
    pinned host memory and the query results copied back inside the timed
    region, double-buffered over two streams (Algorithm 10): step k runs on
    stream k % 2, so one step's copies overlap the other's kernels."""
    import torch
    ctx = ih.ih_create(dev.index or 0, flags=ih.IH_CFG_PROFILE)
    try:
        d_in = torch.from_numpy(spec.frame).to(dev)
        d_rects = torch.from_numpy(spec.rects).to(dev)
        d_wins = torch.from_numpy(spec.wins).to(dev)
        out_r = torch.empty((len(spec.rects), spec.B), dtype=torch.int32, device=dev)
        out_w = torch.empty((len(spec.wins), spec.Bw), dtype=torch.float32, device=dev)

        def step(pix, rects, wins, o_r, o_w, stream=None):
            h, = ih.ih_build(ctx, spec.ih_frame(ih, pix), stream=stream)
            ih.ih_query(ctx, h, rects, o_r, wins, o_w, stream=stream)
            ih.ih_release(ctx, h, stream=stream)

        for _ in range(warmup):
            flush.fill_(1)
            step(d_in, d_rects, d_wins, out_r, out_w)
        ih.ih_sync(ctx)
        prof_all = ih.ih_profile_read(ctx, reset=True)
        dominant = max(prof_all.items(), key=lambda kv: kv[1][1])[0]
        ih.ih_profile_select(ctx, [dominant])
        clocks = ClockSampler(dev.index or 0) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        barrier()
        launches0 = ih.ih_launch_count(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t_wall0 = time.time()
        for i in range(steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record()
            step(d_in, d_rects, d_wins, out_r, out_w)
            ev[i][1].record()
        torch.cuda.synchronize()
        t_wall1 = time.time()
        dev_s = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        barrier()
        launches = ih.ih_launch_count(ctx) - launches0
        if clocks:
            clocks.stop()
        ih.ih_sync(ctx)
        prof = ih.ih_profile_read(ctx, reset=True)
        ih.ih_profile_select(ctx, [])
        # the build alone (ih_build, events around it; release outside), L2 flushed
        nb_ = max(3, min(steps, 20))
        evb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nb_)]
        for k in range(nb_):
            flush.fill_(k & 0xFF)
            evb[k][0].record()
            h, = ih.ih_build(ctx, spec.ih_frame(ih, d_in))
            evb[k][1].record()
            ih.ih_release(ctx, h)
        torch.cuda.synchronize()
        build_ms = sorted(a.elapsed_time(b) for a, b in evb)[nb_ // 2]
        del d_in

        h_in = torch.from_numpy(spec.frame).pin_memory()
        h_rects = torch.from_numpy(spec.rects).pin_memory()
        h_wins = torch.from_numpy(spec.wins).pin_memory()
        bufs = []
        for _ in range(2):
            bufs.append(dict(
                stream=torch.cuda.Stream(device=dev), x=torch.empty(h_in.shape, dtype=h_in.dtype, device=dev),
                rects=torch.empty_like(d_rects), wins=torch.empty_like(d_wins), out_r=torch.empty_like(out_r),
                out_w=torch.empty_like(out_w),
                h_out_r=torch.empty(out_r.shape, dtype=out_r.dtype).pin_memory(),
                h_out_w=torch.empty(out_w.shape, dtype=out_w.dtype).pin_memory()))

        def e2e_run(k_steps):
            main = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            for b in bufs:
                b["stream"].wait_stream(main)
            for k in range(k_steps):
                b = bufs[k % 2]
                st = b["stream"]
                with torch.cuda.stream(st):
                    b["x"].copy_(h_in, non_blocking=True)
                    b["rects"].copy_(h_rects, non_blocking=True)
                    b["wins"].copy_(h_wins, non_blocking=True)
                    step(b["x"], b["rects"], b["wins"], b["out_r"], b["out_w"], stream=st)
                    b["h_out_r"].copy_(b["out_r"], non_blocking=True)
                    b["h_out_w"].copy_(b["out_w"], non_blocking=True)
            for b in bufs:
                main.wait_stream(b["stream"])
            e1.record(main)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3

        e2e_run(max(2, warmup))
        barrier()
        e2e_s = e2e_run(steps)
        barrier()
        ih.ih_sync(ctx)
        ih.ih_profile_read(ctx, reset=True)
        h2d = int(h_in.numel() + h_rects.numel() * 4 + h_wins.numel() * 4)
        d2h = int(bufs[0]["h_out_r"].numel() * 4 + bufs[0]["h_out_w"].numel() * 4)
        del bufs
    finally:
        ih.ih_destroy(ctx)
        torch.cuda.empty_cache()

    dev_max, e2e_max = reduce_max(dev_s), reduce_max(e2e_s)
    nl, tot_ms = prof[dominant]
    per_launch_s = tot_ms / nl / 1e3
    abytes = spec_bytes(spec, dominant)
    achieved = abytes / per_launch_s / 1e9
    peak, peak_src = measured_peak()
    roof = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src, "traffic": dram_traffic(dominant, spec.kind),
            "algorithmic_bytes_per_launch": abytes, "avg_launch_ms": per_launch_s * 1e3}
    total_ms = sum(x[1] for x in prof_all.values())
    kernels = {k: {"launches": v[0], "total_ms": round(v[1], 4), "share": round(v[1] / total_ms, 4),
                   "gbs": round(spec_bytes(spec, k) / (v[1] / v[0] / 1e3) / 1e9, 1)}
               for k, v in sorted(prof_all.items(), key=lambda kv: -kv[1][1])}
    build_bytes = spec_bytes(spec, "tiles/count+moments") + (3 * spec.H * spec.W if spec.rgb_input else 0)
    return {"value": spec.cells * steps * world / dev_max, "ms_per_step": 1e3 * dev_max / steps,
            "build": {"ms_median": round(build_ms, 4), "algorithmic_bytes": build_bytes,
                      "GBs": round(build_bytes / (build_ms / 1e3) / 1e9, 1),
                      "frac_of_peak": round(build_bytes / (build_ms / 1e3) / 1e9 / measured_peak()[0], 4),
                      "what": "ih_build alone (every build kernel of the frame), CUDA events, L2 flushed"},
            "e2e": {"value": spec.cells * steps * world / e2e_max, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": round(1e3 * e2e_max / steps, 4)},
            "roofline": roof, "kernels": kernels, "gpu_launches": int(launches),
            "clocks": clocks.summary(t_wall0, t_wall1) if clocks else None}


def run_engine(args):
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

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    layout = LAYOUTS[args.layout][0]
    # the headline: the wide-area frame, each rank its own frame
    if args.workload == "fmv":  # the FMV step as the line's workload (profiling captures)
        head = Spec("fmv", rank_seed(synth.config_seed(2), rank), layout)
    else:
        head = Spec("wami", rank_seed(synth.config_seed(3), rank), layout, args.wami_side)
    m = measure_step(ih, dev, head, args.steps, args.warmup, world, flush, barrier)
    # the full-motion-video step, the same measurement
    fmv_spec = fmv = None
    if not args.no_fmv:
        fmv_spec = Spec("fmv", rank_seed(synth.config_seed(2), rank), layout)
        fmv = measure_step(ih, dev, fmv_spec, args.fmv_steps, args.warmup, world, flush, barrier,
                           sample_clocks=False)
        fmv = {"workload": fmv_spec.workload, "value": fmv["value"], "unit": UNIT,
               "ms_per_step": fmv["ms_per_step"], "steps": args.fmv_steps, "e2e": fmv["e2e"], "build": fmv["build"],
               "roofline": fmv["roofline"], "kernels": fmv["kernels"], "gpu_launches": fmv["gpu_launches"]}
    del flush
    torch.cuda.empty_cache()

    batched = served = wami = plain = match = median = phog = mma = None
    sections = world == 1  # the side workloads run once, on a single GPU
    if sections and not args.no_wami:
        wami = wami_section(ih, dev, layout)
    if sections and not args.no_plain:
        plain = plain_section(ih, dev)
    if sections and not args.no_mma:
        mma = mma_section(ih, dev, side=args.mma_side)
    if sections and not args.no_match:
        match = match_section(ih, dev, layout)
    if sections and not args.no_median:
        median = median_section(ih, dev, layout)
    if sections and not args.no_phog:
        phog = phog_section(ih, dev)
    if sections and not args.no_batched:
        # the batch and the serving loop have no rectangle-heavy queries: the
        # slab layout (no padding, one channel per group) suits them better
        batched = batched_section(ih, dev, LAYOUTS["slab"][0])
    if sections and not args.no_served:
        served = served_section(ih, dev, LAYOUTS["slab"][0])

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(head)
            if fmv is not None:
                fmv["cpu_baseline"] = cpu_baseline(fmv_spec, 5.0)
        line = {
            "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": head.workload, "global_batch": world, "frames_per_gpu": 1,
                       "l2": "flushed between timed steps (256 MiB write); e2e: host inputs, 77 GB written per step",
                       "e2e_pipeline": "dual buffering over two streams (Algorithm 10)",
                       "parallelism": "replicas: one frame per GPU, no collective",
                       "layout": LAYOUTS[args.layout][1]},
            "roofline": m["roofline"], "cpu_baseline": cpu, "e2e": m["e2e"], "build": m["build"],
            "gpu_launches": m["gpu_launches"], "clocks": m["clocks"], "kernels": m["kernels"],
            "kernels_timed_in": "the warm-up steps (the timed steps carry events around the dominant kernel only)",
            "fmv": fmv, "wami_phases": wami, "plain": plain, "batched": batched, "served": served,
            "match": match, "median": median, "phog": phog, "mma_tiles": mma,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ----------------------------------------------------------------- batched / served

def wami_section(ih, dev, layout, reps=3):
    """One 8192 x 8192 wide-area frame: 32-bin integral histogram (2.15 G int32
    cells) with the four int64 moment planes of its single channel (68.7 GB),
    1,000,000 rectangle queries of side 16..256 and 100,000 Epanechnikov
    windows of side 32..256.  Each phase is timed with events after one
    warm-up, L2 flushed before each repetition."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    hh = ww = 8192
    B = 32
    p = (ww + 3) // 4 * 4
    need = hh * p * (B * 4 + 4 * B * 8) + 64e6 * 4 + 2e9
    free, _ = torch.cuda.mem_get_info(dev)
    if need > free * 0.9:
        return {"skipped": "needs %.1f GB of HBM, %.1f GB free" % (need / 1e9, free / 1e9)}
    img = synth.blob_plane(hh, ww, synth.config_seed(3))
    pix = torch.from_numpy(img).to(dev)[None]
    rects = torch.from_numpy(synth.rects_side_range(hh, ww, 1_000_000, 16, 256, synth.config_seed(3) + 100)).to(dev)
    wins = torch.from_numpy(synth.rects_side_range(hh, ww, 100_000, 32, 256, synth.config_seed(3) + 200)).to(dev)
    r_out = torch.empty((rects.shape[0], B), dtype=torch.int32, device=dev)
    w_out = torch.empty((wins.shape[0], B), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ctx = ih.ih_create(dev.index or 0, flags=ih.IH_CFG_PROFILE)
    frame = ih.Frame(pix, [(B, 0)], weighted_channel=0, layout=layout)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t = {"build": [], "rects": [], "weighted": [], "manhattan": [], "wedding_cake": []}
    ev += [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for rep in range(reps + 1):
        flush.fill_(rep & 0xFF)
        ev[0].record()
        h, = ih.ih_build(ctx, frame)
        ev[1].record()
        ih.ih_query_rects(ctx, h, rects, r_out)
        ev[2].record()
        ih.ih_query_weighted(ctx, h, wins, w_out)
        ev[3].record()
        ih.ih_query_weighted(ctx, h, wins, w_out, kernel=ih.IH_K_MANHATTAN)
        ev[4].record()
        ih.ih_query_weighted(ctx, h, wins, w_out, kernel=ih.IH_K_WEDDING_CAKE, flags=ih.IH_LAYERS(4))
        ev[5].record()
        torch.cuda.synchronize()
        ih.ih_release(ctx, h)
        if rep == 0:
            ih.ih_profile_read(ctx, reset=True)
            continue
        t["build"].append(ev[0].elapsed_time(ev[1]))
        t["rects"].append(ev[1].elapsed_time(ev[2]))
        t["weighted"].append(ev[2].elapsed_time(ev[3]))
        t["manhattan"].append(ev[3].elapsed_time(ev[4]))
        t["wedding_cake"].append(ev[4].elapsed_time(ev[5]))
    torch.cuda.synchronize()
    prof = ih.ih_profile_read(ctx, reset=True)
    ih.ih_destroy(ctx)
    del pix, r_out, w_out, flush
    torch.cuda.empty_cache()
    ms = {k: float(np.median(v)) for k, v in t.items()}
    cells = B * hh * ww
    count_bytes = hh * ww + 4.0 * cells
    moment_bytes = hh * ww + 4 * 8.0 * B * hh * ww
    peak = measured_peak()[0]
    kern = {}
    for name, (n, tot) in prof.items():
        kern[name] = round(tot / n, 3)
    tiles_ms = kern.get("tiles/count+moments")
    out = {"workload": "WAMI 8192x8192 blobs+noise, 32 bins, int64 moment planes, 1,000,000 rects (side 16..256), "
                       "100,000 weighted windows (side 32..256) with the Epanechnikov kernel, the Manhattan "
                       "kernel (Eq. 3.3) and the 4-layer wedding cake (Eq. 3.2)",
           "layout": [k for k, v in LAYOUTS.items() if v[0] == layout][0],
           "build_ms": round(ms["build"], 3), "rect_queries_ms": round(ms["rects"], 3),
           "weighted_queries_ms": round(ms["weighted"], 3),
           "build_cells_per_s": cells / (ms["build"] / 1e3),
           "build_GBs": round((count_bytes + moment_bytes) / (ms["build"] / 1e3) / 1e9, 1),
           "manhattan_queries_ms": round(ms["manhattan"], 3), "wedding_cake_queries_ms": round(ms["wedding_cake"], 3),
           "rects_per_s": 1e6 / (ms["rects"] / 1e3), "windows_per_s": 1e5 / (ms["weighted"] / 1e3),
           "manhattan_windows_per_s": 1e5 / (ms["manhattan"] / 1e3),
           "wedding_cake_windows_per_s": 1e5 / (ms["wedding_cake"] / 1e3),
           "kernel_ms": kern}
    if tiles_ms:
        gbs = (count_bytes + moment_bytes) / (tiles_ms / 1e3) / 1e9
        out["tiles_roofline"] = {"bound": "hbm", "kernel": "tiles/count+moments", "achieved": round(gbs, 1),
                                 "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4)}
    return out


def mma_section(ih, dev, reps=3, side=8192):
    """The count tiles as tensor-core products (ih_build_mma: two chained
    tcgen05 bf16 products per 128 x 128 tile and bin) against the scan-based
    tiles kernel on the same frame: 8192 x 8192 gray, 32 bins, bin-major
    counts, once on the scan path's own tile grid and once on the MMA's
    128 x 128 grid.  Kernel times are CUDA-event averages over `reps` builds
    after one warm-up; the tensors must be equal."""
    import torch
    from paper_1711_01656_gb300 import synth
    hh = ww = side
    B = 32
    free, _ = torch.cuda.mem_get_info(dev)
    if 3 * hh * ww * B * 4 > free * 0.8:
        return {"skipped": "needs %.1f GB of HBM" % (3 * hh * ww * B * 4 / 1e9)}
    img = torch.from_numpy(synth.blob_plane(hh, ww, synth.config_seed(3))).to(dev)[None]
    frame = ih.Frame(img, [(B, 0)], layout=ih.IH_LAYOUT_BIN_MAJOR)
    out = {}
    tensors = []
    for name in ("scan", "scan_128x128", "mma"):
        ctx = ih.ih_create(dev.index or 0, flags=ih.IH_CFG_PROFILE)
        if name == "scan_128x128":
            ih.ih_tune_set(ctx, frame, 128, 128)
        build = (lambda: ih.ih_build_mma(ctx, frame)) if name == "mma" else (lambda: ih.ih_build(ctx, frame)[0])
        for rep in range(reps + 1):
            h = build()
            if rep == reps:
                t = torch.empty((B, hh, ww), dtype=torch.int32, device=dev)
                ih.ih_export(ctx, h, t)
                tensors.append(t)
            ih.ih_release(ctx, h)
            ih.ih_sync(ctx)
            if rep == 0:
                ih.ih_profile_read(ctx, reset=True)
        prof = ih.ih_profile_read(ctx, reset=True)
        ih.ih_destroy(ctx)
        out[name] = {k: round(v[1] / v[0], 4) for k, v in prof.items() if k != "export"}
    equal = all(torch.equal(tensors[0], t) for t in tensors[1:])
    del tensors
    torch.cuda.empty_cache()
    peak, _ = measured_peak()
    abytes = hh * ww + 4.0 * B * hh * ww
    res = {"workload": "%dx%d gray, 32 bins, bin-major int32 counts (no moment planes)" % (hh, ww),
           "kernel_ms": out, "tensors_equal": bool(equal)}
    t_scan, t_scan128, t_mma = (out["scan"].get("tiles/count"), out["scan_128x128"].get("tiles/count"),
                                out["mma"].get("tiles/mma"))
    if t_scan and t_mma:
        flops = 2 * 2 * 128.0 ** 3 * B * (hh // 128) * (ww // 128)
        res.update({"scan_tiles_GBs": round(abytes / (t_scan / 1e3) / 1e9, 1),
                    "scan_128x128_tiles_GBs": round(abytes / (t_scan128 / 1e3) / 1e9, 1) if t_scan128 else None,
                    "mma_tiles_GBs": round(abytes / (t_mma / 1e3) / 1e9, 1),
                    "mma_tiles_tensor_TFLOPs": round(flops / (t_mma / 1e3) / 1e12, 1),
                    "mma_vs_scan_time": round(t_mma / t_scan, 3), "hbm_peak_GBs": peak})
    return res


def match_section(ih, dev, layout, runs=20):
    """Sliding-window histogram matching (Sec. 2.4.3, Eq. 2.22 with p = 1) on
    the FMV frame: a 64 x 64 target window's 91-bin histogram against every
    placement in a 256 x 256 search region (65,536 placements), and the same
    over the whole frame (1017 x 1857 placements) on the intensity bins."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    rgb = torch.from_numpy(synth.blob_rgb(H, W, synth.config_seed(2))).to(dev)
    ctx = ih.ih_create(dev.index or 0)
    h, = ih.ih_build(ctx, ih.Frame(rgb, synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES, layout=layout))
    B = total_bins()
    wh = ww = 64
    target = torch.empty((1, B), dtype=torch.int32, device=dev)
    ih.ih_query_rects(ctx, h, torch.tensor([[500, 900, 500 + wh - 1, 900 + ww - 1]], dtype=torch.int32,
                                           device=dev), target)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(runs):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / runs

    local = (372, 772, 372 + 255, 772 + 255)
    out_l = torch.empty((256, 256), dtype=torch.int32, device=dev)
    ms_l = timed(lambda: ih.ih_match_window(ctx, h, 0, B, target.view(-1), wh, ww, local, out_l))
    full = (0, 0, H - wh, W - ww)
    out_f = torch.empty((H - wh + 1, W - ww + 1), dtype=torch.int32, device=dev)
    t_int = target.view(-1)[48:64].contiguous()  # intensity: channel 3, bins 48..63
    ms_f = timed(lambda: ih.ih_match_window(ctx, h, 48, 16, t_int, wh, ww, full, out_f))
    best = int(out_l.view(-1).argmin().item())
    ih.ih_release(ctx, h)
    ih.ih_destroy(ctx)
    n_l, n_f = 256 * 256, (H - wh + 1) * (W - ww + 1)
    return {"workload": "FMV frame, 64x64 window: 91-bin match over 256x256 placements; 16-bin intensity match "
                        "over all %d placements" % n_f,
            "local_ms": round(ms_l, 4), "local_placements_per_s": n_l / (ms_l / 1e3),
            "local_bin_windows_per_s": n_l * B / (ms_l / 1e3),
            "full_frame_ms": round(ms_f, 4), "full_frame_placements_per_s": n_f / (ms_f / 1e3),
            "best_placement_found": [local[0] + best // 256, local[1] + best % 256], "target_at": [500, 900]}


def median_section(ih, dev, layout, n_frames=24, window=9, box=5):
    """Algorithm 4 on a 1920 x 1080 grayscale video (16 bins): per frame, the
    head frame's integral histogram, the joint-histogram update (head in,
    tail out) and the 5 x 5 x 9 spatio-temporal median of the centre frame;
    frames are built once the window is full, as in the algorithm's loop."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    B = 16
    base = [synth.blob_plane(H, W, synth.config_seed(6) + k) for k in range(4)]
    pix = [torch.from_numpy(np.roll(base[k % 4], 13 * k, axis=1)).to(dev)[None] for k in range(n_frames)]
    ctx = ih.ih_create(dev.index or 0)
    frame = lambda k: ih.Frame(pix[k], [(B, 0)], layout=layout)
    hs = [ih.ih_build(ctx, frame(k))[0] for k in range(window)]
    jih, = ih.ih_build(ctx, frame(0))
    for k in range(1, window):
        ih.ih_accumulate(ctx, jih, add=hs[k])
    out = torch.empty((H, W), dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record()
    steps = 0
    for k in range(window, n_frames):
        head, = ih.ih_build(ctx, frame(k))
        ih.ih_accumulate(ctx, jih, add=head, sub=hs[0])
        ih.ih_release(ctx, hs.pop(0))
        hs.append(head)
        ih.ih_local_median(ctx, jih, 0, B, box, box, out)
        steps += 1
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / steps
    for hd in hs + [jih]:
        ih.ih_release(ctx, hd)
    ih.ih_destroy(ctx)
    return {"workload": "1920x1080 gray video, 16 bins, median over 5x5 pixels x 9 frames (Algorithm 4)",
            "ms_per_frame": round(ms, 4), "frames_per_s": round(1e3 / ms, 1), "frames_timed": steps}


def phog_section(ih, dev, runs=10):
    """Algorithm 2 and Eq. 2.24 on a 512 x 512 grayscale search window: Canny
    edges (thresholds 3 and 9), the magnitude-weighted orientation integral
    histogram over them, a 64 x 64
    target's 3-level pyramid descriptor, and the pyramid match kernel over
    256 x 256 placements."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    sw = torch.from_numpy(synth.blob_plane(512, 512, synth.config_seed(7))).to(dev)
    ctx = ih.ih_create(dev.index or 0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    L, wh, ww = 2, 64, 64
    D = ih.phog_descriptor_len(L)
    target = torch.empty((1, D), dtype=torch.int64, device=dev)
    out = torch.empty((256, 256), dtype=torch.float32, device=dev)
    tw = torch.tensor([[200, 210, 200 + wh - 1, 210 + ww - 1]], dtype=torch.int32, device=dev)
    t_build, t_match = [], []
    for rep in range(runs + 1):
        ev[0].record()
        h = ih.ih_phog_build(ctx, sw, 3, 9)
        ev[1].record()
        ih.ih_phog_descriptors(ctx, h, L, tw, target)
        ev[2].record()
        ih.ih_phog_match(ctx, h, L, target.view(-1), wh, ww, (72, 82, 72 + 255, 82 + 255), out)
        ev[3].record()
        torch.cuda.synchronize()
        ih.ih_release(ctx, h)
        if rep:
            t_build.append(ev[0].elapsed_time(ev[1]))
            t_match.append(ev[2].elapsed_time(ev[3]))
    best = int(out.view(-1).argmax().item())
    ih.ih_destroy(ctx)
    mb, mm = float(np.median(t_build)), float(np.median(t_match))
    return {"workload": "512x512 gray search window, Canny edges (3, 9), 9 orientation bins weighted by "
                        "gradient magnitude, "
                        "3-level pyramid (189 entries), 64x64 windows, 256x256 placements",
            "build_ms": round(mb, 4), "match_ms": round(mm, 4),
            "match_placements_per_s": 65536 / (mm / 1e3),
            "best_placement_found": [72 + best // 256, 82 + best % 256], "target_at": [200, 210]}


def plain_section(ih, dev, runs=400):
    """The plain frame: 640 x 480 uniform grayscale, 16 bins, 10,000 random
    rectangles.  Launch latency dominates, so the build + queries are timed
    both as plain per-frame calls and as one replayed CUDA graph (a one-frame
    batch), in the slab layout (a corner's 8 bins of a group in one sector)
    and in the bin-major layout (Fig. 5.1)."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    hh, ww, B = 480, 640, 16
    img = synth.uniform_plane(hh, ww, synth.config_seed(0))
    pix = torch.from_numpy(img).to(dev)[None]
    rects = torch.from_numpy(synth.rects_uniform_corners(hh, ww, 10_000, synth.config_seed(0) + 1)).to(dev)
    r_out = torch.empty((rects.shape[0], B), dtype=torch.int32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, k):
        fn()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(k):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / k * 1e3

    layouts = {}
    for lname, layout in (("slab", ih.IH_LAYOUT_SLAB), ("bin_major", ih.IH_LAYOUT_BIN_MAJOR)):
        ctx = ih.ih_create(dev.index or 0)
        frame = ih.Frame(pix, [(B, 0)], layout=layout)

        def per_frame():
            h, = ih.ih_build(ctx, frame)
            ih.ih_query_rects(ctx, h, rects, r_out)
            ih.ih_release(ctx, h)

        us_plain = timed(per_frame, runs)
        us = {}
        for name, flags in (("graph", ih.IH_BATCH_GRAPH), ("persistent_graph", ih.IH_BATCH_GRAPH | ih.IH_BATCH_PERSISTENT)):
            batch, handles = ih.ih_batch_create(ctx, [frame], rects=rects, rect_counts=[rects.shape[0]],
                                                rect_out=r_out.view(-1), batch_flags=flags)
            us[name] = timed(lambda: ih.ih_batch_run(ctx, batch), runs)
            ih.ih_batch_destroy(batch)
            for h in handles:
                ih.ih_release(ctx, h)
        ih.ih_destroy(ctx)
        # per-kernel device time of the plain per-frame calls (event pairs around each launch)
        ctxp = ih.ih_create(dev.index or 0, flags=ih.IH_CFG_PROFILE)
        for rep in range(21):
            h, = ih.ih_build(ctxp, frame)
            ih.ih_query_rects(ctxp, h, rects, r_out)
            ih.ih_release(ctxp, h)
            if rep == 0:
                ih.ih_sync(ctxp)
                ih.ih_profile_read(ctxp, reset=True)
        ih.ih_sync(ctxp)
        kern = {k: round(v[1] / v[0] * 1e3, 2) for k, v in ih.ih_profile_read(ctxp, reset=True).items()}
        ih.ih_destroy(ctxp)
        layouts[lname] = {"per_frame_us": round(us_plain, 2), "graph_modes_us": {k: round(v, 2) for k, v in us.items()},
                          "kernel_us_per_frame_calls": kern}
    best = min(layouts, key=lambda k: min(layouts[k]["graph_modes_us"].values()))
    us_graph = min(layouts[best]["graph_modes_us"].values())
    us_plain = min(v["per_frame_us"] for v in layouts.values())
    cells = B * hh * ww
    return {"workload": "plain 640x480 uniform gray, 16 bins, 10,000 rects", "per_frame_us": us_plain,
            "graph_us": round(us_graph, 2), "graph_layout": best, "layouts": layouts,
            "build": "small-frame build: one cooperative launch (tile sums, grid barrier, carries, tiles)",
            "cells_per_s_per_frame": cells / (us_plain / 1e6), "cells_per_s_graph": cells / (us_graph / 1e6)}


def batched_section(ih, dev, layout, n_frames=64, runs=5):
    """64 uneven FMV frames (sizes drawn from {640x480, 1280x720, 1920x1080,
    4096x2160}) with intensity moments and 4,096 weighted windows each: one
    batched launch per kernel replayed from a CUDA graph with autotuned tile
    grids, against 64 per-frame builds and queries on one stream."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    sizes = synth.frame_sizes_batched(n_frames, synth.config_seed(4))
    px = sum(h * w for h, w in sizes)
    need = px * (91 * 4 + 16 * 32) * 1.1 + px * 3
    free, _ = torch.cuda.mem_get_info(dev)
    while need > free * 0.9 and n_frames > 1:  # keep within this GPU's free memory
        n_frames //= 2
        sizes = sizes[:n_frames]
        px = sum(h * w for h, w in sizes)
        need = px * (91 * 4 + 16 * 32) * 1.1 + px * 3
    base = {s: synth.blob_rgb(s[0], s[1], 1000 + s[0]) for s in set(sizes)}
    pix = [torch.from_numpy(np.roll(base[s], 37 * k, axis=2)).to(dev) for k, s in enumerate(sizes)]
    frames = [ih.Frame(p, synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=WEIGHTED_CH,
                       layout=layout) for p in pix]
    nw = 4096
    wins = torch.from_numpy(np.concatenate([synth.rects_side_range(h, w, nw, 32, 256, 77 + k)
                                            for k, (h, w) in enumerate(sizes)])).to(dev)
    w_out = torch.empty(n_frames * nw * 16, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, k):
        ts = []
        for _ in range(k):
            ev[0].record()
            fn()
            ev[1].record()
            torch.cuda.synchronize()
            ts.append(ev[0].elapsed_time(ev[1]))
        return float(np.median(ts))

    ctx = ih.ih_create(dev.index or 0)
    res_b = {}
    for name, flags in (("graph", ih.IH_BATCH_GRAPH | ih.IH_BATCH_AUTOTUNE),
                        ("persistent", ih.IH_BATCH_GRAPH | ih.IH_BATCH_AUTOTUNE | ih.IH_BATCH_PERSISTENT)):
        batch, handles = ih.ih_batch_create(ctx, frames, windows=wins, window_counts=[nw] * n_frames,
                                            weighted_out=w_out, batch_flags=flags)
        timed(lambda: ih.ih_batch_run(ctx, batch), 2)
        l0 = ih.ih_launch_count(ctx)
        res_b[name] = (timed(lambda: ih.ih_batch_run(ctx, batch), runs), (ih.ih_launch_count(ctx) - l0) // runs)
        ih.ih_batch_destroy(batch)
        for h in handles:
            ih.ih_release(ctx, h)
        torch.cuda.synchronize()
    ih.ih_sync(ctx)
    ms_b, launches_b = min(res_b.values())

    def per_frame():
        for k, f in enumerate(frames):
            h, = ih.ih_build(ctx, f)
            ih.ih_query_weighted(ctx, h, wins[nw * k: nw * (k + 1)], w_out[nw * 16 * k: nw * 16 * (k + 1)].view(nw, 16))
            ih.ih_release(ctx, h)

    timed(per_frame, 1)
    l0 = ih.ih_launch_count(ctx)
    ms_p = timed(per_frame, max(2, runs // 2))
    launches_p = (ih.ih_launch_count(ctx) - l0) // max(2, runs // 2)
    ih.ih_sync(ctx)
    ih.ih_destroy(ctx)
    cells = px * 91
    gbytes = px * (91 * 4 + 16 * 32) / 1e9
    return {"workload": "%d uneven FMV frames (%s), 91 bins + intensity moments, %d weighted windows each"
                        % (n_frames, ", ".join("%dx%d:%d" % (w, h, sizes.count((h, w))) for h, w in sorted(set(sizes))), nw),
            "layout": [k for k, v in LAYOUTS.items() if v[0] == layout][0],
            "frames": n_frames, "pixels": px, "output_GB": round(gbytes, 2),
            "batched_graph_ms": round(ms_b, 3), "per_frame_ms": round(ms_p, 3),
            "batched_cells_per_s": cells / (ms_b / 1e3), "per_frame_cells_per_s": cells / (ms_p / 1e3),
            "batched_output_GBs": round(gbytes / (ms_b / 1e3), 1), "speedup_vs_per_frame": round(ms_p / ms_b, 3),
            "launches_per_batch": int(launches_b), "launches_per_frame_loop": int(launches_p),
            "modes": {k: {"ms": round(v[0], 3), "launches_per_batch": int(v[1]),
                          "output_GBs": round(gbytes / (v[0] / 1e3), 1), "speedup_vs_per_frame": round(ms_p / v[0], 3)}
                      for k, v in res_b.items()},
            "fastest_mode": min(res_b, key=lambda k: res_b[k][0])}


def served_section(ih, dev, layout, seconds=2.0, trackers=16, fps=30.0, budget_gb=60):
    """16 tracker streams with Poisson frame arrivals (30 fps each); frames
    drawn from the batched workload's sizes (FMV, 91 bins + intensity int64
    moments) and, with probability 1/16, 8192x8192 WAMI frames (32 bins,
    32-bit moments); 2,000 rectangles and 2,000 weighted windows per frame;
    60 GB budget.  The same arrival trace is served with continuous batching
    (4 streams, 4 ticks in flight, up to 16 requests per tick) and one
    request at a time."""
    import numpy as np
    import torch
    from paper_1711_01656_gb300 import synth
    g = np.random.Generator(np.random.PCG64(synth.config_seed(5)))
    rate = trackers * fps
    n = int(seconds * rate)
    t = np.cumsum(g.exponential(1.0 / rate, size=n))
    tracker = g.integers(0, trackers, size=n)
    sizes = [(480, 640), (720, 1280), (1080, 1920), (2160, 4096)]
    kind = np.where(g.random(n) < 1.0 / 16, 4, g.integers(0, 4, size=n))
    # device-resident inputs: two variants per FMV size, one WAMI frame
    fmv = {s: [torch.from_numpy(synth.blob_rgb(s[0], s[1], 500 + v + s[0])).to(dev) for v in range(2)] for s in sizes}
    wami = torch.from_numpy(synth.blob_plane(8192, 8192, 555)).to(dev)[None]
    qs = {}
    for k, (h, w) in enumerate(sizes + [(8192, 8192)]):
        qs[k] = (torch.from_numpy(synth.rects_uniform_corners(h, w, 2000, 900 + k)).to(dev),
                 torch.from_numpy(synth.rects_side_range(h, w, 2000, 32, 256, 950 + k)).to(dev))

    def frame_of(i):
        if kind[i] == 4:
            return ih.Frame(wami, [(32, 0)], weighted_channel=0, layout=layout, moment_bits=32), 32, 32, \
                8192 * 8192
        s = sizes[kind[i]]
        return ih.Frame(fmv[s][i % 2], synth.FMV_CHANNELS, input=ih.IH_INPUT_RGB_FEATURES, weighted_channel=WEIGHTED_CH,
                        layout=layout), 91, 16, s[0] * s[1]

    def serve(streams, inflight, batch):
        ctx = ih.ih_create(dev.index or 0, hbm_budget_bytes=int(budget_gb * 1e9))
        srv = ih.ih_server_create(ctx, streams=streams, max_inflight=inflight, max_batch=batch)
        keep, lat, cells, done = {}, [], 0, []
        try:
            start = ih.ih_server_clock(srv) + 0.05
            for i in range(n):
                while ih.ih_server_clock(srv) < start + t[i]:
                    for c in ih.ih_server_poll(srv, 256, 0):
                        done.append(c)
                        keep.pop(c["user"], None)
                f, B, Bw, npx = frame_of(i)
                r, w = qs[int(kind[i])]
                ro = torch.empty((2000, B), dtype=torch.int32, device=dev)
                wo = torch.empty((2000, Bw), dtype=torch.float32, device=dev)
                keep[i] = (f, ro, wo)
                ih.ih_server_submit(ctx, srv, int(tracker[i]), f, rects=r, rect_out=ro, windows=w, weighted_out=wo,
                                    user=i)
            ih.ih_server_drain(srv)
            done += ih.ih_server_poll(srv, n + 16, 0)
        finally:
            ih.ih_server_destroy(srv)
            ih.ih_destroy(ctx)
        ok = [c for c in done if c["status"] == 0]
        lat = np.array([c["t_done"] - c["t_submit"] for c in ok]) * 1e3
        span = max(c["t_done"] for c in ok) - min(c["t_submit"] for c in ok)
        for c in ok:
            cells += (91 if kind[c["user"]] < 4 else 32) * (sizes[kind[c["user"]]][0] * sizes[kind[c["user"]]][1]
                                                           if kind[c["user"]] < 4 else 8192 * 8192)
        return {"completed": len(ok), "failed": len(done) - len(ok), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
                "cells_per_s": cells / span, "span_s": round(span, 3)}

    cont = serve(4, 4, 16)
    single = serve(1, 1, 1)
    return {"workload": "%d trackers x %.0f fps Poisson for %.1f s (%d frames, %d WAMI 8192^2), 2,000 rect + "
                        "2,000 weighted queries per frame, %d GB budget" % (trackers, fps, seconds, n,
                                                                            int((kind == 4).sum()), budget_gb),
            "layout": [k for k, v in LAYOUTS.items() if v[0] == layout][0],
            "continuous_batching": cont, "one_request_at_a_time": single}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--fmv-steps", type=int, default=200, help="timed steps of the FMV section")
    ap.add_argument("--no-fmv", action="store_true", help="skip the full-motion-video step")
    ap.add_argument("--impl", choices=["engine", "reference"], default="engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-frame batched comparison")
    ap.add_argument("--no-served", action="store_true", help="skip the serving-loop comparison")
    ap.add_argument("--no-wami", action="store_true", help="skip the per-phase timings of the wide-area frame")
    ap.add_argument("--no-plain", action="store_true", help="skip the 640x480 plain frame")
    ap.add_argument("--no-match", action="store_true", help="skip the sliding-window matching maps")
    ap.add_argument("--no-mma", action="store_true", help="skip the tensor-core count tiles comparison")
    ap.add_argument("--no-median", action="store_true", help="skip the spatio-temporal median video")
    ap.add_argument("--no-phog", action="store_true", help="skip the pyramid-of-orientations matching")
    ap.add_argument("--layout", choices=sorted(LAYOUTS), default="record", help="count-tensor layout")
    ap.add_argument("--workload", choices=["wami", "fmv"], default="wami",
                    help="the workload of the line (wami: the headline; fmv for profiling captures)")
    ap.add_argument("--wami-side", type=int, default=WAMI_H,
                    help="side of the headline frame (smaller only for profiling captures)")
    ap.add_argument("--mma-side", type=int, default=8192, help="side of the frame of the mma_tiles section")
    ap.add_argument("--only-plain", type=int, default=0, metavar="RUNS",
                    help="profiling captures: run only the 640x480 plain-frame section with RUNS timed "
                         "repetitions and print its JSON (no bench line)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "engine":
        ap.error("--warmup must be >= 3")
    if args.only_plain > 0:
        import torch
        from paper_1711_01656_gb300 import ih
        print(json.dumps(plain_section(ih, torch.device("cuda", 0), runs=args.only_plain)))
        return 0
    return run_reference(args) if args.impl == "reference" else run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
