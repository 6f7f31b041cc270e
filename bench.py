#!/usr/bin/env python
"""Throughput of the asymmetric bidirectional optical-flow blend on GB300.

One step = the whole path for one overlap pair: luma + Gaussian pyramids of
both strips, pyramidal LK flow in both directions, and the Code 1 blend
(pano_flow_pair + pano_blend_pair). Workload: a 4000x1500 RGB uint8 pair,
6 pyramid levels, 5 LK steps per level, 5x5 window (synthetic, seeded).
The metric is overlap megapixels per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --workload rig     # all 8 pairs of a 360-degree rig per step
  python bench.py --workload refine_1024

With N > 1 (under torchrun) every rank runs its own pair: the pairs are
independent, there is no data exchange, and the reported value is the pixels
of all ranks over the slowest rank's time. ``--impl reference`` times the
FP64 CPU oracle instead (on rank 0 only), on row bands of the same pair.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "overlap megapixels/sec (bi-flow+warp+blend) on 1 GB300; % HBM roofline; EPE vs oracle"
UNIT = "MP/s"
WORKLOAD = {"workload": "pair_4000x1500_rgb_u8_lv6", "h": 4000, "w": 1500, "channels": 3, "levels": 6,
            "iters": 5, "radius": 2}
# the small single-pair configuration: launch-latency bound, reported, not the headline
SMALL_WORKLOAD = {"workload": "pair_256x512_gray_f32_lv4", "h": 256, "w": 512, "channels": 1, "levels": 4,
                  "iters": 5, "radius": 2}
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2
STREAM_MIN_PIXELS = 50000    # levels with at least this many pixels use the streamed LK kernel
SMALL_TILE_PIXELS = 16000    # tiled levels below this many pixels use 16 x 8 tiles
# DRAM bytes (read + write) per launch of the dominant kernel, averaged over
# its launches in one step, from an ncu capture of the current kernel with
# float32 pyramid planes (the 16-bit instantiations are other kernels: no
# figure); None when the kernel has changed since the counters were taken.
TRAFFIC_PER_LAUNCH = {"lk_stream_kernel": (1.188352e6 + 4.644352e6 + 18.470656e6 + 173.016832e6) / 4}
# Warp instructions per launch of the dominant kernel from the same capture
# (smsp__inst_executed.sum, averaged over its launches in one step).
INST_PER_LAUNCH = {"lk_stream_kernel": (10558682 + 32560009 + 90773349 + 368200597) / 4}
# One warp instruction per scheduler per cycle, four schedulers per SM.
SCHEDULERS_PER_SM = 4
SMS = 152


# ---------------------------------------------------------------------------
# host-side helpers (no GPU needed; covered by the CPU tests)
# ---------------------------------------------------------------------------

def level_pixels(h: int, w: int, levels: int):
    out = []
    for _ in range(levels):
        out.append(h * w)
        h, w = (h + 1) // 2, (w + 1) // 2
    return out


def lk_alg_bytes(h: int, w: int, levels: int, elem: int = 4):
    """Algorithmic bytes of each LK level launch (both directions).

    Per direction and level pixel: read the template and target levels
    (2 elem B), read the coarse flow (8 B per coarse pixel = 2 B per fine
    pixel; none at the coarsest level), write the flow (8 B).
    """
    npx = level_pixels(h, w, levels)
    out = []
    for l, n in enumerate(npx):
        coarse = 8 * npx[l + 1] if l + 1 < levels else 0
        out.append(2 * (2 * elem * n + coarse + 8 * n))
    return out


def path_alg_bytes(h: int, w: int, c: int, levels: int, in_bytes: int = 1, elem: int = 4):
    """Algorithmic bytes of one step of the whole path (each array once);
    elem = bytes of one stored pyramid element."""
    npx = level_pixels(h, w, levels)
    n = h * w
    pyramid = 2 * c * in_bytes * n + 2 * elem * sum(npx) + 2 * elem * sum(npx[:-1])  # read strips, write levels, re-read for REDUCE
    flow = sum(lk_alg_bytes(h, w, levels, elem))
    blend = 2 * c * in_bytes * n + 16 * n + c * in_bytes * n
    return pyramid + flow + blend


RIG_WORKLOAD = {"workload": "rig_8x4000x{800..2000}_rgb_u8_lv6_canvas_9000x4000", "h": 4000,
                "widths": [800, 950, 1100, 1250, 1400, 1600, 1800, 2000], "channels": 3, "levels": 6,
                "iters": 5, "radius": 2, "dmax": 24.0, "canvas": [4000, 9000],
                "canvas_x0": [1125 * k for k in range(8)]}
PANO_LK_AUTO, PANO_LK_STREAM, PANO_LK_TILE = 0, 1, 2
# --pyr-dtype: (pano_dtype of the pyramid storage, oracle storage format, bytes per stored element)
PYR_DTYPES = {"f32": (1, 0, 4), "bf16": (2, 1, 2), "f16": (3, 2, 2)}


def rig_level_kernels(h: int, widths, levels: int, kernels, tiles=None):
    """Kernel launches of each LK level of a rig, in launch order: for level
    l, [(kernel name, [pairs])], the streamed batch first, then one tiled
    launch per tile shape (in the order of the first pair with it).
    kernels[l] is the level's PANO_LK_* tuning and tiles[l] its (tile_w,
    tile_h), (0, 0) for the default; AUTO uses the single-pair rules."""
    out = []
    for l in range(levels):
        hl = h
        ws = list(widths)
        for _ in range(l):
            hl = (hl + 1) // 2
            ws = [(w + 1) // 2 for w in ws]
        tile = tuple(tiles[l]) if tiles else (0, 0)
        st, groups = [], {}
        for k, w in enumerate(ws):
            use = kernels[l] == PANO_LK_STREAM or (kernels[l] == PANO_LK_AUTO and hl * w >= STREAM_MIN_PIXELS)
            if use:
                st.append(k)
                continue
            shape = tile if tile != (0, 0) else ("small" if hl * w < SMALL_TILE_PIXELS else "default")
            groups.setdefault(shape, []).append(k)
        lev = []
        if st:
            lev.append(("lk_stream_batch_kernel", st))
        for members in groups.values():
            lev.append(("lk_level_batch_kernel", members))
        out.append(lev)
    return out


def unfused_stage_bytes(h: int, w: int, levels: int, iters: int, elem: int = 4) -> int:
    """Bytes if every LK step were its own pass: per direction, step and level
    pixel read u, T, J and write u (8 + 2 elem + 8 B)."""
    return sum(2 * iters * (16 + 2 * elem) * n for n in level_pixels(h, w, levels))


def throughput(pixels_per_step: int, steps: int, world: int, max_total_ms: float) -> float:
    """Whole-job MP/s: every rank's pixels over the slowest rank's time."""
    return pixels_per_step * steps * world / (max_total_ms * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def time_oracle(pair, levels: int, budget_s: float, band_rows: int = 500, max_bands: int = 1000):
    """Oracle stitch (flow + blend) on row bands of the pair until budget_s
    of CPU work; returns (MP/s, threads, sample description, seconds)."""
    import oracle
    P = oracle.Params(levels=levels)
    h = pair.L.shape[0]
    done_px, t_total, bands = 0, 0.0, 0
    y = 0
    while (t_total < budget_s or bands == 0) and bands < max_bands:
        y0 = y % max(1, h - band_rows + 1)
        L = pair.L[y0:y0 + band_rows]
        R = pair.R[y0:y0 + band_rows]
        t0 = time.perf_counter()
        oracle.stitch_pair(L, R, P)
        t_total += time.perf_counter() - t0
        done_px += L.shape[0] * L.shape[1]
        bands += 1
        y += band_rows
    desc = f"{bands} bands of {band_rows}x{pair.L.shape[1]} rows of the pair (FP64 oracle, flow + blend)"
    return done_px / t_total / 1e6, oracle.num_threads(), desc, t_total


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, else implementer/part)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info.splitlines():
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = (x.strip() for x in line.split(":", 1))
            fields.setdefault(k, v)
    return f"implementer {fields.get('CPU implementer', '?')} part {fields.get('CPU part', '?')}"


def oracle_baseline(pair, levels: int, budget_s: float, label: str):
    """cpu_baseline object: the oracle on all host cores (the value) and on
    one thread (reported beside it), on row bands of the pair."""
    import oracle
    v, cores, desc, secs = time_oracle(pair, levels, budget_s=budget_s)
    nthreads = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        v1, _, desc1, secs1 = time_oracle(pair, levels, budget_s=budget_s / 4, band_rows=100)
    finally:
        oracle.set_num_threads(nthreads)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc.replace("of the pair", label),
            "seconds": secs, "single_thread": {"value": v1, "sample": desc1.replace("of the pair", label),
                                               "seconds": secs1},
            "cpu": cpu_model(), "nproc": os.cpu_count()}


# The paper's own figure (whole workflow, one 9000x4000 panorama, GPU model
# not stated): context for the rig numbers, not a target.
PAPER_CONTEXT = "under 30 s per 9000x4000 panorama for the whole workflow on an unspecified GPU (abstract, Section IV)"

# FP32 arithmetic of one LK step per level pixel: bilinear sample 8, It 1,
# products 2, separable box sums 8, 2x2 solve 12, update 2, plus gradient
# and normal matrices amortised (about 50 in all).
LK_FLOPS_PER_PIXEL_STEP = 50


def issue_roofline(kernel: str, launch_ms: float, sm_mhz):
    """Warp-instruction issue rate of `kernel` (ncu instruction count per
    launch / live launch time) against the SMs' issue peak at the sampled SM
    clock; None without a counted instruction total or a clock sample."""
    inst = INST_PER_LAUNCH.get(kernel)
    if not inst or not launch_ms or not sm_mhz:
        return None
    achieved = inst / (launch_ms * 1e-3) / 1e9
    peak = SMS * SCHEDULERS_PER_SM * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instr/s", "frac": achieved / peak,
            "inst_per_launch": inst, "kernel": kernel, "peak_source": "152 SMs x 4 schedulers x sampled SM clock"}


def fp32_peak_tflops(sm_mhz: float = 2070.0, sms: int = 152) -> float:
    """FP32 FMA peak: 128 lanes per SM, 2 flops per FMA."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def time_pipeline(pipe, submit, steps: int, world: int, repeats: int = 3):
    """Milliseconds from before the first upload to after the last download of
    `steps` items submitted to a host pipeline (max over ranks), measured
    `repeats` times: (median, all). The copies go through host memory, which
    other jobs on the node share, so one repeat can catch their traffic."""
    import torch
    runs = []
    for r in range(repeats):
        barrier(world)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(pipe.s_in)
        for k in range(steps):
            submit(1000 * (r + 1) + k)
        t1.record(pipe.s_out)
        pipe.drain()
        torch.cuda.synchronize()
        barrier(world)
        runs.append(reduce_max(t0.elapsed_time(t1), world))
    return statistics.median(runs), runs


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    pair = synth.pair_fullres_rgb()
    import oracle
    oracle.build()
    band = 250
    vals = []
    for i in range(args.warmup + args.steps):
        v, cores, desc, _ = time_oracle(pair, WORKLOAD["levels"], 0.0, band_rows=band, max_bands=1)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": band * WORKLOAD["w"] / value / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample=f"one {band}-row band per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"one {band}x{WORKLOAD['w']} band of the pair per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import synth
    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import build as gpu_build

    gpu_build.build()
    pkg.load_library()
    WL = SMALL_WORKLOAD if args.workload == "small" else WORKLOAD
    h, w, c, levels = WL["h"], WL["w"], WL["channels"], WL["levels"]
    if args.workload == "small":
        pair = synth.pair_small_gray(seed=rank, h=h, w=w, levels=levels)
    else:
        pair = synth.pair_fullres_rgb(seed=1 + rank, h=h, w=w, levels=levels)
    pyr_code, pyr_fmt, elem = PYR_DTYPES[args.pyr_dtype]
    ctx = pkg.FlowContext(pkg.Params(levels=levels, iters=WL["iters"], radius=WL["radius"],
                                     pyr_dtype=pyr_code),
                          max_h=h, max_w=w, max_c=c)
    L = torch.from_numpy(pair.L).to(dev)
    R = torch.from_numpy(pair.R).to(dev)
    lr = torch.empty((h, w, 2), dtype=torch.float32, device=dev)
    rl = torch.empty((h, w, 2), dtype=torch.float32, device=dev)
    F = torch.empty_like(L)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ctx.flow_pair(L, R, out=(lr, rl), stream=stream)
        ctx.blend_pair(L, R, lr, rl, out=F, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    # --- timed region: K steps, device-resident inputs, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.launches
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = ctx.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = reduce_max(sum(step_ms), world)
    value = throughput(h * w, args.steps, world, total_ms)

    # --- same loop with every launch bracketed by events: per-kernel times
    ctx.trace_enable(0x3F, 64 * args.steps)
    for k in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    recs = ctx.trace_read(64 * args.steps)
    ctx.trace_enable(0, 0)
    names = {1: "luma_kernel", 2: "pyr_down_kernel", 8: "blend_kernel", 16: "luma_reduce_kernel", 32: "pyr_tail_kernel"}
    npx = level_pixels(h, w, levels)
    lk_bytes = lk_alg_bytes(h, w, levels, elem)
    per_kind = {}
    stream_bytes = 0.0
    for kind, lev, ms in recs:
        if kind == 4:
            # levels of at least STREAM_MIN_PIXELS run the streamed kernel
            name = "lk_stream_kernel" if npx[lev] >= STREAM_MIN_PIXELS else "lk_level_kernel"
            if name == "lk_stream_kernel":
                stream_bytes += lk_bytes[lev]
        else:
            name = names[kind]
        d = per_kind.setdefault(name, {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += ms
    traced_total = sum(d["ms"] for d in per_kind.values())
    for d in per_kind.values():
        d["share"] = d["ms"] / traced_total if traced_total else None
        d["ms_per_step"] = d["ms"] / args.steps
    dominant = max(per_kind, key=lambda k: per_kind[k]["ms"])
    dk = per_kind[dominant]
    launches_per_step = dk["launches"] / args.steps
    if dominant == "lk_stream_kernel":
        bytes_per_launch = stream_bytes / dk["launches"]
    else:
        bytes_per_launch = None
    peak, peak_src = read_peaks()
    launch_ms = dk["ms"] / dk["launches"]
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9 if bytes_per_launch else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": TRAFFIC_PER_LAUNCH.get(dominant) if args.pyr_dtype == "f32" else None, "kernel": dominant,
                "alg_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                "launches_per_step": launches_per_step, "peak_source": f"{peak_src} hbm_gbs"}
    issue = issue_roofline(dominant, launch_ms, clocks["sm_mhz"] if clocks else None) \
        if args.pyr_dtype == "f32" else None
    path_bytes = path_alg_bytes(h, w, c, levels, elem=elem)
    path_gbs = path_bytes / (total_ms / args.steps * 1e-3) / 1e9
    stage_bytes = unfused_stage_bytes(h, w, levels, WL["iters"], elem)
    path_flops = 2 * WL["iters"] * LK_FLOPS_PER_PIXEL_STEP * sum(level_pixels(h, w, levels))

    # --- end to end: pinned host strips in, F back to pinned host memory,
    #     through the library's double-buffered host pipeline (the copies of
    #     neighbouring steps overlap the kernels of the current one)
    Lh = torch.from_numpy(pair.L).pin_memory()
    Rh = torch.from_numpy(pair.R).pin_memory()
    Fh = [torch.empty_like(Lh).pin_memory() for _ in range(2)]
    pipe = ctx.host_pipeline(tuple(L.shape), L.dtype, dev)
    for k in range(max(1, args.warmup)):
        pipe.submit(k, Lh, Rh, Fh[k % 2])
    pipe.drain()
    e2e_ms, e2e_runs = time_pipeline(pipe, lambda k: pipe.submit(k, Lh, Rh, Fh[k % 2]), args.steps, world)
    e2e = {"value": throughput(h * w, args.steps, world, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(Lh.numel() + Rh.numel()), "d2h_bytes_per_step": int(Fh[0].numel()),
           "ms_per_step": e2e_ms / args.steps,
           "pipeline": "two buffer sets; H2D, kernels and D2H on three streams; no L2 flush (inputs arrive by H2D)",
           "repeats_ms": e2e_runs, "timing": "median of 3 timed runs of K steps"}

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(WL, l2="flushed between steps (256 MB write, untimed)",
                               parallelism=f"replicas{world}", pyr_dtype=args.pyr_dtype),
                "roofline": roofline, "issue_roofline": issue,
                "path": {"alg_bytes_per_step": path_bytes, "achieved_gbs": path_gbs, "frac": path_gbs / peak,
                         "unfused_stage_bytes_per_step": stage_bytes,
                         "fp32_tflops": path_flops / (total_ms / args.steps * 1e-3) / 1e12,
                         "fp32_peak_tflops": fp32_peak_tflops(clocks["sm_mhz"] if clocks else 2070.0),
                         "fp32_frac": path_flops / (total_ms / args.steps * 1e-3) / 1e12
                         / fp32_peak_tflops(clocks["sm_mhz"] if clocks else 2070.0),
                         "flops_per_step": path_flops},
                "kernels": per_kind, "dominant_kernel": dominant,
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "paper_context": PAPER_CONTEXT,
                "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms)}
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            # parity of this run's flows against the oracle, and the oracle's speed
            t0 = time.perf_counter()
            olr, orl = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=levels))
            t_full = time.perf_counter() - t0
            g_lr, g_rl = lr.cpu().numpy(), rl.cpu().numpy()
            e_lr = float(np.hypot(*(g_lr - olr).transpose(2, 0, 1)).mean())
            e_rl = float(np.hypot(*(g_rl - orl).transpose(2, 0, 1)).mean())
            line["epe_vs_oracle"] = {"LtoR_mean_px": e_lr, "RtoL_mean_px": e_rl}
            Fo = oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=levels))
            if pair.L.dtype == np.uint8:
                dF = np.abs(F.cpu().numpy().astype(int) - oracle.quantize_u8(Fo).astype(int))
                line["F_u8_vs_oracle"] = {"max_lsb": int(dF.max()), "mean_lsb": float(dF.mean()),
                                          "frac_gt_1lsb": float((dF > 1).mean())}
            else:
                dF = np.abs(F.cpu().numpy().astype(np.float64) - Fo)
                line["F_vs_oracle"] = {"max_abs": float(dF.max()), "mean_abs": float(dF.mean()),
                                       "max_in_u8_lsb": float(dF.max() * 255)}
            if pyr_fmt:
                line["half_precision"] = half_precision_report(pkg, pair, levels, pyr_fmt, g_lr, g_rl,
                                                               F.cpu().numpy(), olr, orl, dev)
            line["cpu_baseline"] = oracle_baseline(pair, levels, args.cpu_budget, f"of the {h}x{w} pair")
            line["cpu_baseline"]["full_pair_flow_s"] = t_full
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def half_precision_report(pkg, pair, levels, pyr_fmt, g_lr, g_rl, g_F, olr, orl, dev):
    """Errors of 16-bit pyramid storage: flows against the exact FP64 oracle,
    the storage-matched oracle and the float32 GPU path; blended pixels
    against the float32 GPU path and the oracle."""
    import numpy as np
    import torch
    import oracle

    def mean_epe(a, b):
        return float(np.hypot(*(a - b).transpose(2, 0, 1)).mean())

    h, w = pair.L.shape[:2]
    c = pair.L.shape[2] if pair.L.ndim == 3 else 1
    with pkg.FlowContext(pkg.Params(levels=levels), max_h=h, max_w=w, max_c=c) as ctx32:
        lr32, rl32, F32 = ctx32.stitch_pair(torch.from_numpy(pair.L).to(dev), torch.from_numpy(pair.R).to(dev))
        torch.cuda.synchronize()
        lr32, rl32, F32 = lr32.cpu().numpy(), rl32.cpu().numpy(), F32.cpu().numpy()
    slr, srl = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=levels, pyr_fmt=pyr_fmt))
    Fo = oracle.quantize_u8(oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=levels)))
    d32 = np.abs(g_F.astype(int) - F32.astype(int))
    do = np.abs(g_F.astype(int) - Fo.astype(int))
    return {"epe_vs_exact_oracle": [mean_epe(g_lr, olr), mean_epe(g_rl, orl)],
            "epe_vs_storage_oracle": [mean_epe(g_lr, slr), mean_epe(g_rl, srl)],
            "epe_vs_gpu_f32": [mean_epe(g_lr, lr32), mean_epe(g_rl, rl32)],
            "gpu_f32_epe_vs_exact_oracle": [mean_epe(lr32, olr), mean_epe(rl32, orl)],
            "F_u8_vs_gpu_f32": {"max_lsb": int(d32.max()), "mean_lsb": float(d32.mean()),
                                "frac_gt_1lsb": float((d32 > 1).mean())},
            "F_u8_vs_exact_oracle": {"max_lsb": int(do.max()), "mean_lsb": float(do.mean()),
                                     "frac_gt_1lsb": float((do > 1).mean())}}


def run_blend_coeff(args):
    """General-mask Eq. (1): the blending coefficient of a 4000 x 9000
    panorama canvas with wavy seams between Area1, Area3 and Area2 and holes
    (exact distance transform + ratio), one pano_blend_coeff per step."""
    import numpy as np
    import torch

    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import binding, build as gpu_build

    gpu_build.build()
    pkg.load_library()
    dev = torch.device("cuda", 0)
    h, w = 4000, 9000
    g = np.random.default_rng(8)
    ys = np.arange(h)[:, None]
    xs = np.arange(w)[None, :]
    a = 0.3 * w + 0.08 * w * np.sin(2 * np.pi * ys / (0.7 * h) + g.uniform(0, 6)) + g.normal(0, 0.01 * w, (h, 1))
    b = 0.7 * w + 0.08 * w * np.sin(2 * np.pi * ys / (0.5 * h) + g.uniform(0, 6))
    lab = np.where(xs < a, 1, np.where(xs >= b, 2, 3)).astype(np.uint8)
    for _ in range(6):
        cy, cx, r = g.integers(0, h), g.integers(0, w), g.integers(1, 400)
        lab[(ys - cy) ** 2 + (xs - cx) ** 2 <= r * r] = 0
    label = torch.from_numpy(lab).to(dev)
    out = torch.empty((h, w), dtype=torch.float32, device=dev)
    scratch = torch.empty(int(binding.load_library().pano_blend_coeff_scratch_bytes(h, w)), dtype=torch.uint8,
                          device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        binding.blend_coeff(label, out=out, scratch=scratch)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        binding.blend_coeff(label, out=out, scratch=scratch)
        ev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(a_.elapsed_time(b_) for a_, b_ in ev) / args.steps
    npx = h * w
    alg = 5 * npx          # label read (1 B) and Blend written (4 B) once per pixel
    peak, src = read_peaks()
    line = {"metric": "general-mask Eq. (1) blending coefficient, canvas megapixels/sec",
            "value": npx / (ms * 1e-3) / 1e6, "unit": "MP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "i32+f32", "data": "synthetic",
            "config": {"workload": "blend_coeff_canvas_4000x9000_wavy_seams_holes",
                       "l2": "flushed between steps (256 MB write, untimed)",
                       "area3_fraction": float((lab == 3).mean())},
            "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": None,
                         "kernel": "edt_cols_kernel + edt_row_kernel (Area1) + edt_row_kernel (Area2)", "alg_bytes_per_launch": alg,
                         "peak_source": f"{src} hbm_gbs"},
            "gpu_launches": 3 * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_refine(args):
    """Differentiable-refinement workload: 1024x1024 gray f32 pair (6 px
    sinusoidal field, 5 levels). Times the energy + adjoint kernel at level 0
    (all three gradients) and a full coarse-to-fine refinement."""
    import numpy as np
    import torch

    import synth
    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import binding, build as gpu_build, refine

    gpu_build.build()
    pkg.load_library()
    dev = torch.device("cuda", 0)
    pair = synth.pair_small_gray(seed=3, h=1024, w=1024, amp_x=6.0, amp_y=3.0, levels=5)
    T = torch.from_numpy(pair.L).to(dev)
    J = torch.from_numpy(pair.R).to(dev)
    u = torch.from_numpy(pair.flow_LtoR.astype(np.float32)).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        binding.energy_grad(T, J, u, 0.05)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(0)
    sampler.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        binding.energy_grad(T, J, u, 0.05)
        ev[k][1].record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    npx = 1024 * 1024
    # per pixel: T 4 B, J taps ~4 B, u 8 B (+ neighbours from cache), dE/du 8 B,
    # dE/dT 4 B, dE/dJ read-modify-write 8 B
    alg = 36 * npx
    peak, src = read_peaks()
    t0 = time.perf_counter()
    uref, trace = refine.refine_flow(T, J, levels=5, steps=20, lr=0.05, alpha=0.05)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    m = 48
    err = np.hypot(*(uref.cpu().numpy() - pair.flow_LtoR).transpose(2, 0, 1))[m:-m, m:-m]
    line = {"metric": "energy + adjoint megapixels/sec (differentiable refinement, level 0)",
            "value": npx / (ms * 1e-3) / 1e6, "unit": "MP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "refine_1024x1024_gray_f32_lv5", "alpha": 0.05,
                       "l2": "flushed between steps (256 MB write, untimed)"},
            "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (ms * 1e-3) / 1e9 / peak, "traffic": None, "kernel": "energy_grad_kernel",
                         "alg_bytes_per_launch": alg, "peak_source": f"{src} hbm_gbs"},
            "refinement": {"levels": 5, "adam_steps_per_level": 20, "seconds": t_ref,
                           "mean_epe_px_vs_truth": float(err.mean()),
                           "energy_per_level": [[l, a, b] for l, a, b in trace]},
            "gpu_launches": args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_rig(args):
    """The 360-degree rig: 8 RGB u8 pairs of 4000 x {800..2000}, 6 levels,
    every step one replay of the rig's CUDA graph (luma, REDUCE, batched LK
    per level, blend into the 9000 x 4000 canvas). The single-pair form
    (pano_flow_pair + pano_blend_pair per pair) is timed beside it."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import synth
    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import binding, build as gpu_build

    gpu_build.build()
    pkg.load_library()
    W = RIG_WORKLOAD
    h, widths, c, levels = W["h"], W["widths"], W["channels"], W["levels"]
    pairs = synth.rig_pairs(h=h, widths=widths, dmax=W["dmax"], levels=levels, seed0=100 + 8 * rank)
    pyr_code, pyr_fmt, elem = PYR_DTYPES[args.pyr_dtype]
    params = pkg.Params(levels=levels, iters=W["iters"], radius=W["radius"], pyr_dtype=pyr_code)
    rig = binding.Rig(params, h, widths, c=c, dtype=torch.uint8, canvas_hw=tuple(W["canvas"]),
                      canvas_x0=W["canvas_x0"])
    Ls = [torch.from_numpy(p.L).to(dev) for p in pairs]
    Rs = [torch.from_numpy(p.R).to(dev) for p in pairs]
    canvas = rig.new_canvas(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    npx = h * sum(widths)

    t0 = time.perf_counter()
    tunings = rig.autotune(Ls, Rs, reps=3, stream=stream) if not args.no_autotune else \
        [rig.get_tuning(l) for l in range(levels)]
    tune_s = time.perf_counter() - t0

    def step():
        rig.run(Ls, Rs, canvas=canvas, use_graph=True, stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = rig.launches
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    launches = rig.launches - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = reduce_max(sum(step_ms), world)
    value = throughput(npx, args.steps, world, total_ms)

    # --- eager runs with every launch bracketed by events: per-kernel times
    rig.trace_enable(0x3F, 64 * args.steps)
    for k in range(args.steps):
        flush.zero_()
        rig.run(Ls, Rs, canvas=canvas, use_graph=False, stream=stream)
    torch.cuda.synchronize()
    recs = rig.trace_read(64 * args.steps)
    rig.trace_enable(0, 0)
    plan = rig_level_kernels(h, widths, levels, [t["kernel"] for t in tunings],
                             [(t["tile_w"], t["tile_h"]) for t in tunings])
    names = {1: "luma_kernel", 2: "pyr_down_kernel", 8: "rig_blend_kernel", 16: "luma_reduce_kernel", 32: "pyr_tail_kernel"}
    per_kind, lk_seen = {}, {}
    stream_bytes = 0.0
    lk_bytes = [lk_alg_bytes(h, w, levels, elem) for w in widths]
    for kind, lev, ms in recs:
        if kind == 4:
            i = lk_seen.get(lev, 0) % len(plan[lev])
            lk_seen[lev] = lk_seen.get(lev, 0) + 1
            name, members = plan[lev][i]
            if name == "lk_stream_batch_kernel":
                stream_bytes += sum(lk_bytes[k][lev] for k in members)
        else:
            name = names[kind]
        d = per_kind.setdefault(name, {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += ms
    traced_total = sum(d["ms"] for d in per_kind.values())
    for d in per_kind.values():
        d["share"] = d["ms"] / traced_total if traced_total else None
        d["ms_per_step"] = d["ms"] / args.steps
    dominant = max(per_kind, key=lambda k: per_kind[k]["ms"])
    dk = per_kind[dominant]
    peak, peak_src = read_peaks()
    launch_ms = dk["ms"] / dk["launches"]
    bytes_per_launch = stream_bytes / dk["launches"] if dominant == "lk_stream_batch_kernel" else None
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9 if bytes_per_launch else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": TRAFFIC_PER_LAUNCH.get(dominant) if args.pyr_dtype == "f32" else None, "kernel": dominant,
                "alg_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                "launches_per_step": dk["launches"] / args.steps, "peak_source": f"{peak_src} hbm_gbs"}
    issue = issue_roofline(dominant, launch_ms, clocks["sm_mhz"] if clocks else None) \
        if args.pyr_dtype == "f32" else None
    path_bytes = sum(path_alg_bytes(h, w, c, levels, elem=elem) for w in widths)

    def time_rig(other):
        """CUDA-event time of K graph replays of another rig on the same strips."""
        cv = other.new_canvas(dev)
        for _ in range(args.warmup):
            flush.zero_()
            other.run(Ls, Rs, canvas=cv, use_graph=True, stream=stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            other.run(Ls, Rs, canvas=cv, use_graph=True, stream=stream)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        return reduce_max(sum(a.elapsed_time(b) for a, b in evs), world), cv

    fp32_form = None
    if pyr_fmt:
        # the float32 batched form beside the 16-bit one, tuned the same way
        rig32 = binding.Rig(pkg.Params(levels=levels, iters=W["iters"], radius=W["radius"]), h, widths, c=c,
                            dtype=torch.uint8, canvas_hw=tuple(W["canvas"]), canvas_x0=W["canvas_x0"])
        if not args.no_autotune:
            rig32.autotune(Ls, Rs, reps=3, stream=stream)
        ms32, canvas32 = time_rig(rig32)
        fp32_form = {"value": throughput(npx, args.steps, world, ms32), "unit": UNIT,
                     "ms_per_step": ms32 / args.steps}

    # --- the single-pair form on the same strips: 8 x (flow_pair + blend_pair)
    ctx = pkg.FlowContext(params, max_h=h, max_w=max(widths), max_c=c)
    outs = [(torch.empty((h, w, 2), device=dev), torch.empty((h, w, 2), device=dev), torch.empty_like(Ls[k]))
            for k, w in enumerate(widths)]

    def pair_step():
        for k in range(len(widths)):
            ctx.flow_pair(Ls[k], Rs[k], out=outs[k][:2], stream=stream)
            ctx.blend_pair(Ls[k], Rs[k], outs[k][0], outs[k][1], out=outs[k][2], stream=stream)

    for _ in range(args.warmup):
        flush.zero_()
        pair_step()
    torch.cuda.synchronize()
    ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        ev3[k][0].record(stream)
        pair_step()
        ev3[k][1].record(stream)
    torch.cuda.synchronize()
    pair_ms = reduce_max(sum(a.elapsed_time(b) for a, b in ev3), world)
    ctx.close()

    # --- end to end: pinned host strips in, the canvas back to pinned host
    #     memory, through the double-buffered host pipeline
    Lh = [torch.from_numpy(p.L).pin_memory() for p in pairs]
    Rh = [torch.from_numpy(p.R).pin_memory() for p in pairs]
    Ch = [torch.empty(tuple(canvas.shape), dtype=canvas.dtype).pin_memory() for _ in range(2)]
    pipe = binding.RigHostPipeline(rig, dev)
    for k in range(max(1, args.warmup)):
        pipe.submit(k, Lh, Rh, Ch[k % 2])
    pipe.drain()
    e2e_ms, e2e_runs = time_pipeline(pipe, lambda k: pipe.submit(k, Lh, Rh, Ch[k % 2]), args.steps, world)
    e2e = {"value": throughput(npx, args.steps, world, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(t.numel() for t in Lh + Rh)), "d2h_bytes_per_step": int(Ch[0].numel()),
           "ms_per_step": e2e_ms / args.steps,
           "pipeline": "two buffer sets; H2D, graph replay and D2H on three streams; no L2 flush (inputs arrive by H2D)",
           "repeats_ms": e2e_runs, "timing": "median of 3 timed runs of K steps"}

    line = None
    if rank == 0:
        line = {"metric": METRIC.replace("(bi-flow+warp+blend)", "(bi-flow+warp+blend, 8-pair rig)"),
                "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(W, l2="flushed between steps (256 MB write, untimed); inputs 262 MB > L2",
                               parallelism=f"replicas{world}", graph=True, pyr_dtype=args.pyr_dtype),
                "roofline": roofline, "issue_roofline": issue,
                "path": {"alg_bytes_per_step": path_bytes,
                         "achieved_gbs": path_bytes / (total_ms / args.steps * 1e-3) / 1e9},
                "kernels": per_kind, "dominant_kernel": dominant,
                "single_pair_form": {"value": throughput(npx, args.steps, world, pair_ms), "unit": UNIT,
                                     "ms_per_step": pair_ms / args.steps},
                "fp32_batched_form": fp32_form,
                "paper_context": PAPER_CONTEXT,
                "autotune": {"seconds": tune_s, "levels": tunings},
                "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
                "step_ms_min": min(step_ms), "step_ms_median": statistics.median(step_ms)}
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            olr, orl = oracle.flow_pair(pairs[0].L, pairs[0].R, oracle.Params(levels=levels))
            g_lr, g_rl = (t.cpu().numpy() for t in rig.flows(0))
            line["epe_vs_oracle"] = {
                "pair": 0,
                "LtoR_mean_px": float(np.hypot(*(g_lr - olr).transpose(2, 0, 1)).mean()),
                "RtoL_mean_px": float(np.hypot(*(g_rl - orl).transpose(2, 0, 1)).mean())}
            if pyr_fmt:
                # pair 1 owns its whole canvas span (columns 1125 .. 2074): pair 0's
                # first columns are overwritten by pair 7, which wraps around the seam
                x1 = W["canvas_x0"][1]
                F1 = canvas[:, x1:x1 + widths[1]].cpu().numpy()
                h_lr, h_rl = (t.cpu().numpy() for t in rig.flows(1))
                x_lr, x_rl = oracle.flow_pair(pairs[1].L, pairs[1].R, oracle.Params(levels=levels))
                line["half_precision"] = half_precision_report(pkg, pairs[1], levels, pyr_fmt, h_lr, h_rl, F1,
                                                               x_lr, x_rl, dev)
                line["half_precision"]["pair"] = 1
                line["half_precision"]["canvas_u8_vs_fp32_rig"] = {
                    "max_lsb": int((canvas.int() - canvas32.int()).abs().max()),
                    "mean_lsb": float((canvas.int() - canvas32.int()).abs().float().mean())}
            line["cpu_baseline"] = oracle_baseline(pairs[0], levels, args.cpu_budget, "of rig pair 0 (4000x800)")
            line["cpu_baseline"]["rig_step_s_extrapolated"] = npx / 1e6 / line["cpu_baseline"]["value"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    rig.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_compose(args):
    """Code 1 on a whole canvas (pano_compose_pair): a 4000x3000 RGB u8 canvas
    holding Area1 (750 columns), the 4000x1500 overlap of the benchmark pair
    (Area3) and Area2 (750 columns). Times the canvas pass alone and the whole
    stitch of the pair onto the canvas (pano_flow_pair on the overlap crop,
    then pano_compose_pair)."""
    import numpy as np
    import torch

    import synth
    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import binding, build as gpu_build

    gpu_build.build()
    pkg.load_library()
    dev = torch.device("cuda", 0)
    pair = synth.pair_fullres_rgb()
    h, ws = pair.shape
    m = 750
    w = ws + 2 * m
    g = np.random.default_rng(7)
    L = np.concatenate([g.integers(0, 256, (h, m, 3), dtype=np.uint8), pair.L, pair.L[:, -m:][:, ::-1]], 1)
    R = np.concatenate([pair.R[:, :m][:, ::-1], pair.R, g.integers(0, 256, (h, m, 3), dtype=np.uint8)], 1)
    lab = np.full((h, w), 3, np.uint8)
    lab[:, :m], lab[:, m + ws:] = 1, 2
    Ld, Rd = torch.from_numpy(np.ascontiguousarray(L)).to(dev), torch.from_numpy(np.ascontiguousarray(R)).to(dev)
    labd = torch.from_numpy(lab).to(dev)
    Bd = binding.blend_coeff(labd)
    params = binding.Params(levels=WORKLOAD["levels"])
    ctx = binding.FlowContext(params, max_h=h, max_w=ws, max_c=3)
    Lc, Rc = Ld[:, m:m + ws], Rd[:, m:m + ws]
    lr, rl = ctx.flow_pair(Lc, Rc)
    F = binding.compose_pair(Ld, Rd, labd, Bd, lr, rl, origin=(0, m), params=params)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            fn()
            ev[k][1].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev) / args.steps

    sampler = ClockSampler(0)
    sampler.start()
    ms = timed(lambda: binding.compose_pair(Ld, Rd, labd, Bd, lr, rl, origin=(0, m), params=params, out=F))
    clocks = sampler.stop()

    def stitch():
        ctx.flow_pair(Lc, Rc, out=(lr, rl))
        binding.compose_pair(Ld, Rd, labd, Bd, lr, rl, origin=(0, m), params=params, out=F)

    ms_stitch = timed(stitch)
    ctx.close()
    # per canvas pixel: label 1 B; Area1/Area2 copy 3 B in, 3 B out; Area3 Blend 4 B,
    # L and R 3 B each, both flows 16 B, F 3 B
    alg = h * (2 * m) * (1 + 3 + 3) + h * ws * (1 + 4 + 6 + 16 + 3)
    peak, src = read_peaks()
    gbs = alg / (ms * 1e-3) / 1e9
    line = {"metric": "canvas megapixels/sec (Code 1, every branch, on one GB300)",
            "value": h * w / (ms * 1e-3) / 1e6, "unit": "MP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "compose_4000x3000_rgb_u8_overlap_1500", "area1_cols": m, "area3_cols": ws,
                       "area2_cols": m, "l2": "flushed between steps (256 MB write, untimed)"},
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "traffic": None, "kernel": "compose_kernel", "alg_bytes_per_launch": alg,
                         "peak_source": f"{src} hbm_gbs"},
            "stitch": {"metric": "overlap megapixels/sec (flow of the overlap + Code 1 on the canvas)",
                       "value": h * ws / (ms_stitch * 1e-3) / 1e6, "unit": "MP/s", "ms_per_step": ms_stitch},
            "gpu_launches": args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="pair",
                    choices=["pair", "small", "rig", "refine_1024", "blend_coeff", "compose"],
                    help="pair: the 4000x1500 overlap pair (default); small: the 256x512 gray pair; "
                         "rig: the 8-pair 360-degree rig; refine_1024: the differentiable refinement; "
                         "blend_coeff: general-mask Eq. (1); compose: Code 1 on a 4000x3000 canvas")
    ap.add_argument("--no-autotune", action="store_true", help="rig: keep the default tuning")
    ap.add_argument("--pyr-dtype", default="f32", choices=sorted(PYR_DTYPES),
                    help="storage of the pyramid levels (arithmetic stays FP32)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "refine_1024":
        return run_refine(args)
    if args.workload == "rig":
        return run_rig(args)
    if args.workload == "blend_coeff":
        return run_blend_coeff(args)
    if args.workload == "compose":
        return run_compose(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
