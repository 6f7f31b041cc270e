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
# ncu counters of the dominant kernels (DRAM bytes and warp instructions per
# launch), written by `--ingest-ncu` from a capture into profiles/ together
# with a digest of the sources the kernel is compiled from. A counter whose
# digest no longer matches those sources belongs to an older kernel and is
# reported as null.
KERNEL_SOURCES = {
    "lk_stream_kernel": ["paper_2006_01201_gb300/csrc/lk_stream_impl.cuh",
                         "paper_2006_01201_gb300/csrc/lk_stream.cu",
                         "paper_2006_01201_gb300/csrc/common.cuh"],
    "blend_kernel": ["paper_2006_01201_gb300/csrc/blend.cu", "paper_2006_01201_gb300/csrc/common.cuh"],
}
KERNEL_SOURCES["lk_stream_batch_kernel"] = KERNEL_SOURCES["lk_stream_kernel"]
KERNEL_SOURCES["rig_blend_kernel"] = KERNEL_SOURCES["blend_kernel"]
COUNTER_FILES = {  # (kernel, workload) -> file under profiles/
    ("lk_stream_kernel", "pair_4000x1500_rgb_u8_lv6"): "counters_lk_stream_kernel_pair_4000x1500_rgb_u8_lv6.json",
    ("lk_stream_batch_kernel", "rig"): "counters_lk_stream_batch_kernel_rig_8x4000_rgb_u8_lv6.json",
}
# One warp instruction per scheduler per cycle, four schedulers per SM.
SCHEDULERS_PER_SM = 4


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


def path_alg_bytes(h: int, w: int, c: int, levels: int, in_bytes: int = 1, elem: int = 4,
                   reduce_reread: bool = False):
    """Algorithmic bytes of one step of the whole path, each persistent array
    read once and written once (the K steps of a level fused on chip):
      pyramid: read both strips (2 C in_bytes per pixel), write both luma
               pyramids (2 elem per level pixel; a one-channel float strip
               is its own level 0);
      flow:    18 B per direction and level pixel with float32 levels (lk_alg_bytes);
      blend:   read L and R (2 C in_bytes), both flows (16 B), write F (C in_bytes).
    reduce_reread=True also counts each REDUCE re-reading its source level
    (2 elem per pixel of every level but the last)."""
    npx = level_pixels(h, w, levels)
    n = h * w
    own_l0 = c == 1 and in_bytes == 4 and elem == 4
    pyramid = 2 * c * in_bytes * n + 2 * elem * (sum(npx) - (npx[0] if own_l0 else 0))
    if reduce_reread:
        pyramid += 2 * elem * sum(npx[:-1])
    flow = sum(lk_alg_bytes(h, w, levels, elem))
    blend = 2 * c * in_bytes * n + 16 * n + c * in_bytes * n
    return pyramid + flow + blend


def source_digest(files) -> str:
    """SHA-256 over the named repository files (path and contents)."""
    import hashlib
    d = hashlib.sha256()
    for f in files:
        d.update(f.encode())
        with open(os.path.join(ROOT, f), "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()


def read_counters(kernel: str, workload: str, profiles_dir: str = None):
    """ncu counters of `kernel` on `workload` from profiles/, or None when
    there are none or they were taken from other sources than the current ones."""
    name = COUNTER_FILES.get((kernel, workload))
    if not name:
        return None
    try:
        with open(os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), name)) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("kernel") != kernel or d.get("sha256") != source_digest(KERNEL_SOURCES[kernel]):
        return None
    return d


def _unit_scale(unit: str) -> float:
    unit = unit.strip()
    for prefix, f in (("K", 1e3), ("M", 1e6), ("G", 1e9), ("T", 1e12)):
        if len(unit) > 1 and unit.startswith(prefix) and unit[1:] in ("byte", "inst", "cycle", "warp"):
            return f
    return 1.0


def parse_ncu_raw_csv(path: str, kernel: str):
    """Per-launch DRAM bytes, warp instructions and durations of the launches
    of `kernel` (its name, as a whole word before the template or parameter
    list) in an `ncu -i REPORT --page raw --csv` export."""
    import csv
    with open(path, newline="") as f:
        rows = list(csv.reader(f))
    hi = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    head, units = rows[hi], rows[hi + 1]
    col = {n: i for i, n in enumerate(head)}

    def val(r, name):
        i = col.get(name)
        if i is None or i >= len(r) or not r[i].strip():
            return None
        return float(r[i].replace(",", "")) * _unit_scale(units[i])

    import re
    pat = re.compile(r"(^|[\s:])" + re.escape(kernel) + r"[<(]")
    out = []
    for r in rows[hi + 2:]:
        if len(r) <= col["Kernel Name"] or not pat.search(r[col["Kernel Name"]]):
            continue
        rd, wr = val(r, "dram__bytes_read.sum"), val(r, "dram__bytes_write.sum")
        out.append({"name": r[col["Kernel Name"]],
                    "dram_bytes": rd + wr if rd is not None and wr is not None else None,
                    "warp_inst": val(r, "smsp__inst_executed.sum"),
                    "duration_ns": val(r, "gpu__time_duration.sum")})
    return out


def ingest_ncu(csv_path: str, kernel: str, workload: str, command: str, profiles_dir: str = None,
               first: int = 0, count: int = 0, tuning=None) -> str:
    """Write profiles/<counters file> for (kernel, workload) from an ncu raw
    CSV export (its launches first .. first + count - 1, all with count 0),
    stamped with the digest of the kernel's current sources. `tuning`
    records the rig tuning the capture ran with, if any."""
    launches = parse_ncu_raw_csv(csv_path, kernel)
    launches = launches[first:first + count] if count else launches[first:]
    if not launches:
        raise SystemExit(f"no launch of {kernel} in {csv_path}")

    def mean(key):
        v = [x[key] for x in launches if x[key] is not None]
        return sum(v) / len(v) if v else None

    d = {"kernel": kernel, "workload": workload, "sources": KERNEL_SOURCES[kernel],
         "sha256": source_digest(KERNEL_SOURCES[kernel]), "command": command, "launches": launches,
         "dram_bytes_per_launch": mean("dram_bytes"), "warp_inst_per_launch": mean("warp_inst")}
    if tuning is not None:
        d["tuning"] = tuning
    path = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), COUNTER_FILES[(kernel, workload)])
    with open(path, "w") as f:
        json.dump(d, f, indent=1)
        f.write("\n")
    return path


def sm_count(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


RIG_WORKLOAD = {"workload": "rig_8x4000x{800..2000}_rgb_u8_lv6_canvas_9000x4000", "h": 4000,
                "widths": [800, 950, 1100, 1250, 1400, 1600, 1800, 2000], "channels": 3, "levels": 6,
                "iters": 5, "radius": 2, "dmax": 24.0, "canvas": [4000, 9000],
                "canvas_x0": [1125 * k for k in range(8)]}
PANO_LK_AUTO, PANO_LK_STREAM, PANO_LK_TILE = 0, 1, 2
# a rig level's tuning as (kernel, seg_rows, tile_w, tile_h); the default is AUTO everywhere
DEFAULT_TUNING = [PANO_LK_AUTO, 0, 0, 0]


def tuning_key(t) -> list:
    return [int(t["kernel"]), int(t["seg_rows"]), int(t["tile_w"]), int(t["tile_h"])]
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


def issue_roofline(counters, launch_ms: float, sm_mhz, sms: int):
    """Warp-instruction issue rate of a kernel (ncu instruction count per
    launch / live launch time) against the SMs' issue peak at the sampled SM
    clock; None without current counters or a clock sample."""
    inst = counters.get("warp_inst_per_launch") if counters else None
    if not inst or not launch_ms or not sm_mhz:
        return None
    achieved = inst / (launch_ms * 1e-3) / 1e9
    peak = sms * SCHEDULERS_PER_SM * sm_mhz * 1e6 / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp-instr/s", "frac": achieved / peak,
            "inst_per_launch": inst, "kernel": counters["kernel"],
            "peak_source": f"{sms} SMs x 4 schedulers x sampled SM clock",
            "counters": "profiles/" + COUNTER_FILES[(counters["kernel"], counters["workload"])]}


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
    import synth
    # the rig and the 16-bit forms ride along with the default single-GPU line
    extras = world == 1 and args.workload == "pair" and args.pyr_dtype == "f32" and not args.no_rig
    W = RIG_WORKLOAD
    rig_pairs = synth.rig_pairs(h=W["h"], widths=W["widths"], dmax=W["dmax"], levels=W["levels"],
                                workers=min(8, os.cpu_count() or 1)) if extras else None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

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
    # counters of the float32 kernel on this workload (16-bit planes run other kernels)
    counters = read_counters(dominant, WL["workload"]) if args.pyr_dtype == "f32" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None,
                "traffic": counters["dram_bytes_per_launch"] if counters else None, "kernel": dominant,
                "alg_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                "launches_per_step": launches_per_step, "peak_source": f"{peak_src} hbm_gbs",
                "counters": "profiles/" + COUNTER_FILES[(dominant, WL["workload"])] if counters else None}
    issue = issue_roofline(counters, launch_ms, clocks["sm_mhz"] if clocks else None, sm_count(dev))
    in_bytes = pair.L.dtype.itemsize
    path_bytes = path_alg_bytes(h, w, c, levels, in_bytes=in_bytes, elem=elem)
    path_bytes_rr = path_alg_bytes(h, w, c, levels, in_bytes=in_bytes, elem=elem, reduce_reread=True)
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
                "path": {"alg_bytes_per_step": path_bytes, "alg_bytes_per_px": path_bytes / (h * w),
                         "achieved_gbs": path_gbs, "frac": path_gbs / peak,
                         "model": "each persistent array read once, written once; K steps of a level fused",
                         "with_reduce_reread": {"alg_bytes_per_step": path_bytes_rr,
                                                "frac": path_bytes_rr / (total_ms / args.steps * 1e-3) / 1e9 / peak},
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
            if extras:
                line["half"] = {"pair": pair_half_report(pkg, dev, pair, levels, args.steps, args.warmup, value,
                                                         g_lr, g_rl, F.cpu().numpy(), olr, orl)}
            line["cpu_baseline"] = oracle_baseline(pair, levels, args.cpu_budget, f"of the {h}x{w} pair")
            line["cpu_baseline"]["full_pair_flow_s"] = t_full
        if extras:
            oflows = None
            if not args.no_cpu_baseline:
                t0 = time.perf_counter()
                oflows = rig_oracle_flows(rig_pairs, W["levels"])
                t_rig_oracle = time.perf_counter() - t0
            rr = rig_report(dev, rig_pairs, args.steps, args.warmup, oracle_flows=oflows)
            if oflows is not None:
                rr["oracle_flow_s"] = t_rig_oracle
            line.setdefault("half", {})["rig"] = rr.pop("half", None)
            line["rig"] = rr
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


def pair_half_report(pkg, dev, pair, levels, steps, warmup, value32, g_lr, g_rl, g_F, olr, orl):
    """The pair in bfloat16 and binary16 pyramid storage: throughput (same
    loop as the float32 line), flows against the exact FP64 oracle, the
    storage-matched oracle and the float32 GPU path, and F against the float32
    GPU path and the oracle's whole path."""
    import numpy as np
    import torch
    import oracle

    h, w = pair.L.shape[:2]
    c = pair.L.shape[2] if pair.L.ndim == 3 else 1
    L = torch.from_numpy(pair.L).to(dev)
    R = torch.from_numpy(pair.R).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    Fo = oracle.quantize_u8(oracle.blend(pair.L, pair.R, olr, orl, oracle.Params(levels=levels)))
    out = {"fp32_value": value32, "bound": "mean EPE <= 0.05 px per direction against the exact FP64 oracle"}
    for dt in ("bf16", "f16"):
        code, fmt, _ = PYR_DTYPES[dt]
        with pkg.FlowContext(pkg.Params(levels=levels, pyr_dtype=code), max_h=h, max_w=w, max_c=c) as ctx:
            lr = torch.empty((h, w, 2), dtype=torch.float32, device=dev)
            rl = torch.empty((h, w, 2), dtype=torch.float32, device=dev)
            F = torch.empty_like(L)

            def step():
                ctx.flow_pair(L, R, out=(lr, rl), stream=stream)
                ctx.blend_pair(L, R, lr, rl, out=F, stream=stream)

            for _ in range(warmup):
                flush.zero_()
                step()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for k in range(steps):
                flush.zero_()
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a_.elapsed_time(b_) for a_, b_ in ev)
            hlr, hrl, hF = lr.cpu().numpy(), rl.cpu().numpy(), F.cpu().numpy()
        slr, srl = oracle.flow_pair(pair.L, pair.R, oracle.Params(levels=levels, pyr_fmt=fmt))
        d32 = np.abs(hF.astype(int) - g_F.astype(int))
        do = np.abs(hF.astype(int) - Fo.astype(int))
        ex = [mean_epe(hlr, olr), mean_epe(hrl, orl)]
        out[dt] = {"value": throughput(h * w, steps, 1, ms), "unit": UNIT, "ms_per_step": ms / steps,
                   "epe_vs_exact_oracle": ex, "epe_vs_storage_oracle": [mean_epe(hlr, slr), mean_epe(hrl, srl)],
                   "epe_vs_gpu_f32": [mean_epe(hlr, g_lr), mean_epe(hrl, g_rl)],
                   "F_u8_vs_gpu_f32": {"max_lsb": int(d32.max()), "mean_lsb": float(d32.mean()),
                                       "frac_gt_1lsb": float((d32 > 1).mean())},
                   "F_u8_vs_exact_oracle": {"max_lsb": int(do.max()), "mean_lsb": float(do.mean()),
                                            "frac_gt_1lsb": float((do > 1).mean())},
                   "meets_epe_bound": max(ex) <= 0.05}
    return out


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


def measure_rig(dev, pairs, pyr_dtype: str, steps: int, warmup: int, world: int = 1, autotune: bool = True,
                single_pair: bool = True, e2e: bool = True, trace: bool = True, sample_clocks: bool = True,
                local: int = 0):
    """The 360-degree rig: every step one replay of the rig's CUDA graph
    (luma, REDUCE, batched LK per level, blend into the 9000 x 4000 canvas)
    with the strips already in HBM and L2 flushed between steps. Returns the
    measurements and the rig (the caller closes it)."""
    import torch

    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import binding

    W = RIG_WORKLOAD
    h, widths, c, levels = W["h"], W["widths"], W["channels"], W["levels"]
    pyr_code, pyr_fmt, elem = PYR_DTYPES[pyr_dtype]
    params = pkg.Params(levels=levels, iters=W["iters"], radius=W["radius"], pyr_dtype=pyr_code)
    rig = binding.Rig(params, h, widths, c=c, dtype=torch.uint8, canvas_hw=tuple(W["canvas"]),
                      canvas_x0=W["canvas_x0"])
    Ls = [torch.from_numpy(p.L).to(dev) for p in pairs]
    Rs = [torch.from_numpy(p.R).to(dev) for p in pairs]
    canvas = rig.new_canvas(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    npx = h * sum(widths)
    out = {"rig": rig, "canvas": canvas, "Ls": Ls, "Rs": Rs}

    t0 = time.perf_counter()
    tunings = rig.autotune(Ls, Rs, reps=3, stream=stream) if autotune else \
        [rig.get_tuning(l) for l in range(levels)]
    out["autotune"] = {"seconds": time.perf_counter() - t0 if autotune else None, "levels": tunings}

    for _ in range(warmup):
        flush.zero_()
        rig.run(Ls, Rs, canvas=canvas, use_graph=True, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    sampler = ClockSampler(local) if sample_clocks else None
    if sampler:
        sampler.start()
    launches0 = rig.launches
    barrier(world)
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        rig.run(Ls, Rs, canvas=canvas, use_graph=True, stream=stream)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    out["clocks"] = sampler.stop() if sampler else None
    out["launches"] = rig.launches - launches0
    step_ms = [a_.elapsed_time(b_) for a_, b_ in ev]
    total_ms = reduce_max(sum(step_ms), world)
    out.update(value=throughput(npx, steps, world, total_ms), ms_per_step=total_ms / steps, total_ms=total_ms,
               step_ms_min=min(step_ms), step_ms_median=statistics.median(step_ms))
    peak, peak_src = read_peaks()
    path_bytes = sum(path_alg_bytes(h, w, c, levels, elem=elem) for w in widths)
    out["path"] = {"alg_bytes_per_step": path_bytes, "alg_bytes_per_px": path_bytes / npx,
                   "achieved_gbs": path_bytes / (total_ms / steps * 1e-3) / 1e9,
                   "frac": path_bytes / (total_ms / steps * 1e-3) / 1e9 / peak}

    if trace:
        # eager runs with every launch bracketed by events: per-kernel times
        rig.trace_enable(0x3F, 64 * steps)
        for k in range(steps):
            flush.zero_()
            rig.run(Ls, Rs, canvas=canvas, use_graph=False, stream=stream)
        torch.cuda.synchronize()
        recs = rig.trace_read(64 * steps)
        rig.trace_enable(0, 0)
        plan = rig_level_kernels(h, widths, levels, [t["kernel"] for t in tunings],
                                 [(t["tile_w"], t["tile_h"]) for t in tunings])
        names = {1: "luma_kernel", 2: "pyr_down_kernel", 8: "rig_blend_kernel", 16: "luma_reduce_kernel",
                 32: "pyr_tail_kernel"}
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
            d["ms_per_step"] = d["ms"] / steps
        dominant = max(per_kind, key=lambda k: per_kind[k]["ms"])
        dk = per_kind[dominant]
        launch_ms = dk["ms"] / dk["launches"]
        bytes_per_launch = stream_bytes / dk["launches"] if dominant == "lk_stream_batch_kernel" else None
        achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9 if bytes_per_launch else None
        counters = read_counters(dominant, "rig") if pyr_dtype == "f32" else None
        note = None
        if counters and counters.get("tuning") != [tuning_key(t) for t in tunings]:
            # taken with another tuning: other launches, other counts
            counters, note = None, "counters were captured with another tuning"
        out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak if achieved else None, "counters_note": note,
                           "traffic": counters["dram_bytes_per_launch"] if counters else None, "kernel": dominant,
                           "alg_bytes_per_launch": bytes_per_launch, "launch_ms": launch_ms,
                           "launches_per_step": dk["launches"] / steps, "peak_source": f"{peak_src} hbm_gbs",
                           "counters": "profiles/" + COUNTER_FILES[(dominant, "rig")] if counters else None}
        clk = out["clocks"]["sm_mhz"] if out["clocks"] else None
        out["issue_roofline"] = issue_roofline(counters, launch_ms, clk, sm_count(dev))
        out["kernels"] = per_kind
        out["dominant_kernel"] = dominant

    if single_pair:
        # the single-pair form on the same strips: 8 x (flow_pair + blend_pair)
        ctx = pkg.FlowContext(params, max_h=h, max_w=max(widths), max_c=c)
        outs = [(torch.empty((h, w, 2), device=dev), torch.empty((h, w, 2), device=dev),
                 torch.empty_like(Ls[k])) for k, w in enumerate(widths)]

        def pair_step():
            for k in range(len(widths)):
                ctx.flow_pair(Ls[k], Rs[k], out=outs[k][:2], stream=stream)
                ctx.blend_pair(Ls[k], Rs[k], outs[k][0], outs[k][1], out=outs[k][2], stream=stream)

        for _ in range(warmup):
            flush.zero_()
            pair_step()
        torch.cuda.synchronize()
        ev3 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            ev3[k][0].record(stream)
            pair_step()
            ev3[k][1].record(stream)
        torch.cuda.synchronize()
        pair_ms = reduce_max(sum(a_.elapsed_time(b_) for a_, b_ in ev3), world)
        out["single_pair_form"] = {"value": throughput(npx, steps, world, pair_ms), "unit": UNIT,
                                   "ms_per_step": pair_ms / steps}
        # the single-pair flows, to compare with the rig's
        out["single_pair_flows"] = [(o[0].cpu().numpy(), o[1].cpu().numpy()) for o in outs]
        ctx.close()

    if e2e:
        # pinned host strips in, the canvas back to pinned host memory,
        # through the double-buffered host pipeline
        Lh = [torch.from_numpy(p.L).pin_memory() for p in pairs]
        Rh = [torch.from_numpy(p.R).pin_memory() for p in pairs]
        Ch = [torch.empty(tuple(canvas.shape), dtype=canvas.dtype).pin_memory() for _ in range(2)]
        pipe = binding.RigHostPipeline(rig, dev)
        for k in range(max(1, warmup)):
            pipe.submit(k, Lh, Rh, Ch[k % 2])
        pipe.drain()
        e2e_ms, e2e_runs = time_pipeline(pipe, lambda k: pipe.submit(k, Lh, Rh, Ch[k % 2]), steps, world)
        out["e2e"] = {"value": throughput(npx, steps, world, e2e_ms), "unit": UNIT,
                      "h2d_bytes_per_step": int(sum(t.numel() for t in Lh + Rh)),
                      "d2h_bytes_per_step": int(Ch[0].numel()), "ms_per_step": e2e_ms / steps,
                      "pipeline": "two buffer sets; H2D, graph replay and D2H on three streams; "
                                  "no L2 flush (inputs arrive by H2D)",
                      "repeats_ms": e2e_runs, "timing": "median of 3 timed runs of K steps"}
        # the last replay of the pipeline wrote its canvas from the same strips
    return out


def mean_epe(a, b) -> float:
    import numpy as np
    return float(np.hypot(*(a - b).transpose(2, 0, 1)).mean())


def rig_oracle_flows(pairs, levels: int, pyr_fmt: int = 0):
    """FP64 oracle flows of every rig pair (storage format pyr_fmt)."""
    import oracle
    return [oracle.flow_pair(p.L, p.R, oracle.Params(levels=levels, pyr_fmt=pyr_fmt)) for p in pairs]


def rig_report(dev, pairs, steps: int, warmup: int, oracle_flows=None, half: bool = True, autotune: bool = True):
    """The rig object of the default line: the float32 rig (graph replay,
    per-kernel times, roofline, single-pair form, end to end), the EPE of
    every pair against the oracle and the single-pair path, and (half=True)
    the bfloat16 and binary16 rigs with their errors."""
    import numpy as np

    W = RIG_WORKLOAD
    levels = W["levels"]
    m = measure_rig(dev, pairs, "f32", steps, warmup, autotune=autotune)
    rig = m.pop("rig")
    g32 = [tuple(t.cpu().numpy() for t in rig.flows(k)) for k in range(len(pairs))]
    canvas32 = m.pop("canvas").cpu().numpy()
    sp = m.pop("single_pair_flows", None)
    Ls, Rs = m.pop("Ls"), m.pop("Rs")
    rig.close()
    if autotune:
        # the same rig with the default tuning of every level: the tuning the
        # committed ncu counters of the batch kernel were captured with
        md = measure_rig(dev, pairs, "f32", steps, warmup, autotune=False, single_pair=False, e2e=False,
                         sample_clocks=True)
        md.pop("rig").close()
        m["default_tuning"] = {k: md[k] for k in ("value", "ms_per_step", "roofline", "issue_roofline", "kernels",
                                                  "dominant_kernel", "clocks")}
        m["default_tuning"]["unit"] = UNIT
    m["npx"] = W["h"] * sum(W["widths"])
    m["config"] = dict(W, graph=True, l2="flushed between steps (256 MB write, untimed); inputs 262 MB > L2")
    m["epe_per_pair"] = []
    converges = [True] * len(pairs)
    if oracle_flows is not None:
        for k, (lr, rl) in enumerate(g32):
            olr, orl = oracle_flows[k]
            # how far the method itself lands from the generator's field (FlowRtoL):
            # with the uncorrected colour gain some pairs' flows wander off (measured
            # 0.3 - 2.2 px on five pairs, 10 - 23 px on the other three)
            truth = mean_epe(orl, pairs[k].flow_RtoL)
            converges[k] = truth <= 5.0
            row = {"pair": k, "w": W["widths"][k], "vs_oracle": [mean_epe(lr, olr), mean_epe(rl, orl)],
                   "oracle_RtoL_vs_truth": truth, "converges": converges[k]}
            if sp is not None:
                row["vs_single_pair_max_abs"] = [float(np.abs(lr - sp[k][0]).max()),
                                                 float(np.abs(rl - sp[k][1]).max())]
            m["epe_per_pair"].append(row)
        m["epe_vs_oracle_max_mean"] = max(max(r["vs_oracle"]) for r in m["epe_per_pair"])
    if half:
        m["half"] = {}
        for dt in ("bf16", "f16"):
            mh = measure_rig(dev, pairs, dt, steps, warmup, autotune=autotune, single_pair=False, e2e=False,
                             trace=False, sample_clocks=False)
            rh = mh.pop("rig")
            gh = [tuple(t.cpu().numpy() for t in rh.flows(k)) for k in range(len(pairs))]
            ch = mh.pop("canvas").cpu().numpy()
            rh.close()
            d = np.abs(ch.astype(int) - canvas32.astype(int))
            entry = {"value": mh["value"], "unit": UNIT, "ms_per_step": mh["ms_per_step"],
                     "fp32_value": m["value"], "canvas_u8_vs_fp32_rig": {"max_lsb": int(d.max()),
                                                                           "mean_lsb": float(d.mean()),
                                                                           "frac_gt_1lsb": float((d > 1).mean())},
                     "per_pair": []}
            _, pyr_fmt, _ = PYR_DTYPES[dt]
            stored = rig_oracle_flows(pairs, levels, pyr_fmt) if oracle_flows is not None else None
            for k, (lr, rl) in enumerate(gh):
                row = {"pair": k, "vs_gpu_f32": [mean_epe(lr, g32[k][0]), mean_epe(rl, g32[k][1])]}
                if oracle_flows is not None:
                    row["vs_exact_oracle"] = [mean_epe(lr, oracle_flows[k][0]), mean_epe(rl, oracle_flows[k][1])]
                    row["vs_storage_oracle"] = [mean_epe(lr, stored[k][0]), mean_epe(rl, stored[k][1])]
                entry["per_pair"].append(row)
            if oracle_flows is not None:
                worst = max(max(r["vs_exact_oracle"]) for r in entry["per_pair"])
                entry["epe_vs_exact_oracle_max_mean"] = worst
                entry["meets_epe_bound"] = worst <= 0.05
                conv = [max(r["vs_exact_oracle"]) for k, r in enumerate(entry["per_pair"]) if converges[k]]
                entry["converging_pairs"] = [k for k in range(len(pairs)) if converges[k]]
                entry["epe_vs_exact_oracle_max_mean_converging"] = max(conv) if conv else None
                entry["meets_epe_bound_on_converging_pairs"] = bool(conv) and max(conv) <= 0.05
            m["half"][dt] = entry
    return m


def run_rig(args):
    """The 360-degree rig: 8 RGB u8 pairs of 4000 x {800..2000}, 6 levels,
    every step one replay of the rig's CUDA graph (luma, REDUCE, batched LK
    per level, blend into the 9000 x 4000 canvas). The single-pair form
    (pano_flow_pair + pano_blend_pair per pair) is timed beside it."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    import synth
    W = RIG_WORKLOAD
    h, widths, c, levels = W["h"], W["widths"], W["channels"], W["levels"]
    # generated before the first CUDA call, in spawned processes
    pairs = synth.rig_pairs(h=h, widths=widths, dmax=W["dmax"], levels=levels, seed0=100 + 8 * rank,
                            workers=min(8, os.cpu_count() or 1))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2006_01201_gb300 as pkg
    from paper_2006_01201_gb300 import build as gpu_build

    gpu_build.build()
    pkg.load_library()
    pyr_code, pyr_fmt, elem = PYR_DTYPES[args.pyr_dtype]
    m = measure_rig(dev, pairs, args.pyr_dtype, args.steps, args.warmup, world=world,
                    autotune=not args.no_autotune, local=local)
    rig, canvas = m["rig"], m["canvas"]
    fp32_form = None
    canvas32 = None
    if pyr_fmt:
        # the float32 batched form beside the 16-bit one, tuned the same way
        m32 = measure_rig(dev, pairs, "f32", args.steps, args.warmup, world=world, autotune=not args.no_autotune,
                          single_pair=False, e2e=False, trace=False, sample_clocks=False, local=local)
        fp32_form = {"value": m32["value"], "unit": UNIT, "ms_per_step": m32["ms_per_step"]}
        canvas32 = m32["canvas"]
        m32["rig"].close()

    line = None
    if rank == 0:
        line = {"metric": METRIC.replace("(bi-flow+warp+blend)", "(bi-flow+warp+blend, 8-pair rig)"),
                "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(W, l2="flushed between steps (256 MB write, untimed); inputs 262 MB > L2",
                               parallelism=f"replicas{world}", graph=True, pyr_dtype=args.pyr_dtype),
                "roofline": m["roofline"], "issue_roofline": m["issue_roofline"], "path": m["path"],
                "kernels": m["kernels"], "dominant_kernel": m["dominant_kernel"],
                "single_pair_form": m["single_pair_form"], "fp32_batched_form": fp32_form,
                "paper_context": PAPER_CONTEXT, "autotune": m["autotune"],
                "e2e": m["e2e"], "gpu_launches": m["launches"], "clocks": m["clocks"],
                "step_ms_min": m["step_ms_min"], "step_ms_median": m["step_ms_median"]}
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            oracle.build()
            olr, orl = oracle.flow_pair(pairs[0].L, pairs[0].R, oracle.Params(levels=levels))
            g_lr, g_rl = (t.cpu().numpy() for t in rig.flows(0))
            line["epe_vs_oracle"] = {"pair": 0, "LtoR_mean_px": mean_epe(g_lr, olr),
                                     "RtoL_mean_px": mean_epe(g_rl, orl)}
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
            line["cpu_baseline"]["rig_step_s_extrapolated"] = h * sum(widths) / 1e6 / line["cpu_baseline"]["value"]
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
    ap.add_argument("--no-rig", action="store_true",
                    help="pair: leave out the rig and the 16-bit forms that the default line carries")
    ap.add_argument("--ingest-ncu", metavar="CSV",
                    help="write the profiles/ counters of --counters-kernel from an `ncu -i REPORT --page raw "
                         "--csv --print-units base` export (no GPU needed) and exit")
    ap.add_argument("--counters-kernel", default="lk_stream_kernel")
    ap.add_argument("--counters-workload", default=WORKLOAD["workload"])
    ap.add_argument("--counters-command", default="", help="the capture command, recorded with the counters")
    ap.add_argument("--counters-launches", default="0:0", help="first:count of the captured launches to keep")
    ap.add_argument("--counters-default-tuning", action="store_true",
                    help="record that the rig ran with the default tuning of every level")
    ap.add_argument("--pyr-dtype", default="f32", choices=sorted(PYR_DTYPES),
                    help="storage of the pyramid levels (arithmetic stays FP32)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.ingest_ncu:
        first, count = (int(v) for v in args.counters_launches.split(":"))
        tuning = [DEFAULT_TUNING] * RIG_WORKLOAD["levels"] if args.counters_default_tuning else None
        print(ingest_ncu(args.ingest_ncu, args.counters_kernel, args.counters_workload, args.counters_command,
                         first=first, count=count, tuning=tuning))
        return 0
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
