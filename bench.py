"""Benchmark: exhaustive PIFS range-domain search on one 512x512 12-bit CT-like slice.

One step = one complete fic_encode of the slice (prep, search, exact
re-score, fallback, map output): 4096 ranges x 15625 domains x 8 symmetries
= 5.12e8 range-domain comparisons.  Metric: comparisons/s (and ms per slice).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank encodes its own slice (weak scaling, no
collective on the data path); the time is the max over ranks.  The reference
arm (--impl reference) times the FP64 CPU oracle on a bounded sample of the
same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fic_synth  # noqa: E402

N_PIX, RANGE, STRIDE, BITS = 512, 8, 4, 12
WORKLOAD = ("512x512 12-bit CT-like synthetic slice; 8x8 ranges (4096); 16x16 domains at stride 4 "
            "(15625) x 8 symmetries; s 5-bit, o 7-bit")
METRIC = "range-domain comparisons/s"
CLOCK_WINDOW_S = 1.0
# untimed warm-up: the W steps asked for, and more of the same step until this
# much wall time has passed (a fresh process's first fraction of a second of
# GPU work runs slower than the steady state)
WARMUP_MIN_S = 0.3
# FP32 operations of the screening key per candidate (the epilogue's
# algorithmic work): s code 4 (scale + saturate, map to the code grid, round
# by magic add, subtract), o residue 4 (z, e: scale + round, w), key 4
# (c*kappa - X, times c, lambda*w*w as a multiply and a fused add), test 1
EPI_OPS_PER_CANDIDATE = 13


def comparisons():
    R = (N_PIX // RANGE) ** 2
    D = ((N_PIX - 2 * RANGE) // STRIDE + 1) ** 2
    return R, D, R * D * 8


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def warm_up(step, w, sync):
    """W untimed steps (at least 3), continued until WARMUP_MIN_S of wall time
    has passed; returns the number of steps run."""
    n, t0 = 0, time.time()
    while n < max(3, w) or time.time() - t0 < WARMUP_MIN_S:
        step()
        n += 1
        if n % 16 == 0:
            sync()
    sync()
    return n


def rank_seed(rank):
    """Every rank encodes its own slice: independent problems, no exchange
    step (weak scaling; the replicas share nothing but the timing)."""
    return fic_synth.CT_SEED + rank


def max_over_ranks(t, ws, device=None):
    """The job's time is its slowest rank's: an all-reduce MAX over the ranks."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_rate(ws, steps, units_per_step, t):
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return ws * steps * units_per_step / t


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def sm_count(dev):
    import torch

    return torch.cuda.get_device_properties(dev).multi_processor_count


def search_traffic():
    """DRAM bytes (read + write) per launch of the tensor-core search from the
    committed ncu capture, or None when the kernel source has changed since."""
    import hashlib

    try:
        with open(os.path.join(ROOT, "profiles", "k_search_tc_ct512.txt")) as fh:
            f = fh.read().split()
        src = os.path.join(ROOT, "paper_1404_0774_gb300", "csrc")
        h = hashlib.sha256()
        for name in ("fic_search_tc.cu", "fic_internal.cuh"):
            with open(os.path.join(src, name), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != f[3]:
            return None
        return int(f[1])
    except (OSError, IndexError, ValueError):
        return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def shadow_mask(img, n):
    """Per range (row-major), whether the n x n block is constant (a shadow
    range: Section V decides it without a search)."""
    h, w = img.shape
    b = img.reshape(h // n, n, w // n, n).transpose(0, 2, 1, 3).reshape(-1, n * n)
    return b.max(1) == b.min(1)


def flat_domains(img, n, t):
    """Number of 2n x 2n domains at stride t whose 2x2-sum block is constant
    (flat: zero variance, s = 0 for every candidate)."""
    from numpy.lib.stride_tricks import sliding_window_view

    q = img.astype(np.int64)
    q = q[0::2, 0::2] + q[1::2, 0::2] + q[0::2, 1::2] + q[1::2, 1::2]
    win = sliding_window_view(q, (n, n))[:: t // 2, :: t // 2] if t % 2 == 0 else None
    if win is None:  # odd stride: domains do not start on the 2x2 grid of q
        h, w = img.shape
        cnt = 0
        for v in range((h - 2 * n) // t + 1):
            for u in range((w - 2 * n) // t + 1):
                blk = img[v * t: v * t + 2 * n, u * t: u * t + 2 * n].astype(np.int64)
                qq = blk[0::2, 0::2] + blk[1::2, 0::2] + blk[0::2, 1::2] + blk[1::2, 1::2]
                cnt += int(qq.max() == qq.min())
        return cnt
    nd_y = (img.shape[0] - 2 * n) // t + 1
    nd_x = (img.shape[1] - 2 * n) // t + 1
    win = win[:nd_y, :nd_x]
    return int((win.max(axis=(2, 3)) == win.min(axis=(2, 3))).sum())


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform

    return platform.processor() or platform.machine()


def psnr_db(ref, x, bits):
    """10 log10(P^2 / MSE) of a decoded image against the original (FP64)."""
    P = float((1 << bits) - 1)
    mse = float(np.mean((np.asarray(x, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(P * P / mse)


def cpu_oracle_baseline(img):
    """The FP64 oracle on the host cores: the whole slice (every range, all
    125000 candidates each; seconds on a many-core host) on all threads, its
    maps decoded by the oracle decoder (10 iterations from 2^(B-1)) for the
    PSNR the GPU arms must match; and single-threaded on the 256x256 8-bit
    MR-like slice (8x8 ranges, domains at stride 8)."""
    import oracle

    oracle.build()
    R, D, _ = comparisons()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.encode(img, n=RANGE, t=STRIDE, bit_depth=BITS, threads=cores)
    dt = time.perf_counter() - t0
    P = float((1 << BITS) - 1)
    x = oracle.decode(ref["d"], ref["k"], ref["c"] / 15.0, ref["e"] * P / 63.0, N_PIX, N_PIX, n=RANGE, t=STRIDE,
                      bit_depth=BITS, iters=10)
    mr = fic_synth.mr_slice()
    t1 = time.perf_counter()
    oracle.encode(mr, n=8, t=8, bit_depth=8, threads=1)
    dt1 = time.perf_counter() - t1
    r1, d1 = oracle.counts(256, 256, 8, 8)
    return {"value": R * D * 8 / dt, "unit": "comparisons/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "ms_per_step": 1e3 * dt,
            "sample": f"the whole 512x512 slice: {R} ranges x {D * 8} candidates, {dt:.1f} s wall on {cores} threads",
            "single_thread_mr256": {"ms": 1e3 * dt1, "comparisons_per_s": r1 * d1 * 8 / dt1,
                                    "workload": "256x256 8-bit MR-like slice, 8x8 ranges, domains at stride 8"}}, \
        psnr_db(img, x, BITS), ref


def cpu_oracle_volume(stack, target_s=15.0):
    """The FP64 oracle on the host cores for the stack: per slice size, a
    sample of ranges of one slice (evenly spaced, all candidates each), scaled
    to whole slices; value in slices/s of the whole 96-slice mix."""
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    sizes = sorted({a.shape[0] for a in stack})
    per_slice, notes = {}, []
    for sz in sizes:
        a = next(x for x in stack if x.shape[0] == sz)
        R, D = oracle.counts(sz, sz, RANGE, STRIDE)
        k = 48
        sel = np.linspace(0, R - 1, k).astype(np.int32)
        t0 = time.perf_counter()
        oracle.encode(a, n=RANGE, t=STRIDE, bit_depth=BITS, ranges=sel, threads=cores)
        dt = time.perf_counter() - t0
        k2 = int(min(R, max(k, k * (target_s / len(sizes)) / max(dt, 1e-3))))
        sel = np.linspace(0, R - 1, k2).astype(np.int32)
        t0 = time.perf_counter()
        oracle.encode(a, n=RANGE, t=STRIDE, bit_depth=BITS, ranges=sel, threads=cores)
        dt = time.perf_counter() - t0
        per_slice[sz] = dt * R / k2
        notes.append(f"{sz}x{sz}: {k2} of {R} ranges in {dt:.1f} s")
    counts = {sz: sum(1 for x in stack if x.shape[0] == sz) for sz in sizes}
    t_stack = sum(counts[sz] * per_slice[sz] for sz in sizes)
    return {"value": len(stack) / t_stack, "unit": "slices/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "ms_per_step": 1e3 * t_stack,
            "sample": "per size, evenly spaced ranges of one slice (all candidates each) scaled to whole slices: "
                      + "; ".join(notes)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    img = fic_synth.ct_slice()
    R, D, comps = comparisons()
    import oracle

    oracle.build()
    cores = os.cpu_count() or 1
    per_step = 64  # ranges per step (bounded sample)
    times = []
    for s in range(args.warmup + args.steps):
        sel = ((np.arange(per_step) * 61 + s * 7) % R).astype(np.int32)
        t0 = time.perf_counter()
        oracle.encode(img, n=RANGE, t=STRIDE, bit_depth=BITS, ranges=sel, threads=cores)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.sum(times))
    value = args.steps * per_step * D * 8 / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "comparisons/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"{per_step} ranges of the slice x 125000 candidates each",
                       "sample_ranges_per_step": per_step,
                       "ms_per_slice_extrapolated": 1e3 * t / args.steps * R / per_step},
            "cpu_baseline": {"value": value, "unit": "comparisons/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{per_step} ranges x 125000 candidates per step"},
            "e2e": {"value": value, "unit": "comparisons/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


QT_WORKLOAD = ("512x512 12-bit CT-like synthetic slice; adaptive quadtree: 16x16 ranges split to 8x8 and 4x4 "
               "while the collage RMS exceeds 8.0; domains 2n x 2n at stride n, 8 symmetries; s 5-bit, o 7-bit")


def quadtree_comparisons(fic, stats):
    """Range-domain comparisons of one quadtree encode: per level, screened
    ranges x domains x 8 (from the library's per-level statistics)."""
    total, per_level = 0, []
    for lvl in range(int(stats[0])):
        n = 16 >> lvl
        _, D = fic.counts(N_PIX, N_PIX, fic.params(range_size=n, domain_stride=n, bit_depth=BITS))
        c = int(stats[3 + 4 * lvl]) * D * 8
        per_level.append({"range_size": n, "ranges": int(stats[3 + 4 * lvl]), "leaves": int(stats[4 + 4 * lvl]),
                          "domains": D, "comparisons": c,
                          "search": {1: "tc", 2: "simt"}.get(int(stats[1 + 4 * lvl]), "?"),
                          "cta_target": int(stats[2 + 4 * lvl])})
        total += c
    return total, per_level


def run_quadtree(args):
    """Adaptive quadtree encode of the 512x512 CT slice: one step = one
    fic_encode_quadtree (3 levels, each an encode over its active ranges,
    plus the split and gather kernels; the call waits for its stream)."""
    import torch

    import __graft_entry__

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    img_np = fic_synth.ct_slice(rank_seed(rank))
    p = fic.params(range_size=16, domain_stride=16, bit_depth=BITS)
    img = torch.from_numpy(img_np.astype(np.int16)).to(dev)
    work = torch.empty(fic.quadtree_workspace_size(N_PIX, N_PIX, p, 4), dtype=torch.uint8, device=dev)
    cap = (N_PIX // 4) ** 2
    maps = torch.empty(cap * fic.QMAP_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        return fic.encode_quadtree(img, p, 4, 8.0, maps=maps, workspace=work, stream=stream)[1]

    # the first call also times the launch shapes of each level
    n_warm = warm_up(step, args.warmup, torch.cuda.synchronize)
    comps, per_level = quadtree_comparisons(fic, fic.last_quadtree_stats())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_clk = time.time()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            n_leaves = step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        while time.time() - t_clk < CLOCK_WINDOW_S:
            flush.zero_()
            step()
        torch.cuda.synchronize()
        clk_window = time.time() - t_clk
    t_total = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    t_total = max_over_ranks(t_total, ws, dev)
    value = job_rate(ws, args.steps, comps, t_total)
    # the search of each level timed alone: events the library records around
    # each level's search launch on the stream (FIC_FLAG_PHASE_TIMING)
    pt = fic.params(range_size=16, domain_stride=16, bit_depth=BITS, flags=fic.FIC_FLAG_PHASE_TIMING)
    lvl_ms = []
    for _ in range(max(5, min(args.steps, 20))):
        flush.zero_()
        fic.encode_quadtree(img, pt, 4, 8.0, maps=maps, workspace=work, stream=stream)
        lvl_ms.append(fic.last_quadtree_phase_ms())
    lvl_ms = np.median(np.array(lvl_ms), axis=0)
    leaves = fic.qmaps_to_numpy(maps, int(n_leaves))
    for lvl, d in enumerate(per_level):
        d["search_ms"] = float(lvl_ms[lvl])
        # screened candidates of the level: its active ranges that are not
        # constant (shadow) x its domains that are not flat x 8
        n = d["range_size"]
        sh = shadow_mask(img_np, n)
        nx = N_PIX // n
        act = np.zeros((N_PIX // n) ** 2, bool)
        for j in range(lvl, 3):  # leaves at this level and below descend from the level's active ranges
            sel = leaves[leaves["level"] == j]
            act[(sel["y"] // n) * nx + sel["x"] // n] = True
        d["screened"] = int((act & ~sh).sum()) * (d["domains"] - flat_domains(img_np, n, n)) * 8
    top = int(np.argmax(lvl_ms[: len(per_level)]))
    peaks, peak_kind = load_peaks()
    alu_peak = sm_count(dev) * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    d = per_level[top]
    kern_s = d["search_ms"] * 1e-3
    if d["search"] == "tc":
        ops = EPI_OPS_PER_CANDIDATE
        roof = {"bound": "alu", "achieved": d["screened"] * ops / kern_s / 1e12, "peak": alu_peak, "unit": "Tops/s",
                "ops_per_unit": ops,
                "tensor": {"bound": "tensor", "achieved": d["screened"] * 2 * d["range_size"] ** 2 / kern_s / 1e12,
                           "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "flops_per_unit": 2 * d["range_size"] ** 2}}
        roof["tensor"]["frac"] = roof["tensor"]["achieved"] / roof["tensor"]["peak"]
    else:
        ops = d["range_size"] ** 2 + EPI_OPS_PER_CANDIDATE
        roof = {"bound": "alu", "achieved": d["screened"] * ops / kern_s / 1e12, "peak": alu_peak, "unit": "Tops/s",
                "ops_per_unit": ops}
    roof.update({"frac": roof["achieved"] / roof["peak"], "units": d["screened"], "traffic": None,
                 "kernel": f"search of level {top} ({d['range_size']}x{d['range_size']} ranges, {d['search']})",
                 "peak_source": peak_kind + "; FP32 lanes x max clock for the ALU view",
                 "search_ms_per_level": [float(x) for x in lvl_ms[: len(per_level)]]})
    # end to end from pinned host memory through the C ABI (image in, leaves out;
    # uint16 views of the pinned buffers, so that the binding passes them as
    # they are)
    h_img_t = torch.from_numpy(img_np.astype(np.int16)).pin_memory()
    h_img = h_img_t.numpy().view(np.uint16)
    h_maps_t = torch.zeros(cap * fic.QMAP_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    h_maps = h_maps_t.numpy().view(fic.QMAP_DTYPE)
    for _ in range(2):
        fic.encode_quadtree(h_img, p, 4, 8.0, maps=h_maps, workspace=work, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        fic.encode_quadtree(h_img, p, 4, 8.0, maps=h_maps, workspace=work, stream=stream)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    clocks = clk.summary()
    clocks["window_s"] = clk_window
    clocks["note"] = "sampled over the timed steps and the identical steps that follow them"
    line = {"metric": METRIC, "value": value, "unit": "comparisons/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp16+fp32", "data": "synthetic",
            "config": {"workload": QT_WORKLOAD, "leaves": int(n_leaves), "comparisons_per_step": comps,
                       "levels": per_level, "l2": "flushed (256 MB write) between steps",
                       "warmup_untimed": {"steps": n_warm, "min_s": WARMUP_MIN_S}},
            "e2e": {"value": job_rate(ws, args.steps, comps, e2e_t), "unit": "comparisons/s",
                    "h2d_bytes_per_step": N_PIX * N_PIX * 2, "d2h_bytes_per_step": int(n_leaves) * 56,
                    "timing": "host wall clock (the call waits for its stream)"},
            # per level the encode kernels (five; six for 16x16 ranges, whose
            # compaction and seed keep a launch of their own) and the split
            # test; then the leaf count and the leaf gather
            "gpu_launches": args.steps * (sum((7 if d["range_size"] == 16 else 6) for d in per_level) + 2),
            "clocks": clocks, "roofline": roof}
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            import oracle

            oracle.build()
            t0 = time.perf_counter()
            lv = oracle.encode_quadtree(img_np, 16, 4, 8.0, bit_depth=BITS)
            tc = time.perf_counter() - t0
            oc = 0
            for lvl in range(3):
                n = 16 >> lvl
                _, D = oracle.counts(N_PIX, N_PIX, n, n)
                # ranges searched at this level: leaves there plus the split ones (4 children each below)
                below = sum(int(np.sum(lv["level"] == j)) / 4 ** (j - lvl) for j in range(lvl + 1, 3))
                oc += int(round(np.sum(lv["level"] == lvl) + below)) * D * 8
            line["cpu_baseline"] = {"value": oc / tc, "unit": "comparisons/s", "cores": os.cpu_count() or 1,
                                    "kind": "oracle", "sample": f"the whole quadtree encode of the slice, {tc:.1f} s"}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


VOL_WORKLOAD = ("12-bit CT-like synthetic stack: 32 slices at 256x256, 32 at 384x384, 32 at 512x512; 8x8 ranges, "
                "16x16 domains at stride 4, 8 symmetries; s 5-bit, o 7-bit; one batch (one CUDA graph) per step")


def batch_launches(sizes, parts=6):
    """Kernel launches of one batched encode: the slices sorted by size are
    dealt round-robin to `parts` concurrent pipelines; in each, the
    statistics, compaction + seed, operand row and output kernels run once per
    group of equal-sized slices, the search, re-score and exact scans once."""
    order = sorted(sizes, reverse=True)
    total = 0
    for k in range(min(parts, len(order))):
        part = order[k::parts]
        total += 4 * len(set(part)) + 3
    return total


def run_volume(args):
    """Batched volume: one step = fic_encode_batch of the whole 96-slice stack
    (a replay of its CUDA graph).  Reports slices/s and the latency of one
    batch replay over the timed replays (p50/p99): every stage covers all
    slices, so a slice's maps are ready when its batch is."""
    import torch

    import __graft_entry__

    ws_n, rank, local = dist_env()
    if ws_n > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    stack = fic_synth.ct_stack(fic_synth.CT_SEED + 7919 * rank)
    p = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS)
    # every slice's image and maps are views of one device buffer each, so that
    # the end-to-end leg moves the stack in and the maps out with one copy each
    npix = [a.size for a in stack]
    nmap = [(a.shape[0] // RANGE) ** 2 * 40 for a in stack]
    img_all = torch.from_numpy(np.concatenate([a.astype(np.int16).ravel() for a in stack])).to(dev)
    maps_all = torch.empty(sum(nmap), dtype=torch.uint8, device=dev)
    imgs, maps = [], []
    o = 0
    for a, k in zip(stack, npix):
        imgs.append(img_all[o:o + k].view(a.shape))
        o += k
    o = 0
    for k in nmap:
        maps.append(maps_all[o:o + k])
        o += k
    tab = fic.slice_table(imgs, maps)
    work = torch.empty(fic.batch_workspace_size(tab, p), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    comps = 0
    for a in stack:
        R, D = fic.counts(a.shape[1], a.shape[0], p)
        comps += R * D * 8
    # the first call runs eagerly and captures the graph
    n_warm = warm_up(lambda: fic.encode_batch(tab, p, work, stream), args.warmup, torch.cuda.synchronize)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    lat = []
    if ws_n > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_clk = time.time()
        for i in range(args.steps):
            ev[i][0].record(stream)
            fic.encode_batch(tab, p, work, stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        while time.time() - t_clk < CLOCK_WINDOW_S:
            fic.encode_batch(tab, p, work, stream)
            torch.cuda.synchronize()
        clk_window = time.time() - t_clk
    t_total = float(np.sum([a.elapsed_time(b) for a, b in ev])) / 1e3
    t_total = max_over_ranks(t_total, ws_n, dev)
    n_sl = len(stack)
    value = job_rate(ws_n, args.steps, n_sl, t_total)
    # latency of a whole batch (every slice's maps are ready when its batch
    # is): events around each of >= 20 separate replays, each waited for
    for _ in range(max(20, args.steps)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fic.encode_batch(tab, p, work, stream)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    # end to end: pinned host stack -> device, batch, maps -> pinned host (one
    # copy each way: the slices sit side by side in one pinned buffer)
    h_img_all = img_all.cpu().pin_memory()
    h_maps_all = torch.empty(maps_all.numel(), dtype=torch.uint8).pin_memory()
    h2d = h_img_all.numel() * 2
    d2h = maps_all.numel()

    def e2e_step():
        img_all.copy_(h_img_all, non_blocking=True)
        fic.encode_batch(tab, p, work, stream)
        h_maps_all.copy_(maps_all, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_t = e0.elapsed_time(e1) / 1e3
    clocks = clk.summary()
    clocks["window_s"] = clk_window
    clocks["note"] = "sampled over the timed steps and the identical steps that follow them"
    lat = np.array(lat)
    # the batch's screened candidates (shadow ranges and flat domains are
    # decided without a cross term); ALU view of the whole batch: the
    # screening key's FP32 operations over the batch's time (the search is
    # the largest stage, not the only one, so this bounds its fraction from below)
    screened = 0
    for a in stack:
        R, D = fic.counts(a.shape[1], a.shape[0], p)
        screened += (R - int(shadow_mask(a, RANGE).sum())) * (D - flat_domains(a, RANGE, STRIDE)) * 8
    peaks, peak_kind = load_peaks()
    alu_peak = sm_count(dev) * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    step_s = t_total / args.steps
    roof = {"bound": "alu", "achieved": screened * EPI_OPS_PER_CANDIDATE / step_s / 1e12, "peak": alu_peak,
            "unit": "Tops/s", "ops_per_unit": EPI_OPS_PER_CANDIDATE, "units": screened, "traffic": None,
            "kernel": "whole batch (one graph replay: statistics, compaction, rows, search, re-score, scans, output)",
            "peak_source": peak_kind + "; FP32 lanes x max clock",
            "tensor": {"bound": "tensor", "achieved": screened * 2 * RANGE * RANGE / step_s / 1e12,
                       "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "flops_per_unit": 2 * RANGE * RANGE}}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["tensor"]["frac"] = roof["tensor"]["achieved"] / roof["tensor"]["peak"]
    line = {"metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": ws_n, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp16+fp32", "data": "synthetic",
            "config": {"workload": VOL_WORKLOAD, "slices": n_sl, "comparisons_per_step": comps,
                       "warmup_untimed": {"steps": n_warm, "min_s": WARMUP_MIN_S},
                       "comparisons_per_s": job_rate(ws_n, args.steps, comps, t_total),
                       "slice_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                            "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                                            "replays": int(lat.size),
                                            "note": "per-replay latency of the batch (CUDA events around each "
                                                    "replay, run one at a time): every stage covers all slices, "
                                                    "so each slice's maps are ready when its batch is"},
                       "screened_comparisons_per_step": screened,
                       "l2": "working set of the batch (several GB) is larger than L2"},
            "e2e": {"value": job_rate(ws_n, args.steps, n_sl, e2e_t), "unit": "slices/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps * batch_launches([a.shape[0] * a.shape[1] for a in stack]), "clocks": clocks,
            "roofline": roof}
    if rank == 0:
        if ws_n == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_oracle_volume(stack)
        print(json.dumps(line), flush=True)
    if ws_n > 1:
        dist.destroy_process_group()


REF_WORKLOAD = ("512x512 12-bit CT-like synthetic slice encoded as the slice workload; s and o as FP32 refined by "
                "Adam (lr 2e-3 on s and o/P) for 200 steps on the MSE of an unrolled 8-iteration decode, adjoint "
                "kernels, iterates checkpointed every 2")


def cpu_oracle_refine(img_np, maps, fic, s0, o0, iters, lr, budget_s=8.0):
    """The FP64 oracle's refinement step on the host: the loss of the unrolled
    decode and its gradient by the adjoint (oracle.refine_grad, one thread),
    then the same Adam update in numpy, repeated for about budget_s seconds
    from the encode's coefficients.  Returns the cpu_baseline record."""
    import oracle

    oracle.build()
    m = fic.maps_to_numpy(maps)
    dom = m["domain_idx"].astype(np.int32)
    sym = m["iso"].astype(np.int32)
    s = s0.double().cpu().numpy().copy()
    o = o0.double().cpu().numpy().copy()
    P = float((1 << BITS) - 1)
    ref = img_np.astype(np.float64)
    ms, vs = np.zeros_like(s), np.zeros_like(s)
    mo, vo = np.zeros_like(o), np.zeros_like(o)
    b1, b2, eps = 0.9, 0.999, 1e-8
    k, t0 = 0, time.time()
    while k < 3 or time.time() - t0 < budget_s:
        _, gs, go = oracle.refine_grad(dom, sym, s, o, ref, n=RANGE, t=STRIDE, bit_depth=BITS, iters=iters)
        k += 1
        go = go * P  # the offset is optimised as o / P
        ms = b1 * ms + (1 - b1) * gs
        vs = b2 * vs + (1 - b2) * gs * gs
        mo = b1 * mo + (1 - b1) * go
        vo = b2 * vo + (1 - b2) * go * go
        s -= lr * (ms / (1 - b1 ** k)) / (np.sqrt(vs / (1 - b2 ** k)) + eps)
        o -= P * lr * (mo / (1 - b1 ** k)) / (np.sqrt(vo / (1 - b2 ** k)) + eps)
    dt = time.time() - t0
    return {"value": k / dt, "unit": "steps/s", "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
            "ms_per_step": 1e3 * dt / k,
            "sample": "%d refinement steps of the slice (FP64 loss and adjoint gradient of the %d-iteration "
                      "unrolled decode, Adam in numpy), %.1f s on one thread" % (k, iters, dt)}


def run_refine(args):
    """Differentiable refinement: one step = forward (8 unrolled iterations),
    loss, reverse sweep (adjoint), Adam update -- one CUDA graph replay."""
    import torch

    import __graft_entry__

    ws_n, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    img_np = fic_synth.ct_slice(rank_seed(rank))
    p = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS)
    img = torch.from_numpy(img_np.astype(np.int16)).to(dev)
    maps = fic.encode(img, p)
    s0, o0 = fic.map_coefficients(maps)
    T, steps, lr = 8, 200, 2e-3
    work = torch.empty(fic.refine_workspace_size(N_PIX, N_PIX, p, T), dtype=torch.uint8, device=dev)
    P = float((1 << BITS) - 1)

    def psnr(s, o):
        with torch.no_grad():
            x = fic.decode_differentiable(s, o, maps, N_PIX, N_PIX, p, T, workspace=work).clamp(0.0, P)
            mse = float(torch.mean((x.double() - img.double()) ** 2))
        return 10.0 * np.log10(P * P / mse)

    for _ in range(max(3, args.warmup)):
        s, o = s0.clone(), o0.clone()
        fic.refine(img, maps, s, o, p, steps=5, iters=T, lr=lr, workspace=work)
    torch.cuda.synchronize()
    s, o = s0.clone(), o0.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t_clk = time.time()
        e0.record()
        loss = fic.refine(img, maps, s, o, p, steps=steps, iters=T, lr=lr, workspace=work)
        e1.record()
        torch.cuda.synchronize()
        while time.time() - t_clk < CLOCK_WINDOW_S:
            fic.refine(img, maps, s0.clone(), o0.clone(), p, steps=20, iters=T, lr=lr, workspace=work)
            torch.cuda.synchronize()
        clk_window = time.time() - t_clk
    t = e0.elapsed_time(e1) / 1e3
    L = loss.cpu().numpy()
    before, after = psnr(s0, o0), psnr(s, o)
    # end to end: the image, the maps and the starting coefficients copied in
    # from pinned host memory, the whole refinement, the refined s, o and the
    # loss curve copied back
    h_img = torch.from_numpy(img_np.astype(np.int16)).pin_memory()
    h_maps = maps.cpu().pin_memory()
    h_s0, h_o0 = s0.cpu().pin_memory(), o0.cpu().pin_memory()
    h_s, h_o, h_loss = (torch.empty_like(h_s0).pin_memory(), torch.empty_like(h_o0).pin_memory(),
                        torch.empty(steps + 1, dtype=torch.float32).pin_memory())
    d_img, d_maps = torch.empty_like(img), torch.empty_like(maps)
    d_s, d_o = torch.empty_like(s0), torch.empty_like(o0)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    d_img.copy_(h_img, non_blocking=True)
    d_maps.copy_(h_maps, non_blocking=True)
    d_s.copy_(h_s0, non_blocking=True)
    d_o.copy_(h_o0, non_blocking=True)
    lo = fic.refine(d_img, d_maps, d_s, d_o, p, steps=steps, iters=T, lr=lr, workspace=work)
    h_s.copy_(d_s, non_blocking=True)
    h_o.copy_(d_o, non_blocking=True)
    h_loss.copy_(lo, non_blocking=True)
    f1.record()
    torch.cuda.synchronize()
    t_e2e = f0.elapsed_time(f1) / 1e3
    h2d = h_img.numel() * 2 + h_maps.numel() + 8 * h_s0.numel()
    d2h = 8 * h_s0.numel() + 4 * (steps + 1)
    clocks = clk.summary()
    clocks["window_s"] = clk_window
    clocks["note"] = "sampled over the timed refinement and identical ones that follow it"
    # algorithmic bytes of one step (W*H pixels, FP32 iterates): the forward
    # reads and writes an iterate per iteration (8 T N), the loss reads x_T and
    # the image and writes dL/dx_T (10 N), the reverse sweep recomputes the odd
    # iterates from the even checkpoints (4 T N) and per iteration reads x_t
    # and the adjoint and writes the next adjoint (12 T N)
    npx = N_PIX * N_PIX
    step_bytes = (24 * T + 10) * npx
    peaks, peak_kind = load_peaks()
    roof = {"bound": "hbm", "achieved": step_bytes / (t / steps) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "bytes_per_unit": step_bytes, "units": 1, "traffic": None,
            "kernel": "whole step (one graph replay of 45 launches; the adjoint item kernel is the largest)",
            "peak_source": peak_kind,
            "note": "the iterates (1 MB each) stay in L2: the step is bound by launch and latency, not by HBM"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    line = {"metric": "refinement steps/s", "value": steps / t, "unit": "steps/s", "n_gpus": 1, "steps": steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": REF_WORKLOAD, "decode_iters": T, "adam_lr": lr,
                       "psnr_collage_optimal_db": before, "psnr_refined_db": after, "psnr_gain_db": after - before,
                       "loss_first": float(L[0]), "loss_last": float(L[-1])},
            # per step: fill + T forward iterations, 2 loss kernels, T/2 recomputed
            # iterates, T per-range gradients, 3 (T - 1) adjoint kernels, Adam
            "psnr_gain_db": after - before, "psnr_refined_db": after,
            "e2e": {"value": steps / t_e2e, "unit": "steps/s", "h2d_bytes_per_step": h2d / steps,
                    "d2h_bytes_per_step": d2h / steps,
                    "timing": "one whole refinement (inputs in, 200 steps, results out), per step"},
            "gpu_launches": steps * (5 * T + T // 2 + 1), "clocks": clocks, "roofline": roof}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_refine(img_np, maps, fic, s0, o0, T, lr)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--search", default="auto", choices=["auto", "tc", "simt"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="slice", choices=["slice", "quadtree", "volume", "refine"],
                    help="slice: the 512x512 CT encode (default); quadtree: its adaptive 16->8->4 quadtree "
                         "encode; volume: a 96-slice CT stack of 256/384/512 slices as one batch; refine: "
                         "200 Adam steps of the differentiable decode after the slice encode")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "quadtree":
        run_quadtree(args)
        return
    if args.workload == "volume":
        run_volume(args)
        return
    if args.workload == "refine":
        run_refine(args)
        return

    import torch

    import __graft_entry__

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    if ws > 1:
        dist.barrier()
    __graft_entry__.build()
    from paper_1404_0774_gb300 import fic

    R, D, comps = comparisons()
    img_np = fic_synth.ct_slice(rank_seed(rank))
    search = {"auto": fic.FIC_SEARCH_AUTO, "tc": fic.FIC_SEARCH_TC, "simt": fic.FIC_SEARCH_SIMT}[args.search]
    p = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS, search=search)
    img = torch.from_numpy(img_np.astype(np.int16)).to(dev)
    wsb = fic.encode_workspace_size(N_PIX, N_PIX, p)
    work = torch.empty(wsb, dtype=torch.uint8, device=dev)
    maps = torch.empty(R * 40, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step():
        fic.encode(img, p, maps=maps, workspace=work, stream=stream)

    n_warm = warm_up(step, args.warmup, torch.cuda.synchronize)
    launches_per_step = 5  # statistics, compaction + operand rows + seed, search, re-score, exact scans + output

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_clk = time.time()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        # the timed steps take milliseconds, nvidia-smi samples every 100 ms:
        # keep the identical load (flush + encode) running so that the sampler
        # sees at least a second of it around the timed region
        while time.time() - t_clk < CLOCK_WINDOW_S:
            for _ in range(20):
                flush.zero_()
                step()
            torch.cuda.synchronize()
        clk_window = time.time() - t_clk
    if ws > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_total = float(np.sum(step_ms)) / 1e3
    t_total = max_over_ranks(t_total, ws, dev)
    value = job_rate(ws, args.steps, comps, t_total)

    stats = fic.last_encode_stats()
    used = {fic.FIC_SEARCH_TC: "tc", fic.FIC_SEARCH_SIMT: "simt"}.get(stats[2], "?")
    mnp = fic.maps_to_numpy(maps)
    n_fallback = int((mnp["info"] & fic.FIC_MAP_FALLBACK).sum())

    # end to end through the C ABI with pinned host buffers
    h_img = torch.from_numpy(img_np.astype(np.int16)).pin_memory()
    h_maps = torch.empty(R * 40, dtype=torch.uint8).pin_memory()
    lib = fic.lib()
    import ctypes

    nm = ctypes.c_int()

    def e2e_step():
        rc = lib.fic_encode(h_img.data_ptr(), N_PIX, N_PIX, N_PIX, ctypes.byref(p), h_maps.data_ptr(), R,
                            ctypes.byref(nm), work.data_ptr(), wsb, stream.cuda_stream)
        assert rc == 0, rc

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        e_ev[i][0].record(stream)
        e2e_step()
        e_ev[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_t = float(np.sum([a.elapsed_time(b) for a, b in e_ev])) / 1e3
    e2e_t = max_over_ranks(e2e_t, ws, dev)
    e2e_value = job_rate(ws, args.steps, comps, e2e_t)

    def timed_arm(pp, wsp, k):
        """k steps of the encode with parameters pp (L2 flushed before each),
        total seconds (max over ranks), after 3 warm-up steps."""
        for _ in range(3):
            fic.encode(img, pp, maps=maps, workspace=wsp, stream=stream)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            flush.zero_()
            evs[i][0].record(stream)
            fic.encode(img, pp, maps=maps, workspace=wsp, stream=stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(float(np.sum([a.elapsed_time(b) for a, b in evs])) / 1e3, ws, dev)

    def phases_of(pp, wsp):
        """Median phase times (ms) of the encode with pp: events the library
        records around each phase on the launching stream, L2 flushed."""
        pt = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS, search=pp.search,
                        flags=pp.flags | fic.FIC_FLAG_PHASE_TIMING)
        ph = []
        for _ in range(max(5, min(args.steps, 20))):
            flush.zero_()
            fic.encode(img, pt, maps=maps, workspace=wsp, stream=stream)
            ph.append(fic.last_encode_phase_ms())
        return {k: float(v) for k, v in zip(["prep", "search", "rescore", "scans_and_output"],
                                            np.median(np.array(ph), axis=0))}

    def decoded_psnr(pp, wsp):
        """PSNR of this arm's maps decoded on the GPU (fic_decode, 10 Jacobi
        iterations from 2^(B-1))."""
        fic.encode(img, pp, maps=maps, workspace=wsp, stream=stream)
        out = fic.decode(maps, N_PIX, N_PIX, pp, stream=stream)
        torch.cuda.synchronize()
        return psnr_db(img_np, out.cpu().numpy(), BITS), fic.maps_to_numpy(maps).copy()

    # the same encode with every range and domain screened (FIC_FLAG_DENSE):
    # the default skips shadow ranges and flat domains (Section V), same maps
    pdense = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS, search=search,
                        flags=fic.FIC_FLAG_DENSE)
    wsd = torch.empty(fic.encode_workspace_size(N_PIX, N_PIX, pdense), dtype=torch.uint8, device=dev)
    dense_t = timed_arm(pdense, wsd, args.steps)
    dense_value = job_rate(ws, args.steps, comps, dense_t)

    # the plain FP32 CUDA-core search on the same slice (the speed-up baseline)
    other = fic.FIC_SEARCH_SIMT if used == "tc" else fic.FIC_SEARCH_TC
    po = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS, search=other)
    wso = torch.empty(fic.encode_workspace_size(N_PIX, N_PIX, po), dtype=torch.uint8, device=dev)
    other_t = timed_arm(po, wso, args.steps)
    podense = fic.params(range_size=RANGE, domain_stride=STRIDE, bit_depth=BITS, search=other,
                         flags=fic.FIC_FLAG_DENSE)
    wsod = torch.empty(fic.encode_workspace_size(N_PIX, N_PIX, podense), dtype=torch.uint8, device=dev)
    other_dense_t = timed_arm(podense, wsod, args.steps)

    # what the skips leave to screen (host-side count from the image itself)
    shadow = int(shadow_mask(img_np, RANGE).sum())
    flat = flat_domains(img_np, RANGE, STRIDE)
    screened = (R - shadow) * (D - flat) * 8

    phase_med = phases_of(p, work)
    phase_other = phases_of(po, wso)
    psnr_main, maps_main = decoded_psnr(p, work)
    psnr_other, maps_other = decoded_psnr(po, wso)
    peaks, peak_kind = load_peaks()
    clocks = clk.summary()
    clocks["window_s"] = clk_window
    clocks["note"] = "sampled over the timed steps and the identical steps that follow them"
    kern_ms = phase_med["search"]
    # algorithmic work of one launch: the candidates it screens (shadow ranges
    # and flat domains are decided without a cross term) x 2m = 128 flops of
    # the cross term each
    useful = screened * 2 * RANGE * RANGE
    # the binding unit of the search is its FP32 epilogue: the launch against
    # the FP32 lane throughput (SMs x 128 lanes x max SM clock)
    alu_peak = sm_count(dev) * 128 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    tensor_tflops = useful / (kern_ms * 1e-3) / 1e12
    if used == "tc":
        alu = screened * EPI_OPS_PER_CANDIDATE / (kern_ms * 1e-3) / 1e12
        executed = screened * 2 * (2 * RANGE * RANGE)  # FP16 MMA flops issued: hi and lo parts
        roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "Tops/s",
                "ops_per_unit": EPI_OPS_PER_CANDIDATE,
                "tensor": {"bound": "tensor", "achieved": tensor_tflops,
                           "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                           "frac": tensor_tflops / peaks["bf16_tflops"],
                           "executed": executed / (kern_ms * 1e-3) / 1e12, "flops_per_unit": 2 * RANGE * RANGE,
                           "executed_frac": executed / (kern_ms * 1e-3) / 1e12 / peaks["bf16_tflops"]}}
    else:
        # the FP32 search: RANGE^2 FMAs of the cross term plus the screening key per candidate
        ops = RANGE * RANGE + EPI_OPS_PER_CANDIDATE
        alu = screened * ops / (kern_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "Tops/s", "ops_per_unit": ops}
    roof["units"] = screened
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = search_traffic() if used == "tc" else None
    roof["peak_source"] = peak_kind + " (bf16 for the tensor view); FP32 lanes x max clock for the ALU view"
    roof["kernel"] = "search"
    roof["phase_ms"] = phase_med

    arms = {used: {"ms_per_step": 1e3 * t_total / args.steps, "value": value, "search_ms": kern_ms,
                   "dense_ms_per_step": 1e3 * dense_t / args.steps, "psnr_db": psnr_main},
            ("simt" if used == "tc" else "tc"): {
                "ms_per_step": 1e3 * other_t / args.steps, "value": job_rate(ws, args.steps, comps, other_t),
                "search_ms": phase_other["search"], "dense_ms_per_step": 1e3 * other_dense_t / args.steps,
                "psnr_db": psnr_other, "phase_ms": phase_other}}
    same_maps = bool(np.array_equal(maps_main[["domain_idx", "iso", "s_code", "o_code"]],
                                    maps_other[["domain_idx", "iso", "s_code", "o_code"]]))
    line = {"metric": METRIC, "value": value, "unit": "comparisons/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "fp16+fp32" if used == "tc" else "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "search": used, "l2": "flushed (256 MB write) between steps",
                       "warmup_untimed": {"steps": n_warm, "min_s": WARMUP_MIN_S},
                       "comparisons_per_step": comps, "ranges_resolved_by_exact_rescan": n_fallback,
                       "shadow_ranges": shadow, "flat_domains": flat, "comparisons_screened_per_step": screened,
                       "screened_comparisons_per_s": job_rate(ws, args.steps, screened, t_total),
                       "dense": {"value": dense_value, "ms_per_step": 1e3 * dense_t / args.steps,
                                 "note": "FIC_FLAG_DENSE: every range and domain screened, same maps"}},
            "tc_over_fp32": arms["simt"]["ms_per_step"] / arms["tc"]["ms_per_step"],
            "tc_over_fp32_dense": arms["simt"]["dense_ms_per_step"] / arms["tc"]["dense_ms_per_step"],
            "tc_over_fp32_search": arms["simt"]["search_ms"] / arms["tc"]["search_ms"],
            "fp32_search": arms["simt"], "tc_search": arms["tc"],
            "psnr_db": {"tc": arms["tc"]["psnr_db"], "fp32": arms["simt"]["psnr_db"]},
            "same_maps_tc_fp32": same_maps,
            "dense_ms_per_step": 1e3 * dense_t / args.steps,
            "tensor_tflops": tensor_tflops if used == "tc" else None,
            "tensor_frac": tensor_tflops / peaks["bf16_tflops"] if used == "tc" else None,
            "e2e": {"value": e2e_value, "unit": "comparisons/s",
                    "h2d_bytes_per_step": N_PIX * N_PIX * 2, "d2h_bytes_per_step": R * 40},
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks, "roofline": roof}
    if abs(arms["tc"]["psnr_db"] - arms["simt"]["psnr_db"]) >= 0.01:
        raise SystemExit(f"decoded PSNR of the two searches differs: {line['psnr_db']}")
    if rank == 0:
        if ws == 1 and not args.no_cpu_baseline:
            cb, psnr_oracle, _ = cpu_oracle_baseline(img_np)
            line["cpu_baseline"] = cb
            line["psnr_db"]["oracle"] = psnr_oracle
            for k in ("tc", "fp32"):
                if abs(line["psnr_db"][k] - psnr_oracle) >= 0.01:
                    raise SystemExit(f"decoded PSNR differs from the oracle's maps: {line['psnr_db']}")
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
