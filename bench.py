#!/usr/bin/env python
"""Benchmark of the Bitmap Filter exact self-join on B300.

Headline workload: self-join of 10,000,000 sets (tokens Zipf(s=1.0) over a
1,000,000-token universe, sizes lognormal(mu=2.0, sigma=0.8) rounded and
clipped to [1, 1000], seed 0, drawn on the device), synthetic, the largest
collection of the paper's range (Section 5: 1e5 to 1e7 sets).  One step = the
two joins at Jaccard thresholds 3/5 and 9/10 with b = 128 bits (Bitmap-Xor),
each through the C ABI with the CSR resident in HBM: size sort, bitmap build,
Bitmap Filter over the length window, exact verification, canonical result
sort.

Metric: pairs filtered/s = window pairs evaluated by the Bitmap Filter
(pairs inside the length-filter window, the inner loop of the paper's GPU
algorithm, Alg. 6) per second of whole-join time.  The filter kernel's own
rate goes into the roofline object, against the bound of its algorithmic
instruction mix on the XU (popcount) and ALU (logic) pipes.

Extras on the same line: the 1,000,000-set workload (four thresholds, b in
{64, 128, 256}), the batched and served forms, prefix-filter candidates, the
cutoff point, the other similarity functions, the RS-join.

--impl reference times the CPU oracle (plain all-pairs join with exact
integer Jaccard) on a bounded row sample of the same 10,000,000-set workload
on the host cores: each step scans the same number of sampled rows per
threshold as the main line's cpu_baseline; ms_per_step is the measured time
of that sample, the full-join time it extrapolates to is reported beside it.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

THRESHOLDS = ((3, 5), (9, 10))                         # headline (10M sets)
B_HEAD = 128
THRESHOLDS_1M = ((1, 2), (3, 4), (9, 10), (19, 20))    # the 1M extra
METRIC = "pairs filtered/s"
UNIT = "pairs/s"
WORKLOAD = ("self-join of 10,000,000 sets, tokens Zipf(s=1.0) over 1,000,000, sizes "
            "lognormal(mu=2.0,sigma=0.8) clipped to [1,1000], Jaccard 3/5 and 9/10, b = 128, "
            "CSR int32 tokens in HBM")
WORKLOAD_1M = ("self-join of 1,000,000 sets, tokens Zipf(s=1.1) over 200,000, sizes "
               "lognormal(mu=2.3,sigma=0.6) clipped to [1,500], Jaccard 1/2, 3/4, 9/10, 19/20")
POPC_PER_CLK_PER_SM = 16      # 32-bit population count (XU pipe) per SM per clock
LOP_PER_CLK_PER_SM = 64       # 32-bit logic operations (ALU pipe) per SM per clock
# Algorithmic instruction mix of the Bitmap Filter per window pair at width b:
# b/32 xors (LOP3) of the 32-bit words, then the fewest popcounts a carry-save
# compression of those words allows (2 words: 2 POPC; 4 words: one carry-save
# adder, 2 LOP3, 3 POPC; 8 words: four carry-save adders, 8 LOP3, 4 POPC).
FILTER_MIX = {64: (2, 2), 128: (3, 6), 256: (4, 16)}   # b -> (POPC, LOP3) per pair
# b = 128 and 256: the folded test every pair meets first (the two halves of the xor folded onto
# each other, 64 or 128 bits: 2 POPC and 2 three-input xors, or 3 POPC, 4 three-input xors and a
# carry-save adder; plus the row's share of the column's fold, 2 words over 5 rows or 4 over 4),
# before the full-width test of FILTER_MIX[b] in the column steps where some pair passes it
FOLD_MIX = {128: (2, 2.4), 256: (3, 7)}
# Bitmap width of the served index: at 128 bits the 20,000 q/s stream had p50 0.032 / p99 0.077 ms
# against 0.034 / 0.079-0.087 at 64 bits (15x fewer survivors to merge) and a saturated capacity of
# 1.0e6 queries/s; at 256 bits p99 0.068-0.072 ms, but the capacity is 6.7e5 queries/s.
SERVE_B = 128
FILTER_KERNEL = {64: "k_filter_tma<1,8,256>", 128: "k_filter_tma<2,5,128>",
                 256: "k_filter_tma<4,4,64>"}
FLUSH_BYTES = 256 << 20       # > 126 MB L2


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=32,
                    help="oracle rows sampled per threshold in one CPU sample (both arms)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="least wall time of the main line's CPU baseline (samples are repeated)")
    ap.add_argument("--budget-s", type=float, default=900.0,
                    help="the extras after the headline start only while the run is younger")
    ap.add_argument("--no-million", action="store_true",
                    help="skip the 1,000,000-set workload (and its prefix/cutoff/sims/RS extras)")
    ap.add_argument("--no-sweep", action="store_true", help="1M workload at b = 64 only")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-joins comparison (512 jobs)")
    ap.add_argument("--no-prefix", action="store_true",
                    help="skip the prefix-filter candidate joins")
    ap.add_argument("--no-cutoff", action="store_true",
                    help="skip the joins with the cutoff point of Section 3.5")
    ap.add_argument("--no-rs", action="store_true",
                    help="skip the RS-joins of two 1,000,000-set collections")
    ap.add_argument("--no-sims", action="store_true",
                    help="skip the joins with Cosine, Dice and Overlap similarity")
    ap.add_argument("--no-combined", action="store_true",
                    help="skip the step with Alg. 4's generation function per threshold")
    ap.add_argument("--no-served", action="store_true",
                    help="skip the served-queries measurement (2,000,000 resident sets)")
    ap.add_argument("--shard", choices=("replicas", "bands"), default="replicas",
                    help="N > 1: every rank runs the whole step (replicas, weak scaling) or "
                         "each rank joins one row band of every join (bands, strong scaling)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="bmj_clocks_", suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = list(csv.reader(open(self.path)))
        os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def strip_comments(src: str) -> str:
    """C/C++ source without its comments, each run of whitespace one blank:
    what the compiler sees, so that a comment edit keeps the digest."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":  # string or character literal, copied whole
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def filter_source_digest() -> str:
    """sha256[:16] of the code (comments and layout stripped) of the sources
    the filter kernel is built from."""
    h = hashlib.sha256()
    for name in ("filter_core.cuh", "kernels.cuh", "filter.cu"):
        with open(os.path.join(ROOT, "paper_1711_07295_b300", "csrc", name)) as f:
            h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:16]


def profile_traffic(name: str):
    """DRAM bytes per filter launch from the committed ncu summary
    profiles/<name>.md, if it was taken on the current filter source."""
    path = os.path.join(ROOT, "profiles", f"{name}.md")
    try:
        text = open(path).read()
        digest = filter_source_digest()
    except OSError:
        return None
    m_hash = re.search(r"filter source sha256\[:16\]:\s*([0-9a-f]{16})", text)
    m_tr = re.search(r"dram bytes per launch, mean over one step:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != digest:
        return None
    return float(m_tr.group(1))


def filter_mix(b: int, full_frac=None):
    """(POPC, LOP3) per window pair: FILTER_MIX[b], or with the folded test
    (b = 128, 256), FOLD_MIX[b] plus the full test's mix for the fraction of
    column steps that took it (counted by the kernel)."""
    if b in FOLD_MIX and full_frac is not None:
        return (FOLD_MIX[b][0] + full_frac * FILTER_MIX[b][0],
                FOLD_MIX[b][1] + full_frac * FILTER_MIX[b][1])
    return FILTER_MIX[b]


def filter_bound(b: int, sms: int, mhz: float, full_frac=None) -> float:
    """Peak window pairs/s of the Bitmap Filter at width b: the XU pipe issues
    POPC_PER_CLK_PER_SM popcounts and the ALU pipe LOP_PER_CLK_PER_SM logic
    operations per SM and clock, and a pair needs filter_mix(b, full_frac) of them."""
    popc, lop = filter_mix(b, full_frac)
    return sms * min(POPC_PER_CLK_PER_SM / popc, LOP_PER_CLK_PER_SM / lop) * mhz * 1e6


def filter_roofline(b, pairs, filter_ms, sms, mhz, median_mhz=None, popc_measured=None,
                    full_frac=None):
    popc, lop = filter_mix(b, full_frac)
    peak = filter_bound(b, sms, mhz, full_frac)
    achieved = pairs / (filter_ms / 1e3)
    binding = "XU (POPC)" if POPC_PER_CLK_PER_SM / popc < LOP_PER_CLK_PER_SM / lop else \
        "ALU (LOP3)" if POPC_PER_CLK_PER_SM / popc > LOP_PER_CLK_PER_SM / lop else "XU and ALU"
    r = {"bound": "alu", "achieved": round(achieved / 1e12, 4), "peak": round(peak / 1e12, 4),
         "unit": "Tpairs/s", "frac": round(achieved / peak, 4),
         "kernel": f"{FILTER_KERNEL[b]} (Bitmap Filter, b = {b}, TMA-staged columns"
                   + (f", folded {b // 2}-bit test first)" if full_frac is not None and b in FOLD_MIX
                      else ")"),
         "work_per_pair": {"popc32": round(popc, 4), "lop3": round(lop, 4), "bits_compared": b},
         "peak_derivation": (f"{sms} SMs x {mhz:.0f} MHz (max SM clock) x min({POPC_PER_CLK_PER_SM}"
                             f" POPC/clk/SM / {popc:.4g}, {LOP_PER_CLK_PER_SM} LOP3/clk/SM / "
                             f"{lop:.4g}) pairs; binding pipe {binding}"),
         "frac_of_popc_only": round(achieved * (b // 32) /
                                    (sms * POPC_PER_CLK_PER_SM * mhz * 1e6), 4)}
    if full_frac is not None and b in FOLD_MIX:
        r["full_test_step_frac"] = round(full_frac, 5)
        r["work_per_pair_note"] = (
            f"every window pair meets the folded {b // 2}-bit test ({FOLD_MIX[b][0]} POPC, "
            f"{FOLD_MIX[b][1]} LOP3); the {full_frac:.2%} of warp column steps in which some pair "
            f"passes it also run the {b}-bit test ({FILTER_MIX[b][0]} POPC, {FILTER_MIX[b][1]} LOP3)")
        r["frac_of_full_test_bound"] = round(achieved / filter_bound(b, sms, mhz), 4)
    if median_mhz:
        r["frac_at_median_clock"] = round(achieved / filter_bound(b, sms, median_mhz, full_frac), 4)
    if popc_measured:
        # the XU side of the bound with the POPC rate measured on this device
        xu = popc_measured / popc
        r["xu_bound_measured"] = round(xu / 1e12, 4)
        r["frac_of_xu_measured"] = round(achieved / xu, 4)
    return r


# ----------------------------------------------------------------------------
# CPU oracle timing
# ----------------------------------------------------------------------------
def oracle_sample(off, tok, thresholds, rows_per_thr: int, seed: int, windowed=False):
    """Times the oracle on ``rows_per_thr`` random rows per threshold.  Each row
    is scanned against all N sets (``windowed``: against the sets of its Table 2
    size window); the full self-join compares N(N-1)/2 pairs (every window pair
    is met from both of its ends in the windowed scan), so the full join at one
    threshold takes (time per row) x N/2.  Returns (seconds measured, seconds of
    the full joins extrapolated, threads used)."""
    import numpy as np
    import oracle
    scan = oracle.join_rows_window if windowed else oracle.join_rows
    n = len(off) - 1
    rng = np.random.default_rng(seed)
    t_cpu = t_full = 0.0
    for (p, q) in thresholds:
        rows = rng.choice(n, size=rows_per_thr, replace=False)
        t0 = time.perf_counter()
        scan(off, tok, p, q, rows)
        dt = time.perf_counter() - t0
        t_cpu += dt
        t_full += dt / rows_per_thr * (n / 2.0)
    return t_cpu, t_full, min(oracle.num_threads(), rows_per_thr)


def oracle_windows(off, thresholds):
    import numpy as np
    import oracle
    sizes = np.diff(off)
    return {thr: oracle.window_pairs(sizes, thr[0], thr[1]) for thr in thresholds}


def cpu_baseline(off, tok, rows_per_thr: int, min_seconds: float, workload: str):
    """The oracle on the host cores: samples of rows_per_thr rows per threshold,
    repeated (new rows each time) until min_seconds of wall time."""
    win = oracle_windows(off, THRESHOLDS)
    total_win = sum(win.values())

    def sampled(windowed, budget):
        t_cpu = t_full = 0.0
        reps, cores = 0, 1
        while t_cpu < budget or reps == 0:
            a, b_, cores = oracle_sample(off, tok, THRESHOLDS, rows_per_thr, seed=reps,
                                         windowed=windowed)
            t_cpu += a
            t_full += b_
            reps += 1
        return total_win * reps / t_full, t_cpu, t_full / reps, cores, reps

    rate, t_cpu, t_step, cores, reps = sampled(False, min_seconds)
    w_rate, w_cpu, w_step, _, w_reps = sampled(True, min_seconds / 3)
    return {"value": round(rate), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} samples of {rows_per_thr} random rows per threshold, each row "
                      f"scanned against all {len(off) - 1:,} sets of the {workload} "
                      f"({t_cpu:.1f} s wall on {cores} threads), extrapolated to the full joins "
                      f"({t_step:.0f} s per step)",
            "with_length_filter": {
                "value": round(w_rate), "unit": UNIT,
                "sample": f"{w_reps} samples of {rows_per_thr} random rows per threshold, each "
                          f"against the sets of its Table 2 size window ({w_cpu:.1f} s wall), "
                          f"extrapolated to the full joins ({w_step:.0f} s per step)"}}


def budget_left(args, t_start) -> bool:
    return time.perf_counter() - t_start < args.budget_s


# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1711_07295_b300 import _bmj, inputs

    t_start = time.perf_counter()
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    t0 = time.perf_counter()
    d_off, d_tok = inputs.gen_collection_device(inputs.spec_10m(), device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    off, tok = d_off.cpu().numpy(), d_tok.cpu().numpy()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    b = B_HEAD

    host_coll = {}
    bands = {}
    if world > 1 and args.shard == "bands":
        from paper_1711_07295_b300 import shard
        for (p, q) in THRESHOLDS:
            bands[(p, q)] = shard.band_split(off, p, q, world)[rank]

    def join(p, q, cap=0, host=False, **kw):
        r0, r1 = bands.get((p, q), (0, 0))
        if host:
            return _bmj.bmj_self_join(host_coll["off"], host_coll["tok"], p, q, b=b,
                                      queue_cap=cap, row_begin=r0, row_end=r1, **kw)
        res, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                        queue_cap=cap, stream=stream.cuda_stream,
                                        row_begin=r0, row_end=r1, **kw)
        res.release()
        return st

    caps = {}
    for _ in range(max(args.warmup, 1)):
        for (p, q) in THRESHOLDS:
            st = join(p, q, caps.get((p, q), 0))
            caps[(p, q)] = max(1, st["survivors"])
    torch.cuda.synchronize()

    # ---- timed region: exactly K steps, L2 flushed between steps (untimed) ----
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    launches0 = _bmj.bmj_kernel_launches()
    step_ms = []
    keys = ("ms_filter", "ms_verify", "ms_total", "ms_prepare", "ms_output")
    per_thr = {thr: {"window": 0, "survivors": 0, "verified": 0, "results": 0,
                     "fold_steps": 0, "fold_full_steps": 0,
                     **{k: 0.0 for k in keys}} for thr in THRESHOLDS}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        ev0.record(stream)
        for thr in THRESHOLDS:
            st = join(thr[0], thr[1], caps[thr])
            d = per_thr[thr]
            for key in ("survivors", "verified", "results", "fold_steps", "fold_full_steps"):
                d[key] = st[key]
            d["window"] = st["window_pairs"]
            for key in keys:
                d[key] += st[key]
        ev1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
    launches = _bmj.bmj_kernel_launches() - launches0
    clk = clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    window_per_step = sum(per_thr[t]["window"] for t in THRESHOLDS)
    units_per_step_all = window_per_step * world          # replicas: every rank the whole step
    if bands:                                             # bands: the ranks' windows add up to one step
        t = torch.tensor([window_per_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        units_per_step_all = float(t.item())
    value = units_per_step_all * args.steps / (total_ms / 1e3)

    # ---- roofline of the dominant kernel (the Bitmap Filter at b = 128) ----
    peaks, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    filt_ms = sum(per_thr[t]["ms_filter"] for t in THRESHOLDS)
    try:  # the POPC rate measured by a POPC-only loop on this device (untimed region)
        popc_meas = _bmj.bmj_measure_popc_rate(stream.cuda_stream)
    except Exception:  # reported as missing, never fatal to the headline line
        popc_meas = None
    fold_steps = sum(per_thr[t]["fold_steps"] for t in THRESHOLDS)
    full_frac = (sum(per_thr[t]["fold_full_steps"] for t in THRESHOLDS) / fold_steps
                 if fold_steps else None)
    roofline = filter_roofline(b, window_per_step * args.steps, filt_ms, sms, max_mhz,
                               clk.get("sm_mhz"), popc_meas, full_frac)
    roofline["traffic"] = profile_traffic(f"filter_10m_b{b}")
    roofline["filter_share_of_step"] = round(filt_ms / sum(step_ms), 4)
    roofline["filter_pairs_per_s"] = round(window_per_step * args.steps / (filt_ms / 1e3))
    if popc_meas:
        roofline["popc_measured_per_s"] = round(popc_meas)
    # verification (HBM/L2): bytes it must read per survivor, at the measured rate
    ver_ms = sum(per_thr[t]["ms_verify"] for t in THRESHOLDS)
    surv = sum(per_thr[t]["survivors"] for t in THRESHOLDS)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pinned = (torch.from_numpy(off).pin_memory(), torch.from_numpy(tok).pin_memory())
        host_coll["off"], host_coll["tok"] = pinned[0].numpy(), pinned[1].numpy()
        e_steps = max(1, min(args.e2e_steps, args.steps))
        for thr in THRESHOLDS:   # one untimed step warms the page-locked result pool
            join(thr[0], thr[1], caps[thr], host=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        d2h = 0
        t0 = time.perf_counter()
        for k in range(e_steps):
            for thr in THRESHOLDS:
                a, bb, st = join(thr[0], thr[1], caps[thr], host=True)
                d2h += a.nbytes + bb.nbytes
                del a, bb
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = len(THRESHOLDS) * (off.nbytes + tok.nbytes)
        e2e = {"value": round(units_per_step_all * e_steps / e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h // e_steps),
               "ms_per_step": round(e2e_s * 1e3 / e_steps, 3), "steps": e_steps,
               "inputs": "pinned host CSR, copied in by the library each call; pairs returned "
                         "in page-locked host memory"}
        del pinned
        host_coll.clear()
        _bmj.bmj_host_pool_trim()

    # ---- bands: the one exchange of a sharded join, gathering the pair lists ----
    gather = None
    if bands:
        from paper_1711_07295_b300 import shard
        gather = []
        for (p, q) in THRESHOLDS:
            r0, r1 = bands[(p, q)]
            a, bb, _ = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, row_begin=r0, row_end=r1,
                                          stream=stream.cuda_stream)
            dist.barrier()
            t0 = time.perf_counter()
            got = shard.gather_pairs(a, bb, dst=0)
            dt = time.perf_counter() - t0
            if rank == 0:
                gather.append({"threshold": f"{p}/{q}", "pairs": int(len(got[0])),
                               "gather_ms": round(dt * 1e3, 2)})
            del a, bb, got

    out = None
    if rank == 0:
        joins = []
        for thr in THRESHOLDS:
            d = per_thr[thr]
            joins.append({"threshold": f"{thr[0]}/{thr[1]}", "window_pairs": d["window"],
                          "survivors": d["survivors"], "verified": d["verified"],
                          "results": d["results"],
                          **{k.replace("ms_", "") + "_ms": round(d[k] / args.steps, 3)
                             for k in keys}})
        out = {"metric": METRIC, "value": round(value), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
               "scaling": "strong" if bands else "weak", "vs_baseline": None, "dtype": "u64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "n_sets": int(len(off) - 1),
                          "tokens": int(len(tok)),
                          "thresholds": [f"{p}/{q}" for p, q in THRESHOLDS],
                          "b": b, "method": "xor",
                          "parallelism": (f"row bands x{world}" if bands else f"replicas x{world}"),
                          "l2": "flushed between steps (256 MB write, untimed); inputs 490 MB",
                          "inputs": "resident in HBM, drawn on the device (seed 0)",
                          "peaks": peak_src},
               "roofline": roofline, "cpu_baseline": None, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clk, "joins": joins,
               "verify": {"survivors_per_s": round(surv * args.steps / (ver_ms / 1e3)),
                          "ms_per_step": round(ver_ms / args.steps, 3)},
               "generation_s": round(gen_s, 2)}
        if gather:
            out["band_gather"] = {"how": "counts, then int64 keys padded to the largest count, "
                                         "one torch.distributed gather to rank 0, merged there",
                                  "joins": gather}

    # ---- extras: the same 10M collection with prefix-filter candidates and the cutoff ----
    if rank == 0 and world == 1:
        extra = {}
        if not args.no_prefix and budget_left(args, t_start):
            rows = []
            for (p, q) in THRESHOLDS:
                for rep in range(2):   # the first call warms the pools
                    r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                                  candidates=_bmj.BMJ_CAND_PREFIX,
                                                  stream=stream.cuda_stream)
                    r.release()
                wj = per_thr[(p, q)]["ms_total"] / args.steps
                r, _, sa = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                              candidates=_bmj.BMJ_CAND_AUTO,
                                              stream=stream.cuda_stream)
                r.release()
                rows.append({"threshold": f"{p}/{q}",
                             "automatic": {"took": "window" if sa["candidates"] == -2 else "prefix",
                                           "join_ms": round(sa["ms_total"], 2)},
                             "candidates": st["candidates"],
                             "candidate_slots": st["candidate_slots"],
                             "candidate_ranges": st["filter_passes"],
                             "survivors": st["survivors"], "results": st["results"],
                             "join_ms": round(st["ms_total"], 2),
                             "candidate_ms": round(st["ms_filter"], 2),
                             "window_join_ms": round(wj, 2),
                             "speedup_vs_window": round(wj / st["ms_total"], 3)})
            extra["prefix_filter"] = rows
        if not args.no_cutoff and budget_left(args, t_start):
            r, _, st = _bmj.bmj_self_join(d_off, d_tok, 3, 5, b=b, output_on_device=True,
                                          cutoff=_bmj.BMJ_CUTOFF_AUTO, stream=stream.cuda_stream)
            r.release()
            wj = per_thr[(3, 5)]["ms_total"] / args.steps
            extra["cutoff_point"] = {"threshold": "3/5", "cutoff": st["cutoff"],
                                     "survivors": st["survivors"], "results": st["results"],
                                     "join_ms": round(st["ms_total"], 2),
                                     "speedup_vs_no_cutoff": round(wj / st["ms_total"], 3)}
        out["ten_million_extras"] = extra
    del d_tok, d_off
    torch.cuda.empty_cache()

    # ---- the other workloads (rank 0, one GPU) ----
    if rank == 0 and world == 1:
        sections = (("million", not args.no_million, run_million),
                    ("batched", not args.no_batched, run_batched),
                    ("served", not args.no_served, run_served))
        for name, on, fn in sections:
            if not on:
                continue
            if not budget_left(args, t_start):
                out[name] = {"skipped": f"run older than --budget-s {args.budget_s:.0f} s"}
                continue
            try:
                out[name] = fn(args, dev)
            except Exception as e:  # reported, never fatal to the headline line
                out[name] = {"error": f"{type(e).__name__}: {e}"}

    # last, so that its host threads disturb none of the GPU measurements above
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(off, tok, args.cpu_rows, args.cpu_seconds,
                                           "10,000,000-set workload")
    if rank == 0:
        out["run_s"] = round(time.perf_counter() - t_start, 1)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_million(args, dev):
    """The 1,000,000-set workload: one step = the four joins at 1/2, 3/4, 9/10
    and 19/20 (b = 64, Xor), timed over --steps steps with the L2 flushed
    between them; then each of b = 128 and 256 for one step (roofline of each
    width), Alg. 4's generation function, the other similarity functions,
    prefix-filter candidates, the cutoff point and an RS-join."""
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    off, tok = inputs.gen_collection(inputs.spec_1m(seed=0))
    d_off = torch.from_numpy(off).to(dev)
    d_tok = torch.from_numpy(tok).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    peaks, _ = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))

    def join(p, q, b, cap=0, method=_bmj.BMJ_XOR, **kw):
        res, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                        queue_cap=cap, stream=stream.cuda_stream, method=method,
                                        **kw)
        res.release()
        return st

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed_step(b, steps, caps, method=_bmj.BMJ_XOR):
        per = {thr: {"ms_total": 0.0, "ms_filter": 0.0, "ms_verify": 0.0} for thr in THRESHOLDS_1M}
        ms = 0.0
        for k in range(steps):
            flush.fill_(k & 0xff)
            torch.cuda.synchronize()
            ev0.record(stream)
            for thr in THRESHOLDS_1M:
                st = join(thr[0], thr[1], b, caps[thr], method=method)
                for key in ("ms_total", "ms_filter", "ms_verify"):
                    per[thr][key] += st[key]
                per[thr]["st"] = st
            ev1.record(stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
        return ms, per

    out = {"workload": WORKLOAD_1M + ", inputs in HBM"}
    widths = (64,) if args.no_sweep else (64, 128, 256)
    by_b = {}
    win = None
    for b in widths:
        caps = {}
        for _ in range(2):
            for thr in THRESHOLDS_1M:
                caps[thr] = max(1, join(thr[0], thr[1], b, caps.get(thr, 0))["survivors"])
        steps = max(1, min(args.steps, 5)) if b == 64 else 1
        ms, per = timed_step(b, steps, caps)
        win = sum(per[t]["st"]["window_pairs"] for t in THRESHOLDS_1M)
        filt = sum(per[t]["ms_filter"] for t in THRESHOLDS_1M)
        fsteps = sum(per[t]["st"]["fold_steps"] for t in THRESHOLDS_1M)
        ffrac = (sum(per[t]["st"]["fold_full_steps"] for t in THRESHOLDS_1M) / fsteps
                 if fsteps else None)
        by_b[str(b)] = {
            "steps": steps, "ms_per_step": round(ms / steps, 3),
            "pairs_per_s": round(win * steps / (ms / 1e3)),
            "roofline": filter_roofline(b, win * steps, filt, sms, max_mhz, full_frac=ffrac),
            "joins": [{"threshold": f"{t[0]}/{t[1]}", "window_pairs": per[t]["st"]["window_pairs"],
                       "survivors": per[t]["st"]["survivors"], "results": per[t]["st"]["results"],
                       "join_ms": round(per[t]["ms_total"] / steps, 3),
                       "filter_ms": round(per[t]["ms_filter"] / steps, 3),
                       "verify_ms": round(per[t]["ms_verify"] / steps, 3)} for t in THRESHOLDS_1M]}
        if b == 64:
            by_b["64"]["roofline"]["traffic"] = profile_traffic("filter_1m_b64")
    out["by_b"] = by_b
    step64 = {t["threshold"]: t for t in by_b["64"]["joins"]}

    if not args.no_combined:
        ccaps = {thr: max(1, join(thr[0], thr[1], 64, method=_bmj.BMJ_COMBINED)["survivors"])
                 for thr in THRESHOLDS_1M}
        ms, per = timed_step(64, 1, ccaps, method=_bmj.BMJ_COMBINED)
        out["combined_method"] = {
            "method": {f"{t[0]}/{t[1]}": ("xor", "set", "next")[per[t]["st"]["method"]]
                       for t in THRESHOLDS_1M},
            "survivors": {f"{t[0]}/{t[1]}": per[t]["st"]["survivors"] for t in THRESHOLDS_1M},
            "ms_per_step": round(ms, 3), "pairs_per_s": round(win / (ms / 1e3))}

    if not args.no_sims:
        sims = {}
        cases = (("cosine", _bmj.BMJ_COSINE, THRESHOLDS_1M), ("dice", _bmj.BMJ_DICE, THRESHOLDS_1M),
                 ("overlap", _bmj.BMJ_OVERLAP, ((10, 1), (20, 1))))
        for name, sim, thr_list in cases:
            rows = []
            for (p, q) in thr_list:
                join(p, q, 64, sim=sim)
                st = join(p, q, 64, sim=sim)
                rows.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                             "survivors": st["survivors"], "results": st["results"],
                             "filter_passes": st["filter_passes"],
                             "join_ms": round(st["ms_total"], 3),
                             "pairs_per_s": round(st["window_pairs"] / (st["ms_total"] / 1e3)),
                             "filter_pairs_per_s": round(st["window_pairs"] /
                                                         max(st["ms_filter"] / 1e3, 1e-9))})
            sims[name] = rows
        out["similarity_functions"] = sims

    if not args.no_prefix:
        rows = []
        for (p, q) in THRESHOLDS_1M:
            join(p, q, 64, candidates=_bmj.BMJ_CAND_PREFIX)
            st = join(p, q, 64, candidates=_bmj.BMJ_CAND_PREFIX)
            sa = join(p, q, 64, candidates=_bmj.BMJ_CAND_AUTO)
            wj = step64[f"{p}/{q}"]["join_ms"]
            rows.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                         "automatic": {"took": "window" if sa["candidates"] == -2 else "prefix",
                                       "join_ms": round(sa["ms_total"], 3)},
                         "candidates": st["candidates"],
                         "candidate_slots": st["candidate_slots"],
                         "candidate_ranges": st["filter_passes"],
                         "survivors": st["survivors"],
                         "results": st["results"], "join_ms": round(st["ms_total"], 3),
                         "candidate_ms": round(st["ms_filter"], 3), "window_join_ms": wj,
                         "speedup_vs_window": round(wj / st["ms_total"], 3)})
        out["prefix_filter"] = rows

    if not args.no_cutoff:
        rows = []
        for (p, q) in THRESHOLDS_1M:
            join(p, q, 64, cutoff=_bmj.BMJ_CUTOFF_AUTO)
            st = join(p, q, 64, cutoff=_bmj.BMJ_CUTOFF_AUTO)
            wj = step64[f"{p}/{q}"]["join_ms"]
            rows.append({"threshold": f"{p}/{q}", "cutoff": st["cutoff"],
                         "survivors": st["survivors"],
                         "survivors_without": step64[f"{p}/{q}"]["survivors"],
                         "results": st["results"], "join_ms": round(st["ms_total"], 3),
                         "window_join_ms": wj,
                         "speedup_vs_no_cutoff": round(wj / st["ms_total"], 3)})
        out["cutoff_point"] = rows

    if not args.no_rs:
        rows = []
        s_off, s_tok = inputs.gen_collection(inputs.spec_1m(seed=1))
        ds_off, ds_tok = torch.from_numpy(s_off).to(dev), torch.from_numpy(s_tok).to(dev)
        for (p, q) in ((9, 10), (3, 4)):
            for rep in range(2):  # the first call warms the pools
                r, _, st = _bmj.bmj_rs_join(d_off, d_tok, ds_off, ds_tok, p, q, b=64,
                                            output_on_device=True, stream=stream.cuda_stream)
                r.release()
            for rep in range(2):
                r, _, sx = _bmj.bmj_rs_join(d_off, d_tok, ds_off, ds_tok, p, q, b=64,
                                            output_on_device=True, stream=stream.cuda_stream,
                                            candidates=_bmj.BMJ_CAND_PREFIX)
                r.release()
            rows.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                         "survivors": st["survivors"], "results": st["results"],
                         "join_ms": round(st["ms_total"], 3), "filter_ms": round(st["ms_filter"], 3),
                         "pairs_per_s": round(st["window_pairs"] / (st["ms_total"] / 1e3)),
                         "prefix_filter": {"candidates": sx["candidates"], "results": sx["results"],
                                           "join_ms": round(sx["ms_total"], 3),
                                           "speedup_vs_window": round(st["ms_total"] /
                                                                      sx["ms_total"], 3)}})
        out["rs_join"] = {"workload": "R = the 1,000,000-set collection, S = a second one (same "
                                      "recipe, seed 1), b = 64", "joins": rows}
    del d_off, d_tok, flush
    torch.cuda.empty_cache()
    return out


def run_batched(args, dev):
    """512 independent joins: one bmj_self_join_batch call (autotuned b,
    graph-captured execute stage) against one bmj_self_join call per job with
    the same b per job."""
    import numpy as np
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    t0 = time.perf_counter()
    off, tok, js, p, q = inputs.gen_batch_device(inputs.BatchSpec(), device=dev)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=0, use_graph=True,
                                               stream=stream.cuda_stream)
    chosen = [s["b"] for s in jst]
    del pairs
    torch.cuda.synchronize()
    times, last = [], None
    for _ in range(max(1, min(args.steps, 3))):
        t0 = time.perf_counter()
        pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=0, use_graph=True,
                                                   stream=stream.cuda_stream)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        last = bst
        del pairs
    batched_s = statistics.median(times)
    jobs = []
    for k in range(len(js) - 1):
        lo, hi = int(js[k]), int(js[k + 1])
        o = (off[lo:hi + 1] - off[lo]).contiguous()
        jobs.append((o, tok[int(off[lo]):int(off[hi])].contiguous(), int(p[k]), int(q[k]), chosen[k]))
    for o, t_, pk, qk, bk in jobs[:8]:
        r, _, _ = _bmj.bmj_self_join(o, t_, pk, qk, b=bk, output_on_device=True,
                                     stream=stream.cuda_stream)
        r.release()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for o, t_, pk, qk, bk in jobs:
        r, _, _ = _bmj.bmj_self_join(o, t_, pk, qk, b=bk, output_on_device=True,
                                     stream=stream.cuda_stream)
        r.release()
    torch.cuda.synchronize()
    single_s = time.perf_counter() - t0
    win = last["window_pairs"]
    return {"workload": "512 independent self-joins, sets per job log-uniform 1,000-200,000, "
                        "sizes U[3,100], Zipf(s=1.0) over 50,000, thresholds from "
                        "{1/2,7/10,4/5,9/10}",
            "sets": int(js[-1]), "tokens": int(tok.numel()), "window_pairs": int(win),
            "survivors": int(last["survivors"]), "results": int(last["results"]),
            "batched_ms": round(batched_s * 1e3, 3),
            "batched_pairs_per_s": round(win / batched_s),
            "batched_stage_ms": {"prepare": round(last["ms_prepare"], 3),
                                 "tune": round(last["ms_tune"], 3),
                                 "execute": round(last["ms_execute"], 3)},
            "one_join_per_call_ms": round(single_s * 1e3, 3),
            "one_join_per_call_pairs_per_s": round(win / single_s),
            "speedup": round(single_s / batched_s, 3),
            "tuned_b": {str(b): chosen.count(b) for b in (64, 128, 256)},
            "window_pairs_by_b": {str(b): int(sum(s["window_pairs"] for s in jst if s["b"] == b))
                                  for b in (64, 128, 256)},
            "graph": int(last["graph"]), "launches": int(last["n_launches"]),
            "filter_passes": int(last["filter_passes"]),
            "generation_s": round(gen_s, 2)}


def run_served(args, dev):
    """A Poisson stream of 20,000 queries/s against a resident index of
    2,000,000 sets: continuous batching (4 slots) against one query per
    launch (1 slot, batches of 1), same arrivals; the saturated capacity
    (three runs, the median reported), with the SM clocks sampled over the
    whole section."""
    import numpy as np
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    t0 = time.perf_counter()
    spec = inputs.spec_resident_2m()
    off_d, tok_d = inputs.gen_collection_device(spec, device=dev)
    off, tok = off_d.cpu().numpy(), tok_d.cpu().numpy()
    qs = inputs.QuerySpec(n_queries=20_000, rate_qps=20_000.0)
    arr, qoff, qtok, p, q = inputs.gen_queries(qs, spec, off, tok)
    gen_s = time.perf_counter() - t0
    idx = _bmj.Index(off_d, tok_d, b=SERVE_B)
    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    clocks.start()
    idx.serve(qoff[:201], qtok[:int(qoff[200])], arr[:200], p[:200], q[:200])   # warm-up
    _, lat, st = idx.serve(qoff, qtok, arr, p, q, n_slots=4, max_batch_queries=4096,
                           want_results=False)
    _, lat1, st1 = idx.serve(qoff, qtok, arr, p, q, n_slots=1, max_batch_queries=1,
                             want_results=False)
    # capacity: the same queries all waiting at time 0
    sat = []
    for _ in range(3):
        sat.append(idx.serve(qoff, qtok, np.zeros_like(arr), p, q, n_slots=4,
                             max_batch_queries=4096, want_results=False)[2])
    st0 = sorted(sat, key=lambda x: x["qps"])[1]
    live = run_live(idx, arr, qoff, qtok, p, q)
    clk = clocks.stop()
    idx.close()
    return {"workload": "resident index of 2,000,000 sets (Zipf(s=1.1) over 300,000, sizes "
                        "lognormal(2.3,0.6) in [1,500]); Poisson arrivals at 20,000 queries/s, "
                        "20,000 probes of size U[2,300] (half edited resident copies), "
                        f"thresholds from {{1/2,3/4,9/10}}, b = {SERVE_B}",
            "continuous_batching": {"p50_ms": round(st["p50_ms"], 4),
                                    "p99_ms": round(st["p99_ms"], 4),
                                    "max_ms": round(st["max_ms"], 4), "qps": round(st["qps"], 1),
                                    "batches": int(st["batches"]),
                                    "window_pairs": int(st["window_pairs"]),
                                    "survivors": int(st["survivors"]),
                                    "results": int(st["results"]), "slots": 4},
            "one_query_per_launch": {"p50_ms": round(st1["p50_ms"], 4),
                                     "p99_ms": round(st1["p99_ms"], 4),
                                     "max_ms": round(st1["max_ms"], 4),
                                     "qps": round(st1["qps"], 1), "batches": int(st1["batches"])},
            "saturated": {"qps": round(st0["qps"], 1), "p50_ms": round(st0["p50_ms"], 4),
                          "p99_ms": round(st0["p99_ms"], 4), "batches": int(st0["batches"]),
                          "qps_runs": [round(x["qps"], 1) for x in sat],
                          "arrivals": "all 20,000 queries at time 0 (median of three runs)"},
            "live_submit_poll": live,
            "clocks": clk,
            "generation_s": round(gen_s, 2)}


def run_live(idx, arr, qoff, qtok, p, q):
    """The same Poisson stream through the live entry points: one host thread
    submits every query at its arrival time (bmj_serve_submit) and, between
    arrivals, polls the oldest tickets (bmj_serve_poll, no wait) while the
    server's own loop thread batches and runs them; latency = completion -
    submission, measured by the library.  Python's cyclic garbage collector is
    paused over the stream and each turn polls at most eight tickets, so that
    neither a collection nor a large finished batch keeps the submitting thread
    from the next arrival."""
    import gc
    import numpy as np
    from paper_1711_07295_b300 import _bmj
    warm = _bmj.Server(idx, n_slots=4, max_batch_queries=4096, max_probe_tokens=512)
    for x in range(200):
        warm.submit(qtok[qoff[x]:qoff[x + 1]], int(p[x]), int(q[x]))
    warm.close()
    srv = _bmj.Server(idx, n_slots=4, max_batch_queries=4096, max_probe_tokens=512)
    n = len(arr)
    tickets = np.full(n, -1, np.int64)
    late = np.zeros(n)
    lat = np.zeros(n)
    n_res = np.zeros(n, np.int64)
    head = 0   # oldest ticket not yet polled

    def poll_some(wait_ms, limit):
        # at most `limit` completed tickets per call, so that a large finished
        # batch does not hold the thread past the next arrival
        nonlocal head
        done = 0
        while head < n and tickets[head] >= 0 and done < limit:
            r = srv.poll(int(tickets[head]), wait_ms=wait_ms)
            if r is None:
                return
            n_res[head] = len(r[0])
            lat[head] = r[1]
            head += 1
            done += 1
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for x in range(n):
            while time.perf_counter() - t0 < arr[x]:
                poll_some(0, 8)
            late[x] = time.perf_counter() - t0 - arr[x]
            tickets[x] = srv.submit(qtok[qoff[x]:qoff[x + 1]], int(p[x]), int(q[x]))
        while head < n:
            poll_some(100, n)
    finally:
        gc.enable()
    st = srv.close()
    return {"p50_ms": round(float(np.percentile(lat, 50)), 4),
            "p99_ms": round(float(np.percentile(lat, 99)), 4),
            "max_ms": round(float(lat.max()), 4), "qps": round(st["qps"], 1),
            "batches": int(st["batches"]), "results": int(n_res.sum()),
            "submit_lateness_p99_ms": round(float(np.percentile(late, 99)) * 1e3, 4),
            "submit_lateness_max_ms": round(float(late.max()) * 1e3, 4),
            "submit_lateness_worst_at_s": round(float(arr[int(np.argmax(late))]), 4),
            "how": "bmj_serve_submit at each arrival time and bmj_serve_poll between arrivals "
                   "from one host thread, the server's loop thread batching; latency = "
                   "completion - submission (library clock)"}


def run_reference(args):
    """The CPU oracle on the host cores on the 10,000,000-set workload: every
    step is one sample of --cpu-rows rows per threshold (the sample size of the
    main line's cpu_baseline), each row scanned against all N sets.  The
    collection is drawn with torch's generator on the device when one is
    present (the main line's collection), on the host otherwise."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_1711_07295_b300 import inputs
    import oracle
    t_start = time.perf_counter()
    try:
        import torch
        have_cuda = torch.cuda.is_available()
    except ImportError:
        have_cuda = False
    if have_cuda:
        d_off, d_tok = inputs.gen_collection_device(inputs.spec_10m())
        off, tok = d_off.cpu().numpy(), d_tok.cpu().numpy()
        del d_off, d_tok
        torch.cuda.empty_cache()
        drawn = "drawn with torch's generator on the device (seed 0), as the main line's"
    else:
        off, tok = inputs.gen_collection(inputs.spec_10m())
        drawn = "drawn by the host sampler (seed 0; no CUDA device: not the main line's sets)"
    win = oracle_windows(off, THRESHOLDS)
    total_win = sum(win.values())
    rows = args.cpu_rows
    for k in range(args.warmup):
        oracle_sample(off, tok, THRESHOLDS, rows, seed=1000 + k)
    t_meas, t_full, cores = [], [], 1
    for k in range(args.steps):
        a, b_, cores = oracle_sample(off, tok, THRESHOLDS, rows, seed=100 + k)
        t_meas.append(a)
        t_full.append(b_)
    value = total_win * args.steps / sum(t_full)
    sample = (f"each step: {rows} random rows per threshold scanned against all "
              f"{len(off) - 1:,} sets ({statistics.mean(t_meas):.2f} s wall on {cores} threads); "
              f"value = the step's window pairs over the full-join time the sample extrapolates "
              f"to (time per row x N/2 per threshold)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(statistics.mean(t_meas) * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_sets": int(len(off) - 1), "tokens": int(len(tok)),
                      "thresholds": [f"{p}/{q}" for p, q in THRESHOLDS],
                      "window_pairs_per_step": int(total_win),
                      "inputs": drawn,
                      "impl": "CPU oracle: plain all-pairs merge join, exact integer Jaccard"},
           "ms_per_step_measured": "wall time of the step's row sample",
           "extrapolated_full_join_ms_per_step": round(statistics.mean(t_full) * 1e3, 1),
           "cpu_baseline": {"value": round(value), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0},
           "run_s": round(time.perf_counter() - t_start, 1)}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
