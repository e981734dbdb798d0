#!/usr/bin/env python
"""Benchmark of the Bitmap Filter exact self-join on B300.

Workload: self-join of 1,000,000 sets (tokens Zipf(s=1.1) over a 200,000-token
universe, sizes lognormal(mu=2.3, sigma=0.6) rounded and clipped to [1, 500],
seed 0), synthetic.  One step = the four joins at Jaccard thresholds 1/2, 3/4,
9/10 and 19/20, each through the C ABI with the collection resident in HBM:
size sort, bitmap build, Bitmap Filter over the length window, exact
verification, canonical result sort.  b = 64 bits, Bitmap-Xor (the fastest
whole join at every one of these thresholds among b in {64, 128, 256}; the
--sweep option times the other widths).

Metric: pairs filtered/s = window pairs evaluated by the Bitmap Filter
(pairs inside the length-filter window, the paper's Alg. 6 inner loop) per
second of whole-join time.  The filter kernel's own rate goes into the
roofline object.

--impl reference times the CPU oracle (plain all-pairs join with exact
integer Jaccard) on a bounded row sample of the same workload, extrapolated
to the full join, on the host cores.
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

THRESHOLDS = ((1, 2), (3, 4), (9, 10), (19, 20))
METRIC = "pairs filtered/s"
UNIT = "pairs/s"
WORKLOAD = ("self-join of 1,000,000 sets, tokens Zipf(s=1.1) over 200,000, sizes "
            "lognormal(mu=2.3,sigma=0.6) clipped to [1,500], Jaccard 1/2, 3/4, 9/10, 19/20")
POPC_PER_CLK_PER_SM = 16      # 32-bit population count throughput per SM per clock
FLUSH_BYTES = 256 << 20       # > 126 MB L2


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--sweep", action="store_true", help="also time b = 128 and 256")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=12,
                    help="least oracle rows sampled per threshold for the CPU baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0,
                    help="target wall time of the CPU baseline's sample (rows are scaled to it)")
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
    ap.add_argument("--no-10m", action="store_true",
                    help="skip the 10,000,000-set joins (b = 128, thresholds 3/5 and 9/10)")
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


def filter_source_digest() -> str:
    """sha256[:16] of the sources the filter kernel is built from."""
    h = hashlib.sha256()
    for name in ("filter_core.cuh", "kernels.cuh", "filter.cu"):
        with open(os.path.join(ROOT, "paper_1711_07295_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_traffic(b: int):
    """DRAM bytes per filter launch (mean over one step's launches) from the
    committed ncu summary, if it was taken on the current filter source."""
    path = os.path.join(ROOT, "profiles", f"filter_1m_b{b}.md")
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


# ----------------------------------------------------------------------------
# CPU oracle timing (rank 0 only)
# ----------------------------------------------------------------------------
def oracle_rate(off, tok, window_by_thr, rows_per_thr: int, seed: int = 0, windowed=False):
    """Time the oracle on ``rows_per_thr`` sampled rows per threshold and
    extrapolate the full self-join time (each sampled row is scanned against
    all N sets; the full join verifies N(N-1)/2 pairs, i.e. N/2 per row).
    ``windowed``: the row scan with the length filter of Table 2 instead
    (each row against its two-sided size window; every window pair of the
    full join is met from both ends, so again half of the rows' sum)."""
    import numpy as np
    import oracle
    scan = oracle.join_rows_window if windowed else oracle.join_rows
    n = len(off) - 1
    rng = np.random.default_rng(seed)
    # enough rows to occupy every oracle thread (rows are its unit of parallelism)
    rows_per_thr = max(rows_per_thr, 2 * oracle.num_threads())
    t_full = 0.0
    t_cpu = 0.0
    for (p, q) in THRESHOLDS:
        rows = rng.choice(n, size=rows_per_thr, replace=False)
        t0 = time.perf_counter()
        scan(off, tok, p, q, rows)
        dt = time.perf_counter() - t0
        t_cpu += dt
        t_full += dt / rows_per_thr * (n / 2.0)
    total_window = sum(window_by_thr.values())
    return total_window / t_full, t_full, t_cpu, min(oracle.num_threads(), rows_per_thr), \
        rows_per_thr


# ----------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1711_07295_b300 import _bmj, inputs

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank)
    off, tok = inputs.gen_collection(inputs.spec_1m(seed=0))
    d_off = torch.from_numpy(off).to(dev)
    d_tok = torch.from_numpy(tok).to(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    host_coll = {}
    bands = {}
    if world > 1 and args.shard == "bands":
        from paper_1711_07295_b300 import shard
        for (p, q) in THRESHOLDS:
            bands[(p, q)] = shard.band_split(off, p, q, world)[rank]

    def join(p, q, b, cap=0, host=False, method=_bmj.BMJ_XOR):
        r0, r1 = bands.get((p, q), (0, 0))
        if host:
            return _bmj.bmj_self_join(host_coll["off"], host_coll["tok"], p, q, b=b,
                                      queue_cap=cap, row_begin=r0, row_end=r1, method=method)
        res, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                        queue_cap=cap, stream=stream.cuda_stream,
                                        row_begin=r0, row_end=r1, method=method)
        res.release()
        return st

    b = args.b
    caps = {}
    for _ in range(max(args.warmup, 1)):
        for (p, q) in THRESHOLDS:
            st = join(p, q, b, caps.get((p, q), 0))
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
    per_thr = {thr: {"window": 0, "survivors": 0, "results": 0, "ms_filter": 0.0,
                     "ms_verify": 0.0, "ms_total": 0.0, "ms_prepare": 0.0, "ms_output": 0.0}
               for thr in THRESHOLDS}
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        torch.cuda.synchronize()
        ev0.record(stream)
        for thr in THRESHOLDS:
            st = join(thr[0], thr[1], b, caps[thr])
            d = per_thr[thr]
            d["window"] = st["window_pairs"]
            d["survivors"] = st["survivors"]
            d["results"] = st["results"]
            for key in ("ms_filter", "ms_verify", "ms_total", "ms_prepare", "ms_output"):
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

    # ---- roofline of the dominant kernel (the Bitmap Filter) ----
    peaks, peak_src = load_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    popc_per_pair = b // 32
    filt_ms = sum(per_thr[t]["ms_filter"] for t in THRESHOLDS)
    popc_ops = window_per_step * args.steps * popc_per_pair
    achieved = popc_ops / (filt_ms / 1e3) / 1e12
    peak = sms * POPC_PER_CLK_PER_SM * max_mhz * 1e6 / 1e12
    # At b = 64 one row in eight counts its bits on the ALU pipe instead of
    # POPC, so the joint bound of the XU and ALU pipes for that mix is 8/7 of
    # the POPC-pipe peak.
    mixed = peak * (8.0 / 7.0) if b == 64 else peak
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4),
                "unit": "Tpopc32/s", "frac": round(achieved / peak, 4),
                "traffic": profile_traffic(b),
                "kernel": f"k_filter_tma<W={b // 64}> (Bitmap Filter, TMA-staged columns)",
                "peak_derivation": f"{sms} SMs x {POPC_PER_CLK_PER_SM} POPC/clk/SM x "
                                   f"{max_mhz:.0f} MHz (max SM clock); work = b/32 32-bit "
                                   f"popcounts per window pair",
                "peak_xu_plus_alu": round(mixed, 4),
                "frac_of_xu_plus_alu": round(achieved / mixed, 4),
                "filter_pairs_per_s": round(window_per_step * args.steps / (filt_ms / 1e3)),
                "filter_share_of_step": round(filt_ms / sum(step_ms), 4)}
    try:  # the same peak measured by a POPC-only loop on this device (untimed region)
        popc_meas = _bmj.bmj_measure_popc_rate(stream.cuda_stream) / 1e12
        roofline["peak_measured"] = round(popc_meas, 4)
        roofline["frac_of_measured"] = round(achieved / popc_meas, 4)
    except Exception as e:  # reported, never fatal to the headline line
        roofline["peak_measured"] = f"unavailable: {type(e).__name__}: {e}"
    if clk.get("sm_mhz"):
        roofline["frac_at_median_clock"] = round(
            achieved / (sms * POPC_PER_CLK_PER_SM * clk["sm_mhz"] * 1e6 / 1e12), 4)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pinned = (torch.from_numpy(off).pin_memory(), torch.from_numpy(tok).pin_memory())
        host_coll["off"], host_coll["tok"] = pinned[0].numpy(), pinned[1].numpy()
        join(1, 2, b, caps[(1, 2)], host=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        d2h = 0
        t0 = time.perf_counter()
        for k in range(args.steps):
            for thr in THRESHOLDS:
                a, bb, st = join(thr[0], thr[1], b, caps[thr], host=True)
                d2h += a.nbytes + bb.nbytes
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = len(THRESHOLDS) * (off.nbytes + tok.nbytes)
        e2e = {"value": round(units_per_step_all * args.steps / e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h // args.steps),
               "ms_per_step": round(e2e_s * 1e3 / args.steps, 3),
               "inputs": "pinned host CSR, copied by the library each call"}

    # ---- the same step with Alg. 4's choice of generation function ----
    # (the paper's GPU runs use Bitmap-Xor, as the headline does; Alg. 4 picks
    # Bitmap-Set at 1/2, which leaves fewer survivors for verification)
    combined = None
    if not args.no_combined:
        ccaps = {}
        for thr in THRESHOLDS:
            st = join(thr[0], thr[1], b, method=_bmj.BMJ_COMBINED)
            ccaps[thr] = max(1, st["survivors"])
        flush.fill_(7)
        torch.cuda.synchronize()
        ev0.record(stream)
        surv, meth = {}, {}
        for thr in THRESHOLDS:
            st = join(thr[0], thr[1], b, ccaps[thr], method=_bmj.BMJ_COMBINED)
            surv[f"{thr[0]}/{thr[1]}"] = st["survivors"]
            meth[f"{thr[0]}/{thr[1]}"] = ("xor", "set", "next")[st["method"]]
        ev1.record(stream)
        torch.cuda.synchronize()
        c_ms = ev0.elapsed_time(ev1)
        combined = {"method": meth, "ms_per_step": round(c_ms, 3),
                    "value": round(window_per_step / (c_ms / 1e3)), "unit": UNIT,
                    "survivors": surv, "steps": 1}

    # ---- the other similarity functions of Table 1 on the same collection ----
    sims = None
    if not args.no_sims:
        sims = {}
        cases = (("cosine", _bmj.BMJ_COSINE, THRESHOLDS), ("dice", _bmj.BMJ_DICE, THRESHOLDS),
                 ("overlap", _bmj.BMJ_OVERLAP, ((10, 1), (20, 1))))
        for name, sim, thr_list in cases:
            rows = []
            for (p, q) in thr_list:
                st0 = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, sim=sim, output_on_device=True,
                                         stream=stream.cuda_stream)
                st0[0].release()
                r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, sim=sim,
                                              output_on_device=True, stream=stream.cuda_stream)
                r.release()
                rows.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                             "survivors": st["survivors"], "results": st["results"],
                             "filter_passes": st["filter_passes"],
                             "join_ms": round(st["ms_total"], 3),
                             "pairs_per_s": round(st["window_pairs"] / (st["ms_total"] / 1e3)),
                             "filter_pairs_per_s": round(st["window_pairs"] /
                                                         max(st["ms_filter"] / 1e3, 1e-9))})
            sims[name] = rows

    # ---- prefix-filter candidates (Section 2.2) against the whole window ----
    prefix = None
    if not args.no_prefix:
        prefix = []
        for (p, q) in THRESHOLDS:
            r, _, _ = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                         candidates=_bmj.BMJ_CAND_PREFIX, stream=stream.cuda_stream)
            r.release()
            r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                          candidates=_bmj.BMJ_CAND_PREFIX,
                                          stream=stream.cuda_stream)
            r.release()
            wj = per_thr[(p, q)]["ms_total"] / args.steps
            prefix.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                           "candidates": st["candidates"], "survivors": st["survivors"],
                           "results": st["results"], "join_ms": round(st["ms_total"], 3),
                           "candidate_ms": round(st["ms_filter"], 3),
                           "window_join_ms": round(wj, 3),
                           "speedup_vs_window": round(wj / st["ms_total"], 3)})

    # ---- the cutoff point (Section 3.5): pairs above it skip the filter ----
    cutoff = None
    if not args.no_cutoff:
        cutoff = []
        for (p, q) in THRESHOLDS:
            for rep in range(2):
                r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True,
                                              cutoff=_bmj.BMJ_CUTOFF_AUTO,
                                              stream=stream.cuda_stream)
                r.release()
            wj = per_thr[(p, q)]["ms_total"] / args.steps
            cutoff.append({"threshold": f"{p}/{q}", "cutoff": st["cutoff"],
                           "window_pairs": st["window_pairs"], "survivors": st["survivors"],
                           "survivors_without": per_thr[(p, q)]["survivors"],
                           "results": st["results"], "join_ms": round(st["ms_total"], 3),
                           "verify_ms": round(st["ms_verify"], 3),
                           "window_join_ms": round(wj, 3),
                           "speedup_vs_no_cutoff": round(wj / st["ms_total"], 3)})

    # ---- RS-join (Section 2.1): the collection against a second one of its kind ----
    rs = None
    if not args.no_rs:
        rs = []
        s_off, s_tok = inputs.gen_collection(inputs.spec_1m(seed=1))
        ds_off, ds_tok = torch.from_numpy(s_off).to(dev), torch.from_numpy(s_tok).to(dev)
        for (p, q) in ((9, 10), (3, 4)):
            for rep in range(2):  # the first call warms the pools
                r, _, st = _bmj.bmj_rs_join(d_off, d_tok, ds_off, ds_tok, p, q, b=b,
                                            output_on_device=True, stream=stream.cuda_stream)
                r.release()
            for rep in range(2):
                r, _, sx = _bmj.bmj_rs_join(d_off, d_tok, ds_off, ds_tok, p, q, b=b,
                                            output_on_device=True, stream=stream.cuda_stream,
                                            candidates=_bmj.BMJ_CAND_PREFIX)
                r.release()
            rs.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                       "survivors": st["survivors"], "results": st["results"],
                       "join_ms": round(st["ms_total"], 3), "filter_ms": round(st["ms_filter"], 3),
                       "pairs_per_s": round(st["window_pairs"] / (st["ms_total"] / 1e3)),
                       "filter_pairs_per_s": round(st["window_pairs"] /
                                                   max(st["ms_filter"] / 1e3, 1e-9)),
                       "prefix_filter": {"candidates": sx["candidates"], "results": sx["results"],
                                         "join_ms": round(sx["ms_total"], 3),
                                         "speedup_vs_window": round(st["ms_total"] /
                                                                    sx["ms_total"], 3)}})
        del ds_off, ds_tok

    # ---- optional b sweep (outside the headline) ----
    sweep = None
    if args.sweep:
        sweep = {}
        for bw in (64, 128, 256):
            tot = 0.0
            filt = 0.0
            for thr in THRESHOLDS:
                st0 = join(thr[0], thr[1], bw)
                st = join(thr[0], thr[1], bw, max(1, st0["survivors"]))
                tot += st["ms_total"]
                filt += st["ms_filter"]
            sweep[str(bw)] = {"step_ms": round(tot, 3), "filter_ms": round(filt, 3),
                              "filter_pairs_per_s": round(window_per_step / (filt / 1e3))}

    batched = None
    if not args.no_batched:
        try:
            batched = run_batched(args, dev)
        except Exception as e:  # reported, never fatal to the headline line
            batched = {"error": f"{type(e).__name__}: {e}"}

    ten_m = None
    if not args.no_10m:
        try:
            ten_m = run_ten_million(args, dev)
        except Exception as e:  # reported, never fatal to the headline line
            ten_m = {"error": f"{type(e).__name__}: {e}"}

    served = None
    if not args.no_served:
        try:
            served = run_served(args, dev)
        except Exception as e:  # reported, never fatal to the headline line
            served = {"error": f"{type(e).__name__}: {e}"}

    # last, so that its host threads disturb none of the GPU measurements above
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        win = {thr: per_thr[thr]["window"] for thr in THRESHOLDS}

        def sampled(windowed, budget_s):
            rate, t_full, t_cpu, cores, nrows = oracle_rate(off, tok, win, args.cpu_rows,
                                                            windowed=windowed)
            if t_cpu < budget_s / 2:  # calibration run: scale the sample to the budget
                rows = int(nrows * budget_s / max(t_cpu, 1e-3))
                rows = max(nrows, min(rows, 256 * nrows, (len(off) - 1) // 2))
                rate, t_full, t_cpu, cores, nrows = oracle_rate(off, tok, win, rows, seed=1,
                                                                windowed=windowed)
            return rate, t_full, t_cpu, cores, nrows

        rate, t_full, t_cpu, cores, nrows = sampled(False, args.cpu_seconds)
        w_rate, w_full, w_cpu, _, w_rows = sampled(True, args.cpu_seconds / 3)
        cpu = {"value": round(rate), "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{nrows} random rows per threshold scanned against all "
                         f"1,000,000 sets ({t_cpu:.1f} s wall on {cores} threads), extrapolated to the "
                         f"full join ({t_full:.0f} s per step)",
               "with_length_filter": {
                   "value": round(w_rate), "unit": UNIT,
                   "sample": f"{w_rows} random rows per threshold, each against the sets of its "
                             f"Table 2 size window ({w_cpu:.1f} s wall), extrapolated to the full "
                             f"join ({w_full:.0f} s per step)"}}

    if rank == 0:
        joins = []
        for thr in THRESHOLDS:
            d = per_thr[thr]
            joins.append({"threshold": f"{thr[0]}/{thr[1]}", "window_pairs": d["window"],
                          "survivors": d["survivors"], "results": d["results"],
                          "join_ms": round(d["ms_total"] / args.steps, 3),
                          "filter_ms": round(d["ms_filter"] / args.steps, 3),
                          "verify_ms": round(d["ms_verify"] / args.steps, 3),
                          "prepare_ms": round(d["ms_prepare"] / args.steps, 3),
                          "output_ms": round(d["ms_output"] / args.steps, 3)})
        out = {"metric": METRIC, "value": round(value), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
               "scaling": "strong" if bands else "weak", "vs_baseline": None, "dtype": "u64",
               "data": "synthetic",
               "config": {"workload": WORKLOAD, "n_sets": int(len(off) - 1),
                          "tokens": int(len(tok)), "thresholds": [f"{p}/{q}" for p, q in THRESHOLDS],
                          "b": b, "method": "xor",
                          "parallelism": (f"row bands x{world}" if bands else f"replicas x{world}"),
                          "l2": "flushed between steps (256 MB write, untimed)",
                          "inputs": "resident in HBM", "peaks": peak_src},
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(launches), "clocks": clk, "joins": joins}
        if sweep:
            out["sweep_b"] = sweep
        if combined:
            out["combined_method"] = combined
        if prefix:
            out["prefix_filter"] = {"workload": "the 1,000,000-set collection at b = " + str(b) +
                                                ", candidates from the prefix filter, one join "
                                                "per threshold, against the step's window joins",
                                    "joins": prefix}
        if cutoff:
            out["cutoff_point"] = {"workload": "the 1,000,000-set collection at b = " + str(b) +
                                               ", cutoff from Eq. 4-6 (Xor, normalised threshold "
                                               "2p/(p+q)), against the step's joins",
                                   "joins": cutoff}
        if rs:
            out["rs_join"] = {"workload": "R = the 1,000,000-set collection, S = a second one "
                                          "(same recipe, seed 1), b = " + str(b) +
                                          ", inputs in HBM, one join per threshold",
                              "joins": rs}
        if sims:
            out["similarity_functions"] = {
                "workload": "the 1,000,000-set collection at b = " + str(b) + ", one join per "
                            "threshold (Overlap thresholds count tokens)", **sims}
        if batched:
            out["batched"] = batched
        if ten_m:
            out["ten_million"] = ten_m
        if served:
            out["served"] = served
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


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


def run_ten_million(args, dev):
    """The 10,000,000-set workload (Zipf(1.0) over 1,000,000 tokens, sizes
    lognormal(2.0,0.8) in [1,1000], CSR in HBM) joined at 3/5 and 9/10 with
    b = 128: one untimed join, then each threshold once (CUDA-event stage
    times reported by the library)."""
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    t0 = time.perf_counter()
    off, tok = inputs.gen_collection_device(inputs.spec_10m(), device=dev)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    r, _, _ = _bmj.bmj_self_join(off, tok, 9, 10, b=128, output_on_device=True,
                                 stream=stream.cuda_stream)
    r.release()
    out = []
    for p, q in ((3, 5), (9, 10)):
        r, _, st = _bmj.bmj_self_join(off, tok, p, q, b=128, output_on_device=True,
                                      stream=stream.cuda_stream)
        r.release()
        out.append({"threshold": f"{p}/{q}", "window_pairs": st["window_pairs"],
                    "survivors": st["survivors"], "results": st["results"],
                    "join_ms": round(st["ms_total"], 2), "filter_ms": round(st["ms_filter"], 2),
                    "verify_ms": round(st["ms_verify"], 2),
                    "pairs_per_s": round(st["window_pairs"] / (st["ms_total"] / 1e3)),
                    "filter_pairs_per_s": round(st["window_pairs"] / (st["ms_filter"] / 1e3))})
    for p, q in ((3, 5), (9, 10)):   # the same joins with prefix-filter candidates
        r, _, st = _bmj.bmj_self_join(off, tok, p, q, b=128, output_on_device=True,
                                      candidates=_bmj.BMJ_CAND_PREFIX, stream=stream.cuda_stream)
        r.release()
        win = next(x for x in out if x["threshold"] == f"{p}/{q}")
        win["prefix_filter"] = {"candidates": st["candidates"], "survivors": st["survivors"],
                                "results": st["results"], "join_ms": round(st["ms_total"], 2),
                                "candidate_ms": round(st["ms_filter"], 2),
                                "speedup_vs_window": round(win["join_ms"] / st["ms_total"], 3)}
    # the cutoff point of Section 3.5 (Eq. 4-6) on the long size tail at 3/5
    if not args.no_cutoff:
        r, _, st = _bmj.bmj_self_join(off, tok, 3, 5, b=128, output_on_device=True,
                                      cutoff=_bmj.BMJ_CUTOFF_AUTO, stream=stream.cuda_stream)
        r.release()
        win = next(x for x in out if x["threshold"] == "3/5")
        win["cutoff_point"] = {"cutoff": st["cutoff"], "survivors": st["survivors"],
                               "results": st["results"], "join_ms": round(st["ms_total"], 2),
                               "filter_ms": round(st["ms_filter"], 2),
                               "verify_ms": round(st["ms_verify"], 2),
                               "speedup_vs_no_cutoff": round(win["join_ms"] / st["ms_total"], 3)}
    del off, tok
    torch.cuda.empty_cache()
    return {"workload": "self-join of 10,000,000 sets, tokens Zipf(s=1.0) over 1,000,000, sizes "
                        "lognormal(mu=2.0,sigma=0.8) clipped to [1,1000], b = 128, inputs in HBM",
            "joins": out, "generation_s": round(gen_s, 2)}


def run_served(args, dev):
    """A Poisson stream of 20,000 queries/s against a resident index of
    2,000,000 sets: continuous batching (4 slots) against one query per
    launch (1 slot, batches of 1), same arrivals."""
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
    idx = _bmj.Index(off_d, tok_d, b=64)
    idx.serve(qoff[:201], qtok[:int(qoff[200])], arr[:200], p[:200], q[:200])   # warm-up
    _, lat, st = idx.serve(qoff, qtok, arr, p, q, n_slots=4, max_batch_queries=4096,
                           want_results=False)
    _, lat1, st1 = idx.serve(qoff, qtok, arr, p, q, n_slots=1, max_batch_queries=1,
                             want_results=False)
    # capacity: the same queries all waiting at time 0
    _, lat0, st0 = idx.serve(qoff, qtok, np.zeros_like(arr), p, q, n_slots=4,
                             max_batch_queries=4096, want_results=False)
    idx.close()
    return {"workload": "resident index of 2,000,000 sets (Zipf(s=1.1) over 300,000, sizes "
                        "lognormal(2.3,0.6) in [1,500]); Poisson arrivals at 20,000 queries/s, "
                        "20,000 probes of size U[2,300] (half edited resident copies), "
                        "thresholds from {1/2,3/4,9/10}, b = 64",
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
                          "arrivals": "all 20,000 queries at time 0"},
            "generation_s": round(gen_s, 2)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_1711_07295_b300 import inputs
    off, tok = inputs.gen_collection(inputs.spec_1m(seed=0))
    sizes = np.diff(off)
    # window pairs per threshold from the size histogram (same count the GPU reports)
    hist = np.bincount(sizes)
    win = {}
    cum = np.concatenate([[0], np.cumsum(hist)])
    for (p, q) in THRESHOLDS:
        tot = 0
        for s in range(1, len(hist)):
            c = int(hist[s])
            if c == 0:
                continue
            lo = -(-p * s // q)
            tot += c * (c - 1) // 2 + c * int(cum[s] - cum[min(lo, s)])
        win[(p, q)] = tot
    rows = max(2, args.cpu_rows // 3)
    for _ in range(args.warmup):
        oracle_rate(off, tok, win, rows, seed=1)
    t_step = []
    cores = 1
    t_cpu_total = 0.0
    for k in range(args.steps):
        rate, t_full, t_cpu, cores, rows = oracle_rate(off, tok, win, rows, seed=100 + k)
        t_step.append(t_full)
        t_cpu_total += t_cpu
    total_window = sum(win.values())
    value = total_window * args.steps / sum(t_step)
    sample = (f"{rows} random rows per threshold per step scanned against all 1,000,000 sets, "
              f"extrapolated to the full join ({t_cpu_total:.1f} s wall on {cores} threads in total)")
    out = {"impl": "reference", "metric": METRIC, "value": round(value), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(statistics.mean(t_step) * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n_sets": int(len(off) - 1),
                      "thresholds": [f"{p}/{q}" for p, q in THRESHOLDS],
                      "impl": "CPU oracle: plain all-pairs merge join, exact integer Jaccard"},
           "cpu_baseline": {"value": round(value), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
