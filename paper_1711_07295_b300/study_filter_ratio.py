"""Filtering ratio of the Bitmap Filter per generation method and bitmap size
on a synthetic collection (the study of the paper's filter-ratio figures,
Section 5, here on the 1,000,000-set synthetic workload).

    python -m paper_1711_07295_b300.study_filter_ratio [--sets 1000000]

For every method (Xor, Set, Next), b in {64, 128, 256} and Jaccard threshold,
one self-join reports window pairs, survivors and results; the filtering
ratio is 1 - survivors / window pairs and the precision results / survivors.
Prints one JSON line per join and a markdown table.

    python -m paper_1711_07295_b300.study_filter_ratio --by-size

gives the filter's pass rate (survivors / window pairs) and precision per
size of the pair's larger set instead (the paper's
filtering-precision study, Section 5.1: b = 64, Xor, Jaccard thresholds 0.5 to
0.8, no cutoff), next to the cutoff point the library derives for each
threshold (Section 3.5), where the precision is expected to fall off.  A size
bucket is a band of rows of the size-sorted collection, joined alone
(``row_begin``/``row_end``: the pairs whose later set, the larger one, lies in
the band).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


SIZE_EDGES = (1, 6, 11, 16, 21, 31, 41, 51, 61, 81, 101, 151)


def size_band_rows(sizes, edges):
    """Row ranges of the size-sorted collection (sizes ascending, ties by id)
    holding the sets of size in [edges[k], edges[k+1]) (the last bucket open
    above): a list of (lo_size, hi_size or None, row_begin, row_end)."""
    import numpy as np
    s = np.asarray(sizes, dtype=np.int64)
    out = []
    for k, lo in enumerate(edges):
        hi = edges[k + 1] if k + 1 < len(edges) else None
        r0 = int(np.count_nonzero(s < lo))
        r1 = int(np.count_nonzero(s < hi)) if hi is not None else len(s)
        out.append((lo, hi, r0, r1))
    return out


def by_size(_bmj, d_off, d_tok, sizes):
    rows = []
    bands = [bd for bd in size_band_rows(sizes, SIZE_EDGES) if bd[3] > bd[2]]
    for p, q in ((1, 2), (3, 5), (7, 10), (4, 5)):
        # the cutoff point the library takes for this threshold (one-row join)
        r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=64, output_on_device=True,
                                      cascade_b=-1, row_begin=0, row_end=1,
                                      cutoff=_bmj.BMJ_CUTOFF_AUTO)
        r.release()
        omega = st["cutoff"]
        for lo, hi, r0, r1 in bands:
            r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=64, output_on_device=True,
                                          cascade_b=-1, row_begin=r0, row_end=r1)
            r.release()
            w, s, res = st["window_pairs"], st["survivors"], st["results"]
            row = {"threshold": f"{p}/{q}", "omega": omega,
                   "larger_size": f"{lo}-{hi - 1}" if hi else f"{lo}+",
                   "window_pairs": w, "survivors": s, "results": res,
                   "pass_rate": s / w if w else None,
                   "precision": res / s if s else None}
            rows.append(row)
            print(json.dumps(row), flush=True)
    print("\n| threshold | ω(64, τ) | larger set size | window pairs | survivors | results | "
          "pass rate | precision |")
    print("|---|---:|---|---:|---:|---:|---:|---:|")
    for r in rows:
        rate = f"{r['pass_rate']:.4f}" if r["pass_rate"] is not None else "-"
        prec = f"{r['precision']:.4f}" if r["precision"] is not None else "-"
        print(f"| {r['threshold']} | {r['omega']} | {r['larger_size']} | {r['window_pairs']:.3e} | "
              f"{r['survivors']} | {r['results']} | {rate} | {prec} |")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=1_000_000)
    ap.add_argument("--by-size", action="store_true",
                    help="precision per size of the larger set (b = 64, Xor) instead")
    ap.add_argument("--planted", type=float, default=0.0,
                    help="fraction of sets replaced by edited copies of others (near duplicates)")
    args = ap.parse_args()
    import numpy as np
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    spec = dataclasses.replace(inputs.spec_1m(), n_sets=args.sets, planted_frac=args.planted)
    off, tok = inputs.gen_collection(spec)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    if args.by_size:
        by_size(_bmj, d_off, d_tok, np.diff(off))
        return
    methods = (("xor", _bmj.BMJ_XOR), ("set", _bmj.BMJ_SET), ("next", _bmj.BMJ_NEXT))
    rows = []
    for p, q in ((1, 2), (3, 4), (9, 10), (19, 20)):
        for b in (64, 128, 256):
            for name, m in methods:
                r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, method=m,
                                              output_on_device=True, cascade_b=-1)
                r.release()
                w, s, res = st["window_pairs"], st["survivors"], st["results"]
                row = {"threshold": f"{p}/{q}", "b": b, "method": name, "window_pairs": w,
                       "survivors": s, "results": res,
                       "filter_ratio": 1.0 - s / w if w else 0.0,
                       "precision": res / s if s else 1.0,
                       "ms_filter": round(st["ms_filter"], 3), "ms_verify": round(st["ms_verify"], 3)}
                rows.append(row)
                print(json.dumps(row), flush=True)
    print("\n| threshold | b | method | filtering ratio | precision | filter ms | verify ms |")
    print("|---|---:|---|---:|---:|---:|---:|")
    for r in rows:
        print(f"| {r['threshold']} | {r['b']} | {r['method']} | {r['filter_ratio']:.5f} | "
              f"{r['precision']:.4f} | {r['ms_filter']} | {r['ms_verify']} |")


if __name__ == "__main__":
    main()
