"""Filtering ratio of the Bitmap Filter per generation method and bitmap size
on a synthetic collection (the study of the paper's filter-ratio figures,
Section 5, here on the 1,000,000-set synthetic workload).

    python -m paper_1711_07295_b300.study_filter_ratio [--sets 1000000]

For every method (Xor, Set, Next), b in {64, 128, 256} and Jaccard threshold,
one self-join reports window pairs, survivors and results; the filtering
ratio is 1 - survivors / window pairs and the precision results / survivors.
Prints one JSON line per join and a markdown table.
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sets", type=int, default=1_000_000)
    args = ap.parse_args()
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    spec = dataclasses.replace(inputs.spec_1m(), n_sets=args.sets)
    off, tok = inputs.gen_collection(spec)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
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
