"""Run the batched workload once (a small driver for profilers).

    python -m paper_1711_07295_b300.profile_batch [--jobs 512] [--repeat 1]

512 independent self-joins (sets per job log-uniform 1,000-200,000, sizes
U[3,100], Zipf(1.0) tokens over 50,000, thresholds from {1/2,7/10,4/5,9/10}),
drawn on the device, joined by bmj_self_join_batch with the autotuner and
the graph-captured execute stage.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=512)
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args()
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    off, tok, js, p, q = inputs.gen_batch_device(inputs.BatchSpec(n_jobs=args.jobs))
    for _ in range(args.repeat):
        pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=0, use_graph=True)
    torch.cuda.synchronize()
    print(json.dumps(bst))


if __name__ == "__main__":
    main()
