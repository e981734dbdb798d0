"""Serve a short query stream against the resident index (a small driver for profilers).

    python -m paper_1711_07295_b300.profile_serve --queries 2000 [--rate 20000]

The index holds the 2,000,000-set served workload (Zipf(s=1.1) tokens over
300,000, sizes lognormal(2.3, 0.6) in [1, 500], drawn on the device); the
probes are the served workload's (sizes U[2,300], half edited copies of
resident sets, thresholds from {1/2, 3/4, 9/10}), arriving as a Poisson
stream at --rate queries/s (0: all at time 0), the index at --b bits (128 by
default, the width the bench serves at).  One warm-up stream of 200
queries runs first, so that a profiler sees steady-state batches.
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
    ap.add_argument("--queries", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=20000.0)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--b", type=int, default=128, help="bitmap width of the index")
    args = ap.parse_args()
    import numpy as np
    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    spec = inputs.spec_resident_2m()
    off_d, tok_d = inputs.gen_collection_device(spec, device="cuda")
    off, tok = off_d.cpu().numpy(), tok_d.cpu().numpy()
    rate = args.rate if args.rate > 0 else 20000.0
    qs = inputs.QuerySpec(n_queries=args.queries + 200, rate_qps=rate)
    arr, qoff, qtok, p, q = inputs.gen_queries(qs, spec, off, tok)
    idx = _bmj.Index(off_d, tok_d, b=args.b)
    w = 200
    idx.serve(qoff[:w + 1], qtok[:int(qoff[w])], arr[:w], p[:w], q[:w])   # warm-up
    o2 = (qoff[w:] - qoff[w]).astype(np.int64)
    t2 = qtok[int(qoff[w]):]
    a2 = arr[w:] - arr[w] if args.rate > 0 else np.zeros(args.queries)
    _, lat, st = idx.serve(o2, t2, a2, p[w:], q[w:], n_slots=args.slots, want_results=False)
    idx.close()
    torch.cuda.synchronize()
    print(json.dumps({"queries": args.queries, "rate": args.rate, **st}))


if __name__ == "__main__":
    main()
