"""Run one self-join (or RS-join) on a synthetic collection (a small driver for profilers).

    python -m paper_1711_07295_b300.profile_join --sets 1000000 --p 19 --q 20 --b 64
    python -m paper_1711_07295_b300.profile_join --sets 1000000 --rs-sets 1000000 --p 9 --q 10

The collection is the 1,000,000-set workload shape (Zipf(s=1.1) tokens over
200,000, sizes lognormal(2.3, 0.6) in [1, 500]) truncated or extended to
--sets sets (seed 0); --shape 10m takes the 10,000,000-set workload's shape
instead (Zipf(s=1.0) over 1,000,000, sizes lognormal(2.0, 0.8) in [1, 1000],
drawn on the device).  The join runs --repeat times with the survivor queue
sized from a first call, so that a profiler sees steady-state launches.
With --rs-sets N the join is an RS-join against a second collection of the
same shape with N sets (seed 1).
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
    ap.add_argument("--sets", type=int, default=1_000_000)
    ap.add_argument("--p", type=int, default=19)
    ap.add_argument("--q", type=int, default=20)
    ap.add_argument("--b", type=int, default=64)
    ap.add_argument("--method", default="xor")
    ap.add_argument("--sim", default="jaccard", choices=("jaccard", "cosine", "dice", "overlap"))
    ap.add_argument("--candidates", default="window", choices=("window", "prefix"))
    ap.add_argument("--cutoff", type=int, default=0, help="cutoff point (-1: from Eq. 4-6)")
    ap.add_argument("--rs-sets", type=int, default=0, help="RS-join against this many sets")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--shape", default="1m", choices=("1m", "10m"))
    args = ap.parse_args()

    import torch
    from paper_1711_07295_b300 import _bmj, inputs
    spec = inputs.spec_1m(seed=0) if args.shape == "1m" else inputs.spec_10m(seed=0)
    spec = inputs.CollectionSpec(args.sets, spec.universe, spec.zipf_s, spec.size_dist, seed=0)
    if args.shape == "10m":
        d_off, d_tok = inputs.gen_collection_device(spec)
    else:
        off, tok = inputs.gen_collection(spec)
        d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    m = _bmj.METHODS[args.method]
    sim = {"jaccard": _bmj.BMJ_JACCARD, "cosine": _bmj.BMJ_COSINE, "dice": _bmj.BMJ_DICE,
           "overlap": _bmj.BMJ_OVERLAP}[args.sim]
    cand = _bmj.BMJ_CAND_PREFIX if args.candidates == "prefix" else _bmj.BMJ_CAND_WINDOW
    kw = dict(b=args.b, method=m, sim=sim, output_on_device=True, candidates=cand,
              cutoff=args.cutoff)
    if args.rs_sets > 0:
        s_spec = inputs.CollectionSpec(args.rs_sets, spec.universe, spec.zipf_s, spec.size_dist,
                                       seed=1)
        s_off, s_tok = inputs.gen_collection(s_spec)
        ds_off, ds_tok = torch.from_numpy(s_off).cuda(), torch.from_numpy(s_tok).cuda()

        def join(**extra):
            return _bmj.bmj_rs_join(d_off, d_tok, ds_off, ds_tok, args.p, args.q, **kw, **extra)
    else:
        def join(**extra):
            return _bmj.bmj_self_join(d_off, d_tok, args.p, args.q, **kw, **extra)
    res, _, st = join()
    res.release()
    # window mode: the survivor queue sized from the first call; prefix mode sizes
    # its candidate ranges itself (a queue_cap there would cut them to that many slots)
    extra = {"queue_cap": max(1, st["survivors"])} if cand == _bmj.BMJ_CAND_WINDOW else {}
    for _ in range(args.repeat):
        res, _, st = join(**extra)
        res.release()
    torch.cuda.synchronize()
    print(json.dumps({"sets": args.sets, "rs_sets": args.rs_sets,
                      "threshold": f"{args.p}/{args.q}", "b": args.b, "sim": args.sim, **st}))


if __name__ == "__main__":
    main()
