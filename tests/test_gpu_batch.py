"""Batched self-joins (many independent jobs in one pass) against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1711_07295_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1711_07295_b300 import _bmj  # noqa: E402

OM = {_bmj.BMJ_XOR: O.XOR, _bmj.BMJ_SET: O.SET, _bmj.BMJ_NEXT: O.NEXT}


def make_batch(n_jobs, seed, lo=40, hi=2500, universe=3000, size_hi=60):
    rng = np.random.default_rng(seed)
    jobs = []
    ths = ((1, 2), (7, 10), (4, 5), (9, 10))
    for k in range(n_jobs):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        off, tok = I.random_collection(n, universe, 3, size_hi, seed=seed * 1000 + k,
                                       planted_frac=0.1)
        p, q = ths[int(rng.integers(0, 4))]
        jobs.append((off, tok, p, q))
    return jobs


def concat(jobs):
    offs, toks, js = [np.zeros(1, np.int64)], [], [0]
    base = 0
    for off, tok, _, _ in jobs:
        offs.append(off[1:] + base)
        toks.append(tok)
        base += int(off[-1])
        js.append(js[-1] + len(off) - 1)
    return (np.concatenate(offs), np.concatenate(toks).astype(np.int32), np.array(js, np.int64),
            np.array([j[2] for j in jobs], np.uint32), np.array([j[3] for j in jobs], np.uint32))


def check(jobs, pairs, jst, method=_bmj.BMJ_XOR, sim=_bmj.BMJ_JACCARD):
    for k, (off, tok, p, q) in enumerate(jobs):
        ra, rb = O.self_join(off, tok, p, q, sim=sim)
        a, b = pairs[k]
        assert np.array_equal(a, ra) and np.array_equal(b, rb), k
        m = OM.get(jst[k]["method"], O.XOR)
        w, s, r = O.filter_counts(off, tok, p, q, jst[k]["b"], m, sim=sim)
        assert (jst[k]["window_pairs"], jst[k]["survivors"], jst[k]["results"]) == (w, s, r), k


@pytest.mark.parametrize("b", [0, 64, 128, 256])
def test_batch_matches_oracle(b):
    jobs = make_batch(24, seed=b + 1)
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    pairs, jst, bst = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=b)
    check(jobs, pairs, jst)
    assert bst["tuned"] == (1 if b == 0 else 0)
    if b:
        assert all(s["b"] == b for s in jst)
    assert bst["results"] == sum(len(x[0]) for x in pairs)


@pytest.mark.parametrize("b,rows", [(0, 0), (0, 1), (64, 1), (128, 1), (256, 1), (64, 8)])
def test_batch_row_tiles(b, rows):
    # The row tile per job: chosen by the tuner's cost model (rows = 0), the small tile
    # forced for every job (rows below the width's default) or the default tile.  Pairs
    # and counts are the oracle's whatever the tile, and the job stats record it.
    jobs = make_batch(18, seed=60 + b + rows, lo=30, hi=4000)
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    pairs, jst, bst = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=b, rows_per_thread=rows,
                                               use_graph=True)
    check(jobs, pairs, jst)
    default = {64: 256, 128: 128, 256: 128}
    small = {64: 64, 128: 32, 256: 32}
    for k, st in enumerate(jst):
        assert st["tile_rows"] in (default[st["b"]], small[st["b"]]) and st["chunk_cols"] > 0
        if rows == 1:
            assert st["tile_rows"] == small[st["b"]]
        if rows == 8:
            assert st["tile_rows"] == default[st["b"]]
    if rows == 0:   # jobs of a few dozen sets take the small tile, the largest the default
        sizes = np.diff(js)
        assert jst[int(np.argmin(sizes))]["tile_rows"] == small[jst[int(np.argmin(sizes))]["b"]]


def test_batch_combined_method_and_host_input():
    jobs = make_batch(12, seed=7)
    off, tok, js, p, q = concat(jobs)
    pairs, jst, _ = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=128, method=_bmj.BMJ_COMBINED)
    for k, (_, _, pk, qk) in enumerate(jobs):
        assert jst[k]["method"] == O.combined_method(pk, qk)
    check(jobs, pairs, jst)


def test_batch_equals_single_joins_and_graph_mode():
    jobs = make_batch(16, seed=3)
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    plain, jst, bst = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=0)
    graphed, jst_g, bst_g = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=0, use_graph=True)
    assert bst_g["graph"] == 1 and bst["graph"] == 0
    for k, (o, t, pk, qk) in enumerate(jobs):
        a, b, st = _bmj.bmj_self_join(o, t, int(pk), int(qk), b=jst[k]["b"])
        assert np.array_equal(plain[k][0], a) and np.array_equal(plain[k][1], b)
        assert np.array_equal(graphed[k][0], a) and np.array_equal(graphed[k][1], b)
        assert st["survivors"] == jst[k]["survivors"] == jst_g[k]["survivors"]


def test_batch_overflow_empty_and_tiny_jobs():
    jobs = make_batch(10, seed=11)
    # an empty job, a one-set job and a job of identical sets
    one = (np.array([0, 3], np.int64), np.array([1, 2, 3], np.int32), 1, 2)
    same = (np.arange(0, 41, 4, dtype=np.int64), np.tile(np.array([5, 9, 70, 200], np.int32), 10), 1, 1)
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32), 3, 4)
    jobs = [empty] + jobs[:4] + [one, same] + jobs[4:] + [empty]
    off, tok, js, p, q = concat(jobs)
    pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=64, queue_cap=1)
    assert bst["filter_passes"] == 2
    check(jobs, pairs, jst)
    assert len(pairs[0][0]) == 0 and len(pairs[5][0]) == 0 and len(pairs[6][0]) == 45


def test_batch_device_output():
    jobs = make_batch(6, seed=5)
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    dev_pairs, jst, _ = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=64, output_on_device=True)
    host_pairs, _, _ = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=64)
    for k in range(len(jobs)):
        dp = dev_pairs[k]
        if isinstance(dp, tuple):
            assert len(dp[0]) == 0 == len(host_pairs[k][0])
            continue
        assert np.array_equal(dp.a.cpu().numpy().view(np.uint32), host_pairs[k][0])
        assert np.array_equal(dp.b.cpu().numpy().view(np.uint32), host_pairs[k][1])
        dp.release()


def test_device_generator_recipe():
    spec = I.CollectionSpec(200_000, 50_000, 1.0, ("uniform", 3, 100), seed=3)
    off, tok = I.gen_collection_device(spec)
    off, tok = off.cpu().numpy(), tok.cpu().numpy()
    sizes = np.diff(off)
    assert sizes.min() >= 3 and sizes.max() <= 100 and off[-1] == len(tok)
    assert tok.min() >= 0 and tok.max() < 50_000
    d = np.diff(tok.astype(np.int64))
    starts = off[1:-1]
    d[starts - 1] = 1                      # differences across set boundaries are free
    assert np.all(d > 0)                   # strictly increasing inside every set
    # Zipf(1): the most frequent token is token 0
    assert np.bincount(tok).argmax() == 0


def test_full_batched_workload_row_sampled():
    # 512 jobs, log-uniform 1,000-200,000 sets, sizes U[3,100], Zipf(1.0) over 50,000,
    # thresholds from {1/2, 7/10, 4/5, 9/10}; autotuned b, graph-captured execute stage.
    off, tok, js, p, q = I.gen_batch_device(I.BatchSpec())
    pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=0, use_graph=True)
    assert bst["tuned"] == 1 and bst["graph"] == 1
    h_off, h_tok = off.cpu().numpy(), tok.cpu().numpy()
    rng = np.random.default_rng(0)
    for k in rng.choice(len(js) - 1, 6, replace=False):
        lo, hi = int(js[k]), int(js[k + 1])
        o = h_off[lo:hi + 1] - h_off[lo]
        t = h_tok[h_off[lo]:h_off[hi]]
        rows = rng.choice(hi - lo, 12, replace=False)
        ra, rb = O.join_rows(o, t, int(p[k]), int(q[k]), rows)
        a, b = pairs[k]
        sel = np.isin(a, rows) | np.isin(b, rows)
        assert np.array_equal(a[sel], ra) and np.array_equal(b[sel], rb), k
        assert jst[k]["results"] == len(a) <= jst[k]["survivors"] <= jst[k]["window_pairs"]
    # every job's window pairs equal the oracle's count from its size histogram
    sizes = np.diff(h_off)
    for k in range(len(js) - 1):
        lo, hi = int(js[k]), int(js[k + 1])
        assert jst[k]["window_pairs"] == O.window_pairs(sizes[lo:hi], int(p[k]), int(q[k])), k
    assert bst["window_pairs"] == sum(s["window_pairs"] for s in jst)


def test_batch_cascade_on_and_off():
    jobs = make_batch(14, seed=17)
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    for b in (0, 64, 128):
        on, jst_on, _ = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=b)
        off_, jst_off, _ = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=b, cascade_b=-1)
        check(jobs, on, jst_on)
        check(jobs, off_, jst_off)


@pytest.mark.parametrize("k,on_device", [(1, True), (4, True), (9, False)])
def test_out_of_memory_batch_retries_in_parts(monkeypatch, k, on_device):
    # An allocation refused inside the batch (injected on the host): the jobs run again
    # in halves of the job list (offsets rebased per part) with the same exact results.
    jobs = make_batch(12, seed=31)
    off, tok, js, p, q = concat(jobs)
    if on_device:
        off, tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    monkeypatch.setenv("BMJ_FAULT", f"alloc:{k}")
    pairs, jst, bst = _bmj.bmj_self_join_batch(off, tok, js, p, q, b=0)
    monkeypatch.delenv("BMJ_FAULT")
    check(jobs, pairs, jst)
    assert bst["n_jobs"] == 12 and bst["results"] == sum(len(x[0]) for x in pairs)
    assert bst["filter_passes"] >= 2   # the two halves ran (one pass or more each)


@pytest.mark.parametrize("sim,b", [(_bmj.BMJ_COSINE, 0), (_bmj.BMJ_DICE, 0), (_bmj.BMJ_COSINE, 128),
                                   (_bmj.BMJ_OVERLAP, 64)])
def test_batch_other_similarity_functions(sim, b):
    jobs = make_batch(16, seed=50 + sim)
    if sim == _bmj.BMJ_OVERLAP:   # token-count thresholds
        jobs = [(off, tok, [3, 5, 8][k % 3], 1) for k, (off, tok, _, _) in enumerate(jobs)]
    off, tok, js, p, q = concat(jobs)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    pairs, jst, bst = _bmj.bmj_self_join_batch(d_off, d_tok, js, p, q, b=b, sim=sim)
    check(jobs, pairs, jst, sim=sim)
    assert bst["results"] == sum(len(x[0]) for x in pairs) > 0
