"""The seeded host input generators follow the recipes the workloads are named
by: set-size distributions and their clipping, distinct sorted tokens inside
the universe, Zipf rank frequencies, batched job counts and thresholds,
Poisson query arrivals and probe sizes (CPU; the device sampler is checked
in tests/test_gpu_batch.py)."""
import numpy as np
import pytest

from paper_1711_07295_b300 import inputs as I


def _check_csr(off, tok, universe):
    assert off[0] == 0 and off[-1] == len(tok) and np.all(np.diff(off) >= 0)
    assert tok.dtype == np.int32 and tok.min() >= 0 and tok.max() < universe
    d = np.diff(tok.astype(np.int64))
    inner = np.ones(len(d), bool)
    inner[off[1:-1][off[1:-1] > 0] - 1] = False   # differences across set boundaries
    assert np.all(d[inner] > 0)                    # strictly increasing inside every set


@pytest.mark.parametrize("make", [I.spec_1m, I.spec_10m, I.spec_resident_2m])
def test_lognormal_recipes(make):
    full = make()
    spec = I.CollectionSpec(40_000, full.universe, full.zipf_s, full.size_dist, seed=0)
    off, tok = I.gen_collection(spec)
    _check_csr(off, tok, spec.universe)
    _, mu, sigma, lo, hi = spec.size_dist
    sizes = np.diff(off)
    assert sizes.min() >= lo and sizes.max() <= hi
    # the log sizes of the unclipped interior follow N(mu, sigma): their median is
    # exp(mu) (clipping at both ends moves neither the median nor the quartiles much)
    assert abs(np.log(np.median(sizes)) - mu) < 0.12
    q1, q3 = np.percentile(np.log(sizes), [25, 75])
    assert abs((q3 - q1) / 1.349 - sigma) < 0.1


def test_uniform_recipe_and_zipf_ranks():
    spec = I.CollectionSpec(30_000, 50_000, 1.0, ("uniform", 3, 100), seed=3)
    off, tok = I.gen_collection(spec)
    _check_csr(off, tok, spec.universe)
    sizes = np.diff(off)
    assert sizes.min() >= 3 and sizes.max() <= 100
    assert abs(sizes.mean() - 51.5) < 1.0
    # Zipf(1): frequency ~ 1/rank, so rank x frequency stays flat over the head
    # (tokens are distinct within a set, which caps the most frequent ones only
    # when a token would appear twice in one set)
    freq = np.bincount(tok, minlength=spec.universe).astype(np.float64)
    assert freq.argmax() == 0
    ranks = np.arange(1, 201)
    prod = ranks * freq[:200]
    assert prod[10:200].max() / prod[10:200].min() < 1.6
    # the slope of log frequency against log rank over ranks 10..1000 is about -s
    r = np.arange(10, 1000)
    slope = np.polyfit(np.log(r + 1), np.log(freq[r]), 1)[0]
    assert abs(slope + 1.0) < 0.15


def test_planted_near_duplicates():
    spec = I.spec_small(planted=True)
    off, tok = I.gen_collection(spec)
    _check_csr(off, tok, spec.universe)
    assert len(off) - 1 == spec.n_sets
    # planted sets are edited copies: many pairs of identical or near-identical sets
    sets = {tuple(tok[off[i]:off[i + 1]]) for i in range(len(off) - 1)}
    assert len(sets) < spec.n_sets


def test_seeds_are_deterministic():
    spec = I.CollectionSpec(5_000, 10_000, 1.1, ("lognormal", 2.3, 0.6, 1, 500), seed=7)
    a = I.gen_collection(spec)
    b = I.gen_collection(spec)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = I.gen_collection(I.CollectionSpec(5_000, 10_000, 1.1, ("lognormal", 2.3, 0.6, 1, 500),
                                          seed=8))
    assert not np.array_equal(a[1][:1000], c[1][:1000])


def test_batch_recipe():
    spec = I.BatchSpec(n_jobs=24, min_sets=1_000, max_sets=20_000)
    jobs = I.gen_batch(spec)
    assert len(jobs) == 24
    ns = []
    for off, tok, p, q in jobs:
        _check_csr(off, tok, spec.universe)
        sizes = np.diff(off)
        assert sizes.min() >= spec.size_lo and sizes.max() <= spec.size_hi
        assert (p, q) in I.THRESHOLDS_BATCH
        ns.append(len(off) - 1)
    ns = np.array(ns)
    assert ns.min() >= spec.min_sets and ns.max() <= spec.max_sets
    assert len({(p, q) for _, _, p, q in jobs}) > 1


def test_query_stream_recipe():
    coll = I.CollectionSpec(20_000, 300_000, 1.1, ("lognormal", 2.3, 0.6, 1, 500), seed=0)
    off, tok = I.gen_collection(coll)
    qs = I.QuerySpec(n_queries=4_000, rate_qps=20_000.0)
    arr, qoff, qtok, p, q = I.gen_queries(qs, coll, off, tok)
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    # Poisson arrivals: exponential gaps of mean 1/rate
    gaps = np.diff(arr)
    assert abs(gaps.mean() * qs.rate_qps - 1.0) < 0.06
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08
    _check_csr(qoff, qtok, coll.universe)
    sizes = np.diff(qoff)
    assert sizes.min() >= 1 and sizes.max() <= max(qs.size_hi, 500 + qs.max_edits)
    assert set(zip(p.tolist(), q.tolist())) <= set(I.THRESHOLDS_SERVE)
    # about half of the probes are edited copies of resident sets: some probe equals
    # a resident set exactly
    resident = {tuple(tok[off[i]:off[i + 1]]) for i in range(len(off) - 1)}
    copies = sum(tuple(qtok[qoff[k]:qoff[k + 1]]) in resident for k in range(len(qoff) - 1))
    assert copies > 0.05 * qs.n_queries
