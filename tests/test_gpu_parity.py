"""Parity of the CUDA path with the CPU oracle (needs a GPU).

Pair lists are compared element by element (bit-exact: the method is integer
work); window-pair and survivor counts are compared with the oracle's Alg. 6
counts, which are deterministic.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_1711_07295_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU, skipped by marker
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1711_07295_b300 import _bmj  # noqa: E402

ORACLE_METHOD = {_bmj.BMJ_XOR: O.XOR, _bmj.BMJ_SET: O.SET, _bmj.BMJ_NEXT: O.NEXT,
                 _bmj.BMJ_COMBINED: O.COMBINED}


def dev(off, tok):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), \
        torch.from_numpy(np.ascontiguousarray(tok)).cuda()


def gpu_join(off, tok, p, q, on_device=True, **kw):
    if on_device:
        d_off, d_tok = dev(off, tok)
        return _bmj.bmj_self_join(d_off, d_tok, p, q, **kw)
    return _bmj.bmj_self_join(off, tok, p, q, **kw)


def check_join(off, tok, p, q, b=64, method=_bmj.BMJ_XOR, counts=True, sim=_bmj.BMJ_JACCARD, **kw):
    a, bb, st = gpu_join(off, tok, p, q, b=b, method=method, sim=sim, **kw)
    ra, rb = O.self_join(off, tok, p, q, sim=sim)
    assert len(a) == len(ra), (len(a), len(ra))
    assert np.array_equal(a, ra) and np.array_equal(bb, rb)
    if counts:
        m = O.combined_method(p, q, sim) if method == _bmj.BMJ_COMBINED else ORACLE_METHOD[method]
        assert st["method"] == m or method != _bmj.BMJ_COMBINED
        w, s, r = O.filter_counts(off, tok, p, q, b, m, sim=sim)
        assert (st["window_pairs"], st["survivors"], st["results"]) == (w, s, r)
    return st


# ------------------------------------------- folded test of the b = 128 filter
@pytest.mark.parametrize("b", [128, 256])
@pytest.mark.parametrize("method", [_bmj.BMJ_XOR, _bmj.BMJ_SET, _bmj.BMJ_NEXT])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 4, 5),
                                     (_bmj.BMJ_COSINE, 3, 4), (_bmj.BMJ_DICE, 9, 10)])
def test_folded_test_keeps_the_survivors(b, method, sim, p, q):
    # b = 128 and 256 run the full-width test only in the warp column steps where some
    # pair passes the folded (64- or 128-bit) test; survivors and results stay the oracle's, and
    # the step counters are consistent with the pairs: a step covers at most one
    # tile's rows (32 x rows per lane) of window pairs, and every survivor lies in a
    # step that took the full test
    off, tok = I.random_collection(6000, 3000, 1, 60, seed=11, planted_frac=0.15)
    st = check_join(off, tok, p, q, b=b, method=method, sim=sim)
    rows = st["tile_rows"]
    assert rows % 32 == 0 and 32 <= rows <= 256
    assert st["survivors"] > 0
    assert 0 <= st["fold_full_steps"] <= st["fold_steps"]
    if st["fold_steps"] or b == 128:  # b = 256 folds only in a build that enables it
        assert st["window_pairs"] <= rows * st["fold_steps"]
        assert st["survivors"] <= rows * st["fold_full_steps"]
    # with a queue too small for the survivors (reruns in item ranges) nothing changes
    check_join(off, tok, p, q, b=b, method=method, sim=sim, queue_cap=97)
    # other widths do not fold
    st64 = check_join(off, tok, p, q, b=64, method=method, sim=sim)
    assert st64["fold_steps"] == 0 and st64["fold_full_steps"] == 0


# --------------------------------------------------------------- config 1
@pytest.mark.parametrize("planted", [False, True])
def test_small_config_literal_and_planted(planted):
    # 10,000 sets, Zipf(1.0) over 5,000 tokens, sizes U[5,50], threshold 4/5, b = 64.
    off, tok = I.gen_collection(I.spec_small(planted=planted))
    st = check_join(off, tok, 4, 5, b=64, method=_bmj.BMJ_XOR)
    if planted:
        assert st["results"] > 0


@pytest.mark.parametrize("p,q", [(1, 2), (3, 5), (7, 10), (9, 10)])
def test_small_config_other_thresholds(p, q):
    off, tok = I.gen_collection(I.spec_small(planted=True))
    check_join(off, tok, p, q, b=64)


# ------------------------------------------------- methods x bitmap sizes
@pytest.mark.parametrize("b", [64, 128, 192, 256, 512, 1024, 4096])
@pytest.mark.parametrize("method", [_bmj.BMJ_XOR, _bmj.BMJ_SET, _bmj.BMJ_NEXT, _bmj.BMJ_COMBINED])
def test_methods_and_widths(b, method):
    # 3,001 sets (a ragged last tile), sizes 1..120 so that Next saturates for b = 64.
    off, tok = I.random_collection(3001, 3000, 1, 120, seed=b + 10 * method, zipf_s=0.9,
                                   planted_frac=0.1)
    for p, q in ((1, 2), (4, 5)):
        check_join(off, tok, p, q, b=b, method=method)


@pytest.mark.parametrize("b", [64, 128, 192, 256, 4096])
@pytest.mark.parametrize("method", [_bmj.BMJ_XOR, _bmj.BMJ_SET, _bmj.BMJ_NEXT])
def test_build_bitmaps_bit_exact(b, method):
    off, tok = I.random_collection(1500, 20 * b, 1, b + 40, seed=b * 3 + method, zipf_s=0.7)
    want = O.bitmaps(off, tok, b, ORACLE_METHOD[method])
    d_off, d_tok = dev(off, tok)
    got = _bmj.bmj_build_bitmaps(d_off, d_tok, b=b, method=method)
    assert np.array_equal(got.cpu().numpy().view(np.uint64), want)
    got_h = _bmj.bmj_build_bitmaps(off, tok, b=b, method=method)
    assert np.array_equal(got_h, want)


# ------------------------------------- other similarity functions (Table 1)
@pytest.mark.parametrize("b", [64, 128, 256, 192])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_COSINE, 1, 2), (_bmj.BMJ_COSINE, 4, 5),
                                     (_bmj.BMJ_DICE, 3, 5), (_bmj.BMJ_DICE, 9, 10),
                                     (_bmj.BMJ_OVERLAP, 3, 1), (_bmj.BMJ_OVERLAP, 9, 2)])
def test_other_similarity_functions(sim, p, q, b):
    # 3,001 sets (a ragged last tile), sizes 1..80; the pair list and the window,
    # survivor and result counts equal the oracle's for the function's window (Table 2)
    # and limit (Cosine: per pair of sizes, the others per size sum).
    off, tok = I.random_collection(3001, 2500, 1, 80, seed=b + 7 * sim + p, zipf_s=0.9,
                                   planted_frac=0.15)
    st = check_join(off, tok, p, q, b=b, sim=sim)
    assert st["results"] > 0


@pytest.mark.parametrize("sim", [_bmj.BMJ_COSINE, _bmj.BMJ_DICE])
def test_other_functions_combined_method_and_host_input(sim):
    off, tok = I.random_collection(2500, 1200, 1, 50, seed=90 + sim, planted_frac=0.1)
    for p, q in ((1, 2), (3, 5), (9, 10)):
        check_join(off, tok, p, q, b=64, sim=sim, method=_bmj.BMJ_COMBINED, on_device=False)


# ------------------------------------------------- cutoff point (Section 3.5)
def _normalised(sim, p, q):
    return 2 * p / (p + q) if sim == _bmj.BMJ_JACCARD else p / q


@pytest.mark.parametrize("b", [64, 128, 256, 1024])
def test_automatic_cutoff_is_the_oracles(b):
    # the library's cutoff point from Eq. 4-6 equals the oracle's, for every method
    # and several functions and thresholds (read from the stats of a two-set join)
    from oracle import expected as E
    off, tok = np.array([0, 2, 4], np.int64), np.array([1, 2, 1, 3], np.int32)
    names = {_bmj.BMJ_SET: "set", _bmj.BMJ_XOR: "xor", _bmj.BMJ_NEXT: "next"}
    for method, name in names.items():
        for sim, p, q in ((_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 3, 4),
                          (_bmj.BMJ_JACCARD, 9, 10), (_bmj.BMJ_DICE, 7, 10),
                          (_bmj.BMJ_COSINE, 3, 5)):
            _, _, st = _bmj.bmj_self_join(off, tok, p, q, b=b, method=method, sim=sim,
                                          cutoff=_bmj.BMJ_CUTOFF_AUTO)
            assert st["cutoff"] == E.cutoff(b, _normalised(sim, p, q), name), (b, name, sim, p, q)
    _, _, st = _bmj.bmj_self_join(off, tok, 2, 1, sim=_bmj.BMJ_OVERLAP, cutoff=_bmj.BMJ_CUTOFF_AUTO)
    assert st["cutoff"] == 0      # Overlap thresholds are not normalised: no cutoff


@pytest.mark.parametrize("b", [64, 128, 256, 192])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 3, 4),
                                     (_bmj.BMJ_COSINE, 3, 5), (_bmj.BMJ_DICE, 7, 10)])
def test_cutoff_point_parity(sim, p, q, b):
    # pairs whose larger set is above the cutoff skip Eq. 2: same pairs, survivors as
    # the oracle's counts with that cutoff (explicit values and the automatic one)
    off, tok = I.random_collection(3001, 2500, 1, 120, seed=b + 3 * sim + q, zipf_s=0.9,
                                   planted_frac=0.15)
    ra, rb = O.self_join(off, tok, p, q, sim=sim)
    base = None
    for cut in (20, 75, _bmj.BMJ_CUTOFF_AUTO):
        a, bb, st = gpu_join(off, tok, p, q, b=b, sim=sim, cutoff=cut)
        assert np.array_equal(a, ra) and np.array_equal(bb, rb)
        w = st["cutoff"]
        assert w == cut or (cut == _bmj.BMJ_CUTOFF_AUTO and w > 0)
        counts = O.filter_counts(off, tok, p, q, b, O.XOR, sim=sim, cutoff=w)
        assert (st["window_pairs"], st["survivors"], st["results"]) == counts
        if base is None:
            base = O.filter_counts(off, tok, p, q, b, O.XOR, sim=sim)
        assert st["survivors"] >= base[1]


def test_cutoff_invalid_combinations():
    off, tok = I.random_collection(200, 100, 1, 10, seed=3)
    for kw in ({"cutoff": -2}, {"cutoff": 5, "candidates": _bmj.BMJ_CAND_PREFIX}):
        with pytest.raises(_bmj.BmjError) as e:
            _bmj.bmj_self_join(off, tok, 1, 2, **kw)
        assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG


# ------------------------------------------------------ host/device paths
def test_host_and_device_paths_agree():
    off, tok = I.random_collection(5000, 2000, 2, 40, seed=5, planted_frac=0.1)
    a1, b1, _ = gpu_join(off, tok, 3, 5, on_device=False)
    a2, b2, _ = gpu_join(off, tok, 3, 5, on_device=True)
    d_off, d_tok = dev(off, tok)
    dp, _, st = _bmj.bmj_self_join(d_off, d_tok, 3, 5, output_on_device=True)
    assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    assert np.array_equal(dp.a.cpu().numpy().view(np.uint32), a1)
    assert np.array_equal(dp.b.cpu().numpy().view(np.uint32), b1)
    dp.release()


def test_pooled_host_lists_are_reused_without_aliasing():
    """Freed page-locked lists go back to the library's pool; a list still held is never reused."""
    off, tok = I.random_collection(5000, 1500, 2, 40, seed=6, planted_frac=0.1)
    ra, rb = O.self_join(off, tok, 1, 2)
    a1, b1, _ = _bmj.bmj_self_join(off, tok, 1, 2)
    keep_a, keep_b = a1.copy(), b1.copy()
    a2, b2, _ = _bmj.bmj_self_join(off, tok, 1, 2)
    span = lambda x: (x.ctypes.data, x.ctypes.data + x.nbytes)  # noqa: E731
    lo1, hi1 = min(span(a1)[0], span(b1)[0]), max(span(a1)[1], span(b1)[1])
    for s0, s1 in (span(a2), span(b2)):
        assert s1 <= lo1 or s0 >= hi1, "a live list was handed out again"
    addr2 = a2.ctypes.data
    del a2, b2  # the last views of the second list: its block goes back to the pool
    a3, b3, _ = _bmj.bmj_self_join(off, tok, 1, 2)
    assert a3.ctypes.data == addr2, "the freed block was not reused"
    assert np.array_equal(a1, keep_a) and np.array_equal(b1, keep_b)
    assert np.array_equal(a1, ra) and np.array_equal(b1, rb)
    assert np.array_equal(a3, ra) and np.array_equal(b3, rb)
    # trimming frees idle blocks only: the held lists stay valid
    del a3, b3
    assert _bmj.bmj_host_pool_trim() > 0
    assert _bmj.bmj_host_pool_trim() == 0
    assert np.array_equal(a1, keep_a) and np.array_equal(b1, keep_b)


def test_queue_overflow_reruns_exactly():
    # A one-entry queue: the work items run in ranges, and an item whose survivors
    # alone overflow the queue gets a queue of exactly its size.
    off, tok = I.random_collection(4000, 300, 1, 30, seed=8, planted_frac=0.2)
    st = check_join(off, tok, 1, 2, b=64, queue_cap=1)
    assert st["filter_passes"] >= 2 and st["survivors"] > 1


@pytest.mark.parametrize("b", [64, 128])
def test_survivors_beyond_the_queue_run_in_item_ranges(b):
    # The survivors need several queue fills: each range of work items is filtered and
    # verified before the next; pairs, window and survivor counts stay exact.
    off, tok = I.random_collection(12000, 3000, 2, 60, seed=21 + b, zipf_s=1.1, planted_frac=0.1)
    full = check_join(off, tok, 1, 2, b=b)   # automatic queue: one pass, or two with exact room
    cap = max(64, full["survivors"] // 7)
    st = check_join(off, tok, 1, 2, b=b, queue_cap=cap)
    assert st["filter_passes"] >= 8
    assert (st["survivors"], st["results"], st["verified"]) == \
        (full["survivors"], full["results"], full["verified"])


def test_repeated_calls_are_deterministic():
    off, tok = I.random_collection(6000, 800, 1, 25, seed=2, planted_frac=0.1)
    d_off, d_tok = dev(off, tok)
    first = _bmj.bmj_self_join(d_off, d_tok, 1, 2)
    for _ in range(3):
        again = _bmj.bmj_self_join(d_off, d_tok, 1, 2)
        assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])
        assert first[2]["survivors"] == again[2]["survivors"]


# ------------------------------------------------------------ edge cases
def test_empty_and_single():
    for n in (0, 1):
        off = np.arange(n + 1, dtype=np.int64) * 3
        tok = np.tile(np.array([1, 4, 9], np.int32), n)
        a, b, st = gpu_join(off, tok, 1, 2)
        assert len(a) == 0 and st["window_pairs"] == 0


def test_identical_sets_and_threshold_one():
    n = 700
    off = np.arange(n + 1, dtype=np.int64) * 4
    tok = np.tile(np.array([3, 70, 134, 9000], np.int32), n)
    a, b, st = gpu_join(off, tok, 1, 1)
    assert len(a) == n * (n - 1) // 2 == st["results"] == st["window_pairs"]
    iu = np.triu_indices(n, 1)
    assert np.array_equal(a, iu[0].astype(np.uint32)) and np.array_equal(b, iu[1].astype(np.uint32))


def test_very_large_sets_among_small_ones():
    # 2,000 small sets plus sets of up to 1,000,000 tokens (near-duplicate pairs among
    # them): 32-bit overlap counts, long merges and saturated bitmaps in one join
    rng = np.random.default_rng(77)
    small_off, small_tok = I.random_collection(2000, 5000, 1, 30, seed=78)
    h1 = np.sort(rng.choice(3_000_000, 1_000_000, replace=False))
    keep = rng.random(len(h1)) > 0.05
    h2 = np.sort(np.concatenate([h1[keep], 3_000_000 + rng.choice(100_000, 20_000, replace=False)]))
    h3 = np.sort(rng.choice(3_000_000, 200_000, replace=False))
    h4 = h3[rng.random(len(h3)) > 0.4]
    h5 = np.arange(5000)
    sets = [small_tok[small_off[i]:small_off[i + 1]] for i in range(len(small_off) - 1)]
    for k, h in enumerate((h1, h2, h3, h4, h5)):
        sets.insert(300 * k + 7, h.astype(np.int32))
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in sets])
    tok = np.concatenate(sets).astype(np.int32)
    for p, q in ((1, 2), (9, 10), (1, 1000)):
        for b in (64, 256):
            st = check_join(off, tok, p, q, b=b)
            assert st["max_set_size"] == 1_000_000 and st["results"] > 0


def test_singletons_and_low_threshold():
    off, tok = I.random_collection(2500, 40, 1, 1, seed=3)
    check_join(off, tok, 1, 1)
    off, tok = I.random_collection(1200, 500, 1, 30, seed=4)
    check_join(off, tok, 1, 100)


def test_exact_bitmaps_survivors_equal_results_on_gpu():
    off, tok = I.random_collection(3000, 64, 1, 30, seed=12, planted_frac=0.1)
    for m in (_bmj.BMJ_XOR, _bmj.BMJ_SET, _bmj.BMJ_NEXT):
        st = check_join(off, tok, 3, 5, b=64, method=m)
        assert st["survivors"] == st["results"]


@pytest.mark.parametrize("case,code", [
    ("unsorted", _bmj.BMJ_ERR_UNSORTED), ("duplicate", _bmj.BMJ_ERR_UNSORTED),
    ("negative", _bmj.BMJ_ERR_NEG_TOKEN), ("empty", _bmj.BMJ_ERR_EMPTY_SET),
    ("bad_offsets", _bmj.BMJ_ERR_UNSORTED), ("past_end", _bmj.BMJ_ERR_UNSORTED),
])
@pytest.mark.parametrize("on_device", [True, False])
def test_invalid_collections(case, code, on_device):
    off = np.array([0, 3, 6, 9], np.int64)
    tok = np.array([1, 5, 9, 2, 4, 6, 1, 5, 9], np.int32)
    if case == "unsorted":
        tok[4], tok[5] = tok[5], tok[4]
    elif case == "duplicate":
        tok[5] = tok[4]
    elif case == "negative":
        tok[3] = -2
    elif case == "empty":
        off = np.array([0, 3, 3, 9], np.int64)
        tok = np.array([1, 5, 9, 1, 2, 4, 5, 6, 9], np.int32)
    elif case == "bad_offsets":
        off = np.array([0, 6, 3, 9], np.int64)
    elif case == "past_end":
        off = np.array([0, 3, 12, 9], np.int64)
    with pytest.raises(_bmj.BmjError) as ei:
        gpu_join(off, tok, 1, 2, on_device=on_device)
    assert ei.value.status == code
    # the context stays usable after a rejected input
    check_join(*I.random_collection(300, 100, 1, 10, seed=1), 1, 2)


# ------------------------------------- full-size configuration, row-sampled
@pytest.fixture(scope="module")
def million():
    return I.gen_collection(I.spec_1m())


@pytest.mark.parametrize("p,q,b", [(1, 2, 64), (3, 4, 128), (9, 10, 256), (19, 20, 64)])
def test_million_sets_row_sampled(million, p, q, b):
    # 1,000,000 sets, Zipf(1.1) over 200,000, sizes lognormal(2.3, 0.6) in [1, 500];
    # the launch configuration is the benchmark's.  The oracle scans 40 sampled
    # rows against all sets; the GPU pairs touching those rows must match exactly.
    off, tok = million
    d_off, d_tok = dev(off, tok)
    a, bb, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b)
    rng = np.random.default_rng(p * 100 + q + b)
    sizes = np.diff(off)
    rows = np.concatenate([rng.choice(len(sizes), 30, replace=False),
                           np.argsort(sizes)[:5], np.argsort(sizes)[-5:]])
    ra, rb = O.join_rows(off, tok, p, q, rows)
    sel = np.isin(a, rows) | np.isin(bb, rows)
    assert np.array_equal(a[sel], ra) and np.array_equal(bb[sel], rb)
    # properties that hold at any size
    assert np.all(a < bb)
    key = a.astype(np.uint64) << np.uint64(32) | bb.astype(np.uint64)
    assert np.all(np.diff(key.astype(np.int64)) > 0)
    assert st["results"] == len(a) <= st["survivors"] <= st["window_pairs"]
    assert st["window_pairs"] == O.window_pairs(sizes, p, q)
    sa, sb = sizes[a], sizes[bb]
    assert np.all(q * np.minimum(sa, sb) >= p * np.maximum(sa, sb))


@pytest.mark.parametrize("b", [64, 128, 256])
def test_million_sets_window_pairs_closed_form(million, b):
    # The headline's numerator: the window pairs the Bitmap Filter evaluated at every
    # threshold of the 1M workload equal the oracle's count from the size histogram
    # (Table 2), at each bitmap width the benchmark times.
    off, tok = million
    d_off, d_tok = dev(off, tok)
    sizes = np.diff(off)
    for p, q in ((1, 2), (3, 4), (9, 10), (19, 20)):
        r, _, st = _bmj.bmj_self_join(d_off, d_tok, p, q, b=b, output_on_device=True)
        r.release()
        assert st["window_pairs"] == O.window_pairs(sizes, p, q), (p, q, b)
        assert st["results"] <= st["survivors"] <= st["window_pairs"]


@pytest.mark.parametrize("b", [64, 128, 256])
def test_cascade_check_changes_nothing_but_merges(b):
    # The second, wider Bitmap Filter in verification is sound (Theorem 1 for any
    # b): the pair list and the first-level survivor count stay the oracle's.
    off, tok = I.random_collection(4000, 1500, 1, 60, seed=31 + b, planted_frac=0.1)
    d_off, d_tok = dev(off, tok)
    ra, rb = O.self_join(off, tok, 1, 2)
    w, s, r = O.filter_counts(off, tok, 1, 2, b, O.XOR)
    seen = []
    for cb in (-1, 0, 512, 1024):
        a, bb, st = _bmj.bmj_self_join(d_off, d_tok, 1, 2, b=b, cascade_b=cb)
        assert np.array_equal(a, ra) and np.array_equal(bb, rb), cb
        assert (st["window_pairs"], st["survivors"], st["results"]) == (w, s, r)
        assert st["results"] <= st["verified"] <= st["survivors"]
        seen.append(st["verified"])
        if cb == -1 or (cb == 0 and b >= 256):
            assert st["cascade_b"] == 0 and st["verified"] == st["survivors"]
    assert seen[2] <= seen[0]


@pytest.fixture(scope="module")
def ten_million():
    # 10,000,000 sets, Zipf(1.0) over 1,000,000 tokens, sizes lognormal(2.0, 0.8) in [1, 1000]
    off_d, tok_d = I.gen_collection_device(I.spec_10m())
    return off_d, tok_d, off_d.cpu().numpy(), tok_d.cpu().numpy()


@pytest.mark.parametrize("p,q", [(9, 10), (3, 5)])
def test_ten_million_sets_row_sampled(ten_million, p, q):
    off_d, tok_d, off, tok = ten_million
    dp, _, st = _bmj.bmj_self_join(off_d, tok_d, p, q, b=128, output_on_device=True)
    a = dp.a.cpu().numpy().view(np.uint32)
    bb = dp.b.cpu().numpy().view(np.uint32)
    dp.release()
    assert st["results"] == len(a) <= st["verified"] <= st["survivors"] <= st["window_pairs"]
    rng = np.random.default_rng(p + q)
    sizes = np.diff(off)
    # the headline's numerator at its full size: 1.8e13 / 3.9e12 window pairs
    assert st["window_pairs"] == O.window_pairs(sizes, p, q)
    rows = np.concatenate([rng.choice(len(sizes), 10, replace=False), np.argsort(sizes)[-2:],
                           np.nonzero(sizes == 1)[0][:2]])
    ra, rb = O.join_rows(off, tok, p, q, rows)
    sel = np.isin(a, rows) | np.isin(bb, rows)
    assert np.array_equal(a[sel], ra) and np.array_equal(bb[sel], rb)
    assert np.all(a < bb)
    key = a.astype(np.uint64) << np.uint64(32) | bb.astype(np.uint64)
    assert np.all(key[1:] > key[:-1])
    # prefix-filter candidates (Section 2.2): the same pair list, from fewer pairs
    xp, _, sx = _bmj.bmj_self_join(off_d, tok_d, p, q, b=128, output_on_device=True,
                                   candidates=_bmj.BMJ_CAND_PREFIX)
    xa = xp.a.cpu().numpy().view(np.uint32)
    xb = xp.b.cpu().numpy().view(np.uint32)
    xp.release()
    assert sx["candidates"] >= 0 and sx["results"] == st["results"]
    assert np.array_equal(xa, a) and np.array_equal(xb, bb)
    assert sx["candidates"] < st["window_pairs"] // 100


def test_measured_popc_rate_matches_the_unit_count():
    # 16 POPC per clock per SM at up to 2032 MHz: the measured rate may fall short of
    # that under a lower clock, never above it by more than timing noise.
    rate = _bmj.bmj_measure_popc_rate()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = sms * 16 * 2032e6
    assert 0.5 * nominal < rate < 1.05 * nominal, (rate, nominal)


# ------------------------------------------ prefix-filter candidates (Section 2.2)
@pytest.mark.parametrize("b", [64, 128, 256])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 4, 5),
                                     (_bmj.BMJ_JACCARD, 19, 20), (_bmj.BMJ_COSINE, 3, 4),
                                     (_bmj.BMJ_DICE, 9, 10), (_bmj.BMJ_OVERLAP, 5, 1)])
def test_prefix_filter_candidates(sim, p, q, b):
    # Only the window pairs whose prefixes share a token reach the Bitmap Filter: the
    # pair list equals the oracle's join, and candidates, survivors and results equal
    # the oracle's prefix-filter counts (ranks by (frequency, token), each pair once).
    off, tok = I.random_collection(4001, 3000, 1, 60, seed=300 + b + sim + p, zipf_s=1.0,
                                   planted_frac=0.15)
    a, bb, st = gpu_join(off, tok, p, q, b=b, sim=sim, candidates=_bmj.BMJ_CAND_PREFIX)
    ra, rb = O.self_join(off, tok, p, q, sim=sim)
    assert np.array_equal(a, ra) and np.array_equal(bb, rb)
    c, s, r = O.prefix_counts(off, tok, p, q, b, O.XOR, sim=sim)
    assert (st["candidates"], st["survivors"], st["results"]) == (c, s, r)
    w, _, _ = O.filter_counts(off, tok, p, q, b, O.XOR, sim=sim)
    assert st["window_pairs"] == w and c <= w


@pytest.mark.parametrize("cap", [1, 97, 5000])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 4, 5),
                                     (_bmj.BMJ_DICE, 3, 4)])
def test_prefix_filter_candidates_in_ranges(sim, p, q, cap):
    # The candidate slots expanded in ranges of at most `cap` slots (a tiny budget
    # forces many ranges, each filtered and verified before the next): candidates,
    # survivors, results and the pair list are the oracle's, whatever the ranges.
    off, tok = I.random_collection(3001, 2000, 1, 50, seed=400 + cap + p, zipf_s=1.0,
                                   planted_frac=0.15)
    a, bb, st = gpu_join(off, tok, p, q, b=64, sim=sim, candidates=_bmj.BMJ_CAND_PREFIX,
                         queue_cap=cap)
    ra, rb = O.self_join(off, tok, p, q, sim=sim)
    assert np.array_equal(a, ra) and np.array_equal(bb, rb)
    c, s, r = O.prefix_counts(off, tok, p, q, 64, O.XOR, sim=sim)
    assert (st["candidates"], st["survivors"], st["results"]) == (c, s, r)
    assert st["candidate_slots"] >= st["candidates"]
    assert st["filter_passes"] == max(1, -(-st["candidate_slots"] // cap))


@pytest.mark.parametrize("large_values", [False, True])
def test_prefix_filter_large_sets_and_token_values(large_values):
    # sets of 2,049 to 6,000 tokens among small ones (their prefixes are ordered by a
    # sort instead of one warp each), and token values of up to 2^30 (ranked by a sort of
    # the occurrences instead of a histogram): same candidates as the oracle
    rng = np.random.default_rng(91 + large_values)
    small_off, small_tok = I.random_collection(1500, 4000, 1, 40, seed=92, planted_frac=0.2)
    sets = [small_tok[small_off[i]:small_off[i + 1]] for i in range(len(small_off) - 1)]
    base = np.sort(rng.choice(20000, 6000, replace=False))
    for k, x in enumerate((2049, 2300, 3000, 3100, 6000)):
        sets.append(np.sort(rng.choice(base[:max(x + 200, 2400)], x, replace=False)))
    if large_values:   # spread the token values up to 2^30, keeping every set sorted
        sets = [(x.astype(np.int64) * 53687 + 7).astype(np.int32) for x in sets]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in sets])
    tok = np.concatenate(sets).astype(np.int32)
    for p, q in ((4, 5), (1, 2)):
        a, bb, st = gpu_join(off, tok, p, q, b=64, candidates=_bmj.BMJ_CAND_PREFIX)
        ra, rb = O.self_join(off, tok, p, q)
        assert np.array_equal(a, ra) and np.array_equal(bb, rb)
        c, s, r = O.prefix_counts(off, tok, p, q, 64, O.XOR)
        assert (st["candidates"], st["survivors"], st["results"]) == (c, s, r) and r > 0


@pytest.mark.parametrize("p,q", [(1, 2), (4, 5), (19, 20)])
def test_automatic_candidates_small(p, q):
    # BMJ_CAND_AUTO takes the prefix filter or the window; either way the pair list is the
    # oracle's, and the counts are those of the mode it took
    off, tok = I.random_collection(4001, 3000, 1, 60, seed=500 + p, zipf_s=1.0, planted_frac=0.15)
    a, bb, st = gpu_join(off, tok, p, q, b=64, candidates=_bmj.BMJ_CAND_AUTO)
    ra, rb = O.self_join(off, tok, p, q)
    assert np.array_equal(a, ra) and np.array_equal(bb, rb)
    assert st["candidate_slots"] > 0
    if st["candidates"] == -2:   # the window
        assert (st["window_pairs"], st["survivors"], st["results"]) == \
            O.filter_counts(off, tok, p, q, 64, O.XOR)
    else:
        assert (st["candidates"], st["survivors"], st["results"]) == \
            O.prefix_counts(off, tok, p, q, 64, O.XOR)


def test_automatic_candidates_on_the_million_set_workload(million):
    # 1M sets: at 1/2 the 6e9 candidate slots cost more than the window (the automatic mode
    # keeps the window), at 9/10 far less (it takes the prefix filter); same pairs either way
    off, tok = million
    off_d, tok_d = dev(off, tok)
    for (p, q), mode in (((1, 2), "window"), ((9, 10), "prefix")):
        w_pairs, _, st_w = _bmj.bmj_self_join(off_d, tok_d, p, q, b=64, output_on_device=True)
        x_pairs, _, st_x = _bmj.bmj_self_join(off_d, tok_d, p, q, b=64, output_on_device=True,
                                              candidates=_bmj.BMJ_CAND_AUTO)
        assert torch.equal(w_pairs.a, x_pairs.a) and torch.equal(w_pairs.b, x_pairs.b)
        assert (st_x["candidates"] == -2) == (mode == "window"), (p, q, st_x["candidates"])
        w_pairs.release()
        x_pairs.release()


def test_prefix_filter_on_the_million_set_workload(million):
    # 1M sets at every threshold of the workload: the same pairs as the window-mode
    # join, fewer pairs through the Bitmap Filter (at 1/2 its billions of candidate
    # slots may go through the buffer in several ranges).
    off, tok = million
    off_d, tok_d = dev(off, tok)
    for p, q in ((1, 2), (3, 4), (9, 10), (19, 20)):
        w_pairs, _, st_w = _bmj.bmj_self_join(off_d, tok_d, p, q, b=64, output_on_device=True)
        x_pairs, _, st_x = _bmj.bmj_self_join(off_d, tok_d, p, q, b=64, output_on_device=True,
                                              candidates=_bmj.BMJ_CAND_PREFIX)
        assert torch.equal(w_pairs.a, x_pairs.a) and torch.equal(w_pairs.b, x_pairs.b)
        assert st_x["results"] == st_w["results"] and 0 < st_x["candidates"] < st_w["window_pairs"] // 10
        assert st_x["candidate_slots"] >= st_x["candidates"] and st_x["filter_passes"] >= 1
        w_pairs.release()
        x_pairs.release()
