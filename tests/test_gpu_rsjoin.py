"""Parity of the RS-join (Section 2.1, Eq. 1 between two collections) with the
CPU oracle (needs a GPU).

The pair lists are compared element by element; window pairs, Bitmap Filter
survivors and results with the oracle's counts over every pair of R x S.
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

ORACLE_METHOD = {_bmj.BMJ_XOR: O.XOR, _bmj.BMJ_SET: O.SET, _bmj.BMJ_NEXT: O.NEXT}


def dev(off, tok):
    return torch.from_numpy(np.ascontiguousarray(off)).cuda(), \
        torch.from_numpy(np.ascontiguousarray(tok)).cuda()


def split(off, tok, n_r):
    """First n_r sets as R, the rest as S; planted near-duplicates of R's sets
    that land in S make similar cross pairs."""
    ro = off[:n_r + 1].copy()
    so = off[n_r:] - off[n_r]
    return ro, tok[:off[n_r]].copy(), so, tok[off[n_r]:].copy()


def check_rs(R, S, p, q, b=64, method=_bmj.BMJ_XOR, sim=_bmj.BMJ_JACCARD, counts=True,
             r_dev=True, s_dev=True, **kw):
    ro, rt = R
    so, st_ = S
    ra = dev(ro, rt) if r_dev else (ro, rt)
    sa = dev(so, st_) if s_dev else (so, st_)
    a, bb, st = _bmj.bmj_rs_join(*ra, *sa, p, q, b=b, method=method, sim=sim, **kw)
    wa, wb = O.rs_join(ro, rt, so, st_, p, q, sim=sim)
    assert len(a) == len(wa), (len(a), len(wa))
    assert np.array_equal(a, wa) and np.array_equal(bb, wb)
    if counts:
        w, s, r = O.rs_filter_counts(ro, rt, so, st_, p, q, b, ORACLE_METHOD[method], sim=sim)
        assert (st["window_pairs"], st["survivors"], st["results"]) == (w, s, r)
    return st


@pytest.mark.parametrize("b", [64, 128, 256, 192, 512])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 4, 5),
                                     (_bmj.BMJ_JACCARD, 9, 10), (_bmj.BMJ_COSINE, 3, 5),
                                     (_bmj.BMJ_DICE, 7, 10), (_bmj.BMJ_OVERLAP, 3, 1)])
def test_rs_join_parity(sim, p, q, b):
    # R of 1,500 sets and S of 2,201 (ragged tiles on both sides), sizes 1..60
    off, tok = I.random_collection(3701, 2500, 1, 60, seed=b + 7 * sim + p, zipf_s=0.9,
                                   planted_frac=0.2)
    R_S = split(off, tok, 1500)
    st = check_rs(R_S[:2], R_S[2:], p, q, b=b, sim=sim)
    assert st["results"] > 0


@pytest.mark.parametrize("method", [_bmj.BMJ_SET, _bmj.BMJ_NEXT])
def test_rs_join_other_generation_methods(method):
    off, tok = I.random_collection(2400, 1500, 1, 90, seed=31 + method, planted_frac=0.2)
    R_S = split(off, tok, 900)
    for p, q in ((1, 2), (3, 4)):
        check_rs(R_S[:2], R_S[2:], p, q, b=64, method=method)


def test_rs_join_host_and_device_inputs():
    off, tok = I.random_collection(2000, 1200, 1, 40, seed=41, planted_frac=0.2)
    R, S = split(off, tok, 700)[:2], split(off, tok, 700)[2:]
    for r_dev, s_dev in ((False, False), (True, False), (False, True)):
        check_rs(R, S, 3, 5, r_dev=r_dev, s_dev=s_dev)
    st = check_rs(R, S, 3, 5, output_on_device=False, cascade_b=-1)
    assert st["results"] > 0
    # pairs left on the device
    dp, _, _ = _bmj.bmj_rs_join(*dev(*R), *dev(*S), 3, 5, output_on_device=True)
    wa, wb = O.rs_join(*R, *S, 3, 5)
    assert np.array_equal(dp.a.cpu().numpy().view(np.uint32), wa)
    assert np.array_equal(dp.b.cpu().numpy().view(np.uint32), wb)
    dp.release()


def test_rs_join_swapped_and_self():
    off, tok = I.random_collection(1800, 900, 1, 30, seed=52, planted_frac=0.25)
    ro, rt, so, st_ = split(off, tok, 800)
    a, b, _ = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), 7, 10)
    a2, b2, _ = _bmj.bmj_rs_join(*dev(so, st_), *dev(ro, rt), 7, 10)
    order = np.lexsort((a, b))
    assert np.array_equal(a2, b[order]) and np.array_equal(b2, a[order]) and len(a) > 0
    # R = S: the self-join's pairs both ways round plus every (r, r)
    sa, sb, _ = _bmj.bmj_self_join(*dev(ro, rt), 7, 10)
    x, y, st = _bmj.bmj_rs_join(*dev(ro, rt), *dev(ro, rt), 7, 10)
    assert np.array_equal(x[x < y], sa) and np.array_equal(y[x < y], sb)
    assert np.count_nonzero(x == y) == len(ro) - 1
    assert len(x) == 2 * len(sa) + len(ro) - 1 == st["results"]


def test_rs_join_edge_cases():
    off, tok = I.random_collection(400, 300, 1, 20, seed=61, planted_frac=0.2)
    ro, rt, so, st_ = split(off, tok, 150)
    empty = (np.zeros(1, np.int64), np.zeros(0, np.int32))
    for R, S in (((ro, rt), empty), (empty, (so, st_)), (empty, empty)):
        a, b, st = _bmj.bmj_rs_join(*R, *S, 1, 2)
        assert len(a) == 0 and st["window_pairs"] == 0
    # one set on each side
    one = (np.array([0, 3], np.int64), np.array([1, 5, 8], np.int32))
    other = (np.array([0, 4], np.int64), np.array([3, 4, 5, 6], np.int32))
    a, b, _ = _bmj.bmj_rs_join(*one, *other, 1, 6)    # J = 1/6 exactly (Section 3.1's pair)
    assert a.tolist() == [0] and b.tolist() == [0]
    a, b, _ = _bmj.bmj_rs_join(*one, *other, 1, 5)
    assert len(a) == 0
    # S's sizes all far below R's: the window is empty at 4/5
    big = I.random_collection(200, 500, 40, 60, seed=62)
    small = I.random_collection(300, 500, 1, 10, seed=63)
    a, b, st = _bmj.bmj_rs_join(*big, *small, 4, 5)
    assert len(a) == 0 and st["window_pairs"] == 0
    check_rs(small, big, 1, 10)   # a low threshold reaches across


def test_rs_join_queue_overflow_is_exact():
    # far more survivors than the queue holds: the filter reruns in item ranges
    off, tok = I.random_collection(5000, 200, 5, 30, seed=71, zipf_s=1.2, planted_frac=0.1)
    R_S = split(off, tok, 2000)
    st = check_rs(R_S[:2], R_S[2:], 1, 4, queue_cap=4096)
    assert st["survivors"] > 4096 and st["filter_passes"] >= 2


@pytest.mark.parametrize("b", [64, 128])
def test_rs_join_with_a_cutoff(b):
    # pairs whose larger set exceeds the cutoff skip Eq. 2 (Section 3.5)
    off, tok = I.random_collection(3000, 2000, 1, 100, seed=91 + b, planted_frac=0.2)
    ro, rt, so, st_ = split(off, tok, 1300)
    for cut in (30, _bmj.BMJ_CUTOFF_AUTO):
        a, bb, st = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), 1, 2, b=b, cutoff=cut)
        wa, wb = O.rs_join(ro, rt, so, st_, 1, 2)
        assert np.array_equal(a, wa) and np.array_equal(bb, wb)
        w = st["cutoff"]
        assert w > 0 and (w == cut or cut == _bmj.BMJ_CUTOFF_AUTO)
        counts = O.rs_filter_counts(ro, rt, so, st_, 1, 2, b, O.XOR, cutoff=w)
        assert (st["window_pairs"], st["survivors"], st["results"]) == counts


def test_rs_join_invalid_arguments():
    off, tok = I.random_collection(100, 100, 1, 10, seed=81)
    ro, rt, so, st_ = split(off, tok, 50)
    with pytest.raises(_bmj.BmjError) as e:
        _bmj.bmj_rs_join(ro, rt, so, st_, 3, 2)
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    bad = so + 1     # S does not start at offset 0
    with pytest.raises(_bmj.BmjError) as e:
        _bmj.bmj_rs_join(ro, rt, bad, np.concatenate([[0], st_]).astype(np.int32), 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_UNSORTED
    x = int(np.flatnonzero(np.diff(so) >= 2)[0])   # a set of S with two tokens or more
    unsorted = st_.copy()
    unsorted[so[x]], unsorted[so[x] + 1] = st_[so[x] + 1], st_[so[x]]
    with pytest.raises(_bmj.BmjError) as e:
        _bmj.bmj_rs_join(ro, rt, so, unsorted, 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_UNSORTED
    with pytest.raises(_bmj.BmjError) as e:   # prefix candidates and a cutoff do not combine
        _bmj.bmj_rs_join(ro, rt, so, st_, 1, 2, candidates=_bmj.BMJ_CAND_PREFIX, cutoff=5)
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    check_rs((ro, rt), (so, st_), 1, 2)   # the context stays usable


def test_rs_join_of_two_million_set_collections_row_sampled():
    # R and S: 1,000,000 sets each (Zipf(1.1) over 200,000, sizes lognormal(2.3, 0.6)
    # in [1, 500]; two seeds).  The oracle scans 40 sampled rows of R against all
    # of S; the GPU pairs of those rows must match exactly.
    ro, rt = I.gen_collection(I.spec_1m(seed=0))
    so, st_ = I.gen_collection(I.spec_1m(seed=1, planted=True))
    for p, q, b in ((9, 10, 64), (3, 4, 128)):
        a, bb, st = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), p, q, b=b)
        rng = np.random.default_rng(p + q + b)
        sizes = np.diff(ro)
        rows = np.unique(np.concatenate([rng.choice(len(sizes), 30, replace=False),
                                         np.argsort(sizes)[:5], np.argsort(sizes)[-5:]]))
        sub_o = np.concatenate([[0], np.cumsum(sizes[rows])]).astype(np.int64)
        sub_t = np.concatenate([rt[ro[r]:ro[r + 1]] for r in rows]).astype(np.int32)
        wa, wb = O.rs_join(sub_o, sub_t, so, st_, p, q)
        sel = np.isin(a, rows)
        assert np.array_equal(a[sel], rows[wa]) and np.array_equal(bb[sel], wb)
        # properties that hold at any size
        key = a.astype(np.uint64) << np.uint64(32) | bb.astype(np.uint64)
        assert np.all(np.diff(key.astype(np.int64)) > 0)
        assert st["results"] == len(a) <= st["survivors"] <= st["window_pairs"]
        # the window pairs of R x S at full size, from the oracle's two size histograms
        assert st["window_pairs"] == O.rs_window_pairs(sizes, np.diff(so), p, q)
        x, y = sizes[a], np.diff(so)[bb]
        assert np.all(q * np.minimum(x, y) >= p * np.maximum(x, y))
        # the automatic candidate mode gives the same pairs
        xa, xb, sx = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), p, q, b=b,
                                      candidates=_bmj.BMJ_CAND_AUTO)
        assert np.array_equal(xa, a) and np.array_equal(xb, bb) and sx["candidate_slots"] > 0


@pytest.mark.parametrize("b", [64, 128, 256])
@pytest.mark.parametrize("sim,p,q", [(_bmj.BMJ_JACCARD, 1, 2), (_bmj.BMJ_JACCARD, 4, 5),
                                     (_bmj.BMJ_COSINE, 3, 5), (_bmj.BMJ_DICE, 9, 10),
                                     (_bmj.BMJ_OVERLAP, 4, 1)])
def test_rs_join_prefix_candidates(sim, p, q, b):
    # prefix-filter candidates of R x S (ranks over R and S together): same pairs, and
    # candidates, survivors and results equal to the oracle's counts
    off, tok = I.random_collection(3200, 2500, 1, 60, seed=400 + b + sim + p, zipf_s=1.0,
                                   planted_frac=0.2)
    ro, rt, so, st_ = split(off, tok, 1300)
    a, bb, st = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), p, q, b=b, sim=sim,
                                 candidates=_bmj.BMJ_CAND_PREFIX)
    wa, wb = O.rs_join(ro, rt, so, st_, p, q, sim=sim)
    assert np.array_equal(a, wa) and np.array_equal(bb, wb) and len(a) > 0
    c, s, r = O.rs_prefix_counts(ro, rt, so, st_, p, q, b, O.XOR, sim=sim)
    assert (st["candidates"], st["survivors"], st["results"]) == (c, s, r)
    w, _, _ = O.rs_filter_counts(ro, rt, so, st_, p, q, b, O.XOR, sim=sim)
    assert st["window_pairs"] == w and c <= w


def test_rs_join_prefix_candidates_with_large_sets():
    # sets of 33 to 6,000 tokens on both sides: every size class of the prefix selection
    # (one thread, one warp, a sort) runs on both of R's and S's size-ordered runs
    rng = np.random.default_rng(97)
    base = np.sort(rng.choice(30000, 8000, replace=False))

    def coll(n_small, bigs, seed):
        o, t = I.random_collection(n_small, 4000, 1, 60, seed=seed, planted_frac=0.2)
        sets = [t[o[i]:o[i + 1]] for i in range(len(o) - 1)]
        sets += [np.sort(rng.choice(base[:x + 400], x, replace=False)) for x in bigs]
        off = np.zeros(len(sets) + 1, np.int64)
        off[1:] = np.cumsum([len(x) for x in sets])
        return off, np.concatenate(sets).astype(np.int32)

    ro, rt = coll(900, (40, 500, 2049, 3000, 6000), 98)
    so, st_ = coll(1200, (33, 2100, 2500, 5900), 99)
    for p, q in ((4, 5), (1, 2)):
        a, bb, st = _bmj.bmj_rs_join(*dev(ro, rt), *dev(so, st_), p, q,
                                     candidates=_bmj.BMJ_CAND_PREFIX)
        wa, wb = O.rs_join(ro, rt, so, st_, p, q)
        assert np.array_equal(a, wa) and np.array_equal(bb, wb) and len(a) > 0
        c, s, r = O.rs_prefix_counts(ro, rt, so, st_, p, q, 64, O.XOR)
        assert (st["candidates"], st["survivors"], st["results"]) == (c, s, r)
