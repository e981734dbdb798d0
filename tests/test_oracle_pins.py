"""Pins of the CPU oracle to facts the paper and mathematics fix (no GPU).

Each test checks the oracle against something other than itself: values the
paper prints for a worked example (fixtures under tests/golden/), brute force
over Python sets with exact fractions, closed forms (Eq. 4-5, the window size
over a size histogram), invariants (Theorem 1, order invariance of the
generation functions) and special cases that reduce to exact binary sets.
"""
from __future__ import annotations

import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from oracle import expected as E
from paper_1711_07295_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fixture(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.rstrip("\n").split("\t", 1)
            out[k] = v
    return out


def _bigrams(s):
    return {s[i:i + 2] for i in range(len(s) - 1)}


def _csr(sets):
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    tok = np.array([t for s in sets for t in sorted(s)], np.int32)
    return off, tok


def _brute_pairs(sets, p, q):
    out = []
    for a, b in itertools.combinations(range(len(sets)), 2):
        A, B = set(sets[a]), set(sets[b])
        if Fraction(len(A & B), len(A | B)) >= Fraction(p, q):
            out.append((a, b))
    return out


# ---------------------------------------------------------------- Section 1
def test_bigram_example_section1():
    g = _fixture("bigrams_section1.txt")
    A, B = _bigrams(g["record_a"]), _bigrams(g["record_b"])
    vocab = {bg: i for i, bg in enumerate(sorted(A | B))}
    x = sorted(vocab[t] for t in A)
    y = sorted(vocab[t] for t in B)
    o = O.overlap(x, y)
    assert o == int(g["overlap_ab"]) == 6
    assert len(_bigrams(g["record_c"])) == int(g["bigrams_c"]) == 13
    # Jaccard = 6 / (8 + 8 - 6) = 3/5: similar at 3/5 (>= is inclusive), not above it.
    assert O.similar(o, len(x), len(y), 3, 5)
    assert not O.similar(o, len(x), len(y), 61, 100)
    off, tok = _csr([x, y])
    a, b = O.self_join(off, tok, 3, 5)
    assert list(zip(a.tolist(), b.tolist())) == [(0, 1)]
    a, b = O.self_join(off, tok, 61, 100)
    assert len(a) == 0


# -------------------------------------------------------------- Section 3.1
def test_binary_set_example_section3_1():
    g = _fixture("binary_sets_section3_1.txt")
    r = [int(t) for t in g["r"].split()]
    s = [int(t) for t in g["s"].split()]
    # Position k (1-based, from the left) of the printed binary set is token k.
    pr = {k + 1 for k, ch in enumerate(g["b_r"]) if ch == "1"}
    ps = {k + 1 for k, ch in enumerate(g["b_s"]) if ch == "1"}
    assert pr == set(r) and ps == set(s)
    for method in (O.SET, O.XOR, O.NEXT):
        br, bs = O.bitmap(r, 64, method), O.bitmap(s, 64, method)
        # No collisions (universe 8 < b = 64): every method gives the exact binary set.
        assert int(br[0]) == sum(1 << t for t in r)
        assert int(bs[0]) == sum(1 << t for t in s)
        assert bin(int(br[0]) & int(bs[0])).count("1") == int(g["and_popcount"]) == 1
        assert bin(int(br[0]) | int(bs[0])).count("1") == int(g["or_popcount"]) == 6
        h = O.hamming(br, bs)
        assert h == 5
        # Eq. 2 is exact without collisions: floor((3 + 4 - 5) / 2) = 1 = |r & s|.
        assert O.upper_bound(3, 4, h) == 1 == O.overlap(r, s)
    j = Fraction(g["jaccard"])
    assert j == Fraction(1, 6)
    assert O.similar(1, 3, 4, j.numerator, j.denominator)          # boundary is inclusive
    assert not O.similar(1, 3, 4, 2, 11)                            # 2/11 > 1/6


# ------------------------------------------------------ brute force, Table 1
@pytest.mark.parametrize("seed,universe,lo,hi,p,q", [
    (1, 12, 1, 6, 1, 2), (2, 30, 2, 10, 3, 5), (3, 8, 1, 8, 4, 5),
    (4, 200, 5, 40, 1, 3), (5, 16, 1, 16, 9, 10), (6, 6, 1, 6, 1, 1),
    (7, 50, 1, 3, 1, 2),
])
def test_self_join_brute_force(seed, universe, lo, hi, p, q):
    rng = np.random.default_rng(seed)
    sets = []
    for _ in range(90):
        n = int(rng.integers(lo, min(hi, universe) + 1))
        sets.append(sorted(rng.choice(universe, size=n, replace=False).tolist()))
    off, tok = _csr(sets)
    a, b = O.self_join(off, tok, p, q)
    assert list(zip(a.tolist(), b.tolist())) == _brute_pairs(sets, p, q)
    # overlap against Python set intersection on every pair
    for x, y in itertools.combinations(range(len(sets)), 2):
        if (x * 7 + y) % 11 == 0:
            assert O.overlap(sets[x], sets[y]) == len(set(sets[x]) & set(sets[y]))


def test_similar_matches_exact_fractions():
    rng = np.random.default_rng(11)
    for _ in range(3000):
        nx, ny = int(rng.integers(1, 60)), int(rng.integers(1, 60))
        o = int(rng.integers(0, min(nx, ny) + 1))
        q = int(rng.integers(1, 40))
        p = int(rng.integers(1, q + 1))
        exact = Fraction(o, nx + ny - o) >= Fraction(p, q)
        assert O.similar(o, nx, ny, p, q) == exact


def test_join_rows_and_search_against_brute_force():
    off, tok = I.random_collection(300, 40, 1, 12, seed=3, planted_frac=0.1)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    p, q = 1, 2
    full = set(_brute_pairs(sets, p, q))
    rows = [0, 5, 17, 17, 299, 150]
    a, b = O.join_rows(off, tok, p, q, rows)
    got = list(zip(a.tolist(), b.tolist()))
    assert got == sorted({pr for pr in full if pr[0] in rows or pr[1] in rows})
    a2, b2 = O.join_rows_window(off, tok, p, q, rows)
    assert list(zip(a2.tolist(), b2.tolist())) == got


@pytest.mark.parametrize("p,q", [(1, 2), (3, 5), (9, 10), (1, 1), (1, 7)])
def test_length_filtered_rows_against_brute_force(p, q):
    # Table 2's size window only drops pairs that cannot be similar: the windowed row
    # scan returns exactly the brute-force pairs of the sampled rows (sizes 1..25, so
    # windows are cut at both ends and at the largest size).
    off, tok = I.random_collection(400, 60, 1, 25, seed=p * 31 + q, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    full = set(_brute_pairs(sets, p, q))
    rows = list(range(0, 400, 7)) + [399]
    a, b = O.join_rows_window(off, tok, p, q, rows)
    assert list(zip(a.tolist(), b.tolist())) == sorted(
        {pr for pr in full if pr[0] in rows or pr[1] in rows})


def test_search_against_brute_force():
    off, tok = I.random_collection(300, 40, 1, 12, seed=3, planted_frac=0.1)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    p, q = 1, 2
    probe = sets[17]
    ids = O.search(probe, off, tok, p, q)
    want = [s for s in range(len(sets))
            if Fraction(len(set(probe) & set(sets[s])), len(set(probe) | set(sets[s]))) >= Fraction(p, q)]
    assert ids.tolist() == want


# ------------------------------------------------------------- Section 3.2
def test_bitmaps_small_examples():
    # h(t) = t mod 64: tokens 0 and 64 collide on bit 0, token 1 hits bit 1.
    x = [0, 1, 64]
    assert int(O.bitmap(x, 64, O.SET)[0]) == 0b11
    assert int(O.bitmap(x, 64, O.XOR)[0]) == 0b10                 # 0 and 64 cancel
    assert int(O.bitmap(x, 64, O.NEXT)[0]) == 0b111               # 64 probes on to bit 1, then 1 to bit 2
    # Next wraps around the end of the bitmap.
    assert int(O.bitmap([63, 127], 64, O.NEXT)[0]) == (1 << 63) | 1
    # n >= b: Next returns all ones (Alg. 3c).
    full = O.bitmap(list(range(0, 64 * 64, 64)), 64, O.NEXT)
    assert int(full[0]) == (1 << 64) - 1
    # Multi-word layout: token 200 with b = 256 is word 3, bit 8.
    bm = O.bitmap([200], 256, O.XOR)
    assert bm.tolist() == [0, 0, 0, 1 << 8]


@pytest.mark.parametrize("b", [64, 128, 256, 192])
def test_bitmaps_exact_when_b_covers_universe(b):
    rng = np.random.default_rng(b)
    for _ in range(200):
        n = int(rng.integers(1, b))
        x = sorted(rng.choice(b, size=n, replace=False).tolist())
        want = [0] * (b // 64)
        for t in x:
            want[t // 64] |= 1 << (t % 64)
        for m in (O.SET, O.XOR, O.NEXT):
            assert [int(w) for w in O.bitmap(x, b, m)] == want


@pytest.mark.parametrize("b", [64, 128, 256])
def test_set_and_xor_by_hash_counts(b):
    # Bit k of Set is "some token hashes to k"; of Xor, "an odd number do".
    rng = np.random.default_rng(5 + b)
    for _ in range(300):
        n = int(rng.integers(1, 4 * b))
        x = sorted(rng.choice(50 * b, size=n, replace=False).tolist())
        cnt = np.bincount(np.array(x) % b, minlength=b)
        bits_set = {k for k in range(b) if cnt[k] > 0}
        bits_xor = {k for k in range(b) if cnt[k] % 2 == 1}

        def bits(bm):
            return {w * 64 + i for w in range(b // 64) for i in range(64) if (int(bm[w]) >> i) & 1}
        assert bits(O.bitmap(x, b, O.SET)) == bits_set
        assert bits(O.bitmap(x, b, O.XOR)) == bits_xor


def _next_by_carry(x, b):
    """Occupied slots of circular linear probing from hash counts (no probing loop).

    c_k tokens hash to slot k; the overflow carried out of slot k is
    carry_k = max(0, carry_{k-1} + c_k - 1), and slot k is occupied iff
    c_k + carry_{k-1} >= 1.  Around the circle the carry into slot 0 is the
    carry out of slot b-1, so the recurrence is iterated to its fixed point.
    """
    n = len(x)
    if n >= b:
        return set(range(b))
    c = np.bincount(np.array(x, dtype=np.int64) % b, minlength=b)
    carry_in = 0
    while True:
        carry = carry_in
        occ = set()
        for k in range(b):
            if c[k] + carry >= 1:
                occ.add(k)
            carry = max(0, carry + c[k] - 1)
        if carry == carry_in:
            return occ
        carry_in = carry


@pytest.mark.parametrize("b", [64, 128])
def test_next_against_carry_form_and_order(b):
    rng = np.random.default_rng(17 + b)
    for trial in range(300):
        n = int(rng.integers(1, b + 8))
        # Adversarial: draw from a few residues so that probing chains are long.
        base = rng.choice(3 + trial % 5, size=n) + b * rng.choice(10 * b, size=n, replace=False)
        x = sorted(set(int(t) for t in base))
        bm = O.bitmap(x, b, O.NEXT)
        bits = {w * 64 + i for w in range(b // 64) for i in range(64) if (int(bm[w]) >> i) & 1}
        assert bits == _next_by_carry(x, b)
        assert len(bits) == min(len(x), b)          # exactly n ones unless n >= b (Alg. 3c)
        # Order invariance of the generation (Section 3.3): any insertion order.
        perm = list(x)
        rng.shuffle(perm)
        for m in (O.SET, O.XOR, O.NEXT):
            assert O.bitmap(perm, b, m).tolist() == O.bitmap(x, b, m).tolist()


# ------------------------------------------------------ Theorem 1 (Eq. 2)
@pytest.mark.parametrize("b", [64, 128, 256])
def test_theorem1_soundness(b):
    rng = np.random.default_rng(100 + b)
    for trial in range(1500):
        nr, ns = int(rng.integers(1, 3 * b)), int(rng.integers(1, 3 * b))
        if trial % 3 == 0:
            # Adversarial collisions: every token is congruent to a few residues mod b.
            pool = (rng.choice(4, size=6 * b) + b * rng.choice(100 * b, size=6 * b)).tolist()
            pool = sorted(set(pool))
        else:
            pool = list(range(4 * b))
        common = int(rng.integers(0, min(nr, ns) + 1))
        picks = rng.choice(len(pool), size=min(len(pool), nr + ns - common), replace=False)
        toks = [pool[i] for i in picks]
        r = sorted(toks[:nr])
        s = sorted(toks[:common] + toks[nr:nr + ns - common])
        o = len(set(r) & set(s))
        for m in (O.SET, O.XOR, O.NEXT):
            h = O.hamming(O.bitmap(r, b, m), O.bitmap(s, b, m))
            assert O.upper_bound(len(r), len(s), h) >= o


# ---------------------------------------------------- Section 3.4, Eq. 4-5
@pytest.mark.parametrize("n", [8, 32, 55, 100])
def test_expected_upper_bound_monte_carlo(n):
    b, M = 64, 4000
    rng = np.random.default_rng(1000 + n)
    # 2M random n-token sets over a universe far larger than b*M*n, so that
    # the two sets of a pair share no token and their hashes are uniform.
    sets = [np.sort(rng.choice(1 << 40, size=n, replace=False) % (1 << 30)) for _ in range(2 * M)]
    sets = [np.unique(s) for s in sets]
    sets = [s for s in sets if len(s) == n][: 2 * (len(sets) // 2)]
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in sets])
    tok = np.concatenate(sets).astype(np.int64)
    assert tok.max() < 2**31
    tok = tok.astype(np.int32)
    for m, ef in ((O.SET, E.e_set), (O.XOR, E.e_xor)):
        bm = O.bitmaps(off, tok, b, m)
        ub = []
        for k in range(0, len(sets) - 1, 2):
            h = O.hamming(bm[k], bm[k + 1])
            ub.append((2 * n - h) / 2.0)          # Eq. 2 without the floor, as in Eq. 4-6
        ub = np.array(ub)
        want = ef(b, n)
        se = ub.std(ddof=1) / np.sqrt(len(ub))
        assert abs(ub.mean() - want) <= 4.5 * se + 1e-9, (m, n, ub.mean(), want, se)
    # Eq. 6 is the paper's approximation for Next: only a loose agreement.
    bm = O.bitmaps(off, tok, b, O.NEXT)
    ub = np.mean([(2 * n - O.hamming(bm[k], bm[k + 1])) / 2.0 for k in range(0, len(sets) - 1, 2)])
    assert abs(ub - E.e_next(b, n)) <= 0.06 * n + 0.1


def test_expected_values_quoted_in_text():
    # Section 3.4: at b = 64, n = 55 the normalised bound of Set and Xor is about 0.72.
    assert abs(E.e_set(64, 55) / 55 - 0.72) < 0.01
    assert abs(E.e_xor(64, 55) / 55 - 0.72) < 0.01
    # With b covering n comfortably the bound tends to 0 (few collisions).
    assert E.e_set(1 << 20, 4) < 1e-4 and E.e_xor(1 << 20, 4) < 1e-4


# --------------------------------------------- Alg. 6 counts (filter oracle)
def _window_closed_form(sizes, p, q):
    hist = np.bincount(sizes)
    total = 0
    for s in range(1, len(hist)):
        c = int(hist[s])
        if c == 0:
            continue
        total += c * (c - 1) // 2
        for t in range(1, s):
            if q * t >= p * s:
                total += c * int(hist[t])
    return total


@pytest.mark.parametrize("p,q", [(1, 2), (4, 5), (9, 10), (3, 4), (1, 1), (1, 100)])
def test_window_count_closed_form(p, q):
    off, tok = I.random_collection(700, 300, 1, 30, seed=p * 31 + q)
    sizes = np.diff(off)
    w, s, r = O.filter_counts(off, tok, p, q, 64, O.XOR)
    assert w == _window_closed_form(sizes, p, q)
    assert r <= s <= w


@pytest.mark.parametrize("method", [O.SET, O.XOR, O.NEXT])
def test_exact_bitmaps_survivors_are_results(method):
    # Universe <= b: bitmaps are the exact binary sets, so the Eq. 2 bound equals
    # the overlap and the filter passes exactly the similar pairs.
    off, tok = I.random_collection(400, 64, 1, 20, seed=9, planted_frac=0.2)
    for p, q in ((1, 2), (3, 5), (4, 5)):
        w, s, r = O.filter_counts(off, tok, p, q, 64, method)
        assert s == r
        assert r == len(O.self_join(off, tok, p, q)[0])


@pytest.mark.parametrize("b", [64, 128, 256])
@pytest.mark.parametrize("method", [O.SET, O.XOR, O.NEXT, O.COMBINED])
def test_filter_pipeline_loses_no_result(b, method):
    # Length filter + Bitmap Filter are sound: the verified survivors are
    # exactly the similar pairs that brute force finds.
    off, tok = I.random_collection(500, 2000, 1, 60, seed=b + method, planted_frac=0.15)
    for p, q in ((1, 2), (7, 10), (9, 10)):
        w, s, r = O.filter_counts(off, tok, p, q, b, method)
        assert r == len(O.self_join(off, tok, p, q)[0])
        assert s <= w


def test_length_window_is_sound():
    off, tok = I.random_collection(300, 30, 1, 25, seed=4, planted_frac=0.2)
    sizes = np.diff(off)
    for p, q in ((1, 2), (3, 4), (9, 10)):
        a, b = O.self_join(off, tok, p, q)
        lo, hi = np.minimum(sizes[a], sizes[b]), np.maximum(sizes[a], sizes[b])
        assert np.all(q * lo >= p * hi)


def test_combined_method_switch_points():
    # Alg. 4 read on the normalised overlap 2p/(p+q).
    assert O.combined_method(1, 2) == O.SET       # 0.667: between the switch points
    assert O.combined_method(4, 5) == O.XOR       # 0.889
    assert O.combined_method(1, 3) == O.NEXT      # 0.5
    assert O.combined_method(7, 18) == O.NEXT     # exactly 0.56 -> Next (<=)
    assert O.combined_method(73, 127) == O.XOR    # exactly 0.73 -> Xor (>=)
    assert O.combined_method(2, 5) == O.SET       # 0.571


def test_degenerate_collections():
    for n in (0, 1):
        off = np.zeros(n + 1, np.int64)
        off[1:] = 3
        tok = np.array([1, 2, 3][: 3 * n], np.int32)
        assert len(O.self_join(off, tok, 1, 2)[0]) == 0
        assert O.filter_counts(off, tok, 1, 2, 64, O.XOR) == (0, 0, 0)
    # identical sets: every pair is similar at any threshold, including 1/1
    off = np.arange(0, 6 * 4 + 1, 4, dtype=np.int64)
    tok = np.tile(np.array([3, 70, 134, 9000], np.int32), 6)
    tok = np.sort(tok.reshape(6, 4), axis=1).ravel()
    a, b = O.self_join(off, tok, 1, 1)
    assert len(a) == 15
    assert O.filter_counts(off, tok, 1, 1, 64, O.XOR) == (15, 15, 15)


# ------------------------------------------- Eq. 2 floor, multi-word Hamming
def test_upper_bound_floor_of_eq2():
    # Eq. 2 floors (|r| + |s| - h) / 2: an odd numerator rounds down.
    assert O.upper_bound(3, 4, 4) == 1
    assert O.upper_bound(5, 8, 0) == 6
    assert O.upper_bound(2, 1, 0) == 1
    assert O.upper_bound(7, 7, 14) == 0


@pytest.mark.parametrize("b", [128, 256, 640])
def test_hamming_is_symmetric_difference_when_exact(b):
    # With b covering the universe the bitmaps are exact and
    # popcount(br xor bs) = |r \ s| + |s \ r| over all words.
    rng = np.random.default_rng(b + 1)
    for _ in range(300):
        r = sorted(rng.choice(b, size=int(rng.integers(1, b // 2)), replace=False).tolist())
        s = sorted(rng.choice(b, size=int(rng.integers(1, b // 2)), replace=False).tolist())
        for m in (O.SET, O.XOR, O.NEXT):
            h = O.hamming(O.bitmap(r, b, m), O.bitmap(s, b, m))
            assert h == len(set(r) ^ set(s))


def _bits_by_counts(x, b, method):
    c = np.bincount(np.asarray(x, dtype=np.int64) % b, minlength=b)
    if method == O.SET:
        occ = {k for k in range(b) if c[k] > 0}
    elif method == O.XOR:
        occ = {k for k in range(b) if c[k] % 2 == 1}
    else:
        occ = _next_by_carry(x, b)
    return occ


@pytest.mark.parametrize("method", [O.SET, O.XOR, O.NEXT])
@pytest.mark.parametrize("b", [64, 128])
def test_survivor_count_brute_force(method, b):
    # Survivors of Alg. 6 recounted over all unordered pairs, without the size
    # order: the pair is in the length window iff q*min >= p*max, and it
    # survives iff floor((|r|+|s|-|br ^ bs|)/2) * (p+q) >= p*(|r|+|s|), with
    # the bitmaps taken from hash counts.
    off, tok = I.random_collection(160, 6 * b, 1, 2 * b, seed=method * 7 + b, zipf_s=0.8,
                                   planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    bits = [_bits_by_counts(x, b, method) for x in sets]
    for p, q in ((1, 2), (2, 3), (4, 5)):
        win = surv = 0
        for x, y in itertools.combinations(range(len(sets)), 2):
            nx, ny = len(sets[x]), len(sets[y])
            if q * min(nx, ny) < p * max(nx, ny):
                continue
            win += 1
            ub = (nx + ny - len(bits[x] ^ bits[y])) // 2
            if ub * (p + q) >= p * (nx + ny):
                surv += 1
        w, s, r = O.filter_counts(off, tok, p, q, b, method)
        assert (w, s) == (win, surv)


# ------------------------------------------------ Table 1 / Table 2: other functions
SIMS = (O.JACCARD, O.COSINE, O.DICE, O.OVERLAP)


def _sim_value(sim, o, x, y):
    """Table 1 evaluated independently: exact fractions, the square root of Cosine
    in 60-digit decimal arithmetic (exact whenever x*y is a perfect square)."""
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    if sim == O.JACCARD:
        return Fraction(o, x + y - o)
    if sim == O.DICE:
        return Fraction(2 * o, x + y)
    if sim == O.OVERLAP:
        return Fraction(o)
    return Decimal(o) / (Decimal(x) * Decimal(y)).sqrt()


def _passes(sim, o, x, y, p, q):
    v = _sim_value(sim, o, x, y)
    if sim == O.COSINE:
        from decimal import Decimal
        return v >= Decimal(p) / Decimal(q)
    return v >= Fraction(p, q)


def _brute_pairs_sim(sets, sim, p, q):
    out = []
    for a, b in itertools.combinations(range(len(sets)), 2):
        A, B = set(sets[a]), set(sets[b])
        if _passes(sim, len(A & B), len(A), len(B), p, q):
            out.append((a, b))
    return out


@pytest.mark.parametrize("sim", SIMS)
def test_similarity_functions_of_table1(sim):
    rng = np.random.default_rng(40 + sim)
    for _ in range(4000):
        x, y = int(rng.integers(1, 90)), int(rng.integers(1, 90))
        o = int(rng.integers(0, min(x, y) + 1))
        q = int(rng.integers(1, 30))
        p = int(rng.integers(1, 3 * q if sim == O.OVERLAP else q + 1))
        assert O.similar_sim(sim, o, x, y, p, q) == _passes(sim, o, x, y, p, q), (sim, o, x, y, p, q)
    # boundary cases that hit the threshold exactly
    assert O.similar_sim(O.COSINE, 6, 9, 16, 1, 2) and not O.similar_sim(O.COSINE, 5, 9, 16, 1, 2)
    assert O.similar_sim(O.DICE, 3, 4, 8, 1, 2) and not O.similar_sim(O.DICE, 2, 4, 8, 1, 2)
    assert O.similar_sim(O.OVERLAP, 3, 5, 5, 3, 1) and not O.similar_sim(O.OVERLAP, 2, 5, 5, 3, 1)
    assert O.similar_sim(O.JACCARD, 4, 6, 6, 1, 2) and not O.similar_sim(O.JACCARD, 3, 6, 6, 1, 2)


@pytest.mark.parametrize("sim", SIMS)
def test_length_window_is_table2(sim):
    # in_window(a, b) for sizes a <= b against the lower bounds printed in Table 2
    # (the larger set r = b): Overlap tau, Jaccard |r| tau_j, Cosine |r| tau_c^2,
    # Dice |r| tau_d / (2 - tau_d).
    for q in (1, 2, 3, 5, 10, 20):
        for p in range(1, (3 * q if sim == O.OVERLAP else q) + 1):
            t = Fraction(p, q)
            lower = {O.OVERLAP: lambda b: t, O.JACCARD: lambda b: b * t,
                     O.COSINE: lambda b: b * t * t, O.DICE: lambda b: b * t / (2 - t)}[sim]
            for b in range(1, 40):
                for a in range(1, b + 1):
                    assert O.in_window(sim, a, b, p, q) == (a >= lower(b)), (sim, p, q, a, b)


def test_dice_and_jaccard_thresholds_are_equivalent():
    # Dice = 2J / (1 + J) is increasing in J, so Dice >= 2t/(1+t) <=> Jaccard >= t:
    # with t = p/q the Dice threshold is 2p/(p+q) (Table 1's equivalences).
    off, tok = I.random_collection(600, 200, 1, 25, seed=61, planted_frac=0.2)
    for p, q in ((1, 2), (3, 5), (4, 5), (9, 10)):
        ja, jb = O.self_join(off, tok, p, q, sim=O.JACCARD)
        da, db = O.self_join(off, tok, 2 * p, p + q, sim=O.DICE)
        assert np.array_equal(ja, da) and np.array_equal(jb, db) and len(ja) > 0


@pytest.mark.parametrize("sim,p,q", [(O.COSINE, 1, 2), (O.COSINE, 4, 5), (O.DICE, 3, 5),
                                     (O.DICE, 9, 10), (O.OVERLAP, 3, 1), (O.OVERLAP, 7, 2)])
def test_other_functions_brute_force(sim, p, q):
    off, tok = I.random_collection(160, 50, 1, 14, seed=sim * 10 + p, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    want = _brute_pairs_sim(sets, sim, p, q)
    a, b = O.self_join(off, tok, p, q, sim=sim)
    assert list(zip(a.tolist(), b.tolist())) == want and len(want) > 0
    rows = [0, 7, 59, 159]
    ra, rb = O.join_rows(off, tok, p, q, rows, sim=sim)
    wa, wb = O.join_rows_window(off, tok, p, q, rows, sim=sim)
    sel = sorted(pr for pr in want if pr[0] in rows or pr[1] in rows)
    assert list(zip(ra.tolist(), rb.tolist())) == sel == list(zip(wa.tolist(), wb.tolist()))
    ids = O.search(sets[7], off, tok, p, q, sim=sim)
    assert ids.tolist() == [s for s in range(len(sets))
                            if _passes(sim, len(set(sets[7]) & set(sets[s])), len(sets[7]),
                                       len(sets[s]), p, q)]


@pytest.mark.parametrize("sim,p,q", [(O.COSINE, 3, 5), (O.DICE, 7, 10), (O.OVERLAP, 4, 1),
                                     (O.JACCARD, 1, 2)])
def test_filter_counts_other_functions(sim, p, q):
    # window pairs = pairs j < i (size order) inside Table 2's window, counted from
    # the size histogram; results = brute force; survivors between the two; exact
    # bitmaps (universe <= b) pass exactly the similar pairs.
    off, tok = I.random_collection(500, 60, 1, 24, seed=70 + sim, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    sizes = sorted(np.diff(off).tolist())
    t = Fraction(p, q)
    lower = {O.OVERLAP: lambda b: t, O.JACCARD: lambda b: b * t,
             O.COSINE: lambda b: b * t * t, O.DICE: lambda b: b * t / (2 - t)}[sim]
    win = sum(1 for i in range(len(sizes)) for j in range(i) if sizes[j] >= lower(sizes[i]))
    n_res = len(_brute_pairs_sim(sets, sim, p, q))
    for method in (O.XOR, O.SET):
        w, s, r = O.filter_counts(off, tok, p, q, 64, method, sim=sim)
        assert w == win and r == n_res and r <= s <= w
        assert s == r   # universe 60 <= b: the bitmaps are exact
    w, s, r = O.filter_counts(off, tok, p, q, 128, O.XOR, sim=sim)
    assert (w, r) == (win, n_res) and s == r


def test_combined_method_of_other_functions():
    # switch points 0.56 / 0.73 on the normalised overlap at the threshold: p/q itself
    # for Dice and Cosine (tau*n / n for two sets of size n); Xor for Overlap
    for sim in (O.DICE, O.COSINE):
        assert O.combined_method(1, 2, sim) == O.NEXT        # 0.50
        assert O.combined_method(14, 25, sim) == O.NEXT      # 0.56
        assert O.combined_method(3, 5, sim) == O.SET         # 0.60
        assert O.combined_method(73, 100, sim) == O.XOR      # 0.73
        assert O.combined_method(9, 10, sim) == O.XOR
    assert O.combined_method(7, 2, O.OVERLAP) == O.XOR
    assert O.combined_method(1, 2, O.JACCARD) == O.SET       # 2/3 normalised


# --------------------------------------- Section 2.2: the prefix filter as candidates
def _prefix_candidates_brute(sets, sim, p, q):
    """Candidates by the definition: tokens ranked by (frequency, id), a set's prefix is
    its x - low(x) + 1 lowest-ranked tokens with low(x) the smallest overlap any similar
    partner can have (found here from Table 1 by search); pairs inside Table 2's window
    whose prefixes intersect."""
    from collections import Counter
    freq = Counter(t for s in sets for t in s)
    rank = {t: r for r, t in enumerate(sorted(freq, key=lambda t: (freq[t], t)))}

    def low(x):   # smallest partner size y <= x that can still reach the threshold
        for y in range(1, x + 1):
            if _passes(sim, y, y, x, p, q):
                return y
        return x + 1

    pre = [set(sorted(rank[t] for t in s)[:max(0, len(s) - low(len(s)) + 1)]) for s in sets]
    cand = 0
    for a, b in itertools.combinations(range(len(sets)), 2):
        x, y = sorted((len(sets[a]), len(sets[b])))
        if not _passes(sim, x, x, y, p, q):
            continue
        if pre[a] & pre[b]:
            cand += 1
    return cand


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 4, 5), (O.COSINE, 3, 5),
                                     (O.DICE, 7, 10), (O.OVERLAP, 3, 1)])
def test_prefix_filter_candidates(sim, p, q):
    off, tok = I.random_collection(220, 90, 1, 16, seed=80 + p + sim, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    c, s, r = O.prefix_counts(off, tok, p, q, 64, O.XOR, sim=sim)
    assert c == _prefix_candidates_brute(sets, sim, p, q)
    # the prefix filter is exact: every similar pair is a candidate
    w, s_w, r_w = O.filter_counts(off, tok, p, q, 64, O.XOR, sim=sim)
    assert r == r_w == len(_brute_pairs_sim(sets, sim, p, q)) and r <= s <= s_w and c <= w


# ------------------------------------------------- Section 2.1: the RS-join (Eq. 1)
def _split(off, tok, n_r):
    """The first n_r sets of a collection as R, the rest as S (each its own CSR)."""
    ro = off[:n_r + 1].copy()
    so = off[n_r:] - off[n_r]
    return ro, tok[:off[n_r]].copy(), so, tok[off[n_r]:].copy()


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 4, 5), (O.COSINE, 3, 5),
                                     (O.DICE, 7, 10), (O.OVERLAP, 3, 1)])
def test_rs_join_brute_force(sim, p, q):
    # every (r, s) of R x S against Table 1 evaluated with Python sets and exact
    # fractions; R and S of different sizes and token mixes
    off, tok = I.random_collection(150, 45, 1, 14, seed=90 + sim * 7 + p, planted_frac=0.25)
    ro, rt, so, st = _split(off, tok, 60)
    R = [set(rt[ro[i]:ro[i + 1]].tolist()) for i in range(len(ro) - 1)]
    S = [set(st[so[j]:so[j + 1]].tolist()) for j in range(len(so) - 1)]
    want = [(i, j) for i in range(len(R)) for j in range(len(S))
            if _passes(sim, len(R[i] & S[j]), len(R[i]), len(S[j]), p, q)]
    a, b = O.rs_join(ro, rt, so, st, p, q, sim=sim)
    assert list(zip(a.tolist(), b.tolist())) == want and len(want) > 0


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 3, 5), (O.DICE, 4, 5), (O.COSINE, 1, 2),
                                     (O.OVERLAP, 5, 2)])
def test_rs_join_is_the_cross_part_of_the_self_join(sim, p, q):
    # the self-join of R and S concatenated holds three kinds of pairs; the ones
    # with one end in each collection are exactly the RS-join (ids of S shifted)
    off, tok = I.random_collection(400, 150, 1, 20, seed=120 + sim, planted_frac=0.2)
    n_r = 170
    ro, rt, so, st = _split(off, tok, n_r)
    sa, sb = O.self_join(off, tok, p, q, sim=sim)
    cross = (sa < n_r) & (sb >= n_r)
    a, b = O.rs_join(ro, rt, so, st, p, q, sim=sim)
    assert np.array_equal(a, sa[cross]) and np.array_equal(b, sb[cross] - n_r) and len(a) > 0
    # and swapping R and S swaps the pairs
    a2, b2 = O.rs_join(so, st, ro, rt, p, q, sim=sim)
    order = np.lexsort((a, b))
    assert np.array_equal(a2, b[order]) and np.array_equal(b2, a[order])


def test_rs_join_of_a_collection_with_itself():
    # S = R: the pairs r < s are the self-join, every (r, r) passes (similarity 1),
    # and the pair list is symmetric
    off, tok = I.random_collection(250, 120, 1, 18, seed=131, planted_frac=0.2)
    for p, q in ((1, 2), (4, 5)):
        a, b = O.rs_join(off, tok, off, tok, p, q)
        sa, sb = O.self_join(off, tok, p, q)
        up = a < b
        assert np.array_equal(a[up], sa) and np.array_equal(b[up], sb)
        assert np.count_nonzero(a == b) == len(off) - 1
        assert len(a) == 2 * len(sa) + len(off) - 1


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 9, 10), (O.COSINE, 3, 5),
                                     (O.DICE, 7, 10), (O.OVERLAP, 4, 1)])
def test_rs_filter_counts(sim, p, q):
    # window pairs from the two size histograms and Table 2's bounds; results =
    # the RS-join's length; exact bitmaps (universe <= b) pass exactly the results
    off, tok = I.random_collection(420, 60, 1, 24, seed=140 + sim, planted_frac=0.2)
    ro, rt, so, st = _split(off, tok, 150)
    t = Fraction(p, q)
    lower = {O.OVERLAP: lambda b: t, O.JACCARD: lambda b: b * t,
             O.COSINE: lambda b: b * t * t, O.DICE: lambda b: b * t / (2 - t)}[sim]
    hr, hs = np.bincount(np.diff(ro)), np.bincount(np.diff(so))
    win = sum(int(hr[x]) * int(hs[y]) for x in range(len(hr)) for y in range(len(hs))
              if hr[x] and hs[y] and min(x, y) >= lower(max(x, y)))
    n_res = len(O.rs_join(ro, rt, so, st, p, q, sim=sim)[0])
    for method in (O.XOR, O.SET, O.NEXT):
        w, s, r = O.rs_filter_counts(ro, rt, so, st, p, q, 64, method, sim=sim)
        assert (w, r) == (win, n_res) and s == r
    # a small universe against b = 64 exceeded: survivors between results and window
    off2, tok2 = I.random_collection(420, 3000, 1, 40, seed=141 + sim, planted_frac=0.3)
    ro, rt, so, st = _split(off2, tok2, 200)
    w, s, r = O.rs_filter_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim)
    assert r == len(O.rs_join(ro, rt, so, st, p, q, sim=sim)[0]) and r <= s <= w


# ------------------------------------------------- Section 3.5: the cutoff point
def test_cutoff_closed_forms_equal_eq4_and_eq5():
    # the fp64 closed forms used for the cutoff search against the exact sums
    for b in (64, 128, 256, 1024):
        for n in (1, 2, 5, 17, 55, 100, 300):
            assert abs(E.e_set_closed(b, n) - E.e_set(b, n)) <= 1e-9 * max(1, n)
            assert abs(E.e_xor_closed(b, n) - E.e_xor(b, n)) <= 1e-9 * max(1, n)


def test_cutoff_values_quoted_in_text():
    # Section 3.5: omega(64, 0.72) = 55; at b = 1024 and Jaccard 0.9 the Set cutoff is
    # 2129 and Xor's is 2.3 times it, at Jaccard 0.8 1.47 times (the normalised
    # threshold of a Jaccard threshold t is 2t/(1+t)).  The paper's Xor value 4983
    # does not follow from Eq. 5 (which gives 4863): parity unpinned for it.
    assert E.cutoff(64, 0.72, "xor") == 55
    u9, u8 = 2 * 0.9 / 1.9, 2 * 0.8 / 1.8
    s9, x9 = E.cutoff(1024, u9, "set"), E.cutoff(1024, u9, "xor")
    assert abs(s9 - 2129) <= 1
    assert round(x9 / s9, 1) == 2.3
    assert round(E.cutoff(1024, u8, "xor") / E.cutoff(1024, u8, "set"), 2) == 1.47


@pytest.mark.parametrize("b", [256, 1024, 4096])
def test_combined_switch_points_follow_from_the_cutoffs(b):
    # Alg. 4 picks the method with the highest cutoff: Next up to 0.56, Set up to
    # 0.73, Xor above (on the normalised threshold), for any b above 64
    def best(u):
        c = {m: E.cutoff(b, u, m) for m in ("set", "xor", "next")}
        return max(c, key=c.get)
    for u in (0.50, 0.53, 0.55):
        assert best(u) == "next", u
    for u in (0.58, 0.62, 0.66, 0.70, 0.72):
        assert best(u) == "set", u
    for u in (0.74, 0.8, 0.9):
        assert best(u) == "xor", u


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 4, 5), (O.COSINE, 3, 5),
                                     (O.DICE, 7, 10)])
def test_filter_counts_with_a_cutoff(sim, p, q):
    # a cutoff changes neither the window nor the results; survivors grow by exactly
    # the pairs above it that the bound rejected (counted by brute force per pair)
    off, tok = I.random_collection(600, 3000, 1, 60, seed=150 + sim + p, planted_frac=0.2)
    sets = [tok[off[i]:off[i + 1]] for i in range(len(off) - 1)]
    bms = O.bitmaps(off, tok, 64, O.XOR)
    sizes = np.diff(off)
    t = Fraction(p, q)
    lower = {O.JACCARD: lambda b: b * t, O.COSINE: lambda b: b * t * t,
             O.DICE: lambda b: b * t / (2 - t)}[sim]
    w0, s0, r0 = O.filter_counts(off, tok, p, q, 64, O.XOR, sim=sim)
    for cut in (10, 30, 59):
        extra = 0
        for a, b in itertools.combinations(range(len(sets)), 2):
            x, y = int(sizes[a]), int(sizes[b])
            if max(x, y) <= cut or min(x, y) < lower(max(x, y)):
                continue
            ub = O.upper_bound(x, y, O.hamming(bms[a], bms[b]))
            extra += not O.similar_sim(sim, ub, x, y, p, q)
        w, s, r = O.filter_counts(off, tok, p, q, 64, O.XOR, sim=sim, cutoff=cut)
        assert (w, r) == (w0, r0) and s == s0 + extra
        assert extra > 0 or cut == 59
    # RS-join of the first 300 sets with the rest: with cutoff 1 only pairs of two
    # single-token sets still meet the bound
    ro, rt = off[:301].copy(), tok[:off[300]].copy()
    so, st = off[300:] - off[300], tok[off[300]:].copy()
    w0, s0, r0 = O.rs_filter_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim)
    w, s, r = O.rs_filter_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim, cutoff=1)
    ones = [a for a in range(len(sets)) if sizes[a] == 1]
    kept = sum(1 for a in ones if a < 300 for b in ones if b >= 300
               and O.similar_sim(sim, O.upper_bound(1, 1, O.hamming(bms[a], bms[b])), 1, 1, p, q))
    n1r, n1s = sum(1 for a in ones if a < 300), sum(1 for a in ones if a >= 300)
    assert (w, r) == (w0, r0) and s == w - (n1r * n1s - kept) and s > s0


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 4, 5), (O.COSINE, 3, 5),
                                     (O.DICE, 7, 10), (O.OVERLAP, 3, 1)])
def test_rs_prefix_filter_candidates(sim, p, q):
    # RS-join candidates by the definition: ranks by (frequency over R and S, id); each
    # set's prefix as in the self-join; pairs (r, s) inside Table 2's window whose
    # prefixes intersect.  Every similar pair is a candidate.
    from collections import Counter
    off, tok = I.random_collection(240, 90, 1, 16, seed=170 + p + sim, planted_frac=0.25)
    ro, rt, so, st = _split(off, tok, 100)
    R = [rt[ro[i]:ro[i + 1]].tolist() for i in range(len(ro) - 1)]
    S = [st[so[j]:so[j + 1]].tolist() for j in range(len(so) - 1)]
    freq = Counter(t for x in R + S for t in x)
    rank = {t: r for r, t in enumerate(sorted(freq, key=lambda t: (freq[t], t)))}

    def low(x):   # smallest partner size y <= x that can still reach the threshold
        for y in range(1, x + 1):
            if _passes(sim, y, y, x, p, q):
                return y
        return x + 1

    def prefix(x):
        return set(sorted(rank[t] for t in x)[:max(0, len(x) - low(len(x)) + 1)])

    pr, ps = [prefix(x) for x in R], [prefix(y) for y in S]
    want = 0
    for i in range(len(R)):
        for j in range(len(S)):
            a, b = sorted((len(R[i]), len(S[j])))
            if _passes(sim, a, a, b, p, q) and pr[i] & ps[j]:
                want += 1
    c, s, r = O.rs_prefix_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim)
    assert c == want
    w, s_w, r_w = O.rs_filter_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim)
    assert r == r_w == len(O.rs_join(ro, rt, so, st, p, q, sim=sim)[0]) and r > 0
    assert r <= s <= s_w and c <= w


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 3, 5), (O.JACCARD, 19, 20),
                                     (O.JACCARD, 1, 1), (O.COSINE, 3, 4), (O.DICE, 7, 10),
                                     (O.OVERLAP, 4, 1), (O.OVERLAP, 1, 3)])
def test_window_pairs_from_the_size_histogram(sim, p, q):
    # The closed form counts, for every pair of sizes t <= s, the set pairs those sizes
    # give; pinned to (1) every pair of sets compared against Table 2's lower bound in
    # exact fractions, (2) the window count of filter_counts (which walks the sets in
    # size order), and (3) the empty and one-set collections.
    off, tok = I.random_collection(450, 80, 1, 40, seed=80 + sim + p, planted_frac=0.1)
    sizes = np.diff(off).tolist()
    t = Fraction(p, q)
    lower = {O.OVERLAP: lambda b: t, O.JACCARD: lambda b: b * t,
             O.COSINE: lambda b: b * t * t, O.DICE: lambda b: b * t / (2 - t)}[sim]
    brute = sum(1 for x, y in itertools.combinations(sizes, 2)
                if min(x, y) >= lower(max(x, y)))
    assert O.window_pairs(sizes, p, q, sim) == brute
    w, _, _ = O.filter_counts(off, tok, p, q, 64, O.XOR, sim=sim)
    assert w == brute
    assert O.window_pairs([], p, q, sim) == 0 and O.window_pairs([7], p, q, sim) == 0


def test_window_pairs_of_equal_sizes_and_large_counts():
    # n sets of one size are all inside each other's window: C(n, 2) pairs, also for
    # counts whose product needs more than 32 bits
    assert O.window_pairs([5] * 1000, 1, 2) == 1000 * 999 // 2
    sizes = np.concatenate([np.full(3_000_000, 10), np.full(2_000_000, 12)])
    # 10 and 12 pair at 4/5 (10 >= 9.6), not at 9/10 (10 < 10.8)
    n10, n12 = 3_000_000, 2_000_000
    same = n10 * (n10 - 1) // 2 + n12 * (n12 - 1) // 2
    assert O.window_pairs(sizes, 4, 5) == same + n10 * n12
    assert O.window_pairs(sizes, 9, 10) == same


@pytest.mark.parametrize("sim,p,q", [(O.JACCARD, 1, 2), (O.JACCARD, 9, 10), (O.COSINE, 3, 5),
                                     (O.DICE, 3, 4), (O.OVERLAP, 3, 1)])
def test_rs_window_pairs_from_the_size_histograms(sim, p, q):
    # every pair of R x S compared against Table 2's lower bound in exact fractions, and
    # the window count of rs_filter_counts
    off, tok = I.random_collection(420, 90, 1, 45, seed=95 + sim + q, planted_frac=0.1)
    ro, rt, so, st = _split(off, tok, 150)
    sr, ss = np.diff(ro).tolist(), np.diff(so).tolist()
    t = Fraction(p, q)
    lower = {O.OVERLAP: lambda b: t, O.JACCARD: lambda b: b * t,
             O.COSINE: lambda b: b * t * t, O.DICE: lambda b: b * t / (2 - t)}[sim]
    brute = sum(1 for x in sr for y in ss if min(x, y) >= lower(max(x, y)))
    assert O.rs_window_pairs(sr, ss, p, q, sim) == brute > 0
    w, _, _ = O.rs_filter_counts(ro, rt, so, st, p, q, 64, O.XOR, sim=sim)
    assert w == brute
    assert O.rs_window_pairs([], ss, p, q, sim) == 0 == O.rs_window_pairs(sr, [], p, q, sim)


def test_folded_bitmap_distance_bounds_the_full_one():
    # The b = 128 filter's first test folds the two 64-bit halves of the xor onto each
    # other.  For Xor bitmaps (h(t) = t mod b) the fold of a 128-bit bitmap is the 64-bit
    # Xor bitmap of the same set, and for every method the folded distance is at most
    # the 128-bit one, so Eq. 2 on the fold never rejects a pair the 128-bit test keeps.
    rng = np.random.default_rng(5)
    for _ in range(300):
        n1, n2 = rng.integers(1, 300, size=2)
        x = np.unique(rng.integers(0, 1 << 31, size=n1)).astype(np.int32)
        y = np.unique(rng.integers(0, 1 << 31, size=n2)).astype(np.int32)
        assert np.array_equal(O.bitmap(x, 128, O.XOR)[0] ^ O.bitmap(x, 128, O.XOR)[1],
                              O.bitmap(x, 64, O.XOR)[0])
        for m in (O.XOR, O.SET, O.NEXT):
            bx, by = O.bitmap(x, 128, m), O.bitmap(y, 128, m)
            h_fold = O.hamming(np.array([bx[0] ^ bx[1]]), np.array([by[0] ^ by[1]]))
            h_full = O.hamming(bx, by)
            assert h_fold <= h_full
            assert O.upper_bound(len(x), len(y), h_fold) >= O.upper_bound(len(x), len(y), h_full)
