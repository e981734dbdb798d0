"""CPU oracle for the Bitmap Filter self-join -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
``cpu_baseline`` / reference leg may import this package.  It shares no code
with the CUDA library: the arithmetic lives in ``oracle.c`` (plain C, int64),
loaded here through ctypes; ``expected.py`` holds the paper's closed forms
(Eq. 4-6) in exact rational / fp64 arithmetic.

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):
  overlap / similar / self_join -- worked examples of Section 1 and Section 3.1,
      brute force with Python ``set`` on tiny inputs, the Table 1 identity
      checked against exact fractions;
  bitmap (Set/Xor/Next) -- exact binary sets when b covers the universe
      (Section 3.1), Next's popcount rule (Alg. 3c), order invariance
      (Section 3.3), Monte Carlo against Eq. 4-5;
  filter_counts -- window count against a closed form over the size
      histogram, survivors == results when bitmaps are exact, Theorem 1
      soundness (results never exceed what brute force finds);
  join_rows / search -- against self_join / brute force on small inputs.
  window_pairs -- against the window count of filter_counts and a brute-force
      count over every pair of sizes with Python integers, for every function.
  rs_window_pairs -- against the window count of rs_filter_counts and a
      brute-force count over every pair of R x S with exact fractions.
  rs_join / rs_filter_counts (Section 2.1) -- brute force with Python ``set``
      and exact fractions; the cross pairs of the self-join of R and S
      concatenated; the self-join itself when S is R (pairs r < s); window
      counts from the two size histograms; survivors == results with exact
      bitmaps.
  similar_sim / in_window (Cosine, Dice, Overlap; Table 1 and Table 2) --
      Table 1 evaluated with exact fractions and 60-digit square roots, the
      bounds printed in Table 2, the Dice-Jaccard threshold equivalence, brute
      force joins, window counts from the size histogram.
  expected.cutoff (Section 3.5, Eq. 4-6 inverted) -- the values the text
      quotes (55 at b = 64; Set 2129 and the Xor/Set ratios 2.3 and 1.47 at
      b = 1024) and Alg. 4's switch points 0.56 / 0.73; the paper's Xor figure
      4983 does not follow from its own Eq. 5: parity unpinned for it.
  rs_prefix_counts -- candidates by the definition over Python sets (ranks by
      frequency over R and S), results equal to the RS-join's.
  filter_counts / rs_filter_counts with a cutoff -- against the counts
      without one: the window and the results are unchanged, the survivors
      grow by exactly the bound-rejected pairs whose larger set is above it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

XOR, SET, NEXT, COMBINED = 0, 1, 2, 3
JACCARD, COSINE, DICE, OVERLAP = 0, 1, 2, 3   # similarity functions (Table 1)
METHODS = {"xor": XOR, "set": SET, "next": NEXT, "combined": COMBINED}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        i64, i32p, i64p, u64p = C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)
        u32pp = C.POINTER(C.POINTER(C.c_uint32))
        L.oracle_overlap.argtypes = [i32p, i64, i32p, i64]
        L.oracle_overlap.restype = i64
        L.oracle_similar.argtypes = [i64, i64, i64, i64, i64]
        L.oracle_similar.restype = C.c_int
        L.oracle_similar_sim.argtypes = [C.c_int, i64, i64, i64, i64, i64]
        L.oracle_similar_sim.restype = C.c_int
        L.oracle_in_window.argtypes = [C.c_int, i64, i64, i64, i64]
        L.oracle_in_window.restype = C.c_int
        L.oracle_self_join.argtypes = [i64, i64p, i32p, C.c_int, i64, i64, u32pp, u32pp]
        L.oracle_self_join.restype = i64
        L.oracle_join_rows.argtypes = [i64, i64p, i32p, C.c_int, i64, i64, i64p, i64, u32pp, u32pp]
        L.oracle_join_rows.restype = i64
        L.oracle_join_rows_window.argtypes = [i64, i64p, i32p, C.c_int, i64, i64, i64p, i64, u32pp,
                                              u32pp]
        L.oracle_join_rows_window.restype = i64
        L.oracle_search.argtypes = [i32p, i64, i64, i64p, i32p, C.c_int, i64, i64, C.POINTER(i64p)]
        L.oracle_search.restype = i64
        L.oracle_bitmap.argtypes = [i32p, i64, C.c_int, C.c_int, u64p]
        L.oracle_bitmap.restype = None
        L.oracle_bitmaps.argtypes = [i64, i64p, i32p, C.c_int, C.c_int, u64p]
        L.oracle_bitmaps.restype = None
        L.oracle_hamming.argtypes = [u64p, u64p, C.c_int]
        L.oracle_hamming.restype = i64
        L.oracle_upper_bound.argtypes = [i64, i64, i64]
        L.oracle_upper_bound.restype = i64
        L.oracle_filter_counts.argtypes = [i64, i64p, i32p, C.c_int, i64, i64, C.c_int, C.c_int,
                                           i64, i64p]
        L.oracle_filter_counts.restype = None
        L.oracle_prefix_counts.argtypes = [i64, i64p, i32p, C.c_int, i64, i64, C.c_int, C.c_int,
                                           i64p]
        L.oracle_prefix_counts.restype = None
        L.oracle_combined_method.argtypes = [i64, i64]
        L.oracle_combined_method.restype = C.c_int
        L.oracle_combined_method_sim.argtypes = [C.c_int, i64, i64]
        L.oracle_combined_method_sim.restype = C.c_int
        L.oracle_rs_join.argtypes = [i64, i64p, i32p, i64, i64p, i32p, C.c_int, i64, i64, u32pp,
                                     u32pp]
        L.oracle_rs_join.restype = i64
        L.oracle_rs_filter_counts.argtypes = [i64, i64p, i32p, i64, i64p, i32p, C.c_int, i64, i64,
                                              C.c_int, C.c_int, i64, i64p]
        L.oracle_rs_filter_counts.restype = None
        L.oracle_rs_prefix_counts.argtypes = [i64, i64p, i32p, i64, i64p, i32p, C.c_int, i64, i64,
                                              C.c_int, C.c_int, i64p]
        L.oracle_rs_prefix_counts.restype = None
        L.oracle_window_pairs_hist.argtypes = [i64p, i64, C.c_int, i64, i64]
        L.oracle_window_pairs_hist.restype = i64
        L.oracle_rs_window_pairs_hist.argtypes = [i64p, i64, i64p, i64, C.c_int, i64, i64]
        L.oracle_rs_window_pairs_hist.restype = i64
        L.oracle_num_threads.argtypes = []
        L.oracle_num_threads.restype = C.c_int
        L.oracle_free.argtypes = [C.c_void_p]
        L.oracle_free.restype = None
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _i32(x):
    return np.ascontiguousarray(x, dtype=np.int32)


def _i64(x):
    return np.ascontiguousarray(x, dtype=np.int64)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def overlap(x, y) -> int:
    """|x & y| of two strictly increasing token arrays."""
    x, y = _i32(x), _i32(y)
    return int(lib().oracle_overlap(_p(x, C.c_int32), len(x), _p(y, C.c_int32), len(y)))


def similar(o: int, nx: int, ny: int, p: int, q: int) -> bool:
    """Jaccard >= p/q given the overlap o and the sizes (Table 1)."""
    return bool(lib().oracle_similar(o, nx, ny, p, q))


def similar_sim(sim: int, o: int, nx: int, ny: int, p: int, q: int) -> bool:
    """sim >= p/q for Jaccard, Cosine, Dice or Overlap given o and the sizes (Table 1)."""
    return bool(lib().oracle_similar_sim(sim, o, nx, ny, p, q))


def in_window(sim: int, a: int, b: int, p: int, q: int) -> bool:
    """Sizes a <= b inside the length filter's window (Table 2)."""
    return bool(lib().oracle_in_window(sim, a, b, p, q))


def _take_pairs(n, A, B):
    L = lib()
    if n < 0:
        raise MemoryError("oracle allocation failed")
    if n == 0:
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32)
    a = np.ctypeslib.as_array(A, shape=(n,)).copy()
    b = np.ctypeslib.as_array(B, shape=(n,)).copy()
    L.oracle_free(C.cast(A, C.c_void_p))
    L.oracle_free(C.cast(B, C.c_void_p))
    return a, b


def self_join(offsets, tokens, p: int, q: int, sim: int = JACCARD):
    """All pairs a<b (original ids) with sim >= p/q, sorted by (a, b)."""
    off, tok = _i64(offsets), _i32(tokens)
    A, B = C.POINTER(C.c_uint32)(), C.POINTER(C.c_uint32)()
    n = lib().oracle_self_join(len(off) - 1, _p(off, C.c_int64), _p(tok, C.c_int32), sim, p, q,
                               C.byref(A), C.byref(B))
    return _take_pairs(n, A, B)


def rs_join(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, sim: int = JACCARD):
    """All pairs (r, s) of R x S with sim >= p/q (Eq. 1, an RS-join), sorted by (r, s)."""
    ro, rt, so, st = _i64(r_offsets), _i32(r_tokens), _i64(s_offsets), _i32(s_tokens)
    A, B = C.POINTER(C.c_uint32)(), C.POINTER(C.c_uint32)()
    n = lib().oracle_rs_join(len(ro) - 1, _p(ro, C.c_int64), _p(rt, C.c_int32), len(so) - 1,
                             _p(so, C.c_int64), _p(st, C.c_int32), sim, p, q, C.byref(A),
                             C.byref(B))
    return _take_pairs(n, A, B)


def rs_filter_counts(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, b: int,
                     method: int, sim: int = JACCARD, cutoff: int = 0):
    """(window pairs, survivors, results) of an RS-join with the Bitmap Filter (pairs whose
    larger set exceeds ``cutoff`` > 0 tokens skip the bound)."""
    ro, rt, so, st = _i64(r_offsets), _i32(r_tokens), _i64(s_offsets), _i32(s_tokens)
    cnt = np.zeros(3, np.int64)
    lib().oracle_rs_filter_counts(len(ro) - 1, _p(ro, C.c_int64), _p(rt, C.c_int32), len(so) - 1,
                                  _p(so, C.c_int64), _p(st, C.c_int32), sim, p, q, b, method,
                                  cutoff, _p(cnt, C.c_int64))
    if cnt[0] < 0:
        raise MemoryError("oracle allocation failed")
    return int(cnt[0]), int(cnt[1]), int(cnt[2])


def rs_prefix_counts(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, b: int,
                     method: int, sim: int = JACCARD):
    """(candidates, survivors, results) of an RS-join with prefix-filter candidates."""
    ro, rt, so, st = _i64(r_offsets), _i32(r_tokens), _i64(s_offsets), _i32(s_tokens)
    cnt = np.zeros(3, np.int64)
    lib().oracle_rs_prefix_counts(len(ro) - 1, _p(ro, C.c_int64), _p(rt, C.c_int32), len(so) - 1,
                                  _p(so, C.c_int64), _p(st, C.c_int32), sim, p, q, b, method,
                                  _p(cnt, C.c_int64))
    if cnt[0] < 0:
        raise MemoryError("oracle allocation failed")
    return int(cnt[0]), int(cnt[1]), int(cnt[2])


def join_rows(offsets, tokens, p: int, q: int, rows, sim: int = JACCARD):
    """Similar pairs (min,max) that touch one of ``rows``, sorted, unique."""
    off, tok, r = _i64(offsets), _i32(tokens), _i64(rows)
    A, B = C.POINTER(C.c_uint32)(), C.POINTER(C.c_uint32)()
    n = lib().oracle_join_rows(len(off) - 1, _p(off, C.c_int64), _p(tok, C.c_int32), sim, p, q,
                               _p(r, C.c_int64), len(r), C.byref(A), C.byref(B))
    return _take_pairs(n, A, B)


def join_rows_window(offsets, tokens, p: int, q: int, rows, sim: int = JACCARD):
    """join_rows with the length filter (Table 2): same output, fewer pairs verified."""
    off, tok, r = _i64(offsets), _i32(tokens), _i64(rows)
    A, B = C.POINTER(C.c_uint32)(), C.POINTER(C.c_uint32)()
    n = lib().oracle_join_rows_window(len(off) - 1, _p(off, C.c_int64), _p(tok, C.c_int32), sim,
                                      p, q, _p(r, C.c_int64), len(r), C.byref(A), C.byref(B))
    return _take_pairs(n, A, B)


def search(probe, offsets, tokens, p: int, q: int, sim: int = JACCARD):
    """Ids of the collection's sets with sim(probe, s) >= p/q, ascending."""
    x, off, tok = _i32(probe), _i64(offsets), _i32(tokens)
    ids = C.POINTER(C.c_int64)()
    n = lib().oracle_search(_p(x, C.c_int32), len(x), len(off) - 1, _p(off, C.c_int64),
                            _p(tok, C.c_int32), sim, p, q, C.byref(ids))
    if n < 0:
        raise MemoryError("oracle allocation failed")
    if n == 0:
        return np.zeros(0, np.int64)
    out = np.ctypeslib.as_array(ids, shape=(n,)).copy()
    lib().oracle_free(C.cast(ids, C.c_void_p))
    return out


def combined_method(p: int, q: int, sim: int = JACCARD) -> int:
    """Alg. 4's choice for threshold p/q (switch points on the normalised overlap:
    2p/(p+q) for Jaccard, p/q for Dice and Cosine; Xor for Overlap)."""
    return int(lib().oracle_combined_method_sim(sim, p, q))


def bitmap(tokens, b: int, method: int):
    """One set's b-bit bitmap (Alg. 3a/3b/3c) as uint64[b/64]."""
    x = _i32(tokens)
    out = np.zeros(b // 64, np.uint64)
    lib().oracle_bitmap(_p(x, C.c_int32), len(x), b, method, _p(out, C.c_uint64))
    return out


def bitmaps(offsets, tokens, b: int, method: int):
    """Bitmaps of a collection in original order, uint64[N, b/64]."""
    off, tok = _i64(offsets), _i32(tokens)
    n = len(off) - 1
    out = np.zeros((n, b // 64), np.uint64)
    lib().oracle_bitmaps(n, _p(off, C.c_int64), _p(tok, C.c_int32), b, method,
                         _p(out, C.c_uint64))
    return out


def hamming(br, bs) -> int:
    br, bs = np.ascontiguousarray(br, np.uint64), np.ascontiguousarray(bs, np.uint64)
    return int(lib().oracle_hamming(_p(br, C.c_uint64), _p(bs, C.c_uint64), 64 * len(br)))


def upper_bound(nr: int, ns: int, h: int) -> int:
    """Eq. 2: floor((|r| + |s| - h) / 2)."""
    return int(lib().oracle_upper_bound(nr, ns, h))


def prefix_counts(offsets, tokens, p: int, q: int, b: int, method: int, sim: int = JACCARD):
    """(candidates, survivors, results) with the prefix filter choosing the candidates."""
    off, tok = _i64(offsets), _i32(tokens)
    cnt = np.zeros(3, np.int64)
    lib().oracle_prefix_counts(len(off) - 1, _p(off, C.c_int64), _p(tok, C.c_int32), sim, p, q,
                               b, method, _p(cnt, C.c_int64))
    if cnt[0] < 0:
        raise MemoryError("oracle allocation failed")
    return int(cnt[0]), int(cnt[1]), int(cnt[2])


def filter_counts(offsets, tokens, p: int, q: int, b: int, method: int, sim: int = JACCARD,
                  cutoff: int = 0):
    """(window pairs, survivors, results) of Alg. 6 + host verification; pairs whose larger
    set exceeds ``cutoff`` > 0 tokens skip the bound (Section 3.5)."""
    off, tok = _i64(offsets), _i32(tokens)
    cnt = np.zeros(3, np.int64)
    lib().oracle_filter_counts(len(off) - 1, _p(off, C.c_int64), _p(tok, C.c_int32), sim, p, q,
                               b, method, cutoff, _p(cnt, C.c_int64))
    if cnt[0] < 0:
        raise MemoryError("oracle allocation failed")
    return int(cnt[0]), int(cnt[1]), int(cnt[2])


def window_pairs(sizes, p: int, q: int, sim: int = JACCARD) -> int:
    """Pairs inside the length window (Table 2) of a self-join of sets with these sizes:
    the window count of ``filter_counts``, from the size histogram alone."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if len(sizes) == 0:
        return 0
    hist = np.bincount(sizes).astype(np.int64)
    w = int(lib().oracle_window_pairs_hist(_p(hist, C.c_int64), len(hist), sim, p, q))
    if w < 0:
        raise ValueError("negative size")
    return w



def rs_window_pairs(sizes_r, sizes_s, p: int, q: int, sim: int = JACCARD) -> int:
    """Pairs of R x S inside the length window (Table 2), from the two size histograms:
    the window count of ``rs_filter_counts`` (and of probe queries against a collection)."""
    sr, ss = np.asarray(sizes_r, dtype=np.int64), np.asarray(sizes_s, dtype=np.int64)
    if len(sr) == 0 or len(ss) == 0:
        return 0
    hr, hs = np.bincount(sr).astype(np.int64), np.bincount(ss).astype(np.int64)
    w = int(lib().oracle_rs_window_pairs_hist(_p(hr, C.c_int64), len(hr), _p(hs, C.c_int64),
                                              len(hs), sim, p, q))
    if w < 0:
        raise ValueError("negative size")
    return w


__all__ = ["XOR", "SET", "NEXT", "COMBINED", "METHODS", "JACCARD", "COSINE", "DICE", "OVERLAP",
           "overlap", "similar", "similar_sim", "in_window", "self_join",
           "join_rows", "join_rows_window", "rs_join", "rs_filter_counts", "rs_prefix_counts",
           "search", "bitmap",
           "bitmaps", "hamming", "upper_bound",
           "filter_counts", "prefix_counts", "window_pairs", "rs_window_pairs", "combined_method", "num_threads", "lib"]
