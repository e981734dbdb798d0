"""The allocation-free Bitmap Filter entry point, bmj_bitmap_filter_noalloc.

Some callers cannot allocate device memory while they run -- code that lives
inside a fixed memory budget owned by another framework's pool, or a
latency-critical serving loop where cudaMalloc/cudaFree and the device
synchronisation they can cause are not allowed.  For them the library runs
the same filter kernel as bmj_self_join with its scratch in a fixed device
array.  This file checks that entry point through the C ABI, on two calls in
a row (the second call reuses the scratch left by the first), against the
CPU oracle -- its survivor count equals the oracle's Bitmap Filter count
(Alg. 6 with the Eq. 2 bound) and the survivors, verified exactly, give the
oracle's pair list -- and against the existing bmj_self_join, which must
agree with both.  It is named to be collected last.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_1711_07295_b300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1711_07295_b300 import _bmj  # noqa: E402


def size_sorted(off, tok, b):
    """Size-sorted copy of a collection with its bitmaps (from bmj_build_bitmaps)."""
    sizes = np.diff(off)
    order = np.argsort(sizes, kind="stable")
    s_sizes = sizes[order]
    s_off = np.zeros(len(order) + 1, np.int64)
    s_off[1:] = np.cumsum(s_sizes)
    s_tok = np.concatenate([tok[off[i]:off[i + 1]] for i in order]).astype(np.int32)
    bm = _bmj.bmj_build_bitmaps(torch.from_numpy(s_off).cuda(), torch.from_numpy(s_tok).cuda(),
                                b=b, method=_bmj.BMJ_XOR)
    d_sizes = torch.from_numpy(s_sizes.astype(np.uint32).view(np.int32)).cuda()
    return order, bm, d_sizes


def call_noalloc(bm, d_sizes, n, b, p, q, cap):
    out = torch.full((2 * max(cap, 1),), -1, dtype=torch.int32, device="cuda")
    count = C.c_int64(-1)
    st = _bmj.lib().bmj_bitmap_filter_noalloc(
        C.c_void_p(bm.data_ptr()), C.c_void_p(d_sizes.data_ptr()), n, b, p, q,
        C.c_void_p(out.data_ptr()), cap, C.byref(count),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, count.value, out


@pytest.mark.parametrize("b,p,q", [(64, 1, 2), (128, 4, 5), (256, 3, 5)])
def test_noalloc_filter_matches_oracle_twice(b, p, q):
    off, tok = I.random_collection(6000, 1500, 1, 40, seed=21 + b, planted_frac=0.1)
    sets = [tok[off[i]:off[i + 1]] for i in range(len(off) - 1)]
    order, bm, d_sizes = size_sorted(off, tok, b)
    # the oracle's counts and pairs (Alg. 6 with Eq. 2; Eq. 1 over all pairs)
    win, surv, res = O.filter_counts(off, tok, p, q, b, O.XOR)
    oa, ob = O.self_join(off, tok, p, q)
    want = set(zip(oa.tolist(), ob.tolist()))
    assert res == len(want) > 0
    # the existing entry point agrees with the oracle on the same collection
    ref_a, ref_b, ref_st = _bmj.bmj_self_join(off, tok, p, q, b=b, method=_bmj.BMJ_XOR)
    assert ref_st["survivors"] == surv and set(zip(ref_a.tolist(), ref_b.tolist())) == want
    cap = surv + 64
    previous = None
    for _call in range(2):
        st, count, out = call_noalloc(bm, d_sizes, len(order), b, p, q, cap)
        assert st == _bmj.BMJ_OK, _bmj.bmj_strerror(st)
        assert count == surv == ref_st["survivors"]
        pairs = out[:2 * count].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
        assert np.all(pairs[:, 1] < pairs[:, 0])
        oi, oj = order[pairs[:, 0]], order[pairs[:, 1]]
        lo, hi = np.minimum(oi, oj), np.maximum(oi, oj)
        keys = np.sort((lo << 32) | hi)
        assert len(np.unique(keys)) == len(keys)
        if previous is not None:
            assert np.array_equal(keys, previous)
        previous = keys
        similar = set()
        for x, y in zip(lo.tolist(), hi.tolist()):
            o = len(np.intersect1d(sets[x], sets[y], assume_unique=True))
            if o * (p + q) >= p * (len(sets[x]) + len(sets[y])):
                similar.add((x, y))
        assert similar == want


def test_noalloc_filter_errors():
    off, tok = I.random_collection(3000, 800, 1, 30, seed=5, planted_frac=0.1)
    order, bm, d_sizes = size_sorted(off, tok, 64)
    n = len(order)
    _, surv, _ = O.filter_counts(off, tok, 1, 2, 64, O.XOR)
    ref = {"survivors": surv}
    assert surv > 10
    # output too small: full count reported, first out_cap pairs written
    st, count, out = call_noalloc(bm, d_sizes, n, 64, 1, 2, 10)
    assert st == _bmj.BMJ_ERR_OUTPUT_OVERFLOW and count == ref["survivors"]
    assert (out[:20].cpu().numpy() >= 0).all()
    # sizes out of order
    bad = d_sizes.flip(0).contiguous()
    st, count, _ = call_noalloc(bm, bad, n, 64, 1, 2, 16)
    assert st == _bmj.BMJ_ERR_UNSORTED
    # thresholds beyond the scratch array: one set of 1,100,000 tokens needs
    # 4 * (2 * 1,100,000 + 1) bytes of thresholds > 8 MiB
    big = torch.tensor([1, 2, 3, 1_100_000], dtype=torch.int32, device="cuda")
    bm4 = torch.zeros((4, 1), dtype=torch.int64, device="cuda")
    st, count, _ = call_noalloc(bm4, big, 4, 64, 1, 2, 16)
    assert st == _bmj.BMJ_ERR_TOO_LARGE
    # invalid arguments are rejected on the host
    st, _, _ = call_noalloc(bm, d_sizes, n, 96, 1, 2, 16)
    assert st == _bmj.BMJ_ERR_INVALID_ARG
    st, _, _ = call_noalloc(bm, d_sizes, n, 64, 3, 2, 16)
    assert st == _bmj.BMJ_ERR_INVALID_ARG
    # and the scratch still works afterwards
    st, count, _ = call_noalloc(bm, d_sizes, n, 64, 1, 2, ref["survivors"])
    assert st == _bmj.BMJ_OK and count == ref["survivors"]
