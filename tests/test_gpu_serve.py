"""Resident index and served probe queries against the oracle."""
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


def small_setup(seed=0, n=20_000, nq=400):
    spec = I.CollectionSpec(n, 3_000, 1.1, ("lognormal", 2.3, 0.6, 1, 200), seed=seed,
                            planted_frac=0.05)
    off, tok = I.gen_collection(spec)
    qs = I.QuerySpec(n_queries=nq, rate_qps=50_000.0, size_lo=2, size_hi=60, seed=seed + 1)
    arr, qoff, qtok, p, q = I.gen_queries(qs, spec, off, tok)
    return off, tok, arr, qoff, qtok, p, q


@pytest.mark.parametrize("b", [64, 128, 256, 192])
def test_index_query_matches_oracle(b):
    # b = 64, 128, 256 keep the probe's bitmap in registers in the query filter;
    # b = 192 takes the filter's path for any width
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=b)
    idx = _bmj.Index(torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda(), b=b)
    assert len(idx) == len(off) - 1
    res, st = idx.query(qoff, qtok, p, q)
    assert st["n_queries"] == len(p) and st["batches"] == 1
    nonempty = 0
    for x in range(len(p)):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(res[x], want), x
        nonempty += len(want) > 0
    assert nonempty > 50
    # batches of at most 8 probes: their bitmaps come from the window kernel
    mixed, _, _ = idx.serve(qoff, qtok, arr, p, q, n_slots=2, max_batch_queries=8)
    assert all(np.array_equal(u, v) for u, v in zip(mixed, res))
    idx.close()


@pytest.mark.parametrize("method", [_bmj.BMJ_SET, _bmj.BMJ_NEXT])
def test_index_with_other_generation_methods(method):
    # Set bitmaps of small batches are built in the window kernel, Next ones by the
    # bitmap kernel; both must equal the oracle's search, alone and batched
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=20 + method, nq=120)
    idx = _bmj.Index(off, tok, b=128, method=method)
    res, _ = idx.query(qoff, qtok, p, q)
    for x in range(len(p)):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(res[x], want), x
    mixed, _, _ = idx.serve(qoff, qtok, arr, p, q, n_slots=2, max_batch_queries=8)
    assert all(np.array_equal(a, b) for a, b in zip(mixed, res))
    idx.close()


def test_each_query_same_alone_and_in_the_mix():
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=3, nq=300)
    idx = _bmj.Index(off, tok, b=64)
    mixed, lat, st = idx.serve(qoff, qtok, arr, p, q, n_slots=3, max_batch_queries=64)
    assert st["n_queries"] == len(p) and st["batches"] >= 2
    assert np.all(lat > 0) and st["p99_ms"] >= st["p50_ms"] > 0
    # every query waiting from the start, at most 5 per batch
    tight, _, st2 = idx.serve(qoff, qtok, np.zeros_like(arr), p, q, n_slots=2,
                              max_batch_queries=5, max_batch_window_pairs=1)
    assert st2["batches"] >= -(-len(p) // 5)
    for x in range(0, len(p), 7):
        alone, _ = idx.query(qoff[x:x + 2] - qoff[x], qtok[qoff[x]:qoff[x + 1]], p[x:x + 1], q[x:x + 1])
        assert np.array_equal(alone[0], mixed[x]) and np.array_equal(alone[0], tight[x]), x
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(mixed[x], want)
    idx.close()


@pytest.mark.parametrize("copies", [300, 5000])
def test_small_and_large_result_batches(copies):
    # A batch's first 2048 result keys come back with its counters and are sorted on
    # the host; a batch with more results is sorted on the device.  `copies` identical
    # resident sets equal to the probe put the batch on one side or the other.
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=11, n=4000, nq=6)
    dup = np.array([5, 17, 99, 1000, 4242], np.int32)
    off2 = np.concatenate([off, off[-1] + len(dup) * np.arange(1, copies + 1, dtype=np.int64)])
    tok2 = np.concatenate([tok, np.tile(dup, copies)])
    qoff2 = np.concatenate([qoff, [qoff[-1] + len(dup)]]).astype(np.int64)
    qtok2 = np.concatenate([qtok, dup]).astype(np.int32)
    p2 = np.concatenate([p, [4]]).astype(np.uint32)
    q2 = np.concatenate([q, [5]]).astype(np.uint32)
    idx = _bmj.Index(off2, tok2, b=64)
    res, st = idx.query(qoff2, qtok2, p2, q2)
    assert st["batches"] == 1 and (st["results"] > 2048) == (copies > 2048)
    for x in range(len(p2)):
        want = O.search(qtok2[qoff2[x]:qoff2[x + 1]], off2, tok2, int(p2[x]), int(q2[x]))
        assert np.array_equal(res[x], want), x
    assert len(res[-1]) >= copies
    idx.close()


def test_invalid_probes_and_empty_batch():
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=5, n=2000, nq=10)
    idx = _bmj.Index(off, tok)
    res, st = idx.query(np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.uint32),
                        np.zeros(0, np.uint32))
    assert res == [] and st["n_queries"] == 0
    bad = qtok.copy()
    a = int(qoff[0])
    if qoff[1] - qoff[0] >= 2:
        bad[a], bad[a + 1] = bad[a + 1], bad[a]
        with pytest.raises(_bmj.BmjError) as e:
            idx.query(qoff, bad, p, q)
        assert e.value.status == _bmj.BMJ_ERR_UNSORTED
    with pytest.raises(_bmj.BmjError) as e:
        idx.query(qoff, qtok, q, p if np.any(p < q) else p)   # p > q somewhere
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    idx.close()


@pytest.mark.parametrize("b", [64, 128])
def test_full_served_workload_sampled(b):
    # 2,000,000 resident sets (Zipf 1.1 over 300,000, lognormal(2.3, 0.6)); a Poisson
    # stream at 20,000 queries/s of probes of size 2..300 (half edited resident copies);
    # the index at 128 bits (the width the bench serves at) and at 64.
    spec = I.spec_resident_2m()
    off_d, tok_d = I.gen_collection_device(spec)
    off, tok = off_d.cpu().numpy(), tok_d.cpu().numpy()
    qs = I.QuerySpec(n_queries=4000)
    arr, qoff, qtok, p, q = I.gen_queries(qs, spec, off, tok)
    idx = _bmj.Index(off_d, tok_d, b=b)
    res, lat, st = idx.serve(qoff, qtok, arr, p, q)
    assert st["n_queries"] == 4000 and st["p99_ms"] > 0
    # window pairs = every (probe, resident set) pair inside Table 2's two-sided window,
    # counted by the oracle from the size histograms, one threshold at a time
    psz, rsz = np.diff(qoff), np.diff(off)
    want_win = sum(O.rs_window_pairs(psz[(p == pk) & (q == qk)], rsz, int(pk), int(qk))
                   for pk, qk in set(zip(p.tolist(), q.tolist())))
    assert st["window_pairs"] == want_win
    rng = np.random.default_rng(0)
    for x in rng.choice(4000, 24, replace=False):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(res[x], want), x
    # small batches at 1/2 whose windows are wide (millions of resident sets each):
    # one probe (survivors verified inside the filter) and four (the window total
    # is above the in-filter bound, so a verification kernel runs) give the oracle's ids
    wide = np.nonzero((psz >= 8) & (psz <= 16))[0][:4]
    for sel in (wide[:1], wide):
        o2 = np.zeros(len(sel) + 1, np.int64)
        o2[1:] = np.cumsum(psz[sel])
        t2 = np.concatenate([qtok[qoff[x]:qoff[x + 1]] for x in sel])
        half = np.ones(len(sel), np.uint32)
        got, st2 = idx.query(o2, t2, half, 2 * half)
        assert st2["window_pairs"] == O.rs_window_pairs(psz[sel], rsz, 1, 2) > 1_000_000 * len(sel)
        for k, x in enumerate(sel):
            want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, 1, 2)
            assert np.array_equal(got[k], want), x
    idx.close()


@pytest.mark.parametrize("sim", [_bmj.BMJ_COSINE, _bmj.BMJ_DICE, _bmj.BMJ_OVERLAP])
def test_index_other_similarity_functions(sim):
    # The index's function (set at creation) decides the two-sided window (Table 2),
    # the Eq. 2 limit per pair and the exact test; every probe equals the oracle's
    # search, alone and in the continuous mix.
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=20 + sim, nq=200)
    if sim == _bmj.BMJ_OVERLAP:          # token-count thresholds
        p = (3 + np.arange(len(p)) % 6).astype(np.uint32)
        q = np.ones(len(p), np.uint32)
    idx = _bmj.Index(torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda(), b=64, sim=sim)
    res, st = idx.query(qoff, qtok, p, q)
    mixed, lat, _ = idx.serve(qoff, qtok, arr, p, q, n_slots=3, max_batch_queries=32)
    nonempty = 0
    for x in range(len(p)):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]), sim=sim)
        assert np.array_equal(res[x], want) and np.array_equal(mixed[x], want), x
        nonempty += len(want) > 0
    assert nonempty > 20
    if sim != _bmj.BMJ_OVERLAP:
        with pytest.raises(_bmj.BmjError) as e:   # p > q is no valid threshold for it
            idx.query(qoff[:2], qtok[:int(qoff[1])], np.array([5], np.uint32), np.array([4], np.uint32))
        assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    idx.close()


def test_live_server_submissions_while_batches_run():
    # bmj_serve_open / submit / poll / close: a second host thread submits queries
    # while earlier batches are on the device and the main thread polls; every result
    # equals the oracle's search, in that mix and alone (one query in flight at a time).
    import threading
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=41, nq=300)
    idx = _bmj.Index(torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda(), b=64)
    srv = _bmj.Server(idx, n_slots=3, max_batch_queries=16, max_probe_tokens=64)
    tickets = [None] * len(p)
    done = threading.Event()

    def producer():
        for x in range(len(p)):
            tickets[x] = srv.submit(qtok[qoff[x]:qoff[x + 1]], int(p[x]), int(q[x]))
            if x % 16 == 15:
                done.wait(0.0003)   # let some batches start before the next submissions
    th = threading.Thread(target=producer)
    th.start()
    got = {}
    while len(got) < len(p):
        for x in range(len(p)):
            if x not in got and tickets[x] is not None:
                r = srv.poll(tickets[x])
                if r is not None:
                    got[x] = r
    th.join()
    st = srv.close()
    assert st["n_queries"] == len(p) and 1 <= st["batches"] <= len(p)
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    psz, rsz = np.diff(qoff), np.diff(off)
    assert st["window_pairs"] == sum(
        O.rs_window_pairs(psz[(p == pk) & (q == qk)], rsz, int(pk), int(qk))
        for pk, qk in set(zip(p.tolist(), q.tolist())))
    alone = _bmj.Server(idx, n_slots=1)
    nonempty = 0
    for x in range(len(p)):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(got[x][0], want), x
        assert got[x][1] > 0
        nonempty += len(want) > 0
        if x < 60:
            t = alone.submit(qtok[qoff[x]:qoff[x + 1]], int(p[x]), int(q[x]))
            ids, _ = alone.poll(t, wait_ms=20_000)
            assert np.array_equal(ids, want), x
    assert nonempty > 30
    alone.close()
    idx.close()


def test_live_server_errors():
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=43, nq=10)
    idx = _bmj.Index(off, tok, b=64)
    srv = _bmj.Server(idx, n_slots=2, max_probe_tokens=8)
    with pytest.raises(_bmj.BmjError) as e:
        srv.submit(np.array([3, 2, 5]), 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_UNSORTED
    with pytest.raises(_bmj.BmjError) as e:
        srv.submit(np.arange(9), 1, 2)            # above max_probe_tokens
    assert e.value.status == _bmj.BMJ_ERR_TOO_LARGE
    with pytest.raises(_bmj.BmjError) as e:
        srv.submit(np.array([1, 2]), 3, 2)        # p > q
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    with pytest.raises(_bmj.BmjError) as e:
        srv.submit(np.zeros(0, np.int32), 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_EMPTY_SET
    x = int(np.nonzero((np.diff(off) >= 2) & (np.diff(off) <= 8))[0][0])   # a resident set
    t = srv.submit(tok[off[x]:off[x + 1]], 1, 2)
    ids, lat = srv.poll(t, wait_ms=20_000)
    assert np.array_equal(ids, O.search(tok[off[x]:off[x + 1]], off, tok, 1, 2)) and x in ids.tolist()
    with pytest.raises(_bmj.BmjError) as e:     # a result is handed out once
        srv.poll(t)
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG
    # close finishes what was submitted; nothing can be submitted after it
    last = [srv.submit(qtok[qoff[x]:qoff[x + 1]][:8], 1, 2) for x in range(5)]
    st = srv.close()
    assert st["n_queries"] == 6 and len(last) == 5
    idx.close()


def test_live_server_many_submitters_and_pollers():
    # Four host threads submit concurrently and four others poll their tickets with
    # waits: every ticket is unique, every result equals the oracle's search.
    import threading
    off, tok, arr, qoff, qtok, p, q = small_setup(seed=47, nq=240)
    idx = _bmj.Index(torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda(), b=128)
    srv = _bmj.Server(idx, n_slots=4, max_batch_queries=8, max_probe_tokens=64)
    tickets = {}
    lock = threading.Lock()
    got = {}

    def submitter(part):
        for x in range(part, len(p), 4):
            t = srv.submit(qtok[qoff[x]:qoff[x + 1]], int(p[x]), int(q[x]))
            with lock:
                tickets[x] = t

    def poller(part):
        for x in range(part, len(p), 4):
            while True:
                with lock:
                    t = tickets.get(x)
                if t is not None:
                    break
            r = srv.poll(t, wait_ms=20_000)
            assert r is not None
            got[x] = r[0]

    threads = [threading.Thread(target=f, args=(k,)) for f in (submitter, poller) for k in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    st = srv.close()
    assert st["n_queries"] == len(p)
    assert sorted(tickets.values()) == list(range(len(p)))
    for x in range(len(p)):
        want = O.search(qtok[qoff[x]:qoff[x + 1]], off, tok, int(p[x]), int(q[x]))
        assert np.array_equal(got[x], want), x
    idx.close()
