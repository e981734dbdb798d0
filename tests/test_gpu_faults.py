"""Failure paths without a GPU fault: an injected allocation failure (host)
and a bounded device wait that runs out (one copy is never issued, so the
mbarrier it would complete stays unset).  Both must come back as status codes
with the context still usable."""
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


def test_injected_timeout_and_allocation_failures(monkeypatch):
    off, tok = I.random_collection(20_000, 3_000, 1, 40, seed=77, planted_frac=0.05)
    d_off, d_tok = torch.from_numpy(off).cuda(), torch.from_numpy(tok).cuda()
    monkeypatch.setenv("BMJ_FAULT", "timeout")
    with pytest.raises(_bmj.BmjError) as e:
        _bmj.bmj_self_join(d_off, d_tok, 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_TIMEOUT
    for k in (1, 2, 5, 9):
        monkeypatch.setenv("BMJ_FAULT", f"alloc:{k}")
        with pytest.raises(_bmj.BmjError) as e:
            _bmj.bmj_self_join(d_off, d_tok, 1, 2)
        assert e.value.status == _bmj.BMJ_ERR_OOM
    monkeypatch.delenv("BMJ_FAULT")
    a, b, st = _bmj.bmj_self_join(d_off, d_tok, 1, 2)
    ra, rb = O.self_join(off, tok, 1, 2)
    assert np.array_equal(a, ra) and np.array_equal(b, rb)
    torch.cuda.synchronize()


def test_refused_key_buffer_verifies_the_queue_in_slices(monkeypatch):
    # A key buffer as long as the survivor queue is refused: verification runs over
    # the queue in slices and appends their results; the pairs and counts are exact.
    off, tok = I.random_collection(6_000, 1_500, 1, 40, seed=78, planted_frac=0.1)
    ra, rb = O.self_join(off, tok, 1, 2)
    w, s, r = O.filter_counts(off, tok, 1, 2, 64, O.XOR)
    monkeypatch.setenv("BMJ_FAULT", "keys")
    a, b, st = _bmj.bmj_self_join(off, tok, 1, 2, b=64)
    monkeypatch.delenv("BMJ_FAULT")
    assert np.array_equal(a, ra) and np.array_equal(b, rb)
    assert (st["window_pairs"], st["survivors"], st["results"]) == (w, s, r) and s >= 5


def test_device_failures_stick_to_an_index(monkeypatch):
    # a call on an index that fails as a CUDA runtime error would (injected on the
    # host) leaves every later call on that index failing with the same status;
    # argument errors do not stick, and a fresh index is unaffected
    off, tok = I.random_collection(5000, 1000, 1, 30, seed=78, planted_frac=0.1)
    qoff, qtok = off[:41].copy(), tok[:off[40]].copy()
    p, q = np.full(40, 3, np.uint32), np.full(40, 4, np.uint32)
    idx = _bmj.Index(off, tok, b=64)
    want, _ = idx.query(qoff, qtok, p, q)
    with pytest.raises(_bmj.BmjError) as e:      # an argument error: not sticky
        idx.query(qoff, qtok, np.full(40, 5, np.uint32), q)
    assert e.value.status == _bmj.BMJ_ERR_INVALID_ARG and idx.status() == _bmj.BMJ_OK
    monkeypatch.setenv("BMJ_FAULT", "serve")
    with pytest.raises(_bmj.BmjError) as e:
        idx.query(qoff, qtok, p, q)
    assert e.value.status == _bmj.BMJ_ERR_CUDA
    monkeypatch.delenv("BMJ_FAULT")
    assert idx.status() == _bmj.BMJ_ERR_CUDA
    with pytest.raises(_bmj.BmjError) as e:      # sticky: the fault is gone, the status stays
        idx.query(qoff, qtok, p, q)
    assert e.value.status == _bmj.BMJ_ERR_CUDA
    with pytest.raises(_bmj.BmjError) as e:
        idx.serve(qoff, qtok, np.zeros(40), p, q)
    assert e.value.status == _bmj.BMJ_ERR_CUDA
    idx.close()
    fresh = _bmj.Index(off, tok, b=64)
    got, _ = fresh.query(qoff, qtok, p, q)
    assert fresh.status() == _bmj.BMJ_OK
    assert len(got) == len(want) and all(np.array_equal(x, y) for x, y in zip(got, want))
    fresh.close()


def test_live_server_device_failure_fails_its_queries(monkeypatch):
    # A live server whose first batch fails as a CUDA runtime error would (injected on
    # the host at open: nothing is launched): every submitted query comes back with that
    # status, later submissions are refused with it, close reports it, and it sticks to
    # the index; a fresh index serves the same queries correctly.
    off, tok = I.random_collection(5000, 1000, 1, 30, seed=79, planted_frac=0.1)
    idx = _bmj.Index(off, tok, b=64)
    monkeypatch.setenv("BMJ_FAULT", "serve")
    srv = _bmj.Server(idx, n_slots=2)
    monkeypatch.delenv("BMJ_FAULT")
    tickets = [srv.submit(tok[off[x]:off[x + 1]], 1, 2) for x in range(5)]
    for t in tickets:
        with pytest.raises(_bmj.BmjError) as e:
            srv.poll(t, wait_ms=20_000)
        assert e.value.status == _bmj.BMJ_ERR_CUDA
    with pytest.raises(_bmj.BmjError) as e:
        srv.submit(tok[off[0]:off[1]], 1, 2)
    assert e.value.status == _bmj.BMJ_ERR_CUDA
    with pytest.raises(_bmj.BmjError) as e:
        srv.close()
    assert e.value.status == _bmj.BMJ_ERR_CUDA
    assert idx.status() == _bmj.BMJ_ERR_CUDA
    idx.close()
    fresh = _bmj.Index(off, tok, b=64)
    srv = _bmj.Server(fresh, n_slots=2)
    ids, _ = srv.poll(srv.submit(tok[off[3]:off[4]], 1, 2), wait_ms=20_000)
    assert np.array_equal(ids, O.search(tok[off[3]:off[4]], off, tok, 1, 2))
    srv.close()
    fresh.close()
