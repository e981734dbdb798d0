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
