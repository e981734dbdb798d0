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
