"""C ABI checks that need no GPU: the library loads, exports every entry point
declared in include/bmj.h, and rejects bad arguments before touching CUDA."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1711_07295_b300 import _bmj

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bmj.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][\w\s\*]*?\b(bmj_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bmj_build_bitmaps", "bmj_self_join", "bmj_pairs_free", "bmj_strerror",
                     "bmj_default_options"):
        assert required in names


def test_library_exports_every_declared_symbol():
    L = _bmj.lib()
    for name in declared_functions():
        assert hasattr(L, name), f"libbmj.so does not export {name}"
        assert name in _bmj.SIGNATURES, f"binding lacks {name}"


def test_host_pool_trim_on_an_empty_pool():
    # nothing has been returned to the pool in this process on the CPU: no CUDA call is made
    assert _bmj.bmj_host_pool_trim() == 0


def test_strerror_and_defaults():
    assert _bmj.bmj_strerror(0) == "ok"
    for code in range(-9, 0):
        assert _bmj.bmj_strerror(code) != "unknown status"
    o = _bmj.bmj_default_options()
    assert (o.b, o.method, o.validate, o.output_on_device, o.queue_cap) == (64, 0, 1, 0, 0)


def _join_status(off, tok, p, q, **kw):
    coll, keep = _bmj.make_collection(off, tok)
    o = _bmj.bmj_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    pairs = _bmj.bmj_pairs()
    return _bmj.lib().bmj_self_join(C.byref(coll), 0, p, q, C.byref(o), C.byref(pairs), None)


@pytest.mark.parametrize("p,q,kw", [
    (0, 5, {}), (3, 0, {}), (6, 5, {}), (1, 2, {"b": 100}), (1, 2, {"b": 0}),
    (1, 2, {"b": 4160}), (1, 2, {"method": 7}), (1, 2, {"queue_cap": -1}),
])
def test_invalid_arguments_rejected_on_host(p, q, kw):
    off = np.array([0, 2, 4], np.int64)
    tok = np.array([1, 2, 1, 3], np.int32)
    assert _join_status(off, tok, p, q, **kw) == _bmj.BMJ_ERR_INVALID_ARG


@pytest.mark.parametrize("sim,p,q,ok", [
    (_bmj.BMJ_COSINE, 3, 4, True), (_bmj.BMJ_COSINE, 1, 70000, False), (_bmj.BMJ_COSINE, 5, 4, False),
    (_bmj.BMJ_DICE, 9, 10, True), (_bmj.BMJ_DICE, 11, 10, False), (_bmj.BMJ_OVERLAP, 7, 2, True),
    (_bmj.BMJ_OVERLAP, 0, 1, False), (4, 1, 2, False), (-1, 1, 2, False),
])
def test_similarity_function_thresholds_checked_on_host(sim, p, q, ok):
    off = np.array([0, 2, 4], np.int64)
    tok = np.array([1, 3, 1, 3], np.int32)
    coll, keep = _bmj.make_collection(off, tok)
    o = _bmj.bmj_default_options()
    o.validate = 0
    st = _bmj.lib().bmj_self_join(C.byref(coll), sim, p, q, C.byref(o), C.byref(_bmj.bmj_pairs()),
                                  None)
    if ok:
        assert st != _bmj.BMJ_ERR_INVALID_ARG   # without a GPU the call fails later, not here
    else:
        assert st == _bmj.BMJ_ERR_INVALID_ARG


def test_null_pointers_rejected():
    L = _bmj.lib()
    assert L.bmj_index_status(None) == _bmj.BMJ_ERR_INVALID_ARG
    pairs = _bmj.bmj_pairs()
    assert L.bmj_self_join(None, 0, 1, 2, None, C.byref(pairs), None) == _bmj.BMJ_ERR_INVALID_ARG
    coll = _bmj.bmj_collection(-1, None, None, 0, 0)
    assert L.bmj_self_join(C.byref(coll), 0, 1, 2, None, C.byref(pairs), None) == _bmj.BMJ_ERR_INVALID_ARG
    coll = _bmj.bmj_collection(1 << 31, None, None, 0, 0)
    assert L.bmj_self_join(C.byref(coll), 0, 1, 2, None, C.byref(pairs), None) == _bmj.BMJ_ERR_TOO_LARGE
    assert L.bmj_build_bitmaps(None, 64, 0, None, None) == _bmj.BMJ_ERR_INVALID_ARG
    off = np.array([0, 1], np.int64)
    tok = np.array([1], np.int32)
    coll, keep = _bmj.make_collection(off, tok)
    assert L.bmj_build_bitmaps(C.byref(coll), 64, _bmj.BMJ_COMBINED, None, None) == _bmj.BMJ_ERR_INVALID_ARG
    assert L.bmj_build_bitmaps(C.byref(coll), 96, 0, None, None) == _bmj.BMJ_ERR_INVALID_ARG
    # freeing an empty list is a no-op
    L.bmj_pairs_free(C.byref(pairs))
    L.bmj_pairs_free(None)


def test_batch_arguments_rejected_on_host():
    L = _bmj.lib()
    off = np.array([0, 2, 4, 6], np.int64)
    tok = np.array([1, 2, 1, 3, 2, 3], np.int32)
    coll, keep = _bmj.make_collection(off, tok)
    outs = (_bmj.bmj_pairs * 4)()
    p = np.array([1, 1, 1, 1], np.uint32)
    q = np.array([2, 2, 2, 2], np.uint32)

    def call(js, pp=p, qq=q, n_jobs=2, **kw):
        o = _bmj.bmj_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        js = np.array(js, np.int64)
        return L.bmj_self_join_batch(C.byref(coll), n_jobs, js.ctypes.data_as(C.c_void_p), 0,
                                     pp.ctypes.data_as(C.c_void_p), qq.ctypes.data_as(C.c_void_p),
                                     C.byref(o), outs, None, None)
    assert call([0, 1, 2]) == _bmj.BMJ_ERR_INVALID_ARG          # does not end at n_sets
    assert call([1, 2, 3]) == _bmj.BMJ_ERR_INVALID_ARG          # does not start at 0
    assert call([0, 2, 1, 3], n_jobs=3) == _bmj.BMJ_ERR_INVALID_ARG  # decreasing
    assert call([0, 1, 3], pp=np.array([1, 3, 1, 1], np.uint32)) == _bmj.BMJ_ERR_INVALID_ARG  # p > q
    assert call([0, 1, 3], b=100) == _bmj.BMJ_ERR_INVALID_ARG
    assert call([0, 1, 3], n_jobs=0) == _bmj.BMJ_ERR_INVALID_ARG
    for kw in ({"cutoff": 5}, {"candidates": _bmj.BMJ_CAND_PREFIX}, {"row_end": 2}):
        assert call([0, 1, 3], **kw) == _bmj.BMJ_ERR_INVALID_ARG   # single-join options


def test_rs_join_arguments_rejected_on_host():
    L = _bmj.lib()
    off = np.array([0, 2, 4], np.int64)
    tok = np.array([1, 2, 1, 3], np.int32)
    r, keep_r = _bmj.make_collection(off, tok)
    s, keep_s = _bmj.make_collection(off, tok)
    pairs = _bmj.bmj_pairs()

    def call(p=1, q=2, sim=0, rr=r, ss=s, **kw):
        o = _bmj.bmj_default_options()
        for k, v in kw.items():
            setattr(o, k, v)
        return L.bmj_rs_join(C.byref(rr) if rr is not None else None,
                             C.byref(ss) if ss is not None else None, sim, p, q, C.byref(o),
                             C.byref(pairs), None)
    assert call(rr=None) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(ss=None) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(p=3, q=2) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(b=100) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(candidates=_bmj.BMJ_CAND_PREFIX, cutoff=4) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(candidates=7) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(row_begin=0, row_end=1) == _bmj.BMJ_ERR_INVALID_ARG
    assert call(cutoff=-2) == _bmj.BMJ_ERR_INVALID_ARG
    big = _bmj.bmj_collection(1 << 30, off.ctypes.data_as(C.c_void_p), tok.ctypes.data_as(C.c_void_p), 0, 0)
    assert call(rr=big, ss=big) == _bmj.BMJ_ERR_TOO_LARGE       # |R| + |S| >= 2^31
    assert _join_status(off, tok, 1, 2, cutoff=-2) == _bmj.BMJ_ERR_INVALID_ARG
    assert _join_status(off, tok, 1, 2, cutoff=3, candidates=_bmj.BMJ_CAND_PREFIX) == \
        _bmj.BMJ_ERR_INVALID_ARG


STRUCTS = ("bmj_collection", "bmj_pairs", "bmj_options", "bmj_stats", "bmj_batch_stats",
           "bmj_id_lists", "bmj_serve_options", "bmj_serve_stats")


def test_binding_structs_match_the_header_layout(tmp_path):
    # Every struct the binding marshals has the size and field offsets that a C compiler
    # gives the header's declaration (gcc, the host ABI the library is built for).
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bmj.h"', 'int main(void) {']
    for name in STRUCTS:
        cls = getattr(_bmj, name)
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name in STRUCTS:
        cls = getattr(_bmj, name)
        assert int(got[name]) == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
