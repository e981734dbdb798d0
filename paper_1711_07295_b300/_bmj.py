"""ctypes binding of ``libbmj.so`` (the C ABI declared in include/bmj.h).

Argument marshalling only: every step of the join runs in the library's CUDA
kernels.  Functions keep the C names.  Arrays may be torch tensors (CUDA or
CPU) or numpy arrays; CUDA tensors are passed as device pointers on the
current torch stream, everything else as host pointers.  There is no CPU
fallback: if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbmj.so")

BMJ_OK = 0
BMJ_ERR_INVALID_ARG = -1
BMJ_ERR_UNSORTED = -2
BMJ_ERR_EMPTY_SET = -3
BMJ_ERR_NEG_TOKEN = -4
BMJ_ERR_OOM = -5
BMJ_ERR_OUTPUT_OVERFLOW = -6
BMJ_ERR_TIMEOUT = -7
BMJ_ERR_CUDA = -8
BMJ_ERR_TOO_LARGE = -9
BMJ_PENDING = 1   # bmj_serve_poll: the query has not completed yet (not an error)

BMJ_XOR, BMJ_SET, BMJ_NEXT, BMJ_COMBINED = 0, 1, 2, 3
BMJ_JACCARD, BMJ_COSINE, BMJ_DICE, BMJ_OVERLAP = 0, 1, 2, 3   # similarity functions (Table 1)
BMJ_CAND_WINDOW, BMJ_CAND_PREFIX = 0, 1   # candidate pairs: the whole window, or the prefix filter
BMJ_CAND_AUTO = 2   # the prefix filter or the window, whichever the slot count says is faster
BMJ_CUTOFF_AUTO = -1   # bmj_options.cutoff: the cutoff point from Eq. 4-6 (Section 3.5)
METHODS = {"xor": BMJ_XOR, "set": BMJ_SET, "next": BMJ_NEXT, "combined": BMJ_COMBINED}


class bmj_collection(C.Structure):
    _fields_ = [("n_sets", C.c_int64), ("offsets", C.c_void_p), ("tokens", C.c_void_p),
                ("on_device", C.c_int32), ("reserved", C.c_int32)]


class bmj_pairs(C.Structure):
    _fields_ = [("n", C.c_int64), ("a", C.c_void_p), ("b", C.c_void_p),
                ("on_device", C.c_int32), ("host_pinned", C.c_int32)]


class _HostPairsOwner:
    """Keeps a library-owned host pair list alive while numpy views of it exist."""

    def __init__(self, pairs):
        self.pairs = pairs

    def __del__(self):
        try:
            lib().bmj_pairs_free(C.byref(self.pairs))
        except Exception:
            pass


def _host_views(pairs):
    """numpy views (no copy) of a host pair list; freed with the last view."""
    n = int(pairs.n)
    owner = _HostPairsOwner(pairs)
    views = []
    for ptr in (pairs.a, pairs.b):
        buf = (C.c_uint32 * n).from_address(ptr)
        buf._owner = owner
        views.append(np.frombuffer(buf, dtype=np.uint32))
    return views[0], views[1]


class bmj_options(C.Structure):
    _fields_ = [("b", C.c_int32), ("method", C.c_int32), ("output_on_device", C.c_int32),
                ("validate", C.c_int32), ("queue_cap", C.c_int64), ("stream", C.c_void_p),
                ("rows_per_thread", C.c_int32), ("use_graph", C.c_int32),
                ("cascade_b", C.c_int32), ("sim", C.c_int32), ("row_begin", C.c_int64),
                ("row_end", C.c_int64), ("candidates", C.c_int32),
                ("cutoff", C.c_int32)]


class bmj_stats(C.Structure):
    _fields_ = [("window_pairs", C.c_int64), ("survivors", C.c_int64), ("results", C.c_int64),
                ("filter_passes", C.c_int64), ("verified", C.c_int64), ("n_launches", C.c_int32),
                ("b", C.c_int32), ("method", C.c_int32), ("max_set_size", C.c_int32),
                ("cascade_b", C.c_int32), ("cutoff", C.c_int32), ("ms_prepare", C.c_float),
                ("ms_filter", C.c_float), ("ms_verify", C.c_float), ("ms_output", C.c_float),
                ("ms_total", C.c_float), ("reserved_f", C.c_float), ("candidates", C.c_int64),
                ("candidate_slots", C.c_int64), ("tile_rows", C.c_int32), ("chunk_cols", C.c_int32),
                ("fold_steps", C.c_int64), ("fold_full_steps", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class bmj_batch_stats(C.Structure):
    _fields_ = [("n_jobs", C.c_int64), ("window_pairs", C.c_int64), ("survivors", C.c_int64),
                ("results", C.c_int64), ("n_launches", C.c_int32), ("filter_passes", C.c_int32),
                ("graph", C.c_int32), ("tuned", C.c_int32), ("ms_prepare", C.c_float),
                ("ms_tune", C.c_float), ("ms_execute", C.c_float), ("ms_output", C.c_float),
                ("ms_total", C.c_float), ("reserved_f", C.c_float * 3)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class bmj_id_lists(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("offsets", C.c_void_p), ("ids", C.c_void_p)]


class bmj_serve_options(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("reserved0", C.c_int32),
                ("max_batch_queries", C.c_int64), ("max_batch_window_pairs", C.c_int64),
                ("max_probe_tokens", C.c_int64), ("reserved", C.c_int64 * 3)]


class bmj_serve_stats(C.Structure):
    _fields_ = [("n_queries", C.c_int64), ("batches", C.c_int64), ("window_pairs", C.c_int64),
                ("survivors", C.c_int64), ("results", C.c_int64), ("wall_s", C.c_double),
                ("qps", C.c_double), ("p50_ms", C.c_double), ("p99_ms", C.c_double),
                ("max_ms", C.c_double), ("reserved", C.c_double * 4)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class BmjError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {bmj_strerror(status)} (status {status})")


_lib = None

# Every exported entry point of include/bmj.h with its ctypes signature.
SIGNATURES = {
    "bmj_default_options": (None, [C.POINTER(bmj_options)]),
    "bmj_strerror": (C.c_char_p, [C.c_int]),
    "bmj_build_bitmaps": (C.c_int, [C.POINTER(bmj_collection), C.c_int, C.c_int, C.c_void_p,
                                    C.c_void_p]),
    "bmj_self_join": (C.c_int, [C.POINTER(bmj_collection), C.c_int, C.c_uint32, C.c_uint32,
                                C.POINTER(bmj_options), C.POINTER(bmj_pairs),
                                C.POINTER(bmj_stats)]),
    "bmj_rs_join": (C.c_int, [C.POINTER(bmj_collection), C.POINTER(bmj_collection), C.c_int,
                              C.c_uint32, C.c_uint32, C.POINTER(bmj_options), C.POINTER(bmj_pairs),
                              C.POINTER(bmj_stats)]),
    "bmj_self_join_batch": (C.c_int, [C.POINTER(bmj_collection), C.c_int64, C.c_void_p, C.c_int,
                                      C.c_void_p, C.c_void_p, C.POINTER(bmj_options),
                                      C.POINTER(bmj_pairs), C.POINTER(bmj_stats),
                                      C.POINTER(bmj_batch_stats)]),
    "bmj_pairs_free": (None, [C.POINTER(bmj_pairs)]),
    "bmj_index_create": (C.c_int, [C.POINTER(bmj_collection), C.POINTER(bmj_options),
                                   C.POINTER(C.c_void_p)]),
    "bmj_index_destroy": (None, [C.c_void_p]),
    "bmj_index_size": (C.c_int64, [C.c_void_p]),
    "bmj_index_status": (C.c_int, [C.c_void_p]),
    "bmj_default_serve_options": (None, [C.POINTER(bmj_serve_options)]),
    "bmj_index_query": (C.c_int, [C.c_void_p, C.POINTER(bmj_collection), C.c_void_p, C.c_void_p,
                                  C.POINTER(bmj_id_lists), C.POINTER(bmj_serve_stats)]),
    "bmj_serve": (C.c_int, [C.c_void_p, C.POINTER(bmj_collection), C.c_void_p, C.c_void_p,
                            C.c_void_p, C.POINTER(bmj_serve_options), C.POINTER(bmj_id_lists),
                            C.c_void_p, C.POINTER(bmj_serve_stats)]),
    "bmj_id_lists_free": (None, [C.POINTER(bmj_id_lists)]),
    "bmj_serve_open": (C.c_int, [C.c_void_p, C.POINTER(bmj_serve_options), C.POINTER(C.c_void_p)]),
    "bmj_serve_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_uint32, C.c_uint32,
                                   C.POINTER(C.c_int64)]),
    "bmj_serve_poll": (C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(bmj_id_lists),
                                 C.POINTER(C.c_double)]),
    "bmj_serve_close": (C.c_int, [C.c_void_p, C.POINTER(bmj_serve_stats)]),
    "bmj_kernel_launches": (C.c_int64, []),
    "bmj_host_pool_trim": (C.c_int64, []),
    "bmj_measure_popc_rate": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "bmj_bitmap_filter_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_uint32,
                                            C.c_uint32, C.c_void_p, C.c_int64,
                                            C.POINTER(C.c_int64), C.c_void_p]),
}


def lib():
    """Load ``libbmj.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ----------------------------------------------------------------------------
def _is_cuda_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


def _host_array(x, dtype):
    if hasattr(x, "numpy"):
        x = x.numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _stream_of(stream, on_device):
    if stream is not None:
        return C.c_void_p(int(stream))
    if on_device:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def make_collection(offsets, tokens):
    """Marshal (offsets, tokens) into a bmj_collection; returns (struct, keepalive)."""
    if _is_cuda_tensor(offsets) != _is_cuda_tensor(tokens):
        raise ValueError("offsets and tokens must both be CUDA tensors or both host arrays")
    on_dev = _is_cuda_tensor(offsets)
    if on_dev:
        import torch
        if offsets.dtype != torch.int64 or tokens.dtype != torch.int32:
            raise TypeError("offsets must be int64 and tokens int32")
        offsets, tokens = offsets.contiguous(), tokens.contiguous()
    else:
        offsets, tokens = _host_array(offsets, np.int64), _host_array(tokens, np.int32)
    coll = bmj_collection(len(offsets) - 1, _ptr(offsets), _ptr(tokens), 1 if on_dev else 0, 0)
    return coll, (offsets, tokens)


def bmj_default_options() -> bmj_options:
    o = bmj_options()
    lib().bmj_default_options(C.byref(o))
    return o


def bmj_strerror(status: int) -> str:
    return lib().bmj_strerror(int(status)).decode()


def bmj_kernel_launches() -> int:
    return int(lib().bmj_kernel_launches())


def bmj_measure_popc_rate(stream=None) -> float:
    """32-bit popcounts per second of the device (the Bitmap Filter's roofline peak)."""
    out = C.c_double(0.0)
    st = lib().bmj_measure_popc_rate(_stream_of(stream, True), C.byref(out))
    if st != BMJ_OK:
        raise BmjError(st, "bmj_measure_popc_rate")
    return float(out.value)


def bmj_host_pool_trim() -> int:
    """Releases the idle page-locked blocks the library keeps for host pair lists (bytes freed)."""
    return int(lib().bmj_host_pool_trim())


def bmj_build_bitmaps(offsets, tokens, b: int = 64, method: int = BMJ_XOR, out=None,
                      stream=None):
    """Bitmaps uint64[N, b/64] of a collection in original set order.

    Device tensors in -> device tensor out (torch.int64 viewed as uint64 words);
    host arrays in -> numpy uint64 out.
    """
    coll, keep = make_collection(offsets, tokens)
    n = coll.n_sets
    W = b // 64 if b > 0 else 0
    if out is None:
        if coll.on_device:
            import torch
            out = torch.empty((max(n, 0), max(W, 1)), dtype=torch.int64, device=offsets.device)
        else:
            out = np.zeros((max(n, 0), max(W, 1)), np.uint64)
    st = lib().bmj_build_bitmaps(C.byref(coll), int(b), int(method), _ptr(out),
                                 _stream_of(stream, coll.on_device))
    del keep
    if st != BMJ_OK:
        raise BmjError(st, "bmj_build_bitmaps")
    return out


class DevicePairs:
    """Library-owned device pair list; freed with bmj_pairs_free on release()."""

    def __init__(self, pairs: bmj_pairs, device):
        self._p = pairs
        self.n = int(pairs.n)
        self.device = device

    def _view(self, ptr):
        import torch
        if self.n == 0:
            return torch.zeros(0, dtype=torch.int32, device=self.device)

        class _CAI:
            __cuda_array_interface__ = {"shape": (self.n,), "typestr": "<u4",
                                        "data": (int(ptr), False), "version": 3}
        return torch.as_tensor(_CAI(), device=self.device).view(torch.int32)

    @property
    def a(self):
        return self._view(self._p.a)

    @property
    def b(self):
        return self._view(self._p.b)

    def release(self):
        if self._p is not None:
            lib().bmj_pairs_free(C.byref(self._p))
            self._p = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def bmj_self_join(offsets, tokens, p: int, q: int, b: int = 64, method: int = BMJ_XOR,
                  output_on_device: bool = False, queue_cap: int = 0, validate: bool = True,
                  stream=None, sim: int = BMJ_JACCARD, cascade_b: int = 0,
                  row_begin: int = 0, row_end: int = 0, candidates: int = 0, cutoff: int = 0):
    """Exact Jaccard self-join at threshold p/q.

    Returns ``(a, b, stats)``: original ids with a < b sorted by (a, b), as
    numpy uint32 arrays (host output) or a :class:`DevicePairs` as ``a`` with
    ``b`` None (device output); ``stats`` is a dict of the bmj_stats fields.
    """
    coll, keep = make_collection(offsets, tokens)
    o = bmj_default_options()
    o.b = int(b)
    o.method = int(method)
    o.output_on_device = 1 if output_on_device else 0
    o.validate = 1 if validate else 0
    o.queue_cap = int(queue_cap)
    o.cascade_b = int(cascade_b)
    o.row_begin = int(row_begin)
    o.row_end = int(row_end)
    o.candidates = int(candidates)
    o.cutoff = int(cutoff)
    o.stream = _stream_of(stream, coll.on_device)
    pairs = bmj_pairs()
    st_ = bmj_stats()
    st = lib().bmj_self_join(C.byref(coll), int(sim), C.c_uint32(int(p)), C.c_uint32(int(q)),
                             C.byref(o), C.byref(pairs), C.byref(st_))
    del keep
    if st != BMJ_OK:
        raise BmjError(st, "bmj_self_join")
    return _pairs_out(pairs, st_.as_dict(), output_on_device, offsets)


def _pairs_out(pairs, stats, output_on_device, like):
    if output_on_device:
        dev = like.device if hasattr(like, "device") else "cuda"
        return DevicePairs(pairs, dev), None, stats
    n = int(pairs.n)
    if n == 0:
        lib().bmj_pairs_free(C.byref(pairs))
        return np.zeros(0, np.uint32), np.zeros(0, np.uint32), stats
    a, bb = _host_views(pairs)
    return a, bb, stats


def bmj_rs_join(r_offsets, r_tokens, s_offsets, s_tokens, p: int, q: int, b: int = 64,
                method: int = BMJ_XOR, output_on_device: bool = False, queue_cap: int = 0,
                validate: bool = True, stream=None, sim: int = BMJ_JACCARD, cascade_b: int = 0,
                candidates: int = 0, cutoff: int = 0):
    """Exact RS-join of R = (r_offsets, r_tokens) and S = (s_offsets, s_tokens) at p/q.

    Returns ``(a, b, stats)`` as :func:`bmj_self_join` does, with ``a`` ids of R
    and ``b`` ids of S, sorted by (a, b).
    """
    rc, keep_r = make_collection(r_offsets, r_tokens)
    sc, keep_s = make_collection(s_offsets, s_tokens)
    o = bmj_default_options()
    o.b = int(b)
    o.method = int(method)
    o.output_on_device = 1 if output_on_device else 0
    o.validate = 1 if validate else 0
    o.queue_cap = int(queue_cap)
    o.cascade_b = int(cascade_b)
    o.candidates = int(candidates)
    o.cutoff = int(cutoff)
    o.stream = _stream_of(stream, rc.on_device or sc.on_device)
    pairs = bmj_pairs()
    st_ = bmj_stats()
    st = lib().bmj_rs_join(C.byref(rc), C.byref(sc), int(sim), C.c_uint32(int(p)),
                           C.c_uint32(int(q)), C.byref(o), C.byref(pairs), C.byref(st_))
    del keep_r, keep_s
    if st != BMJ_OK:
        raise BmjError(st, "bmj_rs_join")
    like = r_offsets if hasattr(r_offsets, "device") else s_offsets
    return _pairs_out(pairs, st_.as_dict(), output_on_device, like)


def bmj_self_join_batch(offsets, tokens, job_sets, p, q, b: int = 0, method: int = BMJ_XOR,
                        output_on_device: bool = False, queue_cap: int = 0,
                        validate: bool = True, use_graph: bool = False, stream=None,
                        sim: int = BMJ_JACCARD, cascade_b: int = 0, rows_per_thread: int = 0):
    """Independent self-joins of the jobs ``job_sets`` of one concatenated collection.

    ``job_sets`` int64[n_jobs+1] set boundaries, ``p``/``q`` per-job thresholds;
    ``b = 0`` autotunes b per job; ``rows_per_thread`` 0 picks each job's row
    tile, a value below a width's default forces the small tile.  Returns
    ``(pairs, job_stats, batch_stats)``
    where ``pairs[k]`` is ``(a, b)`` numpy uint32 arrays in job-local ids.
    """
    coll, keep = make_collection(offsets, tokens)
    js = np.ascontiguousarray(job_sets, dtype=np.int64)
    n_jobs = len(js) - 1
    pp = np.ascontiguousarray(p, dtype=np.uint32)
    qq = np.ascontiguousarray(q, dtype=np.uint32)
    if len(pp) != n_jobs or len(qq) != n_jobs:
        raise ValueError("p and q need one entry per job")
    o = bmj_default_options()
    o.b = int(b)
    o.method = int(method)
    o.output_on_device = 1 if output_on_device else 0
    o.validate = 1 if validate else 0
    o.queue_cap = int(queue_cap)
    o.use_graph = 1 if use_graph else 0
    o.cascade_b = int(cascade_b)
    o.rows_per_thread = int(rows_per_thread)
    o.stream = _stream_of(stream, coll.on_device)
    outs = (bmj_pairs * max(n_jobs, 1))()
    jst = (bmj_stats * max(n_jobs, 1))()
    bst = bmj_batch_stats()
    st = lib().bmj_self_join_batch(C.byref(coll), n_jobs, _ptr(js), int(sim), _ptr(pp), _ptr(qq),
                                   C.byref(o), outs, jst, C.byref(bst))
    del keep
    if st != BMJ_OK:
        raise BmjError(st, "bmj_self_join_batch")
    pairs = []
    for k in range(n_jobs):
        m = int(outs[k].n)
        if m == 0:
            pairs.append((np.zeros(0, np.uint32), np.zeros(0, np.uint32)))
        elif output_on_device:
            pairs.append(DevicePairs(outs[k], offsets.device if hasattr(offsets, "device") else "cuda"))
            continue
        else:
            a = np.ctypeslib.as_array(C.cast(outs[k].a, C.POINTER(C.c_uint32)), shape=(m,)).copy()
            bb = np.ctypeslib.as_array(C.cast(outs[k].b, C.POINTER(C.c_uint32)), shape=(m,)).copy()
            pairs.append((a, bb))
        lib().bmj_pairs_free(C.byref(outs[k]))
    return pairs, [jst[k].as_dict() for k in range(n_jobs)], bst.as_dict()


def _take_id_lists(lists: bmj_id_lists):
    n = int(lists.n_queries)
    if n == 0 or not lists.offsets:
        lib().bmj_id_lists_free(C.byref(lists))
        return []
    off = np.ctypeslib.as_array(C.cast(lists.offsets, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    tot = int(off[-1])
    ids = (np.ctypeslib.as_array(C.cast(lists.ids, C.POINTER(C.c_int64)), shape=(tot,)).copy()
           if tot else np.zeros(0, np.int64))
    lib().bmj_id_lists_free(C.byref(lists))
    return [ids[off[k]:off[k + 1]] for k in range(n)]


class Index:
    """A resident index (bmj_index_create / bmj_index_destroy)."""

    def __init__(self, offsets, tokens, b: int = 64, method: int = BMJ_XOR, validate: bool = True,
                 sim: int = BMJ_JACCARD):
        coll, keep = make_collection(offsets, tokens)
        o = bmj_default_options()
        o.b = int(b)
        o.method = int(method)
        o.sim = int(sim)
        o.validate = 1 if validate else 0
        o.stream = _stream_of(None, coll.on_device)
        h = C.c_void_p()
        st = lib().bmj_index_create(C.byref(coll), C.byref(o), C.byref(h))
        del keep
        if st != BMJ_OK:
            raise BmjError(st, "bmj_index_create")
        self._h = h

    def __len__(self):
        return int(lib().bmj_index_size(self._h))

    def close(self):
        if self._h is not None and self._h.value:
            lib().bmj_index_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self) -> int:
        """bmj_index_status: BMJ_OK, or the device failure that stuck to the index."""
        return int(lib().bmj_index_status(self._h))

    def query(self, offsets, tokens, p, q):
        """bmj_index_query: per-probe arrays of resident ids (ascending) and stats."""
        coll, keep = make_collection(offsets, tokens)
        pp = np.ascontiguousarray(p, dtype=np.uint32)
        qq = np.ascontiguousarray(q, dtype=np.uint32)
        out = bmj_id_lists()
        st_ = bmj_serve_stats()
        st = lib().bmj_index_query(self._h, C.byref(coll), _ptr(pp), _ptr(qq), C.byref(out),
                                   C.byref(st_))
        del keep
        if st != BMJ_OK:
            raise BmjError(st, "bmj_index_query")
        return _take_id_lists(out), st_.as_dict()

    def serve(self, offsets, tokens, arrival_s, p, q, n_slots: int = 4,
              max_batch_queries: int = 4096, max_batch_window_pairs: int = 1 << 25,
              want_results: bool = True):
        """bmj_serve: (per-query ids or None, latency_ms array, stats dict)."""
        coll, keep = make_collection(offsets, tokens)
        arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
        pp = np.ascontiguousarray(p, dtype=np.uint32)
        qq = np.ascontiguousarray(q, dtype=np.uint32)
        so = bmj_serve_options()
        lib().bmj_default_serve_options(C.byref(so))
        so.n_slots = int(n_slots)
        so.max_batch_queries = int(max_batch_queries)
        so.max_batch_window_pairs = int(max_batch_window_pairs)
        lat = np.zeros(len(arr), np.float64)
        out = bmj_id_lists()
        st_ = bmj_serve_stats()
        st = lib().bmj_serve(self._h, C.byref(coll), _ptr(arr), _ptr(pp), _ptr(qq), C.byref(so),
                             C.byref(out) if want_results else None, _ptr(lat), C.byref(st_))
        del keep
        if st != BMJ_OK:
            raise BmjError(st, "bmj_serve")
        return (_take_id_lists(out) if want_results else None), lat, st_.as_dict()


class Server:
    """A live request loop over an index (bmj_serve_open / _submit / _poll /
    _close): queries submitted from any thread while other batches run."""

    def __init__(self, index: Index, n_slots: int = 4, max_batch_queries: int = 4096,
                 max_batch_window_pairs: int = 1 << 25, max_probe_tokens: int = 4096):
        so = bmj_serve_options()
        lib().bmj_default_serve_options(C.byref(so))
        so.n_slots = int(n_slots)
        so.max_batch_queries = int(max_batch_queries)
        so.max_batch_window_pairs = int(max_batch_window_pairs)
        so.max_probe_tokens = int(max_probe_tokens)
        h = C.c_void_p()
        st = lib().bmj_serve_open(index._h, C.byref(so), C.byref(h))
        if st != BMJ_OK:
            raise BmjError(st, "bmj_serve_open")
        self._h = h
        self._index = index   # the index must outlive the server

    def submit(self, tokens, p: int, q: int) -> int:
        """Returns the query's ticket."""
        t = np.ascontiguousarray(tokens, dtype=np.int32)
        ticket = C.c_int64(-1)
        st = lib().bmj_serve_submit(self._h, _ptr(t), len(t), C.c_uint32(int(p)),
                                    C.c_uint32(int(q)), C.byref(ticket))
        if st != BMJ_OK:
            raise BmjError(st, "bmj_serve_submit")
        return int(ticket.value)

    def poll(self, ticket: int, wait_ms: int = 0):
        """(ids ascending, latency_ms) when the query has completed, else None."""
        out = bmj_id_lists()
        lat = C.c_double(0.0)
        st = lib().bmj_serve_poll(self._h, int(ticket), int(wait_ms), C.byref(out), C.byref(lat))
        if st == BMJ_PENDING:
            return None
        if st != BMJ_OK:
            raise BmjError(st, "bmj_serve_poll")
        return _take_id_lists(out)[0], float(lat.value)

    def close(self):
        """Finishes every submitted query; returns the stats dict."""
        if self._h is None:
            return None
        st_ = bmj_serve_stats()
        st = lib().bmj_serve_close(self._h, C.byref(st_))
        self._h = None
        if st != BMJ_OK:
            raise BmjError(st, "bmj_serve_close")
        return st_.as_dict()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
