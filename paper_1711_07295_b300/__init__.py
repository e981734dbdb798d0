"""Bitmap Filter exact set-similarity self-joins on B300 (sm_103a).

The join runs in the CUDA library ``libbmj.so`` behind the C ABI of
``include/bmj.h``; ``_bmj`` is its ctypes binding (same function names).
``inputs`` draws seeded synthetic collections.  Importing this package does
not load the library; the first call of a binding function does, and fails
loudly when it is missing.
"""
from importlib import import_module

_BINDING = {
    "bmj_build_bitmaps", "bmj_self_join", "bmj_rs_join", "bmj_default_options", "bmj_strerror",
    "bmj_kernel_launches", "BmjError", "DevicePairs", "BMJ_XOR", "BMJ_SET", "BMJ_NEXT",
    "BMJ_COMBINED", "BMJ_JACCARD", "METHODS", "lib",
}


def __getattr__(name):
    if name in _BINDING:
        return getattr(import_module("._bmj", __name__), name)
    raise AttributeError(name)
