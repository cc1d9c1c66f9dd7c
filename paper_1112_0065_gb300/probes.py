"""ctypes binding of the measurement probes (``_build/libddprobe.so``,
declared in ``csrc/probe/dd_probe.h``).

The probes measure the GPU at hand (integer and float issue rates, a
tensor-core self-check); the tests and the benchmark's roofline figures use
them.  They are a library of their own: nothing in the product library or in
the rest of this package calls them.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from ._lib import DDError

HERE = os.path.dirname(os.path.abspath(__file__))
PROBE_LIB_PATH = os.path.join(HERE, "_build", "libddprobe.so")

_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "dd_probe_int_rates": (_I, [_P]),
    "dd_probe_fp_rates": (_I, [_P, _P]),
    "dd_probe_tc_gemm": (_I, [_P, _P, _P, _I, _I]),
    "dd_probe_wait_giveup": (_I, [ctypes.c_uint, ctypes.POINTER(ctypes.c_uint)]),
    "dd_probe_tile_giveup": (_I, [ctypes.c_uint, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(ctypes.c_longlong)]),
    "dd_probe_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(PROBE_LIB_PATH):
                raise ImportError(f"probe library {PROBE_LIB_PATH} is missing; build with "
                                  "`python -m paper_1112_0065_gb300._build`")
            L = ctypes.CDLL(PROBE_LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(status: int, where: str):
    if status != 0:
        msg = load().dd_probe_last_error()
        raise DDError(status, where, msg.decode() if msg else "")


def int_rates():
    """Measured integer issue rates (Tops/s): lop3, add, mad, lop3+mad mix."""
    out = (ctypes.c_double * 4)()
    _check(load().dd_probe_int_rates(out), "dd_probe_int_rates")
    return {"lop3": out[0], "iadd": out[1], "imad": out[2], "lop3_imad_mix": out[3]}


def fp_rates():
    """Measured float FMA rates (T FMA/s): scalar and packed-pair forms, and
    the number of packed results that differ from fmaf's (expected 0)."""
    out = (ctypes.c_double * 2)()
    mm = ctypes.c_ulonglong()
    _check(load().dd_probe_fp_rates(out, ctypes.byref(mm)), "dd_probe_fp_rates")
    return {"ffma": out[0], "ffma2": out[1], "ffma2_mismatches": mm.value}


def tc_gemm(a, b):
    """Tensor-core self-check: a (128 x k) and b (n x k) bfloat16 bit patterns
    (uint16 arrays) -> float32 a @ b.T (128 x n), computed with tcgen05 MMAs."""
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(b, dtype=np.uint16)
    assert a.ndim == 2 and b.ndim == 2 and a.shape[0] == 128 and a.shape[1] == b.shape[1]
    d = np.empty((128, b.shape[0]), dtype=np.float32)
    _check(load().dd_probe_tc_gemm(a.ctypes.data, b.ctypes.data, d.ctypes.data, b.shape[0], a.shape[1]),
           "dd_probe_tc_gemm")
    return d


def wait_giveup(poll_limit: int = 1000):
    """Run a bounded tensor-core wait that cannot complete: -> (status code,
    per-warp give-up bits, message)."""
    flags = ctypes.c_uint()
    L = load()
    st = L.dd_probe_wait_giveup(int(poll_limit), ctypes.byref(flags))
    msg = L.dd_probe_last_error()
    return st, flags.value, msg.decode() if msg else ""


def tile_giveup(poll_limit: int = 1000):
    """Run the dedispersion tile with stage waits that cannot complete: ->
    (status code, the tile's error word, output words it wrote, message)."""
    err = ctypes.c_uint()
    written = ctypes.c_longlong()
    L = load()
    st = L.dd_probe_tile_giveup(int(poll_limit), ctypes.byref(err), ctypes.byref(written))
    msg = L.dd_probe_last_error()
    return st, err.value, written.value, msg.decode() if msg else ""
