"""ctypes binding of the C ABI in include/dd.h (argument marshalling only).

Every computation happens in the CUDA library ``_build/libdd.so``.  If the
library has not been built, importing the binding raises: there is no
Python or CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdd.so")

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double
_F = ctypes.c_float
_PI = ctypes.POINTER(ctypes.c_int)
_PF = ctypes.POINTER(ctypes.c_float)

# name -> (restype, argtypes); mirrors include/*.h
SIGNATURES = {
    "dd_status_string": (ctypes.c_char_p, [_I]),
    "dd_last_error": (ctypes.c_char_p, []),
    "dd_version": (_I, []),
    "dd_compute_delays": (_I, [_I, _P, _D, _I, _P, _P]),
    "dd_plan_create": (_I, [ctypes.POINTER(_P), _I, _P, _D, _I, _P, _P]),
    "dd_plan_info": (_I, [_P, _PI, _PI, _PI]),
    "dd_plan_delay_table": (_I, [_P, _P]),
    "dd_plan_kernel_shape": (_I, [_P, _PI, _PI, _PI, _PI]),
    "dd_plan_autotune": (_I, [_P, _SZ, _P, _PF]),
    "dd_execute": (_I, [_P, _P, _SZ, _SZ, _P, _SZ, _P]),
    "dd_execute_host": (_I, [_P, _P, _SZ, _SZ, _P, _SZ, _P]),
    "dd_destroy": (None, [_P]),
    "dd_dedisp_status": (_I, [_P]),
    "dd_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, _I]),
    "dd_batch_set": (_I, [_P, _I, _P, _P]),
    "dd_batch_launch": (_I, [_P, _P]),
    "dd_batch_info": (_I, [_P, _PI, ctypes.POINTER(ctypes.c_longlong), _PI, _PI, _PI]),
    "dd_batch_destroy": (None, [_P]),
    "dd_execute_batch": (_I, [_I, _P, _P]),
    "dd_search_create": (_I, [ctypes.POINTER(_P), _P]),
    "dd_search_run": (_I, [_P, _P, _SZ, _I, _SZ, _I, _P]),
    "dd_search_result": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), _PI, ctypes.POINTER(ctypes.c_uint), _P]),
    "dd_search_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), _P]),
    "dd_search_candidates": (_I, [_P, _P, _I, _PI, _P]),
    "dd_search_device_candidates": (_I, [_P, ctypes.POINTER(_P)]),
    "dd_search_buffers": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "dd_snippets": (_I, [_P, _SZ, _I, _SZ, _P, _I, _P, _P, _P]),
    "dd_search_snippets": (_I, [_P, _I, _P, _P]),
    "dd_search_destroy": (None, [_P]),
    "dd_nn_create": (_I, [ctypes.POINTER(_P), _I]),
    "dd_nn_set_params": (_I, [_P, _P]),
    "dd_nn_get_params": (_I, [_P, _P]),
    "dd_nn_forward": (_I, [_P, _P, _I, _P, _P]),
    "dd_nn_forward_tc": (_I, [_P, _P, _I, _P, _P]),
    "dd_nn_status": (_I, [_P, _P]),
    "dd_nn_backward": (_I, [_P, _P, _P, _I, _P]),
    "dd_nn_get_grads": (_I, [_P, _P, _P]),
    "dd_nn_set_grads": (_I, [_P, _P]),
    "dd_nn_get_loss": (_I, [_P, _PF, _P]),
    "dd_nn_adamw": (_I, [_P, _F, _F, _F, _F, _F, _P]),
    "dd_nn_get_state": (_I, [_P, _P, _P, _P, _PI]),
    "dd_nn_save": (_I, [_P, ctypes.c_char_p]),
    "dd_nn_load": (_I, [_P, ctypes.c_char_p]),
    "dd_nn_destroy": (None, [_P]),
    "dd_server_create": (_I, [ctypes.POINTER(_P), _P, _P]),
    "dd_server_submit": (_I, [_P, _I, _P, _SZ, ctypes.POINTER(ctypes.c_longlong)]),
    "dd_server_poll": (_I, [_P, _P, _I, _PI, _P, _I, _PI, _D]),
    "dd_server_drain": (_I, [_P, _D]),
    "dd_server_info": (_I, [_P, _PI, _PI, ctypes.POINTER(_SZ)]),
    "dd_server_set_tap": (_I, [_P, _I, _P, _SZ, _SZ]),
    "dd_server_destroy": (None, [_P]),
    "dd_corner_turn": (_I, [_P, _SZ, _I, _SZ, _P, _SZ, _P]),
    "dd_rfi_create": (_I, [_P, _I, _I, _SZ]),
    "dd_rfi_run": (_I, [_P, _P, _I, _SZ, _SZ, _I, _I, _I, _P]),
    "dd_rfi_result": (_I, [_P, _P, _P]),
    "dd_rfi_buffers": (_I, [_P, _P, _P, _P]),
    "dd_rfi_destroy": (None, [_P]),
    "dd_execute_noalloc": (_I, [_I, _P, _D, _I, _P, _P, _SZ, _SZ, _P, _SZ, _P]),
}

_lock = threading.Lock()
_lib = None


class DDError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {status_name(status)}: {message}")
        self.status = status


def load() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"native library {LIB_PATH} is missing; build it with "
                    "`python -m paper_1112_0065_gb300._build` (there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


STATUS = {0: "DD_OK", -1: "DD_ERR_INVALID_ARG", -2: "DD_ERR_NOMEM", -3: "DD_ERR_CUDA",
          -4: "DD_ERR_TOO_SHORT", -5: "DD_ERR_TIMEOUT", -6: "DD_ERR_INTERNAL", -7: "DD_ERR_BUSY"}
DD_OK, DD_ERR_INVALID_ARG, DD_ERR_NOMEM, DD_ERR_CUDA, DD_ERR_TOO_SHORT, DD_ERR_TIMEOUT, DD_ERR_INTERNAL, \
    DD_ERR_BUSY = 0, -1, -2, -3, -4, -5, -6, -7


def status_name(s: int) -> str:
    return STATUS.get(int(s), f"status {s}")


def check(status: int, where: str):
    if status != 0:
        msg = load().dd_last_error()
        raise DDError(status, where, msg.decode() if msg else "")
    return status


class Beam(ctypes.Structure):
    _fields_ = [("plan", _P), ("d_in", _P), ("ld_in_bytes", _SZ), ("nsamp_in", _SZ), ("d_out", _P),
                ("ld_out", _SZ)]


class Candidate(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int32), ("d", ctypes.c_int32), ("t", ctypes.c_int32), ("w", ctypes.c_int32),
                ("snr", ctypes.c_float), ("score", ctypes.c_float), ("ncells", ctypes.c_int64)]


SEARCH_MAX_WIDTHS = 16
SEARCH_MAX_CANDS = 1 << 20


class SearchConfig(ctypes.Structure):
    _fields_ = [("ndm_max", _I), ("n_max", _SZ), ("nchan", _I), ("half_window", _I), ("nwidths", _I),
                ("widths", _I * SEARCH_MAX_WIDTHS), ("thresh", _F), ("max_cands", _I),
                ("full_map", _I), ("baseline", _I)]


class Trigger(ctypes.Structure):
    _fields_ = [("beam", _I), ("nchan", _I), ("seq", ctypes.c_longlong), ("cand", Candidate),
                ("t0", ctypes.c_longlong), ("nsamp", ctypes.c_longlong), ("ld", _SZ)]


TRIGGER_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.POINTER(Trigger), ctypes.POINTER(ctypes.c_uint8))


class ServerConfig(ctypes.Structure):
    _fields_ = [("nbeams", _I), ("gulp_nsamp", _SZ), ("max_slots", _I), ("hbm_reserve_bytes", _SZ),
                ("half_window", _I), ("nwidths", _I), ("widths", _I * SEARCH_MAX_WIDTHS), ("thresh", _F),
                ("max_cands", _I), ("classifier_path", ctypes.c_char_p), ("nn_batch", _I),
                ("trigger_snr", _F), ("trigger_max", _I), ("trigger_fn", TRIGGER_FN), ("trigger_user", _P)]


class GulpResult(ctypes.Structure):
    _fields_ = [("beam", _I), ("ncand", _I), ("seq", ctypes.c_longlong), ("t0", ctypes.c_longlong),
                ("nout", ctypes.c_longlong), ("t_submit", _D), ("t_done", _D), ("ngroups", _I),
                ("flags", ctypes.c_uint), ("cand_offset", _I), ("reserved", _I)]


class Options(ctypes.Structure):
    _fields_ = [("kernel", _I), ("dms_per_block", _I), ("words_per_thread", _I), ("chan_chunk", _I),
                ("reserved", _I), ("tune_cache_path", ctypes.c_char_p)]
