"""Multi-beam batches (C ABI: dd_batch_create / dd_batch_set /
dd_batch_launch): every beam's gulp dedispersed by one persistent launch,
optionally replayed from a CUDA graph."""
from __future__ import annotations

import ctypes

from . import _lib
from .dedisp import _stream_handle


def _beams(items):
    """items: iterable of (plan, d_in tensor, nsamp_in, d_out tensor)."""
    items = list(items)
    arr = (_lib.Beam * len(items))()
    for k, (plan, d_in, nsamp, out) in enumerate(items):
        assert d_in.is_cuda and out.is_cuda and d_in.stride(1) == 1 and out.stride(1) == 1
        arr[k] = _lib.Beam(plan.handle, d_in.data_ptr(), d_in.stride(0), nsamp, out.data_ptr(), out.stride(0))
    return arr, len(items)


class Batch:
    def __init__(self, items, use_graph: bool = True):
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        arr, n = _beams(items)
        _lib.check(self._L.dd_batch_create(ctypes.byref(self._h), n, arr, 1 if use_graph else 0), "dd_batch_create")

    def set(self, items, stream=None):
        arr, n = _beams(items)
        _lib.check(self._L.dd_batch_set(self._h, n, arr, _stream_handle(stream)), "dd_batch_set")

    def launch(self, stream=None):
        _lib.check(self._L.dd_batch_launch(self._h, _stream_handle(stream)), "dd_batch_launch")

    def info(self):
        nb, gr, dpb, wpt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nt = ctypes.c_longlong()
        _lib.check(self._L.dd_batch_info(self._h, ctypes.byref(nb), ctypes.byref(nt), ctypes.byref(gr),
                                         ctypes.byref(dpb), ctypes.byref(wpt)), "dd_batch_info")
        return {"nbeams": nb.value, "ntiles": nt.value, "grid": gr.value, "dms_per_block": dpb.value,
                "words_per_thread": wpt.value}

    def close(self):
        if self._h:
            self._L.dd_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def execute_batch(items, stream=None):
    arr, n = _beams(items)
    L = _lib.load()
    _lib.check(L.dd_execute_batch(n, arr, _stream_handle(stream)), "dd_execute_batch")
