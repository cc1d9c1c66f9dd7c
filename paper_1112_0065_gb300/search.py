"""Python face of the search stage (C ABI dd_search_*): running-median
baseline, boxcar matched filter, sigma cut + grouping, snippets."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .dedisp import _stream_handle

CAND_DTYPE = np.dtype([("beam", np.int32), ("d", np.int32), ("t", np.int32), ("w", np.int32), ("snr", np.float32),
                       ("score", np.float32), ("ncells", np.int64)])
DEFAULT_WIDTHS = tuple(1 << k for k in range(11))  # 1 .. 1024


class _DeviceView:
    """Zero-copy __cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


def _view(ptr, shape, typestr, owner):
    import torch

    return torch.as_tensor(_DeviceView(ptr, shape, typestr, owner), device="cuda")


class Search:
    def __init__(self, ndm_max: int, n_max: int, nchan: int, half_window: int = 4096,
                 widths=DEFAULT_WIDTHS, thresh: float = 6.0, max_cands: int = 4096,
                 full_map: bool = True, baseline: str = "median"):
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        cfg = _lib.SearchConfig()
        cfg.ndm_max, cfg.n_max, cfg.nchan, cfg.half_window = ndm_max, n_max, nchan, half_window
        cfg.nwidths = len(widths)
        for k, w in enumerate(widths):
            cfg.widths[k] = int(w)
        cfg.thresh, cfg.max_cands = float(thresh), max_cands
        cfg.full_map = 1 if full_map else 0
        cfg.baseline = {"median": 0, "mean": 1}[baseline]
        _lib.check(self._L.dd_search_create(ctypes.byref(self._h), ctypes.byref(cfg)), "dd_search_create")
        self.widths = tuple(int(w) for w in widths)
        self.max_cands = max_cands
        self.ndm = 0
        self.n = 0

    @property
    def handle(self):
        return self._h

    def run(self, d_x, ndm: int, n: int, beam: int = 0, stream=None):
        """d_x: int32-typed CUDA tensor [>= ndm, ld] holding uint32 dedispersed sums."""
        assert d_x.is_cuda and d_x.stride(1) == 1
        _lib.check(self._L.dd_search_run(self._h, ctypes.c_void_p(d_x.data_ptr()), d_x.stride(0), ndm, n, beam,
                                         _stream_handle(stream)), "dd_search_run")
        self.ndm, self.n = ndm, n

    def result(self, stream=None):
        nh, ng, fl = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_uint()
        _lib.check(self._L.dd_search_result(self._h, ctypes.byref(nh), ctypes.byref(ng), ctypes.byref(fl),
                                            _stream_handle(stream)), "dd_search_result")
        return {"nhot": nh.value, "ngroups": ng.value, "flags": fl.value}

    def stats(self, stream=None):
        """Work counters of the last run: median histogram rebuilds."""
        nr = ctypes.c_longlong()
        _lib.check(self._L.dd_search_stats(self._h, ctypes.byref(nr), _stream_handle(stream)), "dd_search_stats")
        return {"median_rebuilds": nr.value}

    def candidates(self, stream=None) -> np.ndarray:
        out = np.zeros(self.max_cands, dtype=CAND_DTYPE)
        cnt = ctypes.c_int()
        _lib.check(self._L.dd_search_candidates(self._h, out.ctypes.data, self.max_cands, ctypes.byref(cnt),
                                                _stream_handle(stream)), "dd_search_candidates")
        return out[: cnt.value].copy()

    def buffers(self):
        """(y int32 [ndm, n], sumsq int64 [ndm], best float32 [ndm, n], bestw int16 [ndm, n]) device views."""
        py, ps, pb, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _lib.check(self._L.dd_search_buffers(self._h, ctypes.byref(py), ctypes.byref(ps), ctypes.byref(pb),
                                             ctypes.byref(pw)), "dd_search_buffers")
        return (_view(py.value, (self.ndm, self.n), "<i4", self), _view(ps.value, (self.ndm,), "<i8", self),
                _view(pb.value, (self.ndm, self.n), "<f4", self), _view(pw.value, (self.ndm, self.n), "<u2", self))

    def snippets(self, ncand: int, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty((max(ncand, 1), 64, 64), dtype=torch.bfloat16, device="cuda")
        _lib.check(self._L.dd_search_snippets(self._h, ncand, ctypes.c_void_p(out.data_ptr()),
                                              _stream_handle(stream)), "dd_search_snippets")
        return out[:ncand]

    def snippets_from_y(self, ncand: int, out=None, stream=None):
        """The same snippets computed straight from the y rows (dd_snippets)."""
        import torch

        if out is None:
            out = torch.empty((max(ncand, 1), 64, 64), dtype=torch.bfloat16, device="cuda")
        py, ps = ctypes.c_void_p(), ctypes.c_void_p()
        _lib.check(self._L.dd_search_buffers(self._h, ctypes.byref(py), ctypes.byref(ps), None, None),
                   "dd_search_buffers")
        _lib.check(self._L.dd_snippets(py, self.n, self.ndm, self.n, ps, ncand,
                                       ctypes.c_void_p(self.device_candidates_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)), "dd_snippets")
        return out[:ncand]

    def device_candidates_ptr(self) -> int:
        p = ctypes.c_void_p()
        _lib.check(self._L.dd_search_device_candidates(self._h, ctypes.byref(p)), "dd_search_device_candidates")
        return p.value

    def close(self):
        if self._h:
            self._L.dd_search_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
