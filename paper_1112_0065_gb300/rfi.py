"""Python face of the multibeam coincidence RFI mask (C ABI: dd_rfi_*); all
arithmetic runs in the CUDA library."""
from __future__ import annotations

import ctypes

from . import _lib
from .dedisp import _stream_handle
from .search import _view


class RfiMask:
    """Coincidence rejection across beams (a sample exceeding k_sigma standard
    deviations of its beam's total power in at least min_beams beams)."""

    def __init__(self, nbeams_max: int, nchan: int, nsamp_max: int):
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        _lib.check(self._L.dd_rfi_create(ctypes.byref(self._h), nbeams_max, nchan, nsamp_max), "dd_rfi_create")
        self.nchan = nchan
        self.nbeams = 0
        self.nsamp = 0

    def run(self, gulps, nsamp: int, k_sigma: int = 3, min_beams: int = 4, apply: bool = False, stream=None):
        """gulps: list of uint8 CUDA tensors [nchan, ld_bytes] (same ld); with
        apply=True the masked samples are replaced in place."""
        ptrs = (ctypes.c_void_p * len(gulps))(*[g.data_ptr() for g in gulps])
        _lib.check(self._L.dd_rfi_run(self._h, ptrs, len(gulps), gulps[0].stride(0), nsamp, k_sigma, min_beams,
                                      1 if apply else 0, _stream_handle(stream)), "dd_rfi_run")
        self.nbeams, self.nsamp = len(gulps), nsamp

    def nmasked(self, stream=None) -> int:
        v = ctypes.c_longlong()
        _lib.check(self._L.dd_rfi_result(self._h, ctypes.byref(v), _stream_handle(stream)), "dd_rfi_result")
        return v.value

    def buffers(self):
        """(zero-DM series [nbeams, nsamp] as int32-typed uint32 values, mask uint8
        [nsamp]) device views."""
        pz, pm = ctypes.c_void_p(), ctypes.c_void_p()
        ld = ctypes.c_size_t()
        _lib.check(self._L.dd_rfi_buffers(self._h, ctypes.byref(pz), ctypes.byref(ld), ctypes.byref(pm)),
                   "dd_rfi_buffers")
        z = _view(pz.value, (self.nbeams, ld.value), "<i4", self)[:, :self.nsamp]
        return z, _view(pm.value, (self.nsamp,), "|u1", self)

    def close(self):
        if self._h:
            self._L.dd_rfi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
