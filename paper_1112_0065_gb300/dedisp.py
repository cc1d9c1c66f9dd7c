"""Python face of the dedispersion plan (C ABI: dd_plan_create / dd_execute /
dd_destroy).  Device memory and streams come from PyTorch; all arithmetic runs
in the CUDA library."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib

KERNEL_AUTO, KERNEL_SIMPLE, KERNEL_TILED = 0, 1, 2


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def compute_delays(freqs_mhz, tsamp_s: float, dms) -> np.ndarray:
    f, d = _f64(freqs_mhz), _f64(dms)
    out = np.empty((d.size, f.size), dtype=np.int32)
    L = _lib.load()
    _lib.check(L.dd_compute_delays(f.size, f.ctypes.data, float(tsamp_s), d.size, d.ctypes.data, out.ctypes.data),
               "dd_compute_delays")
    return out


def row_bytes(nsamp: int) -> int:
    """Smallest legal ld_in_bytes for nsamp samples (multiple of 16)."""
    return ((nsamp + 3) // 4 + 15) // 16 * 16


def out_stride(nout: int) -> int:
    return (nout + 3) // 4 * 4


class Plan:
    def __init__(self, freqs_mhz, tsamp_s: float, dms, kernel: int = KERNEL_AUTO, dms_per_block: int = 0,
                 words_per_thread: int = 0, chan_chunk: int = 0, tune_cache: str | None = None):
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        self._cache = tune_cache.encode() if tune_cache else None
        opt = _lib.Options(kernel, dms_per_block, words_per_thread, chan_chunk, 0, self._cache)
        f, d = _f64(freqs_mhz), _f64(dms)
        _lib.check(self._L.dd_plan_create(ctypes.byref(self._h), f.size, f.ctypes.data, float(tsamp_s), d.size,
                                          d.ctypes.data, ctypes.byref(opt)), "dd_plan_create")
        nc, nd, md = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(self._L.dd_plan_info(self._h, ctypes.byref(nc), ctypes.byref(nd), ctypes.byref(md)), "dd_plan_info")
        self.nchan, self.ndm, self.maxdelay = nc.value, nd.value, md.value
        self.freqs = f
        self.dms = d
        self.tsamp = float(tsamp_s)

    @property
    def handle(self):
        return self._h

    def nout(self, nsamp_in: int) -> int:
        return nsamp_in - self.maxdelay

    def delay_table(self) -> np.ndarray:
        out = np.empty((self.ndm, self.nchan), dtype=np.int32)
        _lib.check(self._L.dd_plan_delay_table(self._h, out.ctypes.data), "dd_plan_delay_table")
        return out

    def kernel_shape(self):
        v = [ctypes.c_int() for _ in range(4)]
        _lib.check(self._L.dd_plan_kernel_shape(self._h, *[ctypes.byref(x) for x in v]), "dd_plan_kernel_shape")
        return tuple(x.value for x in v)

    def autotune(self, nsamp_in: int, stream=None) -> float:
        ms = ctypes.c_float()
        _lib.check(self._L.dd_plan_autotune(self._h, nsamp_in, _stream_handle(stream), ctypes.byref(ms)),
                   "dd_plan_autotune")
        return ms.value

    def alloc_output(self, nsamp_in: int, device="cuda"):
        import torch

        n = self.nout(nsamp_in)
        return torch.empty((self.ndm, out_stride(n)), dtype=torch.int32, device=device)

    def execute(self, d_in, nsamp_in: int, out=None, stream=None):
        """d_in: uint8 CUDA tensor [nchan, ld_in_bytes]; returns the int32-typed
        output tensor [ndm, ld_out] holding the uint32 sums."""
        if out is None:
            out = self.alloc_output(nsamp_in, d_in.device)
        assert d_in.is_cuda and out.is_cuda and d_in.dim() == 2 and out.dim() == 2
        assert d_in.shape[0] == self.nchan and out.shape[0] == self.ndm
        assert d_in.stride(1) == 1 and out.stride(1) == 1
        _lib.check(self._L.dd_execute(self._h, ctypes.c_void_p(d_in.data_ptr()), d_in.stride(0), nsamp_in,
                                      ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
                   "dd_execute")
        return out

    def execute_host(self, h_in, nsamp_in: int, h_out=None, stream=None):
        """Host buffers in and out (numpy or pinned CPU tensors); synchronous."""
        import torch

        nout = self.nout(nsamp_in)
        if h_out is None:
            h_out = torch.empty((self.ndm, out_stride(nout)), dtype=torch.int32, pin_memory=True)
        pin = h_in.data_ptr() if isinstance(h_in, torch.Tensor) else h_in.ctypes.data
        pout = h_out.data_ptr() if isinstance(h_out, torch.Tensor) else h_out.ctypes.data
        ld_in = h_in.stride(0) if isinstance(h_in, torch.Tensor) else h_in.strides[0]
        ld_out = h_out.stride(0) if isinstance(h_out, torch.Tensor) else h_out.strides[0] // 4
        _lib.check(self._L.dd_execute_host(self._h, ctypes.c_void_p(pin), ld_in, nsamp_in, ctypes.c_void_p(pout),
                                           ld_out, _stream_handle(stream)), "dd_execute_host")
        return h_out

    def close(self):
        if self._h:
            self._L.dd_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dedisp_status() -> int:
    """Device error flags of the tiled dedispersion kernels on the current
    device, read and cleared (bit 0: a tile stopped waiting for its staged
    input and left its outputs unwritten).  Synchronises the device."""
    L = _lib.load()
    f = ctypes.c_uint()
    _lib.check(L.dd_dedisp_status(ctypes.byref(f)), "dd_dedisp_status")
    return f.value


def as_uint32(t) -> np.ndarray:
    """int32-typed torch tensor (device or host) -> numpy uint32 view copy."""
    return t.detach().cpu().numpy().view(np.uint32)


def corner_turn(d_tm, nchan: int, nsamp: int, out=None, stream=None):
    """Time-major packed 2-bit data (uint8 CUDA tensor [nsamp, ld_tm]) ->
    channel-major rows (uint8 [nchan, row_bytes(nsamp)]) for Plan.execute."""
    import torch

    if out is None:
        out = torch.empty((nchan, row_bytes(nsamp)), dtype=torch.uint8, device=d_tm.device)
    L = _lib.load()
    _lib.check(L.dd_corner_turn(ctypes.c_void_p(d_tm.data_ptr()), d_tm.stride(0), nchan, nsamp,
                                ctypes.c_void_p(out.data_ptr()), out.stride(0), _stream_handle(stream)),
               "dd_corner_turn")
    return out
