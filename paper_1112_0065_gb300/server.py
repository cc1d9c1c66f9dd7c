"""Python face of the streaming server (C ABI dd_server_*)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from .search import CAND_DTYPE, DEFAULT_WIDTHS

RESULT_FIELDS = ("beam", "ncand", "seq", "t0", "nout", "t_submit", "t_done", "ngroups", "flags", "cand_offset")


class Server:
    def __init__(self, plans, gulp_nsamp: int, max_slots: int = 8, hbm_reserve: int = 0, half_window: int = 4096,
                 widths=DEFAULT_WIDTHS, thresh: float = 6.0, max_cands: int = 16384, classifier_path=None,
                 nn_batch: int = 1024, trigger_snr: float = 0.0, trigger_max: int = 4, on_trigger=None):
        """on_trigger(info dict, raw uint8 array [nchan, ld]) is called on the
        server's worker thread for every dump (candidates with snr >=
        trigger_snr); it must not call back into the server."""
        self._L = _lib.load()
        self._h = ctypes.c_void_p()
        self.plans = list(plans)  # keep the plans alive as long as the server
        cfg = _lib.ServerConfig()
        cfg.nbeams, cfg.gulp_nsamp, cfg.max_slots, cfg.hbm_reserve_bytes = len(self.plans), gulp_nsamp, max_slots, \
            hbm_reserve
        cfg.half_window, cfg.nwidths = half_window, len(widths)
        for k, w in enumerate(widths):
            cfg.widths[k] = int(w)
        cfg.thresh, cfg.max_cands, cfg.nn_batch = float(thresh), max_cands, nn_batch
        self._trigger_cb = None
        if on_trigger is not None and trigger_snr > 0:
            def _cb(user, trig, raw):
                t = trig.contents
                info = {"beam": t.beam, "seq": t.seq, "t0": t.t0, "nsamp": t.nsamp, "nchan": t.nchan,
                        "d": t.cand.d, "t": t.cand.t, "w": t.cand.w, "snr": t.cand.snr}
                buf = np.ctypeslib.as_array(raw, shape=(t.nchan * t.ld,)).reshape(t.nchan, t.ld).copy()
                on_trigger(info, buf)

            self._trigger_cb = _lib.TRIGGER_FN(_cb)   # kept alive as long as the server
            cfg.trigger_snr, cfg.trigger_max, cfg.trigger_fn = float(trigger_snr), trigger_max, self._trigger_cb
        self._cpath = classifier_path.encode() if classifier_path else None
        cfg.classifier_path = self._cpath
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        _lib.check(self._L.dd_server_create(ctypes.byref(self._h), ctypes.byref(cfg), arr), "dd_server_create")
        self.gulp_nsamp = gulp_nsamp
        self.max_cands = max_cands
        self._held = {}

    def submit(self, beam: int, h_new):
        """h_new: host uint8 array/tensor [nchan, >= gulp_nsamp/4].  Returns the
        gulp's sequence number, or None when the server is busy."""
        import torch

        if isinstance(h_new, torch.Tensor):
            ptr, pitch = h_new.data_ptr(), h_new.stride(0)
        else:
            ptr, pitch = h_new.ctypes.data, h_new.strides[0]
        seq = ctypes.c_longlong()
        st = self._L.dd_server_submit(self._h, beam, ctypes.c_void_p(ptr), pitch, ctypes.byref(seq))
        if st == _lib.DD_ERR_BUSY:
            return None
        _lib.check(st, "dd_server_submit")
        self._held[(beam, seq.value)] = h_new  # the copy is asynchronous: keep the buffer alive
        return seq.value

    def poll(self, wait_s: float = 0.0, max_results: int = 64):
        """-> list of (result dict, candidates structured array)."""
        res = (_lib.GulpResult * max_results)()
        cap = max_results * self.max_cands
        cands = np.zeros(cap, dtype=CAND_DTYPE)
        nr, nc = ctypes.c_int(), ctypes.c_int()
        _lib.check(self._L.dd_server_poll(self._h, res, max_results, ctypes.byref(nr), cands.ctypes.data, cap,
                                          ctypes.byref(nc), float(wait_s)), "dd_server_poll")
        out = []
        for i in range(nr.value):
            r = {f: getattr(res[i], f) for f in RESULT_FIELDS}
            c = cands[r["cand_offset"]:r["cand_offset"] + r["ncand"]].copy()
            self._held.pop((r["beam"], r["seq"]), None)
            out.append((r, c))
        return out

    def drain(self, timeout_s: float = 120.0):
        _lib.check(self._L.dd_server_drain(self._h, float(timeout_s)), "dd_server_drain")

    def info(self):
        ns, fl, sb = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _lib.check(self._L.dd_server_info(self._h, ctypes.byref(ns), ctypes.byref(fl), ctypes.byref(sb)),
                   "dd_server_info")
        return {"slots": ns.value, "in_flight": fl.value, "slot_bytes": sb.value}

    def set_tap(self, beam: int, d_dst, capacity: int):
        _lib.check(self._L.dd_server_set_tap(self._h, beam, ctypes.c_void_p(d_dst.data_ptr()), d_dst.stride(0),
                                             capacity), "dd_server_set_tap")

    def close(self):
        if self._h:
            self._L.dd_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
