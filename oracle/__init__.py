"""CPU oracle for the dedispersion pipeline -- TEST INFRASTRUCTURE ONLY.

Plain C (``*_oracle.c``, built with gcc into ``_build/liboracle.so``) plus
this numpy-facing wrapper.  It states, slowly and directly, what each step of
the paper's pipeline computes (Section 2.2 dedispersion, Section 2.3 baseline
removal, matched filtering and peak finding) and the candidate classifier's
forward/backward pass.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library under ``paper_1112_0065_gb300/`` and never imports it.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP over independent rows).
    Rebuilt when a SHA-256 over the command, the machine and the sources
    changes (never by modification time)."""
    srcs = sorted(os.path.join(_HERE, s) for s in os.listdir(_HERE) if s.endswith("_oracle.c"))
    flags = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]
    h = hashlib.sha256((" ".join(flags) + "\0" + platform.machine()).encode())
    for src in srcs:
        with open(src, "rb") as fh:
            h.update(os.path.basename(src).encode() + b"\0" + fh.read())
    key = h.hexdigest()
    key_path = _LIB_PATH + ".key"
    if not force and os.path.exists(_LIB_PATH) and os.path.exists(key_path):
        with open(key_path) as fh:
            if fh.read() == key:
                return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc"] + flags + ["-o", tmp] + srcs + ["-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    with open(key_path, "w") as fh:
        fh.write(key)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _declare(_lib)
        return _lib


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_D = ctypes.c_double
_F = ctypes.c_float


def _declare(L):
    L.oracle_delay_table.argtypes = [_I, _P, _D, _I, _P, _P]
    L.oracle_max_delay.argtypes = [_I, _I, _P]
    L.oracle_max_delay.restype = ctypes.c_int32
    L.oracle_dedisperse.argtypes = [_I, _I, _P, _P, _SZ, _SZ, _P, _SZ]
    L.oracle_dedisperse_points.argtypes = [_I, _I, _P, _P, _SZ, _SZ, _SZ, _P, _P, _P]
    L.oracle_corner_turn.argtypes = [_P, _SZ, _I, _SZ, _P, _SZ]
    L.oracle_num_threads.restype = _I
    L.oracle_running_median.argtypes = [_P, _I64, _I64, _P]
    L.oracle_baseline_row.argtypes = [_P, _I64, _I64, _P]
    L.oracle_baseline_rows.argtypes = [_P, _I, _I64, _I64, _I64, _P]
    L.oracle_best_snr_rows.argtypes = [_P, _I, _I64, _I, _P, _P, _P]
    L.oracle_running_mean.argtypes = [_P, _I64, _I64, _P]
    L.oracle_baseline_mean_row.argtypes = [_P, _I64, _I64, _P]
    L.oracle_sumsq.argtypes = [_P, _I64]
    L.oracle_sumsq.restype = _I64
    L.oracle_sigma.argtypes = [_P, _I64]
    L.oracle_sigma.restype = _D
    L.oracle_boxcar_snr.argtypes = [_P, _I64, _I, _P]
    L.oracle_best_snr_row.argtypes = [_P, _I64, _I, _P, _P, _P]
    L.oracle_find_peaks.argtypes = [_P, _P, _I, _I64, _F, _P, _I64]
    L.oracle_find_peaks.restype = _I64
    L.oracle_snippets.argtypes = [_P, _P, _I, _I64, _I64, _P, _P, _P, _P]
    _declare_nn(L)
    _declare_rfi(L)


def _declare_rfi(L):
    L.oracle_zero_dm.argtypes = [_P, _I, _SZ, _SZ, _P]
    L.oracle_rfi_mask.argtypes = [_P, _I, _SZ, _I, _I, _P, _P]
    L.oracle_rfi_apply.argtypes = [_P, _I, _SZ, _SZ, _P]


def _declare_nn(L):
    L.oracle_nn_param_count.restype = ctypes.c_long
    L.oracle_nn_forward.argtypes = [_P, _I, _P, _P, _I]
    L.oracle_nn_loss.argtypes = [_P, _P, _I]
    L.oracle_nn_loss.restype = _F
    L.oracle_nn_backward.argtypes = [_P, _I, _P, _P, _P, _P, _I]
    L.oracle_nn_backward.restype = _F
    L.oracle_adamw_step.argtypes = [ctypes.c_long, _P, _P, _P, _P, _P, _F, _F, _F, _F, _F, _I]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(lib().oracle_num_threads())


# ---- dedispersion ---------------------------------------------------------

def delay_table(freqs_mhz, tsamp_s: float, dms) -> np.ndarray:
    f = _c(freqs_mhz, np.float64)
    dm = _c(dms, np.float64)
    out = np.empty((dm.size, f.size), dtype=np.int32)
    rc = lib().oracle_delay_table(f.size, _ptr(f), float(tsamp_s), dm.size, _ptr(dm), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_delay_table rejected its arguments")
    return out


def dedisperse(delays: np.ndarray, packed: np.ndarray, nsamp_in: int) -> np.ndarray:
    """packed: uint8 [nchan, ld_in] (2-bit, 4 samples/byte, earliest in the LSBs)."""
    delays = _c(delays, np.int32)
    packed = _c(packed, np.uint8)
    ndm, nchan = delays.shape
    assert packed.shape[0] == nchan
    maxdelay = int(delays.max()) if delays.size else 0
    nout = nsamp_in - maxdelay
    if nout <= 0:
        raise ValueError("input shorter than the largest delay")
    out = np.empty((ndm, nout), dtype=np.uint32)
    rc = lib().oracle_dedisperse(nchan, ndm, _ptr(delays), _ptr(packed), packed.shape[1],
                                 nsamp_in, _ptr(out), nout)
    if rc != 0:
        raise RuntimeError(f"oracle_dedisperse failed ({rc})")
    return out


def dedisperse_points(delays, packed, nsamp_in: int, d_idx, t_idx) -> np.ndarray:
    delays = _c(delays, np.int32)
    packed = _c(packed, np.uint8)
    d_idx = _c(d_idx, np.int32)
    t_idx = _c(t_idx, np.int64)
    ndm, nchan = delays.shape
    vals = np.empty(d_idx.size, dtype=np.uint32)
    rc = lib().oracle_dedisperse_points(nchan, ndm, _ptr(delays), _ptr(packed), packed.shape[1],
                                        nsamp_in, d_idx.size, _ptr(d_idx), _ptr(t_idx), _ptr(vals))
    if rc != 0:
        raise ValueError(f"oracle_dedisperse_points failed ({rc})")
    return vals


# ---- search stage -----------------------------------------------------------

def running_median(x, half: int) -> np.ndarray:
    x = _c(x, np.int32)
    med = np.empty_like(x)
    rc = lib().oracle_running_median(_ptr(x), x.size, int(half), _ptr(med))
    if rc != 0:
        raise RuntimeError("oracle_running_median failed")
    return med


def running_mean(x, half: int) -> np.ndarray:
    x = _c(x, np.int32)
    out = np.empty(x.size, dtype=np.float64)
    lib().oracle_running_mean(_ptr(x), x.size, int(half), _ptr(out))
    return out


def baseline(rows, half: int) -> np.ndarray:
    """rows: uint32 [ndm, n] (or a row-strided view) -> int32 y = x - running
    lower median, row by row (rows in parallel)."""
    rows = np.atleast_2d(np.asarray(rows))
    if rows.dtype != np.uint32 or rows.strides[1] != 4 or rows.strides[0] % 4:
        rows = _c(rows, np.uint32)
    ndm, n = rows.shape
    y = np.empty((ndm, n), dtype=np.int32)
    if ndm and lib().oracle_baseline_rows(_ptr(rows), ndm, n, rows.strides[0] // 4, int(half), _ptr(y)) != 0:
        raise RuntimeError("oracle_baseline_rows failed")
    return y


def baseline_mean(rows, half: int) -> np.ndarray:
    """rows: uint32 [ndm, n] -> int32 y = x - running mean rounded half up."""
    rows = np.atleast_2d(_c(rows, np.uint32))
    y = np.empty(rows.shape, dtype=np.int32)
    for d in range(rows.shape[0]):
        r = np.ascontiguousarray(rows[d])
        yd = np.empty(r.size, dtype=np.int32)
        if lib().oracle_baseline_mean_row(_ptr(r), r.size, int(half), _ptr(yd)) != 0:
            raise RuntimeError("oracle_baseline_mean_row failed")
        y[d] = yd
    return y


def sumsq(y) -> int:
    y = _c(y, np.int32)
    return int(lib().oracle_sumsq(_ptr(y), y.size))


def sigma(y) -> float:
    y = _c(y, np.int32)
    return float(lib().oracle_sigma(_ptr(y), y.size))


def boxcar_snr(y, w: int) -> np.ndarray:
    y = _c(y, np.int32)
    out = np.full(y.size, np.nan, dtype=np.float32)
    rc = lib().oracle_boxcar_snr(_ptr(y), y.size, int(w), _ptr(out))
    if rc != 0:
        raise ValueError("bad width")
    return out[: y.size - w + 1]


def best_snr(y2d, widths):
    """Per-cell best snr and its width over an ascending widths list (rows in
    parallel)."""
    y2d = np.atleast_2d(_c(y2d, np.int32))
    ws = _c(widths, np.int32)
    ndm, n = y2d.shape
    best = np.empty(y2d.shape, dtype=np.float32)
    bw = np.empty(y2d.shape, dtype=np.int32)
    if ndm and lib().oracle_best_snr_rows(_ptr(y2d), ndm, n, ws.size, _ptr(ws), _ptr(best), _ptr(bw)) != 0:
        raise MemoryError("oracle_best_snr_rows")
    return best, bw


CAND_DTYPE = np.dtype([("d", np.int32), ("t", np.int32), ("w", np.int32), ("snr", np.float32),
                       ("ncells", np.int64)])


def find_peaks(best, bestw, thresh: float) -> np.ndarray:
    best = _c(best, np.float32)
    bestw = _c(bestw, np.int32)
    ndm, n = best.shape
    cap = 1 << 16
    while True:
        out = np.zeros(cap, dtype=CAND_DTYPE)
        k = lib().oracle_find_peaks(_ptr(best), _ptr(bestw), ndm, n, float(thresh), _ptr(out), cap)
        if k < 0:
            raise MemoryError("oracle_find_peaks")
        if k <= cap:
            return out[:k]
        cap = int(k)


def snippets(y2d, sumsq_rows, cd, ct, cw) -> np.ndarray:
    """-> uint16 bfloat16 bit patterns [ncand, 64, 64]."""
    y2d = np.atleast_2d(_c(y2d, np.int32))
    ss = _c(sumsq_rows, np.int64)
    cd = _c(cd, np.int32)
    ct = _c(ct, np.int32)
    cw = _c(cw, np.int32)
    ndm, n = y2d.shape
    out = np.empty((cd.size, 64, 64), dtype=np.uint16)
    lib().oracle_snippets(_ptr(y2d), _ptr(ss), ndm, n, cd.size, _ptr(cd), _ptr(ct), _ptr(cw), _ptr(out))
    return out


def bf16_bits_to_float(u16) -> np.ndarray:
    return (np.asarray(u16, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


# ---- candidate classifier -------------------------------------------------------

NN_SHAPES = [("conv1.w", (16, 1, 3, 3)), ("conv1.b", (16,)), ("conv2.w", (32, 16, 3, 3)), ("conv2.b", (32,)),
             ("conv3.w", (64, 32, 3, 3)), ("conv3.b", (64,)), ("conv4.w", (64, 64, 3, 3)), ("conv4.b", (64,)),
             ("fc1.w", (128, 1024)), ("fc1.b", (128,)), ("fc2.w", (1, 128)), ("fc2.b", (1,))]


def nn_param_count() -> int:
    return int(lib().oracle_nn_param_count())


def nn_split(flat):
    out, o = {}, 0
    for name, shp in NN_SHAPES:
        k = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + k]).reshape(shp)
        o += k
    return out


def nn_forward(params, x_bf16_bits, round_bf16: bool = True) -> np.ndarray:
    p = _c(params, np.float32)
    x = _c(x_bf16_bits, np.uint16)
    n = x.shape[0]
    out = np.empty(n, dtype=np.float32)
    rc = lib().oracle_nn_forward(_ptr(p), n, _ptr(x), _ptr(out), 1 if round_bf16 else 0)
    if rc != 0:
        raise MemoryError("oracle_nn_forward")
    return out


def nn_loss(logits, labels) -> float:
    z = _c(logits, np.float32)
    y = _c(labels, np.float32)
    return float(lib().oracle_nn_loss(_ptr(z), _ptr(y), z.size))


def nn_backward(params, x_bf16_bits, labels, round_bf16: bool = True):
    """-> (loss, grads float32 [P], logits)"""
    p = _c(params, np.float32)
    x = _c(x_bf16_bits, np.uint16)
    y = _c(labels, np.float32)
    g = np.zeros(p.size, dtype=np.float32)
    z = np.empty(x.shape[0], dtype=np.float32)
    loss = lib().oracle_nn_backward(_ptr(p), x.shape[0], _ptr(x), _ptr(y), _ptr(g), _ptr(z), 1 if round_bf16 else 0)
    return float(loss), g, z


def adamw_step(master, grads, m, v, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.01, step=1):
    """In place on master/m/v (float32 arrays); returns the bfloat16 copy (uint16 bits)."""
    out = np.empty(master.size, dtype=np.uint16)
    g = _c(grads, np.float32)
    lib().oracle_adamw_step(master.size, _ptr(master), _ptr(g), _ptr(m), _ptr(v), _ptr(out), lr, beta1, beta2, eps,
                            wd, step)
    return out


def float_to_bf16_bits(a) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16 bit patterns (numpy)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


# ---- multibeam coincidence RFI mask (paper Section 2.1) ---------------------

def zero_dm(packed, nsamp: int) -> np.ndarray:
    """uint32 zero-DM series of one beam's packed rows [nchan, ld]."""
    packed = _c(packed, np.uint8)
    z = np.empty(nsamp, dtype=np.uint32)
    if lib().oracle_zero_dm(_ptr(packed), packed.shape[0], packed.shape[1], nsamp, _ptr(z)) != 0:
        raise ValueError("oracle_zero_dm")
    return z


def rfi_mask(z2d, k: int, min_beams: int):
    """(uint8 mask [nsamp], number masked) for zero-DM series z2d [nbeams, nsamp]."""
    z2d = np.atleast_2d(_c(z2d, np.uint32))
    mask = np.empty(z2d.shape[1], dtype=np.uint8)
    n = ctypes.c_int64()
    if lib().oracle_rfi_mask(_ptr(z2d), z2d.shape[0], z2d.shape[1], int(k), int(min_beams), _ptr(mask),
                             ctypes.byref(n)) != 0:
        raise ValueError("oracle_rfi_mask")
    return mask, int(n.value)


def rfi_apply(packed, nsamp: int, mask) -> np.ndarray:
    """Copy of one beam's packed rows with the masked samples replaced."""
    out = np.array(packed, dtype=np.uint8, copy=True, order="C")
    mask = _c(mask, np.uint8)
    if lib().oracle_rfi_apply(_ptr(out), out.shape[0], out.shape[1], nsamp, _ptr(mask)) != 0:
        raise ValueError("oracle_rfi_apply")
    return out


def corner_turn(tm, nchan: int, nsamp: int, ld_cm: int) -> np.ndarray:
    """Time-major packed bytes [nsamp, ld_tm] -> channel-major [nchan, ld_cm]."""
    tm = _c(tm, np.uint8)
    out = np.empty((nchan, ld_cm), dtype=np.uint8)
    if lib().oracle_corner_turn(_ptr(tm), tm.shape[1], nchan, nsamp, _ptr(out), ld_cm) != 0:
        raise ValueError("oracle_corner_turn")
    return out
