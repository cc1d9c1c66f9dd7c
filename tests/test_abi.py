"""The C-ABI library loads, exports every entry point its headers declare,
and rejects bad arguments on the host before touching the GPU (CPU only)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(headers=None):
    names = set()
    for h in headers or glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \t\*]*?\b(dd_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1112_0065_gb300 import _build, _lib

    _build.build()
    return _lib.load()


def test_headers_declare_entry_points():
    names = declared_symbols()
    for n in ("dd_plan_create", "dd_execute", "dd_destroy", "dd_compute_delays"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert missing == []


PROBE_HEADER = os.path.join(ROOT, "paper_1112_0065_gb300", "csrc", "probe", "dd_probe.h")


def test_probes_live_outside_the_product_library(lib):
    """The measurement probes are a library of their own: libddprobe.so
    exports what its header declares, libdd.so exports none of it, and the
    binding of the product library does not name them."""
    from paper_1112_0065_gb300 import _lib, probes

    probe_names = declared_symbols([PROBE_HEADER])
    assert set(probe_names) == set(probes.SIGNATURES)
    plib = probes.load()
    assert [n for n in probe_names if not hasattr(plib, n)] == []
    assert [n for n in probe_names if hasattr(lib, n)] == []
    assert not (set(probe_names) & set(declared_symbols())) and not (set(probe_names) & set(_lib.SIGNATURES))


def test_build_keys_follow_content(tmp_path):
    """Objects are rebuilt when a key over the compiler command, the machine
    and the text of the source and headers changes, not by modification time."""
    from paper_1112_0065_gb300 import _build

    obj = tmp_path / "x.o"
    obj.write_bytes(b"object")
    _build._write_key(str(obj), "k1")
    assert _build._key_ok(str(obj), "k1") and not _build._key_ok(str(obj), "k2")
    os.utime(obj, (0, 0))   # an old timestamp alone changes nothing
    assert _build._key_ok(str(obj), "k1")
    assert any(h.endswith(".cuh") for h in _build._headers())


def test_binding_covers_every_symbol():
    from paper_1112_0065_gb300 import _lib

    assert sorted(set(declared_symbols()) - set(_lib.SIGNATURES)) == []


def test_status_strings(lib):
    from paper_1112_0065_gb300 import _lib

    for code, name in _lib.STATUS.items():
        assert lib.dd_status_string(code).decode() == name
    assert lib.dd_version() >= 10000


def _plan_create(lib, freqs, tsamp, dms, opt=None):
    from paper_1112_0065_gb300 import _lib

    h = ctypes.c_void_p()
    f = np.ascontiguousarray(freqs, np.float64)
    d = np.ascontiguousarray(dms, np.float64)
    st = lib.dd_plan_create(ctypes.byref(h), f.size, f.ctypes.data, tsamp, d.size, d.ctypes.data,
                            ctypes.byref(opt) if opt is not None else None)
    if st == 0:
        lib.dd_destroy(h)
    return st


@pytest.mark.parametrize("case", ["descending", "dup_freq", "neg_dm", "unsorted_dm", "tsamp", "nan", "nchan"])
def test_invalid_plans_rejected_before_cuda(lib, case):
    f = synth.band_freqs(16)
    dms = np.linspace(0, 10, 5)
    tsamp = 64e-6
    if case == "descending":
        f = f[::-1]
    elif case == "dup_freq":
        f[3] = f[2]
    elif case == "neg_dm":
        dms[0] = -1
    elif case == "unsorted_dm":
        dms = dms[::-1]
    elif case == "tsamp":
        tsamp = 0.0
    elif case == "nan":
        f[5] = np.nan
    elif case == "nchan":
        f = f[:0]
    assert _plan_create(lib, f, tsamp, dms) == -1
    assert lib.dd_last_error()


def test_bad_options_rejected(lib):
    from paper_1112_0065_gb300 import _lib

    opt = _lib.Options(7, 0, 0, 0, 0, None)
    assert _plan_create(lib, synth.band_freqs(8), 64e-6, [0.0, 1.0], opt) == -1
    opt = _lib.Options(2, 12, 2, 64, 0, None)  # DMs per CTA must be 8 * trials per warp
    assert _plan_create(lib, synth.band_freqs(8), 64e-6, [0.0, 1.0], opt) == -1


def test_compute_delays_matches_oracle_and_rejects_null(lib):
    import oracle
    from paper_1112_0065_gb300 import compute_delays

    f = synth.band_freqs(256)
    dms = synth.dm_list_piecewise(500.0)
    np.testing.assert_array_equal(compute_delays(f, 64e-6, dms), oracle.delay_table(f, 64e-6, dms))
    assert lib.dd_compute_delays(4, None, 64e-6, 1, None, None) == -1


def test_execute_rejects_null_plan(lib):
    assert lib.dd_execute(None, None, 16, 100, None, 100, None) == -1
    lib.dd_destroy(None)
