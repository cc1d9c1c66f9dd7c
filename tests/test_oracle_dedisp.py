"""Pins for the dedispersion oracle (CPU only).

The oracle is checked against things other than itself: numpy brute force on
tiny inputs, closed forms (DM 0 is a plain channel sum, constant input gives
nchan*k), the exact sum of an injected dispersed pulse on a zero background
(paper Section 2.2: a trial integrates the whole band along the pulse's
dispersion sweep), linearity and time-shift equivariance, the physical
dispersion constant derived from CODATA values, and the paper's ~4 MB/s
per-beam data rate for 1024 channels x 2 bits x 64 us (Section 1).
"""
import math
import os

import numpy as np
import pytest

import oracle
import synth


def brute(levels, delays):
    ndm, nchan = delays.shape
    nout = levels.shape[1] - int(delays.max())
    out = np.zeros((ndm, nout), dtype=np.int64)
    for d in range(ndm):
        for c in range(nchan):
            out[d] += levels[c, delays[d, c]:delays[d, c] + nout]
    return out


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_oracle_matches_brute_force_random_delays(seed):
    rng = np.random.default_rng(seed)
    nchan = int(rng.integers(1, 17))
    ndm = int(rng.integers(1, 9))
    nsamp = int(rng.integers(40, 257))
    maxd = int(rng.integers(0, nsamp // 2))
    delays = rng.integers(0, maxd + 1, size=(ndm, nchan)).astype(np.int32)
    delays[0, 0] = 0
    delays[-1, -1] = maxd
    levels = rng.integers(0, 4, size=(nchan, nsamp)).astype(np.uint8)
    packed = synth.pack2(levels)
    got = oracle.dedisperse(delays, packed, nsamp)
    np.testing.assert_array_equal(got.astype(np.int64), brute(levels, delays))
    # sampled-point form agrees with the full form
    d_idx = rng.integers(0, ndm, 50)
    t_idx = rng.integers(0, got.shape[1], 50)
    pts = oracle.dedisperse_points(delays, packed, nsamp, d_idx, t_idx)
    np.testing.assert_array_equal(pts, got[d_idx, t_idx])


def test_dm_zero_is_channel_sum():
    f = synth.band_freqs(64)
    dms = synth.dm_list_linear(8, 100.0)
    delays = oracle.delay_table(f, 64e-6, dms)
    assert np.all(delays[0] == 0)
    packed, lv = synth.make_gulp(5, 64, 4096)
    out = oracle.dedisperse(delays, packed, 4096)
    np.testing.assert_array_equal(out[0], lv[:, : out.shape[1]].astype(np.uint32).sum(axis=0))


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_constant_input(k):
    f = synth.band_freqs(32)
    delays = oracle.delay_table(f, 64e-6, synth.dm_list_linear(16, 100.0))
    lv = np.full((32, 3000), k, dtype=np.uint8)
    out = oracle.dedisperse(delays, synth.pack2(lv), 3000)
    assert np.all(out == 32 * k)


def test_injected_pulse_sums_exactly_at_its_dm_and_arrival():
    """Tiny configuration: 64 channels 1581.8->1181.8 MHz, 64 us, 8192
    samples, 64 DMs i*100/64, pulse at DM 50 (trial 32), arrival sample 1000,
    amplitude 2 on a zero background."""
    nchan, nsamp = 64, 8192
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(64, 100.0)
    assert dms[32] == 50.0
    delays = oracle.delay_table(f, 64e-6, dms)
    assert int(delays.max()) == 1984
    rec = synth.BeamRecipe(pulses=[synth.Pulse(t0=1000, offsets=delays[32], amp=2, width=1, dm=50.0)])
    packed, _ = synth.make_gulp(0, nchan, nsamp, rec, background="zero")
    out = oracle.dedisperse(delays, packed, nsamp)
    assert out.shape == (64, nsamp - 1984)
    assert out[32, 1000] == nchan * 2
    # the full sum appears nowhere else
    flat = out.copy()
    flat[32, 1000] = 0
    assert flat.max() < nchan * 2


def test_injected_pulse_stands_out_in_noise():
    nchan, nsamp = 64, 8192
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_linear(64, 100.0)
    delays = oracle.delay_table(f, 64e-6, dms)
    rec = synth.BeamRecipe(pulses=[synth.Pulse(t0=1000, offsets=delays[32], amp=2, width=1, dm=50.0)])
    packed, _ = synth.make_gulp(synth.BASE_SEED, nchan, nsamp, rec)
    out = oracle.dedisperse(delays, packed, nsamp).astype(np.int64)
    d, t = np.unravel_index(np.argmax(out), out.shape)
    assert (d, t) == (32, 1000)


def test_linearity_and_shift_equivariance():
    rng = np.random.default_rng(7)
    nchan, nsamp = 24, 900
    f = synth.band_freqs(nchan)
    delays = oracle.delay_table(f, 64e-6, synth.dm_list_linear(12, 30.0))
    a = rng.integers(0, 2, size=(nchan, nsamp)).astype(np.uint8)
    b = 2 * rng.integers(0, 2, size=(nchan, nsamp)).astype(np.uint8)
    oa = oracle.dedisperse(delays, synth.pack2(a), nsamp).astype(np.int64)
    ob = oracle.dedisperse(delays, synth.pack2(b), nsamp).astype(np.int64)
    oab = oracle.dedisperse(delays, synth.pack2(a + b), nsamp).astype(np.int64)
    np.testing.assert_array_equal(oa + ob, oab)
    s = 37
    osh = oracle.dedisperse(delays, synth.pack2(a[:, s:]), nsamp - s).astype(np.int64)
    np.testing.assert_array_equal(osh, oa[:, s:])


def test_delay_table_structure():
    f = synth.band_freqs(1024)
    dms = synth.dm_list_piecewise(1000.0)
    assert dms.size == 1500 and dms[-1] == 999.0
    delays = oracle.delay_table(f, 64e-6, dms)
    assert np.all(delays[:, 0] == 0)
    assert np.all(np.diff(delays, axis=0) >= 0)   # non-decreasing in DM
    assert np.all(np.diff(delays, axis=1) >= 0)   # non-decreasing as frequency falls
    assert int(delays.max()) == 20464


def test_dispersion_constant_from_physical_constants():
    """k_DM = e^2 / (2 pi m_e c) (Gaussian units) turned into s MHz^2 per
    pc cm^-3 reproduces the delay of a DM=1000 sweep across the band."""
    e = 4.80320471e-10          # statC
    m_e = 9.1093837015e-28      # g
    c = 2.99792458e10           # cm/s
    pc = 3.0856775814913673e18  # cm
    k = e * e / (2 * math.pi * m_e * c) * pc / 1e12
    f = np.array([1581.8, 1181.8])
    tsamp = 64e-6
    want = k * 1000.0 * (1 / f[1] ** 2 - 1 / f[0] ** 2) / tsamp
    got = oracle.delay_table(f, tsamp, [1000.0])[0, 1]
    assert abs(got - want) <= 1.0 + 2e-5 * want


def test_paper_data_rate_per_beam():
    """1024 channels x 2 bits every 64 us is ~4 MB/s per beam (paper Section 1)."""
    nsamp = int(round(1.0 / 64e-6))
    bytes_per_s = 1024 * nsamp / 4
    assert nsamp == 15625
    assert bytes_per_s == 4.0e6
    lv = np.zeros((4, 64), dtype=np.uint8)
    assert synth.pack2(lv).shape == (4, 16)   # 4 samples per byte


def test_packing_order_low_bits_first():
    lv = np.array([[1, 2, 3, 0, 3]], dtype=np.uint8)
    p = synth.pack2(lv)
    assert p[0, 0] == (1 | (2 << 2) | (3 << 4))
    assert p[0, 1] == 3
    np.testing.assert_array_equal(synth.unpack2(p, 5), lv)


def test_level_distribution_matches_quantiser():
    rng = np.random.default_rng(3)
    lv = synth.noise_levels(rng, 64, 20000)
    freq = np.bincount(lv.ravel(), minlength=4) / lv.size
    z = rng.standard_normal(2_000_000)
    q = (z >= -0.98).astype(int) + (z >= 0) + (z >= 0.98)
    ref = np.bincount(q, minlength=4) / q.size
    np.testing.assert_allclose(freq, ref, atol=3e-3)
    assert abs(lv.mean() - 1.5) < 5e-3


def test_piecewise_dm_grid_counts():
    assert synth.dm_list_piecewise(250.0).size == 700
    assert synth.dm_list_piecewise(500.0).size == 1000
    assert synth.dm_list_piecewise(1000.0).size == 1500


def test_corner_turn_against_numpy_transpose():
    """Time-major to channel-major: the oracle against unpack / transpose /
    pack in numpy, for channel counts off the 4-channel byte grid."""
    rng = np.random.default_rng(17)
    for nchan, nsamp in [(64, 1000), (7, 33), (130, 257)]:
        lv = rng.integers(0, 4, size=(nsamp, nchan)).astype(np.uint8)     # [t][c]
        ld_tm = (nchan + 3) // 4 + 3
        tm = synth.pack2(lv, ld_tm)                                         # rows are time samples
        ld_cm = synth.padded_row_bytes(nsamp)
        cm = oracle.corner_turn(tm, nchan, nsamp, ld_cm)
        np.testing.assert_array_equal(cm, synth.pack2(lv.T.copy(), ld_cm))


def _delay_rounding_golden():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "delay_rounding.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            nchan, grid, d, c, exact, rounded, fl, ce = line.split()
            rows.append((int(nchan), grid, int(d), int(c), float(exact), int(rounded), int(fl), int(ce)))
    return rows


def golden_delay_grid(nchan, grid):
    f = synth.band_freqs(nchan)
    dms = synth.dm_list_piecewise(1000.0) if grid == "piecewise1000" else synth.dm_list_linear(64, 100.0)
    return f, dms


def test_delay_rounding_mode_golden():
    """Delays whose exact rational value (tests/golden/delay_rounding.txt,
    written without floating point) has a fractional part in [0.55, 0.95] or
    [0.05, 0.45]: the table must hold the nearest integer, so a floor,
    truncating or ceiling delay table fails here."""
    rows = _delay_rounding_golden()
    assert sum(r[5] != r[6] for r in rows) >= 8      # entries where floor / truncation differ
    assert sum(r[5] != r[7] for r in rows) >= 5      # entries where ceil differs
    tables = {}
    for nchan, grid, d, c, exact, rounded, _, _ in rows:
        if (nchan, grid) not in tables:
            f, dms = golden_delay_grid(nchan, grid)
            tables[(nchan, grid)] = oracle.delay_table(f, 64e-6, dms)
        assert rounded == math.floor(exact + 0.5)
        assert tables[(nchan, grid)][d, c] == rounded, (nchan, grid, d, c, exact)


def test_delay_rounding_golden_is_reproducible():
    """The committed golden file is exactly what its script writes (rational
    arithmetic only, no floating point in the values it checks)."""
    import importlib.util

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_delay_rounding", os.path.join(here, "make_delay_rounding.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rows = mod.pick(1024, mod.piecewise_dms(), "piecewise1000", 8, 3) + \
        mod.pick(64, mod.linear_dms(64, 100), "linear64x100", 4, 2)
    stored = _delay_rounding_golden()
    assert len(rows) == len(stored)
    for (nchan, grid, d, c, v), (snchan, sgrid, sd, sc, exact, rounded, fl, ce) in zip(rows, stored):
        assert (nchan, grid, d, c) == (snchan, sgrid, sd, sc)
        assert abs(float(v) - exact) < 1e-9
        assert rounded == (math.floor(v) + 1 if v - math.floor(v) >= mod.Fraction(1, 2) else math.floor(v))
