"""Pins of the multibeam coincidence RFI oracle (paper Section 2.1): the
zero-DM series against a numpy unpack, the exact-integer threshold against a
float64 evaluation away from the boundary, coincident broadband bursts masked
exactly where at least min_beams beams carry them, single-beam signals left
alone, the false-alarm rate on noise against the binomial tail, the paper's
printed bound, and the substitution pattern."""
import math

import numpy as np

import oracle
import synth


def beams_with_bursts(seed, nbeams, nchan, nsamp, events):
    """events: list of (t0, dur, beams) broadband bursts (level 3, all channels)."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(nbeams):
        lv = synth.noise_levels(rng, nchan, nsamp)
        for t0, dur, bs in events:
            if b in bs:
                lv[:, t0:t0 + dur] = 3
        out.append(synth.pack2(lv))
    return out


def test_paper_false_alarm_bound():
    # 3 sigma in 4 or more of 13 beams with 0.01 per beam: C(13,4) * 0.01^4
    assert abs(math.comb(13, 4) * 0.01 ** 4 - 7.15e-6) < 5e-9
    # the exact Gaussian one-sided 3-sigma tail is far below the paper's 0.01
    p1 = 0.5 * math.erfc(3 / math.sqrt(2))
    exact = sum(math.comb(13, j) * p1 ** j * (1 - p1) ** (13 - j) for j in range(4, 14))
    assert exact < 7.15e-6 and abs(p1 - 1.3499e-3) < 1e-6


def test_zero_dm_against_unpack():
    packed = beams_with_bursts(1, 1, 37, 1001, [])[0]
    z = oracle.zero_dm(packed, 1001)
    np.testing.assert_array_equal(z, synth.unpack2(packed, 1001).astype(np.uint32).sum(axis=0))


def test_threshold_matches_float_away_from_the_boundary():
    rng = np.random.default_rng(2)
    z = rng.integers(1400, 1700, size=(13, 5000)).astype(np.uint32)
    for k in (1, 2, 3):
        mask, _ = oracle.rfi_mask(z, k, 1)   # one beam suffices: mask = any beam over
        zf = z.astype(np.float64)
        mu = zf.mean(axis=1, keepdims=True)
        sd = zf.std(axis=1, keepdims=True)
        over = zf > mu + k * sd
        safe = np.all(np.abs(zf - (mu + k * sd)) > 1e-6, axis=0)
        np.testing.assert_array_equal(mask[safe].astype(bool), over.any(axis=0)[safe])


def test_coincident_bursts_masked_single_beam_signals_kept():
    nchan, nsamp = 64, 6000
    events = [(1000, 40, set(range(5))),          # 5 beams: RFI
              (2500, 30, {0, 4, 8, 12}),          # exactly 4 beams: RFI
              (4000, 50, {1, 2, 3}),              # 3 beams: kept
              (5000, 20, {7})]                    # one beam (a sky signal): kept
    beams = beams_with_bursts(3, 13, nchan, nsamp, events)
    z = np.stack([oracle.zero_dm(p, nsamp) for p in beams])
    mask, nm = oracle.rfi_mask(z, 3, 4)
    want = np.zeros(nsamp, np.uint8)
    want[1000:1040] = 1
    want[2500:2530] = 1
    np.testing.assert_array_equal(mask, want)
    assert nm == 70


def test_noise_false_alarms_follow_the_binomial_tail():
    """With k = 1 a beam exceeds often enough to count coincidences: the mask
    rate for >= 4 of 13 beams matches the tail of the Poisson-binomial
    distribution of the 13 measured per-beam rates (independent beams)."""
    nchan, nsamp = 64, 40000
    beams = beams_with_bursts(4, 13, nchan, nsamp, [])
    z = np.stack([oracle.zero_dm(p, nsamp) for p in beams])
    dist = np.array([1.0])
    for b in range(13):
        pb = oracle.rfi_mask(z[b:b + 1], 1, 1)[0].mean()
        dist = np.convolve(dist, [1 - pb, pb])
    tail = float(dist[4:].sum())
    _, nm = oracle.rfi_mask(z, 1, 4)
    sd = math.sqrt(tail * (1 - tail) / nsamp)
    assert abs(nm / nsamp - tail) < 5 * sd + 1e-4, (nm / nsamp, tail)
    _, nm3 = oracle.rfi_mask(z, 3, 4)
    assert nm3 == 0


def test_apply_substitutes_the_alternating_mean_level():
    nchan, nsamp = 40, 777
    beams = beams_with_bursts(5, 1, nchan, nsamp, [(100, 30, {0})])
    mask = np.zeros(nsamp, np.uint8)
    mask[100:130] = 1
    mask[776] = 1
    out = oracle.rfi_apply(beams[0], nsamp, mask)
    lv_in, lv = synth.unpack2(beams[0], nsamp), synth.unpack2(out, nsamp)
    keep = mask == 0
    np.testing.assert_array_equal(lv[:, keep], lv_in[:, keep])
    c, t = np.meshgrid(np.arange(nchan), np.flatnonzero(mask), indexing="ij")
    np.testing.assert_array_equal(lv[:, mask == 1], 1 + ((c + t) & 1))
    # the zero-DM sum of a masked sample is 1.5 * nchan (nchan even)
    assert np.all(oracle.zero_dm(out, nsamp)[mask == 1] == 3 * nchan // 2)
    # bytes past nsamp are untouched
    np.testing.assert_array_equal(out[:, (nsamp + 3) // 4:], beams[0][:, (nsamp + 3) // 4:])
