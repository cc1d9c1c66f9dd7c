"""Pins for the search-stage oracle (CPU only): running median against a
numpy sort of every window, the paper's running mean against a prefix-sum
statement of it (Section 2.3), boxcar sums against numpy cumulative sums,
closed-form S/N cases, Gaussian-noise S/N statistics, hand-built peak maps
for the grouping rules, and a hand-computed snippet."""
import numpy as np
import pytest

import oracle


def np_lower_median(x, half):
    n = x.size
    out = np.empty(n, dtype=np.int64)
    for t in range(n):
        w = np.sort(x[max(0, t - half):min(n, t + half)])
        out[t] = w[(w.size - 1) // 2]
    return out


@pytest.mark.parametrize("seed,n,half", [(0, 50, 4), (1, 301, 16), (2, 128, 64), (3, 33, 100)])
def test_running_median_vs_sort(seed, n, half):
    rng = np.random.default_rng(seed)
    x = rng.integers(-50, 300, size=n).astype(np.int32)
    np.testing.assert_array_equal(oracle.running_median(x, half), np_lower_median(x, half))


def test_running_median_closed_forms():
    x = np.full(100, 7, dtype=np.int32)
    assert np.all(oracle.running_median(x, 8) == 7)
    ramp = np.arange(200, dtype=np.int32)
    med = oracle.running_median(ramp, 10)
    # interior windows [t-10, t+10) of a ramp: lower median of 20 values = t - 1
    np.testing.assert_array_equal(med[10:190], np.arange(10, 190) - 1)


def test_running_mean_vs_prefix_sum():
    rng = np.random.default_rng(4)
    x = rng.integers(0, 100, size=500).astype(np.int32)
    half = 13
    P = np.concatenate([[0], np.cumsum(x.astype(np.int64))])
    t = np.arange(500)
    lo = np.maximum(t - half, 0)
    hi = np.minimum(t + half, 500)
    np.testing.assert_allclose(oracle.running_mean(x, half), (P[hi] - P[lo]) / (hi - lo), rtol=0, atol=1e-12)


def test_mean_baseline_rounds_half_up():
    """The integer mean baseline: x - round-half-up(window mean), against the
    float mean (a different computation) and at exact halves."""
    rng = np.random.default_rng(9)
    x = rng.integers(1400, 1700, size=(2, 3000)).astype(np.uint32)
    half = 57
    y = oracle.baseline_mean(x, half)
    for d in range(2):
        mean = oracle.running_mean(x[d].astype(np.int32), half)
        frac = mean - np.floor(mean)
        ok = np.abs(frac - 0.5) > 1e-9
        np.testing.assert_array_equal(y[d][ok], (x[d].astype(np.int64) - np.floor(mean + 0.5).astype(np.int64))[ok])
    # half 1: windows [t-1, t+1); means 1, 1.5 -> 2, 3.5 -> 4; constant rows -> 0
    np.testing.assert_array_equal(oracle.baseline_mean(np.array([[1, 2, 5]], np.uint32), 1), [[0, 0, 1]])
    np.testing.assert_array_equal(oracle.baseline_mean(np.full((1, 50), 7, np.uint32), 5), np.zeros((1, 50)))


def test_baseline_removes_constant_offset():
    rows = np.full((2, 400), 1536, dtype=np.uint32)
    rows[1, 100] = 1600
    y = oracle.baseline(rows, 32)
    assert np.all(y[0] == 0)
    assert y[1, 100] == 64 and np.count_nonzero(y[1]) == 1


@pytest.mark.parametrize("w", [1, 2, 4, 8, 16, 64])
def test_boxcar_sums_vs_cumsum(w):
    rng = np.random.default_rng(w)
    y = rng.integers(-40, 40, size=777).astype(np.int32)
    sig = np.sqrt(np.sum(y.astype(np.int64) ** 2) / y.size)
    P = np.concatenate([[0], np.cumsum(y.astype(np.int64))])
    S = P[w:] - P[:-w]
    want = S.astype(np.float32) / np.float32(sig * np.sqrt(w))
    np.testing.assert_array_equal(oracle.boxcar_snr(y, w), want)
    assert oracle.sumsq(y) == int(np.sum(y.astype(np.int64) ** 2))


def test_snr_closed_forms():
    y = np.array([1, -1] * 50, dtype=np.int32)
    assert oracle.sigma(y) == 1.0
    np.testing.assert_array_equal(oracle.boxcar_snr(y, 1), y.astype(np.float32))
    assert np.all(oracle.boxcar_snr(y, 2) == 0.0)
    z = np.zeros(10, dtype=np.int32)
    assert np.all(oracle.boxcar_snr(z, 3) == 0.0)


def test_snr_of_white_noise_is_unit_variance():
    rng = np.random.default_rng(11)
    y = np.round(rng.standard_normal(200_000) * 30).astype(np.int32)
    for w in (1, 4, 32):
        s = oracle.boxcar_snr(y, w)
        assert abs(float(np.std(s)) - 1.0) < 0.02


def test_best_snr_prefers_smaller_width_on_ties():
    y = np.array([0, 0, 5, 0, 0, 0], dtype=np.int32)
    best, bw = oracle.best_snr(y, [1, 2, 4])
    # at t=2: w=1 -> 5/s, w=2 -> 5/(s*sqrt2), w=4 -> 5/(2s): w=1 wins
    assert bw[0, 2] == 1
    # at t=1: w=1 -> 0, w=2 -> 5/(s sqrt2), w=4 -> 5/(2s) => w=2
    assert bw[0, 1] == 2
    # last cells only have the widths that fit
    assert bw[0, 5] == 1


def test_find_peaks_hand_built_map():
    best = np.zeros((5, 8), dtype=np.float32)
    bw = np.ones((5, 8), dtype=np.int32)
    # group A: L-shape, max 9 at (1,2)
    best[0, 1] = 6.0
    best[1, 1] = 7.0
    best[1, 2] = 9.0
    # group B: diagonal neighbour of A only -> separate group
    best[2, 3] = 6.5
    # group C: tie between (4,6) and (4,7) -> earlier t wins; 5.999 excluded
    best[4, 6] = 8.0
    best[4, 7] = 8.0
    best[3, 7] = 5.999
    bw[4, 6] = 4
    c = oracle.find_peaks(best, bw, 6.0)
    got = [(int(r["d"]), int(r["t"]), int(r["w"]), float(r["snr"]), int(r["ncells"])) for r in c]
    assert got == [(1, 2, 1, 9.0, 3), (2, 3, 1, 6.5, 1), (4, 6, 4, 8.0, 2)]


def test_find_peaks_tie_prefers_lower_dm():
    best = np.zeros((3, 3), dtype=np.float32)
    best[1, 2] = 7.0
    best[2, 2] = 7.0
    best[2, 1] = 7.0
    c = oracle.find_peaks(best, np.ones_like(best, dtype=np.int32), 6.0)
    assert len(c) == 1 and (c[0]["d"], c[0]["t"], c[0]["ncells"]) == (1, 2, 3)


def test_snippet_hand_computed():
    n = 300
    y = np.zeros((3, n), dtype=np.int32)
    y[1, 100:104] = [4, 4, -2, 6]
    y[1, 200] = 10
    ss = np.array([oracle.sumsq(r) for r in y], dtype=np.int64)
    snip = oracle.snippets(y, ss, [1], [100], [4])
    f = oracle.bf16_bits_to_float(snip[0])
    sig = np.sqrt(ss[1] / n)
    # row index 32 holds DM row 1; bin 32 starts at t=100 and sums 4+4-2+6
    exact = 12 / (sig * 2)
    assert abs(f[32, 32] - exact) <= 2.0**-8 * exact   # within bf16 rounding
    # bin 57 covers t = 200..203 -> 10
    assert abs(f[32, 57] - 10 / (sig * 2)) <= 2.0**-8 * 10 / (sig * 2)
    # rows 31 and 33 are DM rows 0 and 2 with zero variance -> 0; rows outside -> 0
    assert np.all(f[31] == 0) and np.all(f[33] == 0) and np.all(f[:31] == 0) and np.all(f[34:] == 0)
    # every other bin of row 32 is zero
    mask = np.ones(64, bool)
    mask[[32, 57]] = False
    assert np.all(f[32, mask] == 0)


def test_bf16_rounding_is_nearest_even():
    # 1 + 2^-8 is halfway between two bf16 values: ties to even -> 1.0
    y = np.zeros((1, 64), dtype=np.int32)
    y[0, 0] = 1
    # sigma = sqrt(1/64) = 1/8; bin value = 1/(1/8) = 8 exactly
    snip = oracle.snippets(y, np.array([1], dtype=np.int64), [0], [0], [1])
    assert oracle.bf16_bits_to_float(snip[0, 32, 32]) == 8.0
