/*
 * Multibeam coincidence RFI oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain CPU statement of the coincidence-rejection step of paper Section 2.1:
 * the beams of the multibeam receiver act as reference antennas, a sample is
 * flagged as interference when the signal exceeds k sigma in at least
 * min_beams beams (the paper's example: 3 sigma in 4 or more of 13 beams),
 * and the result is a boolean mask per sample, computed independently for
 * every sample.  Only the test-suite and the CPU legs of the benchmark load
 * this library; it shares nothing with the CUDA path.
 *
 * Readings (the paper gives the rule in words only):
 *  - The per-beam time series is the zero-DM sum z_b[t] = sum_c x_b[c][t] of
 *    the 2-bit levels, i.e. the beam's total power per sample.
 *  - Mean and standard deviation are those of the gulp: S1 = sum_t z_b[t],
 *    S2 = sum_t z_b[t]^2 over the n samples, mu = S1 / n,
 *    sigma^2 = S2 / n - mu^2.
 *  - "Exceeds k sigma" is z > mu + k sigma, decided exactly in integers:
 *    n z - S1 > 0 and (n z - S1)^2 > k^2 (n S2 - S1^2).
 *  - A masked sample is replaced, in every beam and channel, by the level
 *    1 + ((c + t) mod 2): the channel's mean level 1.5 over pairs of samples,
 *    keeping every dedispersed sum an integer.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>

static inline unsigned level(const uint8_t *row, size_t t) { return (row[t >> 2] >> (2 * (t & 3))) & 3u; }

/* z[t] = sum over the nchan rows (row stride ld bytes) of sample t. */
int oracle_zero_dm(const uint8_t *packed, int nchan, size_t ld, size_t nsamp, uint32_t *z)
{
    if (nchan <= 0 || ld * 4 < nsamp) return -1;
    for (size_t t = 0; t < nsamp; ++t) z[t] = 0;
    for (int c = 0; c < nchan; ++c) {
        const uint8_t *row = packed + (size_t)c * ld;
        for (size_t t = 0; t < nsamp; ++t) z[t] += level(row, t);
    }
    return 0;
}

/* mask[t] = 1 when at least min_beams of the nbeams series z ([nbeams][nsamp])
 * exceed their mean by more than k standard deviations; *nmasked counts them. */
int oracle_rfi_mask(const uint32_t *z, int nbeams, size_t nsamp, int k, int min_beams, uint8_t *mask,
                    int64_t *nmasked)
{
    if (nbeams <= 0 || nsamp == 0 || k < 0 || min_beams <= 0) return -1;
    int64_t s1[64];
    unsigned __int128 lim[64];
    if (nbeams > 64) return -1;
    const int64_t n = (int64_t)nsamp;
    for (int b = 0; b < nbeams; ++b) {
        int64_t a = 0;
        unsigned __int128 q = 0;
        for (size_t t = 0; t < nsamp; ++t) {
            const uint32_t v = z[(size_t)b * nsamp + t];
            a += v;
            q += (unsigned __int128)((uint64_t)v * v);
        }
        s1[b] = a;
        /* n S2 - S1^2 >= 0 (Cauchy-Schwarz) */
        const unsigned __int128 var_n = (unsigned __int128)n * q - (unsigned __int128)a * (unsigned __int128)a;
        lim[b] = (unsigned __int128)((int64_t)k * k) * var_n;
    }
    int64_t cnt = 0;
    for (size_t t = 0; t < nsamp; ++t) {
        int over = 0;
        for (int b = 0; b < nbeams; ++b) {
            const int64_t dev = n * (int64_t)z[(size_t)b * nsamp + t] - s1[b];
            if (dev > 0 && (unsigned __int128)dev * (unsigned __int128)dev > lim[b]) ++over;
        }
        mask[t] = (uint8_t)(over >= min_beams);
        cnt += mask[t];
    }
    *nmasked = cnt;
    return 0;
}

/* Replace the masked samples of one beam's rows by 1 + ((c + t) mod 2). */
int oracle_rfi_apply(uint8_t *packed, int nchan, size_t ld, size_t nsamp, const uint8_t *mask)
{
    if (nchan <= 0 || ld * 4 < nsamp) return -1;
    for (int c = 0; c < nchan; ++c) {
        uint8_t *row = packed + (size_t)c * ld;
        for (size_t t = 0; t < nsamp; ++t) {
            if (!mask[t]) continue;
            const unsigned v = 1u + (unsigned)((c + t) & 1);
            const unsigned sh = 2 * (unsigned)(t & 3);
            row[t >> 2] = (uint8_t)((row[t >> 2] & ~(3u << sh)) | (v << sh));
        }
    }
    return 0;
}
