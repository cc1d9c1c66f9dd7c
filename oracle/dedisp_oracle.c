/*
 * Dedispersion oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU statement of direct incoherent
 * dedispersion (paper Section 2.2, "Incoherent dedispersion": every trial DM
 * is a complete integration over the frequency channels; the "direct"
 * algorithm).  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load this file's library.  It shares no code, header
 * or table with the CUDA path and must never be linked into it.
 *
 * The paper describes the frequency-dependent dispersive delay in words only
 * (Section 2.2); the formula applied here is the standard cold-plasma delay
 *
 *     delay[d][c] = round( 4.148808e3 s * DM_d * (f_c^-2 - f_max^-2) / t_samp )
 *
 * with f in MHz, DM in pc cm^-3, t_samp in seconds, f_max the largest channel
 * frequency, and round = half away from zero (C's llround).  f^-2 is evaluated
 * as 1.0/(f*f) and the product left to right, in double precision.
 *
 * Input layout: 2-bit samples (paper Section 1: filterbank data stored with
 * 2 bits per sample), channel-major, 4 samples per byte along time, the
 * earliest sample in the least-significant bits.  Sample t of channel c is
 * bits 2*(t%4)..2*(t%4)+1 of byte c*ld_in + t/4.
 *
 * Output: out[d][t] = sum over channels c of x[c][t + delay[d][c]] as an
 * exact uint32, for 0 <= t < nsamp_in - maxdelay, maxdelay = max over the
 * whole table.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

/* The dispersion constant in seconds * MHz^2 / (pc cm^-3). */
#define ORACLE_KDM 4.148808e3

int oracle_delay_table(int nchan, const double *freqs_mhz, double tsamp_s,
                       int ndm, const double *dms, int32_t *delays)
{
    if (nchan <= 0 || ndm <= 0 || !freqs_mhz || !dms || !delays || !(tsamp_s > 0))
        return -1;
    double fmax = freqs_mhz[0];
    for (int c = 1; c < nchan; ++c)
        if (freqs_mhz[c] > fmax) fmax = freqs_mhz[c];
    for (int d = 0; d < ndm; ++d) {
        for (int c = 0; c < nchan; ++c) {
            double f = freqs_mhz[c];
            double v = ORACLE_KDM * dms[d] * (1.0 / (f * f) - 1.0 / (fmax * fmax)) / tsamp_s;
            delays[(size_t)d * nchan + c] = (int32_t)llround(v);
        }
    }
    return 0;
}

int32_t oracle_max_delay(int nchan, int ndm, const int32_t *delays)
{
    int32_t m = 0;
    for (size_t i = 0; i < (size_t)nchan * ndm; ++i)
        if (delays[i] > m) m = delays[i];
    return m;
}

/* One 2-bit sample, read straight from the packed layout described above. */
static unsigned sample_at(const uint8_t *in, size_t ld_in, int c, size_t t)
{
    unsigned byte = in[(size_t)c * ld_in + t / 4];
    return (byte >> (2 * (t % 4))) & 3u;
}

/* Full dedispersion: out must hold ndm rows of ld_out uint32. */
int oracle_dedisperse(int nchan, int ndm, const int32_t *delays,
                      const uint8_t *in, size_t ld_in, size_t nsamp_in,
                      uint32_t *out, size_t ld_out)
{
    int32_t maxdelay = oracle_max_delay(nchan, ndm, delays);
    if ((size_t)maxdelay >= nsamp_in) return -4;
    size_t nout = nsamp_in - (size_t)maxdelay;
    if (ld_out < nout) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        uint32_t *row = out + (size_t)d * ld_out;
        memset(row, 0, nout * sizeof(uint32_t));
        for (int c = 0; c < nchan; ++c) {
            size_t shift = (size_t)delays[(size_t)d * nchan + c];
            for (size_t t = 0; t < nout; ++t)
                row[t] += sample_at(in, ld_in, c, t + shift);
        }
    }
    return 0;
}

/* The same sum at selected (DM index, output sample) points only. */
int oracle_dedisperse_points(int nchan, int ndm, const int32_t *delays,
                             const uint8_t *in, size_t ld_in, size_t nsamp_in,
                             size_t npts, const int32_t *d_idx,
                             const int64_t *t_idx, uint32_t *vals)
{
    int32_t maxdelay = oracle_max_delay(nchan, ndm, delays);
    if ((size_t)maxdelay >= nsamp_in) return -4;
    size_t nout = nsamp_in - (size_t)maxdelay;
    for (size_t p = 0; p < npts; ++p) {
        if (d_idx[p] < 0 || d_idx[p] >= ndm || t_idx[p] < 0 || (size_t)t_idx[p] >= nout)
            return -1;
    }
#pragma omp parallel for schedule(static)
    for (long long p = 0; p < (long long)npts; ++p) {
        int d = d_idx[p];
        size_t t = (size_t)t_idx[p];
        uint32_t s = 0;
        for (int c = 0; c < nchan; ++c)
            s += sample_at(in, ld_in, c, t + (size_t)delays[(size_t)d * nchan + c]);
        vals[p] = s;
    }
    return 0;
}

/* Threads the OpenMP runtime will use (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Time-major 2-bit data (sample t's channels consecutive, channel c in bits
 * 2(c%4) of byte t*ld_tm + c/4) to the channel-major rows dedispersion reads
 * (sample t in bits 2(t%4) of byte c*ld_cm + t/4); padding samples are 0. */
int oracle_corner_turn(const uint8_t *tm, size_t ld_tm, int nchan, size_t nsamp, uint8_t *cm, size_t ld_cm)
{
    if (nchan <= 0 || ld_tm * 4 < (size_t)nchan || ld_cm * 4 < nsamp) return -1;
    memset(cm, 0, (size_t)nchan * ld_cm);
    for (size_t t = 0; t < nsamp; ++t)
        for (int c = 0; c < nchan; ++c) {
            const unsigned v = (tm[t * ld_tm + (size_t)c / 4] >> (2 * (c % 4))) & 3u;
            cm[(size_t)c * ld_cm + t / 4] |= (uint8_t)(v << (2 * (t % 4)));
        }
    return 0;
}
