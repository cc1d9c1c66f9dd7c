/*
 * Measurement probes: a separate library (libddprobe.so) that the tests and
 * the benchmark's roofline figures load.  It is not part of the product
 * library libdd.so and nothing in libdd.so calls it.  The paper has no
 * counterpart to any of these; they measure the GPU at hand.
 *
 * Every call is synchronous on the current device, allocates and frees its
 * own small device buffers, and returns DD_OK or a dd_status error whose
 * message dd_probe_last_error() returns (thread-local).
 */
#ifndef DD_PROBE_H
#define DD_PROBE_H

#include "../../../include/dd.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Measured integer issue rates of the current GPU in tera-operations per
 * second, for the roofline of the dedispersion kernel (its additions are
 * integer work; the paper has no counterpart): tops[0] 3-input logic ops,
 * tops[1] 32-bit additions (the compiler may fuse two into one instruction),
 * tops[2] integer multiply-adds, tops[3] an even logic / multiply-add mix.
 * Synchronous; allocates and frees a small device buffer.
 */
dd_status dd_probe_int_rates(double *tops);

/*
 * Float FMA issue rates (no paper counterpart; they back the classifier's
 * kernel choice): tops[0] single-precision FMAs per second (T) from scalar
 * fma.rn.f32, tops[1] from packed fma.rn.f32x2 (two per instruction).
 * *mismatches counts, over 2^24 pseudo-random operand sets, packed results
 * that differ from fmaf's.  Synchronous; allocates small device buffers.
 */
dd_status dd_probe_fp_rates(double *tops, unsigned long long *mismatches);

/*
 * Tensor-core self-check (no paper counterpart; it backs the classifier's
 * tensor-core convolutions): D = A * B^T for bfloat16 A (128 x k, row-major,
 * host h_a) and B (n x k, row-major, host h_b) with a float accumulator, run
 * as k/16 tcgen05 MMAs of one CTA from shared-memory descriptors into tensor
 * memory; D (128 x n, row-major float) is written to host h_d.  n in 16..256
 * and k in 16..256, multiples of 16.  Synchronous; allocates and frees small
 * device buffers.  DD_ERR_TIMEOUT if the MMA completion was not observed.
 */
dd_status dd_probe_tc_gemm(const uint16_t *h_a, const uint16_t *h_b, float *h_d, int n, int k);

/*
 * The give-up path of the classifier's bounded tensor-core waits, run without
 * any fault (no paper counterpart): one CTA allocates tensor memory, waits
 * with at most poll_limit polls (1..2^20) on an mbarrier phase that never
 * completes, records the give-up of each of its 4 warps in *h_status (bit w:
 * warp w gave up), frees the tensor memory and returns.  Synchronous; returns
 * DD_ERR_TIMEOUT when a wait gave up (always, by construction), DD_OK never
 * in practice, DD_ERR_INVALID_ARG for bad arguments.
 */
dd_status dd_probe_wait_giveup(unsigned poll_limit, unsigned *h_status);

/*
 * The give-up path of the dedispersion tile's bounded stage waits, run
 * without any fault (no paper counterpart): one CTA dedisperses a 64-channel,
 * 16-trial, 1536-sample tile whose stage mbarriers expect one arrival more
 * than the stage copies make, so no stage ever completes; every wait stops
 * after poll_limit polls (1..2^20).  *h_err receives the tile's error word
 * (bit 0: gave up), *h_written the number of output words the tile wrote
 * (expected 0).  Synchronous; DD_ERR_TIMEOUT when the tile gave up (always, by
 * construction), DD_ERR_INVALID_ARG for bad arguments.
 */
dd_status dd_probe_tile_giveup(unsigned poll_limit, unsigned *h_err, long long *h_written);

/* Message of the calling thread's last failed probe call ("" if none). */
const char *dd_probe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DD_PROBE_H */
