/*
 * dd.h -- C ABI of the GB300 (sm_103a) direct-dedispersion library.
 *
 * The library implements the hot path of the real-time transient pipeline of
 * Barsdell, Bailes, Barnes & Fluke, "Spotting Radio Transients with the help
 * of GPUs" (ADASS XXI): direct incoherent dedispersion of 2-bit filterbank
 * data (Section 2.2), followed by the search steps of Section 2.3 (baseline
 * removal, boxcar matched filtering, sigma-cut peak finding with grouping of
 * contiguous regions), a learned candidate classifier and a streaming server.
 *
 * Conventions shared by every entry point
 *  - Plain C types only.  Pointers documented "device" must point to CUDA
 *    device memory of the current device; "host" pointers to host memory.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  Work is enqueued asynchronously on it unless stated.
 *  - Argument errors are detected on the host before anything is launched and
 *    returned as a dd_status; nothing is enqueued then.  CUDA failures are
 *    returned as DD_ERR_CUDA.  dd_last_error() gives a message for the most
 *    recent failure on the calling thread.  No C++ exception crosses the ABI.
 *  - The caller owns every buffer it passes; handles (plans, batches, search
 *    and classifier contexts, servers) own what they allocate and free it in
 *    their destroy call, which accepts NULL.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dd_status {
    DD_OK = 0,
    DD_ERR_INVALID_ARG = -1, /* a pointer, size, ordering or alignment rule broken */
    DD_ERR_NOMEM = -2,       /* a device or host allocation failed */
    DD_ERR_CUDA = -3,        /* a CUDA runtime call failed (message in dd_last_error) */
    DD_ERR_TOO_SHORT = -4,   /* input shorter than or equal to the plan's maximum delay */
    DD_ERR_TIMEOUT = -5,     /* a bounded device or host wait ran out */
    DD_ERR_INTERNAL = -6,    /* an internal consistency check failed */
    DD_ERR_BUSY = -7         /* no capacity right now (server admission); retry later */
} dd_status;

/* Human-readable name of a status code (static string). */
const char *dd_status_string(dd_status s);

/* Message for the most recent failure on the calling thread (static per
 * thread; valid until the thread's next failing call). */
const char *dd_last_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int dd_version(void);

/* ------------------------------------------------------------------------ */
/* Delay table (paper Section 2.2: the dispersive delay grows with the free  */
/* electron column, the DM, and with falling frequency).                      */
/* ------------------------------------------------------------------------ */

/*
 * Dispersive delays in whole samples, computed on the host in double:
 *
 *   delay[d][c] = round(4.148808e3 * dms[d] * (1/(f_c*f_c) - 1/(f_max*f_max)) / tsamp_s)
 *
 * freqs_mhz: host, nchan channel frequencies in MHz, strictly descending
 *            (channel 0 is the highest, so f_max = freqs_mhz[0]).
 * dms:       host, ndm trial DMs in pc cm^-3, finite, >= 0, non-decreasing.
 * out:       host, ndm*nchan int32, row-major [d][c].
 * round is half away from zero.  Errors: DD_ERR_INVALID_ARG for NULL
 * pointers, nchan/ndm <= 0, tsamp_s not > 0, unsorted or non-finite inputs,
 * or a delay that does not fit in int32.
 */
dd_status dd_compute_delays(int nchan, const double *freqs_mhz, double tsamp_s, int ndm,
                            const double *dms, int32_t *out);

/* ------------------------------------------------------------------------ */
/* Plans and single-gulp dedispersion                                        */
/* ------------------------------------------------------------------------ */

typedef struct dd_plan dd_plan;

/* Kernel selection for a plan. */
enum {
    DD_KERNEL_AUTO = 0,   /* the tiled sm_103a kernel, shape from the autotuner */
    DD_KERNEL_SIMPLE = 1, /* one thread per (DM, 4 samples), global loads; for checking */
    DD_KERNEL_TILED = 2   /* the tiled kernel with the shape given in dd_options */
};

typedef struct dd_options {
    int kernel;          /* DD_KERNEL_* */
    int dms_per_block;   /* tiled kernel: DM trials per CTA (0 = tuned) */
    int words_per_thread;/* tiled kernel: 16-sample words per thread along time (0 = tuned) */
    int chan_chunk;      /* tiled kernel: channels per shared-memory stage, 32, 64 or 128
                            (0 = tuned; bands of 2048 channels or more use 64) */
    int reserved;        /* must be 0 */
    const char *tune_cache_path; /* autotune cache file (NULL = none) */
} dd_options;

/*
 * Create a plan: validates the band and the DM list, computes the delay
 * table (as dd_compute_delays) and uploads it to the current device, where it
 * stays for the plan's lifetime.
 * out:  host, receives the plan (NULL on failure).
 * opt:  host, may be NULL (all defaults).
 * Errors: DD_ERR_INVALID_ARG (as dd_compute_delays, or bad options),
 * DD_ERR_NOMEM / DD_ERR_CUDA (device upload).
 */
dd_status dd_plan_create(dd_plan **out, int nchan, const double *freqs_mhz, double tsamp_s,
                         int ndm, const double *dms, const dd_options *opt);

/* Sizes of a plan: channels, DM trials, largest delay in samples. */
dd_status dd_plan_info(const dd_plan *plan, int *nchan, int *ndm, int *maxdelay);

/* Copy the plan's delay table to host memory (ndm*nchan int32, [d][c]). */
dd_status dd_plan_delay_table(const dd_plan *plan, int32_t *host_out);

/* The tiled kernel's shape chosen for this plan (after tuning, if any). */
dd_status dd_plan_kernel_shape(const dd_plan *plan, int *kernel, int *dms_per_block,
                               int *words_per_thread, int *chan_chunk);

/*
 * Run the autotuner for this plan on a gulp of nsamp_in samples: times the
 * candidate tile shapes -- DM trials per CTA x 16-sample words per thread (8
 * pairs) x channels per shared-memory stage (32, 64, 128) -- on `stream` with
 * scratch buffers it allocates and frees, keeps the fastest, and writes it to
 * opt->tune_cache_path if one was given at plan creation.  The tables of the
 * other shapes are freed, unless a batch built on this plan still points at
 * them (they then live until dd_destroy).  Synchronous.  Returns the best
 * time in *best_ms (0 when the shape came from the cache).
 */
dd_status dd_plan_autotune(dd_plan *plan, size_t nsamp_in, void *stream, float *best_ms);

/*
 * Direct dedispersion of one gulp (paper Section 2.2):
 *
 *   out[d][t] = sum_{c < nchan} x[c][t + delay[d][c]],  0 <= t < nsamp_in - maxdelay
 *
 * as exact uint32 sums.
 * d_in:   device, nchan rows of ld_in_bytes bytes; sample t of channel c is
 *         bits 2*(t%4)..2*(t%4)+1 of byte d_in[c*ld_in_bytes + t/4] (4 samples
 *         per byte, earliest in the least-significant bits).  d_in must be
 *         16-byte aligned and ld_in_bytes a multiple of 16 that is at least
 *         ceil(nsamp_in/4); bytes past the last sample are read but ignored.
 * d_out:  device, ndm rows of ld_out uint32, ld_out >= nsamp_in - maxdelay,
 *         d_out 16-byte aligned and ld_out a multiple of 4.  Only the first
 *         nsamp_in - maxdelay entries of each row are written.
 * Errors: DD_ERR_TOO_SHORT if nsamp_in <= maxdelay; DD_ERR_INVALID_ARG for
 * NULL pointers or broken layout rules.  The call is asynchronous on stream.
 * A plan is read-only during execution: concurrent calls on different streams
 * with different outputs are safe.
 */
dd_status dd_execute(const dd_plan *plan, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                     uint32_t *d_out, size_t ld_out, void *stream);

/*
 * The same with HOST buffers: h_in (nchan*ld_in_bytes, pinned memory gives
 * the full copy rate) is copied to plan-owned device staging, dedispersed,
 * and the result copied back to h_out (ndm rows of ld_out uint32).
 * Synchronous: returns after the result is in h_out.
 */
dd_status dd_execute_host(dd_plan *plan, const uint8_t *h_in, size_t ld_in_bytes, size_t nsamp_in,
                          uint32_t *h_out, size_t ld_out, void *stream);

/* Free a plan and its device memory (NULL-safe).  Work that uses the plan
 * must have completed. */
void dd_destroy(dd_plan *plan);

/*
 * Device-side error flags of the tiled dedispersion kernels (dd_execute,
 * dd_execute_host, batches, dd_execute_noalloc) on the current device, read
 * and cleared: bit 0 means some tile stopped waiting for its channel windows
 * (copied into shared memory by the copy engine) after a fixed poll limit,
 * and left its outputs unwritten.  Synchronises the device first.
 * Errors: DD_ERR_INVALID_ARG for a NULL flags, DD_ERR_CUDA.
 */
dd_status dd_dedisp_status(unsigned *flags);

/* ------------------------------------------------------------------------ */
/* Multi-beam batches: many gulps in one persistent launch                   */
/* ------------------------------------------------------------------------ */

/*
 * One beam's gulp in a batch.  The paper's receiver has 13 beams (Section 1)
 * and its goal is real-time processing of all of them (Section 3); a batch
 * dedisperses the gulps of several beams -- each with its own plan, DM range
 * and gulp length -- in one launch of a persistent kernel whose CTAs take
 * output tiles from a global work counter.
 * plan:  the beam's plan (not const: the batch may add the tile tables of its
 *        kernel shape to the plan).
 * d_in, ld_in_bytes, nsamp_in, d_out, ld_out: as for dd_execute.
 */
typedef struct dd_beam {
    dd_plan *plan;
    const uint8_t *d_in;
    size_t ld_in_bytes;
    size_t nsamp_in;
    uint32_t *d_out;
    size_t ld_out;
} dd_beam;

typedef struct dd_batch dd_batch;

/* Largest number of beams in one batch. */
#define DD_BATCH_MAX_BEAMS 64

/*
 * Create a batch for nbeams (1..DD_BATCH_MAX_BEAMS) beams.  All beams run the
 * tiled kernel with one tile shape (the first beam's plan's shape).  With
 * use_graph != 0 the launch (work-counter reset + persistent kernel) is
 * captured once in a CUDA graph and replayed by dd_batch_launch.  The beam
 * descriptors are uploaded synchronously.  The batch owns its device
 * descriptor block and work counter; its descriptors point at the plans'
 * tables, so every plan of the batch must outlive it (dd_plan_autotune on
 * such a plan keeps those tables).  The input and output buffers belong to
 * the caller and must stay valid while launches may run.
 * Errors: DD_ERR_INVALID_ARG (as dd_execute for any beam, or a plan that uses
 * the simple kernel), DD_ERR_NOMEM, DD_ERR_CUDA.
 */
dd_status dd_batch_create(dd_batch **out, int nbeams, const dd_beam *beams, int use_graph);

/*
 * Replace the beams of a batch (count, buffers, lengths; plans must keep the
 * batch's tile shape).  The new descriptors are copied to the device on
 * `stream`, so launches enqueued later on the same stream see them; no graph
 * re-capture is needed.  Launches on other streams must be ordered by the
 * caller.
 */
dd_status dd_batch_set(dd_batch *batch, int nbeams, const dd_beam *beams, void *stream);

/* Enqueue one batched dedispersion of every beam on `stream` (graph replay
 * when the batch was created with use_graph). */
dd_status dd_batch_launch(dd_batch *batch, void *stream);

/* Batch facts: beams, output tiles, persistent grid size, tile shape. */
dd_status dd_batch_info(const dd_batch *batch, int *nbeams, long long *ntiles, int *grid, int *dms_per_block,
                        int *words_per_thread);

/* Free a batch (NULL-safe).  Its launches must have completed. */
void dd_batch_destroy(dd_batch *batch);

/* One-shot batch without a graph: create, launch on `stream`, wait for it,
 * destroy.  Synchronous. */
dd_status dd_execute_batch(int nbeams, const dd_beam *beams, void *stream);

/* ------------------------------------------------------------------------ */
/* Search stage (paper Section 2.3)                                          */
/* ------------------------------------------------------------------------ */

/* Largest number of groups (candidates) a search context can hold. */
#define DD_SEARCH_MAX_CANDS (1 << 20)
/* Largest number of boxcar widths. */
#define DD_SEARCH_MAX_WIDTHS 16

/* One event: a group of 4-connected (DM, time) cells whose best boxcar S/N
 * reached the threshold, reported at its cell of largest S/N (ties: lower DM
 * index, then earlier sample). */
typedef struct dd_candidate {
    int32_t beam;     /* tag passed to dd_search_run */
    int32_t d;        /* DM trial index of the representative cell */
    int32_t t;        /* output sample of the representative cell */
    int32_t w;        /* boxcar width (samples) giving its S/N */
    float snr;        /* S/N of the representative cell */
    float score;      /* classifier logit when scored by a server, else 0 */
    int64_t ncells;   /* cells in the group */
} dd_candidate;

typedef struct dd_search_config {
    int ndm_max;       /* capacity: DM rows */
    size_t n_max;      /* capacity: samples per row (ndm_max * n_max < 2^31) */
    int nchan;         /* channels summed into each value: values lie in 0..3*nchan (nchan <= 21844) */
    int half_window;   /* baseline window [t - half_window, t + half_window) (clipped to the row), 1..32767 */
    int nwidths;       /* number of boxcar widths, 1..DD_SEARCH_MAX_WIDTHS */
    int widths[DD_SEARCH_MAX_WIDTHS]; /* ascending powers of two <= 1024 */
    float thresh;      /* S/N threshold (cells with S/N >= thresh are hot) */
    int max_cands;     /* candidate capacity, 1..DD_SEARCH_MAX_CANDS */
    int full_map;      /* 1: store best S/N and width for every cell; 0: only for hot cells */
    int baseline;      /* 0: running lower median; 1: the paper's running mean (Section 2.3),
                          rounded half up: y = x - floor((S + floor(m/2)) / m) for the window's
                          sum S of its m values */
} dd_search_config;

typedef struct dd_search dd_search;

/*
 * Create a search context owning its device buffers: baseline-removed rows y
 * (int32, ndm_max*n_max), per-row sum of y^2 (int64), per-cell best S/N
 * (float) and its width (uint16), group labels (int32), a hot-cell bitmask and
 * the candidate lists.  Errors: DD_ERR_INVALID_ARG, DD_ERR_NOMEM.
 */
dd_status dd_search_create(dd_search **out, const dd_search_config *cfg);

/*
 * Run the search on ndm dedispersed rows of n samples (d_x: device, uint32,
 * row stride ld_x >= n), asynchronously on stream:
 *  1. baseline (Section 2.3 removes a running mean; the default is the robust
 *     running lower median): y[t] = x[t] - median(x[t-h .. t+h-1] clipped to
 *     the row), or with baseline = 1 x[t] minus the window mean rounded half
 *     up; exact int32;
 *  2. sigma_d = sqrt(sum_t y^2 / n) per row (sum exact in int64, rest double);
 *  3. matched filter (Section 2.3: boxcars of growing width): for each width w
 *     S_w[t] = sum_{i<w} y[t+i] for t + w <= n, snr = (float)S_w /
 *     (float)(sigma_d*sqrt(w)) (0 for a constant row); per cell the largest
 *     snr over the widths (ties keep the smaller width; -inf and width 0 where
 *     no width fits before the row end);
 *  4. peak finding (Section 2.3: sigma cut, then contiguous regions grouped
 *     into events): cells with snr >= thresh grouped by 4-connectivity in
 *     (DM, time), one dd_candidate per group, sorted by (d, t).
 * `beam` is copied into the candidates.  Results are exact and deterministic
 * while the number of groups stays <= max_cands (see dd_search_result).
 */
dd_status dd_search_run(dd_search *search, const uint32_t *d_x, size_t ld_x, int ndm, size_t n, int beam,
                        void *stream);

/* Counts of the last run (synchronises stream): hot cells, groups found, and
 * flags: bit 0 = a value beyond 3*nchan was clipped, bit 2 = union-find retry
 * cap reached (bit 1 is unused). */
dd_status dd_search_result(const dd_search *search, long long *nhot, int *ngroups, unsigned *flags, void *stream);

/* Work counters of the last run (synchronises stream): how many times a lane
 * of the running-median baseline recounted its histogram from the window
 * (its median had walked to an edge of the counted range; 0 with the mean
 * baseline).  NULL pointers are skipped. */
dd_status dd_search_stats(const dd_search *search, long long *median_rebuilds, void *stream);

/* Copy up to max sorted candidates to host memory; *count = candidates
 * available (min(groups, max_cands)).  Synchronises stream. */
dd_status dd_search_candidates(const dd_search *search, dd_candidate *host_out, int max, int *count, void *stream);

/* Device pointer to the sorted candidate list (valid until the next run). */
dd_status dd_search_device_candidates(const dd_search *search, const dd_candidate **d_cands);

/* Device pointers to the context's buffers (row stride n of the last run). */
dd_status dd_search_buffers(const dd_search *search, const int32_t **d_y, const int64_t **d_sumsq,
                            const float **d_best, const uint16_t **d_bestw);

/*
 * DM-time snippets for a classifier: for each of ncand candidates (device
 * list), 64 DM rows (d-32 .. d+31) x 64 bins of w samples, bin k starting at
 * t + (k-32)*w; a bin is (float)(sum of the row's y samples inside the data)
 * / (float)(sigma_row*sqrt(w)), rounded to bfloat16 (nearest even); rows
 * outside 0..ndm-1 or with sigma 0 are 0.  d_out: device, ncand*64*64
 * bfloat16 bit patterns.  Widths must be powers of two.
 */
dd_status dd_snippets(const int32_t *d_y, size_t ld_y, int ndm, size_t n, const int64_t *d_sumsq, int ncand,
                      const dd_candidate *d_cands, uint16_t *d_out, void *stream);

/* dd_snippets on a search context's own buffers and first ncand candidates. */
dd_status dd_search_snippets(const dd_search *search, int ncand, uint16_t *d_out, void *stream);

/* Free a search context (NULL-safe).  Its work must have completed. */
void dd_search_destroy(dd_search *search);

/* ------------------------------------------------------------------------ */
/* Candidate classifier                                                      */
/* ------------------------------------------------------------------------ */

/*
 * A small CNN scoring 64x64 bfloat16 DM-time snippets (dd_snippets) as
 * astrophysical (logit > 0) or interference/noise; the paper motivates
 * separating true signals from RFI (Section 2.1) but has no classifier, so
 * the network is this library's own.
 *
 * Parameters: DD_NN_PARAMS floats, in this order: conv1 w[16][1][3][3] b[16],
 * conv2 w[32][16][3][3] b[32], conv3 w[64][32][3][3] b[64], conv4
 * w[64][64][3][3] b[64], fc1 w[128][1024] b[128], fc2 w[1][128] b[1].  Each conv
 * is 3x3, zero padding 1, then ReLU and 2x2 max pooling; conv4's [64][4][4]
 * output is flattened as c*16 + y*4 + x; fc1 has a ReLU.
 * Numerics: weights and activations are bfloat16 (nearest-even rounding of the
 * float master weights and of every post-ReLU activation), sums are float,
 * accumulated from the bias in increasing (channel, ky, kx) / input order;
 * pooling keeps the first maximum.  Training minimises the mean binary
 * cross-entropy with logits with float gradients (each bfloat16 rounding
 * treated as the identity) and AdamW on the float master copy.
 */
#define DD_NN_PARAMS 191553

typedef struct dd_nn dd_nn;

/* Create a classifier for batches of up to max_batch snippets; parameters
 * and optimiser state start at zero. */
dd_status dd_nn_create(dd_nn **out, int max_batch);

/* Set the float master parameters from host memory (DD_NN_PARAMS floats);
 * resets the AdamW moments and step count.  Synchronous. */
dd_status dd_nn_set_params(dd_nn *nn, const float *h_master);

/* Copy the float master parameters to host memory.  Synchronous. */
dd_status dd_nn_get_params(const dd_nn *nn, float *h_master);

/* Logits of n snippets (d_x: device, n*64*64 bfloat16 bit patterns, 4-byte
 * aligned) into d_logits (device, n floats; may be NULL to keep them
 * internal).  CUDA-core
 * kernels with a fixed summation order: every sum starts at the bias and adds
 * products in (input channel, ky, kx) / input order with one rounding per
 * step, so the logits are reproducible bit for bit and equal a float CPU
 * evaluation in that order (the forward that training uses). */
dd_status dd_nn_forward(dd_nn *nn, const uint16_t *d_x, int n, float *d_logits, void *stream);

/* The same network with the convolutions on the tensor cores (tcgen05 implicit
 * GEMM, bf16 x bf16 -> fp32 in the tensor cores' own summation order; d_x
 * 16-byte aligned).  Sums differ from dd_nn_forward's by float round-off,
 * which now and then moves a bfloat16-rounded activation by one unit; the
 * logits therefore agree to about 1e-2, not bit for bit.  An MMA whose
 * completion is not observed sets a flag read by dd_nn_status. */
dd_status dd_nn_forward_tc(dd_nn *nn, const uint16_t *d_x, int n, float *d_logits, void *stream);

/* Error flags of the tensor-core forward (bit 0: an MMA completion was not
 * observed within the wait limit).  Synchronous. */
dd_status dd_nn_status(const dd_nn *nn, unsigned *flags);

/* Forward + backward on n snippets with labels in {0,1} (d_labels: device, n
 * floats): the mean loss and the gradients stay on the device. */
dd_status dd_nn_backward(dd_nn *nn, const uint16_t *d_x, const float *d_labels, int n, void *stream);

/* Copy the gradients (DD_NN_PARAMS floats) / the last loss to host memory
 * (synchronise stream).  dd_nn_set_grads overwrites the device gradients. */
dd_status dd_nn_get_grads(const dd_nn *nn, float *h_grads, void *stream);
dd_status dd_nn_set_grads(dd_nn *nn, const float *h_grads);
dd_status dd_nn_get_loss(const dd_nn *nn, float *h_loss, void *stream);

/* One AdamW step with the current gradients:
 * m = b1*m + (1-b1)*g; v = b2*v + (1-b2)*g*g; w -= lr*((m/c1)/(sqrt(v/c2)+eps) + wd*w),
 * c1 = 1-b1^t, c2 = 1-b2^t (t counts steps from 1); refreshes the bfloat16 copy. */
dd_status dd_nn_adamw(dd_nn *nn, float lr, float beta1, float beta2, float eps, float wd, void *stream);

/* Optimiser state for inspection: moments (floats), the bfloat16 weights the
 * forward pass uses (bit patterns) and the step count; NULL outputs skipped. */
dd_status dd_nn_get_state(const dd_nn *nn, float *h_m, float *h_v, uint16_t *h_bf16, int *step);

/* Checkpoint: magic "DDNNCKP1", int64 parameter count, int64 step, then the
 * float master weights, first and second moments (little-endian). */
dd_status dd_nn_save(const dd_nn *nn, const char *path);
dd_status dd_nn_load(dd_nn *nn, const char *path);

/* Free a classifier (NULL-safe). */
void dd_nn_destroy(dd_nn *nn);

/* ------------------------------------------------------------------------ */
/* Streaming server                                                          */
/* ------------------------------------------------------------------------ */

/*
 * Real-time serving of many beams (the paper's goal of processing the 13-beam
 * receiver's data as it arrives, Sections 1 and 3): each beam is a stream of
 * gulps of gulp_nsamp new 2-bit samples.  Per beam the device carries the
 * last L >= maxdelay input samples from gulp to gulp, so the dedispersed
 * outputs of successive gulps join into exactly the one-shot result: gulp k
 * yields absolute outputs [k*G - maxdelay, (k+1)*G - maxdelay) (gulp 0:
 * [0, G - maxdelay)), G = gulp_nsamp.  Each gulp is then searched
 * (dd_search_run on its outputs; the baseline window is clipped at the gulp's
 * edges) and its candidates scored by the classifier when one is loaded.
 *
 * Gulps are admitted as they are submitted: each runs on an execution slot
 * (stream + buffers); slots are created on demand while free device memory
 * stays above hbm_reserve_bytes plus one slot's needs, up to max_slots.
 * Gulps of different beams run concurrently; gulps of one beam are ordered on
 * the device.  Results come back through dd_server_poll in completion order.
 */
/*
 * Triggered dumps (paper Sections 1 and 3: a buffer of the raw data kept for
 * a short time and saved around events of interest).  The server keeps each
 * beam's input window on the device; when a gulp's candidate reaches the
 * trigger S/N, the raw 2-bit rows of its sweep are copied out before the
 * window is reused and handed to the callback on the server's worker thread.
 */
typedef struct dd_trigger {
    int beam;
    int nchan;
    long long seq;      /* gulp of the beam */
    dd_candidate cand;  /* the candidate that fired (score 0: scores come later) */
    long long t0;       /* absolute input sample of the dump's first sample (< 0: before the stream, zeros) */
    long long nsamp;    /* samples per channel in the dump: maxdelay + 1024 rounded up to 64 */
    size_t ld;          /* bytes per channel row of the dump (nsamp / 4) */
} dd_trigger;

/* raw: nchan rows of ld bytes packed as dd_execute's input; valid during the call only. */
typedef void (*dd_trigger_fn)(void *user, const dd_trigger *trig, const uint8_t *raw);

typedef struct dd_server_config {
    int nbeams;               /* 1..DD_BATCH_MAX_BEAMS */
    size_t gulp_nsamp;        /* new samples per gulp: a multiple of 64 above every beam's maxdelay */
    int max_slots;            /* gulps in flight at most (1..256) */
    size_t hbm_reserve_bytes; /* admission keeps this much device memory free */
    int half_window;          /* search configuration, as dd_search_config */
    int nwidths;
    int widths[DD_SEARCH_MAX_WIDTHS];
    float thresh;
    int max_cands;            /* candidates kept per gulp */
    const char *classifier_path; /* dd_nn_save checkpoint, or NULL: candidates keep score 0 */
    int nn_batch;             /* classifier batch (0 = 1024) */
    float trigger_snr;        /* dump the raw sweep of candidates with snr >= trigger_snr (0 = off) */
    int trigger_max;          /* dumps per gulp at most (first candidates in (d, t) order; 0 = 4) */
    dd_trigger_fn trigger_fn; /* called once per dump, on the worker thread, before the gulp's result is polled */
    void *trigger_user;
} dd_server_config;

typedef struct dd_gulp_result {
    int beam;
    int ncand;            /* candidates returned for this gulp */
    long long seq;        /* gulp number within its beam, from 0 */
    long long t0;         /* absolute output sample of the gulp's first output */
    long long nout;       /* outputs searched */
    double t_submit;      /* host steady-clock seconds at dd_server_submit */
    double t_done;        /* host steady-clock seconds when its candidates were on the host */
    int ngroups;          /* groups the search found */
    unsigned flags;       /* dd_search_result flags; bit 31 = a CUDA error in this gulp */
    int cand_offset;      /* index of its first candidate in dd_server_poll's array */
    int reserved;
} dd_gulp_result;

typedef struct dd_server dd_server;

/* Create a server for nbeams beams, plans[b] being beam b's plan (host array
 * of nbeams plans, which must outlive the server). */
dd_status dd_server_create(dd_server **out, const dd_server_config *cfg, dd_plan *const *plans);

/*
 * Submit beam `beam`'s next gulp: h_new is host memory, nchan rows of
 * gulp_nsamp/4 bytes at pitch h_pitch bytes (pinned memory gives the full
 * copy rate; the copy is asynchronous, so keep the buffer unchanged until the
 * gulp's result is polled).  *seq receives the gulp's number.
 * Returns DD_ERR_BUSY when no slot is free and no new slot fits (retry after
 * polling); nothing is enqueued then.
 */
dd_status dd_server_submit(dd_server *server, int beam, const uint8_t *h_new, size_t h_pitch, long long *seq);

/*
 * Collect finished gulps (up to max_results), waiting up to wait_s seconds
 * for the first one.  Their candidates (beam, d, t, w, snr, classifier score
 * in `score`) are copied to cands (up to max_cands_total); result r's start
 * at cands[r.cand_offset].
 */
dd_status dd_server_poll(dd_server *server, dd_gulp_result *results, int max_results, int *nresults,
                         dd_candidate *cands, int max_cands_total, int *ncands, double wait_s);

/* Wait (up to timeout_s) until no gulp is in flight. */
dd_status dd_server_drain(dd_server *server, double timeout_s);

/* Slots created, gulps in flight, device bytes one slot is budgeted at. */
dd_status dd_server_info(const dd_server *server, int *nslots, int *in_flight, size_t *slot_bytes);

/* Debug tap: also copy every later gulp's dedispersed outputs of `beam` into
 * d_dst (device, ndm rows of ld_dst uint32) at their absolute output columns,
 * for outputs below `capacity`. */
dd_status dd_server_set_tap(dd_server *server, int beam, uint32_t *d_dst, size_t ld_dst, size_t capacity);

/* Stop the server and free it (NULL-safe); waits for gulps in flight. */
void dd_server_destroy(dd_server *server);

/* ------------------------------------------------------------------------ */
/* Input layouts                                                              */
/* ------------------------------------------------------------------------ */

/*
 * Corner turn of time-major 2-bit data (backends that emit each time sample's
 * channels together): d_tm holds nsamp samples of ld_tm_bytes bytes, channel
 * c of sample t in bits 2*(c%4) of byte t*ld_tm_bytes + c/4.  Writes the
 * channel-major rows dd_execute reads into d_cm (nchan rows of ld_cm_bytes:
 * sample t of channel c in bits 2*(t%4) of byte c*ld_cm_bytes + t/4); the
 * whole rows are written, samples past nsamp as 0.  Both device, not
 * overlapping; asynchronous on stream.  A permutation of 2-bit values.
 */
dd_status dd_corner_turn(const uint8_t *d_tm, size_t ld_tm_bytes, int nchan, size_t nsamp, uint8_t *d_cm,
                         size_t ld_cm_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Multibeam coincidence RFI mask (paper Section 2.1)                         */
/* ------------------------------------------------------------------------ */

typedef struct dd_rfi dd_rfi;

/* Context for up to nbeams_max beams (<= 64) of nchan channels (<= 21844) and
 * up to nsamp_max samples (<= 2^31): owns the zero-DM series, the per-beam
 * sums and the mask.  Errors: DD_ERR_INVALID_ARG, DD_ERR_NOMEM. */
dd_status dd_rfi_create(dd_rfi **out, int nbeams_max, int nchan, size_t nsamp_max);

/*
 * Coincidence rejection across the beams (paper Section 2.1: a signal
 * exceeding k sigma in min_beams or more beams is interference; the paper's
 * example is 3 sigma in 4 of 13), asynchronously on stream:
 *  1. z_b[t] = sum over the channels of beam b's 2-bit sample t (the beam's
 *     total power per sample);
 *  2. S1_b = sum_t z_b[t], S2_b = sum_t z_b[t]^2 over the nsamp samples;
 *  3. beam b exceeds at t when n z - S1 > 0 and (n z - S1)^2 > k^2 (n S2 - S1^2)
 *     (z > mean + k sigma, decided exactly in integers);
 *  4. mask[t] = 1 when at least min_beams beams exceed;
 *  5. with apply != 0, every masked sample of every beam and channel c is
 *     replaced in place by the level 1 + ((c + t) mod 2) (the channel mean 1.5
 *     over pairs of samples).
 * d_in: host array of nbeams device pointers, each to nchan rows of
 * ld_in_bytes bytes (16-byte aligned, a multiple of 16) packed as for
 * dd_execute.  Results are exact.
 */
dd_status dd_rfi_run(dd_rfi *rfi, uint8_t *const *d_in, int nbeams, size_t ld_in_bytes, size_t nsamp, int k_sigma,
                     int min_beams, int apply, void *stream);

/* Masked samples of the last run (synchronises stream). */
dd_status dd_rfi_result(const dd_rfi *rfi, long long *nmasked, void *stream);

/* Device views of the last run: zero-DM series (uint32, [nbeams][ld_zerodm])
 * and the mask (uint8, [nsamp]); valid until the next run. */
dd_status dd_rfi_buffers(const dd_rfi *rfi, const uint32_t **d_zerodm, size_t *ld_zerodm, const uint8_t **d_mask);

void dd_rfi_destroy(dd_rfi *rfi);

/* ------------------------------------------------------------------------ */
/* Allocation-free dedispersion                                              */
/* ------------------------------------------------------------------------ */

/* Size of the fixed device scratch array behind dd_execute_noalloc. */
#define DD_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)

/*
 * dd_execute without a plan and without allocating anything (the paper has no
 * counterpart; this serves callers that may not call cudaMalloc or cudaFree,
 * e.g. a real-time loop where cudaFree would synchronise the device, or a host
 * framework that owns all device memory through its own pool).
 *
 * Computes the same exact sums as dd_execute for the band (freqs_mhz, host,
 * strictly descending), tsamp_s and DM list (dms, host, non-decreasing) given,
 * with the same input and output layout rules.  The kernel's offset tables
 * are built on the host in fixed static buffers and copied on `stream` into a
 * fixed device array of DD_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library reserves until the process exits; bands whose tables need more
 * (roughly ndm*nchan*4 bytes, plus padding) are rejected with
 * DD_ERR_INVALID_ARG.  Every call reuses that one array: calls whose kernels
 * may overlap on the GPU race and must be ordered (one stream, or events).
 * The first call on each device looks up the array's device address with that
 * device current; make it before any stream capture.  The kernel runs
 * asynchronously on `stream`, but the table upload comes from pageable host
 * memory, so the call may wait for work already queued on `stream` before it
 * returns; host threads are serialised by an internal mutex.
 * Errors: as dd_compute_delays and dd_execute, plus DD_ERR_INVALID_ARG for
 * tables beyond the scratch size.
 */
dd_status dd_execute_noalloc(int nchan, const double *freqs_mhz, double tsamp_s, int ndm, const double *dms,
                             const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out,
                             size_t ld_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
