// Plans, delay table, error reporting and the single-gulp execute entry
// points of the C ABI (include/dd.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "dd_internal.h"

namespace dd {

static thread_local char g_last_error[512] = "";

dd_status fail(dd_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

dd_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return DD_OK;
    dd_status s = (e == cudaErrorMemoryAllocation) ? DD_ERR_NOMEM : DD_ERR_CUDA;
    return fail(s, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Dispersion constant, s MHz^2 per (pc cm^-3).
static const double kDM = 4.148808e3;

dd_status compute_delays(int nchan, const double *freqs, double tsamp, int ndm, const double *dms,
                         int32_t *out, int *maxdelay) {
    if (nchan <= 0 || ndm <= 0) return fail(DD_ERR_INVALID_ARG, "nchan and ndm must be positive");
    if (!freqs || !dms) return fail(DD_ERR_INVALID_ARG, "NULL frequency or DM list");
    if (!(tsamp > 0) || !isfinite(tsamp)) return fail(DD_ERR_INVALID_ARG, "tsamp must be > 0");
    for (int c = 0; c < nchan; ++c) {
        if (!isfinite(freqs[c]) || !(freqs[c] > 0))
            return fail(DD_ERR_INVALID_ARG, "channel %d frequency is not a positive number", c);
        if (c > 0 && !(freqs[c] < freqs[c - 1]))
            return fail(DD_ERR_INVALID_ARG, "frequencies must be strictly descending (channel %d)", c);
    }
    for (int d = 0; d < ndm; ++d) {
        if (!isfinite(dms[d]) || dms[d] < 0)
            return fail(DD_ERR_INVALID_ARG, "DM %d is negative or not finite", d);
        if (d > 0 && dms[d] < dms[d - 1])
            return fail(DD_ERR_INVALID_ARG, "DMs must be non-decreasing (trial %d)", d);
    }
    const double fmax = freqs[0];
    int32_t mx = 0;
    for (int d = 0; d < ndm; ++d) {
        for (int c = 0; c < nchan; ++c) {
            const double f = freqs[c];
            const double v = kDM * dms[d] * (1.0 / (f * f) - 1.0 / (fmax * fmax)) / tsamp;
            if (!(v < 2147483647.0)) return fail(DD_ERR_INVALID_ARG, "delay overflows int32 (DM %d)", d);
            const int32_t dl = (int32_t)llround(v);
            if (out) out[(size_t)d * nchan + c] = dl;
            mx = std::max(mx, dl);
        }
    }
    if (maxdelay) *maxdelay = mx;
    return DD_OK;
}

dd_status check_exec_args(const Plan *p, const void *d_in, size_t ld_in_bytes, size_t nsamp_in,
                          const void *d_out, size_t ld_out) {
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL plan");
    if (!d_in || !d_out) return fail(DD_ERR_INVALID_ARG, "NULL input or output");
    if (nsamp_in <= (size_t)p->maxdelay)
        return fail(DD_ERR_TOO_SHORT, "nsamp_in (%zu) must exceed the plan's maximum delay (%d)", nsamp_in,
                    p->maxdelay);
    if (ld_in_bytes % 16 != 0 || ld_in_bytes < (nsamp_in + 3) / 4)
        return fail(DD_ERR_INVALID_ARG, "ld_in_bytes (%zu) must be a multiple of 16 and >= ceil(nsamp_in/4)",
                    ld_in_bytes);
    if (((uintptr_t)d_in) % 16 != 0) return fail(DD_ERR_INVALID_ARG, "input must be 16-byte aligned");
    const size_t nout = nsamp_in - (size_t)p->maxdelay;
    if (ld_out < nout || ld_out % 4 != 0)
        return fail(DD_ERR_INVALID_ARG, "ld_out (%zu) must be >= %zu and a multiple of 4", ld_out, nout);
    if (((uintptr_t)d_out) % 16 != 0) return fail(DD_ERR_INVALID_ARG, "output must be 16-byte aligned");
    return DD_OK;
}

int max_block_spread(const Plan *p, int dpb) {
    int best = 0;
    for (int d0 = 0; d0 < p->ndm; d0 += dpb) {
        const int d1 = std::min(d0 + dpb, p->ndm) - 1;
        const int32_t *a = p->delays_host.data() + (size_t)d0 * p->nchan;
        const int32_t *b = p->delays_host.data() + (size_t)d1 * p->nchan;
        for (int c = 0; c < p->nchan; ++c) best = std::max(best, (int)(b[c] - a[c]));
    }
    return best;
}

static dd_status run(const Plan *p, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out,
                     size_t ld_out, cudaStream_t stream) {
    if (p->kernel == DD_KERNEL_SIMPLE) return launch_simple(p, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    return launch_tiled(p, p->shape, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
}

}  // namespace dd

using namespace dd;

extern "C" {

const char *dd_status_string(dd_status s) {
    switch (s) {
        case DD_OK: return "DD_OK";
        case DD_ERR_INVALID_ARG: return "DD_ERR_INVALID_ARG";
        case DD_ERR_NOMEM: return "DD_ERR_NOMEM";
        case DD_ERR_CUDA: return "DD_ERR_CUDA";
        case DD_ERR_TOO_SHORT: return "DD_ERR_TOO_SHORT";
        case DD_ERR_TIMEOUT: return "DD_ERR_TIMEOUT";
        case DD_ERR_INTERNAL: return "DD_ERR_INTERNAL";
        case DD_ERR_BUSY: return "DD_ERR_BUSY";
    }
    return "DD_ERR_UNKNOWN";
}

const char *dd_last_error(void) { return g_last_error; }

int dd_version(void) { return 10000; }

dd_status dd_compute_delays(int nchan, const double *freqs_mhz, double tsamp_s, int ndm, const double *dms,
                            int32_t *out) {
    if (!out) return fail(DD_ERR_INVALID_ARG, "NULL output");
    return compute_delays(nchan, freqs_mhz, tsamp_s, ndm, dms, out, nullptr);
}

dd_status dd_plan_create(dd_plan **out, int nchan, const double *freqs_mhz, double tsamp_s, int ndm,
                         const double *dms, const dd_options *opt) {
    if (!out) return fail(DD_ERR_INVALID_ARG, "NULL plan pointer");
    *out = nullptr;
    dd_options o;
    memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.kernel < DD_KERNEL_AUTO || o.kernel > DD_KERNEL_TILED || o.reserved != 0 || o.dms_per_block < 0 ||
        o.words_per_thread < 0 || o.chan_chunk < 0)
        return fail(DD_ERR_INVALID_ARG, "bad dd_options");
    int maxdelay = 0;
    dd_status st = compute_delays(nchan, freqs_mhz, tsamp_s, ndm, dms, nullptr, &maxdelay);
    if (st != DD_OK) return st;
    Plan *p = new (std::nothrow) Plan();
    if (!p) return fail(DD_ERR_NOMEM, "host allocation failed");
    p->nchan = nchan;
    p->ndm = ndm;
    p->maxdelay = maxdelay;
    p->tsamp = tsamp_s;
    p->freqs.assign(freqs_mhz, freqs_mhz + nchan);
    p->dms.assign(dms, dms + ndm);
    p->delays_host.resize((size_t)nchan * ndm);
    compute_delays(nchan, freqs_mhz, tsamp_s, ndm, dms, p->delays_host.data(), nullptr);
    p->kernel = o.kernel;
    if (o.tune_cache_path) p->tune_cache = o.tune_cache_path;
    if (p->kernel != DD_KERNEL_SIMPLE && nchan > tiled_max_nchan()) {
        if (p->kernel == DD_KERNEL_TILED) {
            delete p;
            return fail(DD_ERR_INVALID_ARG, "the tiled kernel supports at most %d channels", tiled_max_nchan());
        }
        p->kernel = DD_KERNEL_SIMPLE;
    }
    if (o.dms_per_block || o.words_per_thread || o.chan_chunk) {
        TiledShape s = p->shape;
        if (o.dms_per_block) s.dms_per_warp = o.dms_per_block / 8;
        if (o.words_per_thread) s.words_per_lane = o.words_per_thread;
        if (o.chan_chunk) s.chan_chunk = o.chan_chunk;
        if (o.dms_per_block % 8 != 0 || !tiled_shape_supported(s)) {
            delete p;
            return fail(DD_ERR_INVALID_ARG, "unsupported tiled kernel shape");
        }
        p->shape = s;
    }
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaMalloc(&p->delays_dev, p->delays_host.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->delays_dev, p->delays_host.data(), p->delays_host.size() * sizeof(int32_t),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        dd_status s = cuda_fail(e, "uploading the delay table");
        if (p->delays_dev) cudaFree(p->delays_dev);
        delete p;
        return s;
    }
    if (p->kernel != DD_KERNEL_SIMPLE) {
        dd_status ts = ensure_shape_table(p, p->shape);
        if (ts != DD_OK) {
            if (p->kernel == DD_KERNEL_TILED) {
                cudaFree(p->delays_dev);
                free_shape_tables(p);
                delete p;
                return ts;
            }
            p->kernel = DD_KERNEL_SIMPLE;  // delay spread beyond the tiled kernel's shared memory
        }
    }
    *out = reinterpret_cast<dd_plan *>(p);
    return DD_OK;
}

dd_status dd_plan_info(const dd_plan *plan, int *nchan, int *ndm, int *maxdelay) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL plan");
    if (nchan) *nchan = p->nchan;
    if (ndm) *ndm = p->ndm;
    if (maxdelay) *maxdelay = p->maxdelay;
    return DD_OK;
}

dd_status dd_plan_delay_table(const dd_plan *plan, int32_t *host_out) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p || !host_out) return fail(DD_ERR_INVALID_ARG, "NULL plan or output");
    memcpy(host_out, p->delays_host.data(), p->delays_host.size() * sizeof(int32_t));
    return DD_OK;
}

dd_status dd_plan_kernel_shape(const dd_plan *plan, int *kernel, int *dms_per_block, int *words_per_thread,
                               int *chan_chunk) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL plan");
    if (kernel) *kernel = p->kernel;
    if (dms_per_block) *dms_per_block = p->shape.dms_per_warp * 8;
    if (words_per_thread) *words_per_thread = p->shape.words_per_lane;
    if (chan_chunk) *chan_chunk = p->shape.chan_chunk;
    return DD_OK;
}

dd_status dd_execute(const dd_plan *plan, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                     uint32_t *d_out, size_t ld_out, void *stream) {
    const Plan *p = reinterpret_cast<const Plan *>(plan);
    dd_status st = check_exec_args(p, d_in, ld_in_bytes, nsamp_in, d_out, ld_out);
    if (st != DD_OK) return st;
    return run(p, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, (cudaStream_t)stream);
}

dd_status dd_execute_host(dd_plan *plan, const uint8_t *h_in, size_t ld_in_bytes, size_t nsamp_in,
                          uint32_t *h_out, size_t ld_out, void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !h_in || !h_out) return fail(DD_ERR_INVALID_ARG, "NULL plan, input or output");
    const size_t in_bytes = (size_t)p->nchan * ld_in_bytes;
    const size_t out_bytes = (size_t)p->ndm * ld_out * sizeof(uint32_t);
    if (p->stage_in_bytes < in_bytes) {
        if (p->stage_in) cudaFree(p->stage_in);
        p->stage_in = nullptr;
        p->stage_in_bytes = 0;
        DD_CUDA_TRY(cudaMalloc(&p->stage_in, in_bytes));
        p->stage_in_bytes = in_bytes;
    }
    if (p->stage_out_bytes < out_bytes) {
        if (p->stage_out) cudaFree(p->stage_out);
        p->stage_out = nullptr;
        p->stage_out_bytes = 0;
        DD_CUDA_TRY(cudaMalloc(&p->stage_out, out_bytes));
        p->stage_out_bytes = out_bytes;
    }
    dd_status st = check_exec_args(p, p->stage_in, ld_in_bytes, nsamp_in, p->stage_out, ld_out);
    if (st != DD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    DD_CUDA_TRY(cudaMemcpyAsync(p->stage_in, h_in, in_bytes, cudaMemcpyHostToDevice, s));
    st = run(p, p->stage_in, ld_in_bytes, nsamp_in, p->stage_out, ld_out, s);
    if (st != DD_OK) return st;
    DD_CUDA_TRY(cudaMemcpyAsync(h_out, p->stage_out, out_bytes, cudaMemcpyDeviceToHost, s));
    DD_CUDA_TRY(cudaStreamSynchronize(s));
    return DD_OK;
}

void dd_destroy(dd_plan *plan) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return;
    if (p->delays_dev) cudaFree(p->delays_dev);
    free_shape_tables(p);
    if (p->stage_in) cudaFree(p->stage_in);
    if (p->stage_out) cudaFree(p->stage_out);
    delete p;
}

dd_status dd_dedisp_status(unsigned *flags) {
    if (!flags) return fail(DD_ERR_INVALID_ARG, "NULL flags");
    unsigned *word = nullptr;
    dd_status st = tile_error_word(&word);
    if (st != DD_OK) return st;
    DD_CUDA_TRY(cudaDeviceSynchronize());
    DD_CUDA_TRY(cudaMemcpy(flags, word, 4, cudaMemcpyDeviceToHost));
    DD_CUDA_TRY(cudaMemset(word, 0, 4));
    return DD_OK;
}

}  // extern "C"
