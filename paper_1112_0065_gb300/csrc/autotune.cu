// Autotuner for the tiled dedispersion kernel: times every supported tile
// shape (DM trials per CTA x 16-sample words per lane) on the plan's own
// delay table and a scratch gulp, keeps the fastest, and caches the choice
// in a small text file keyed by (device name, nchan, ndm, maxdelay, gulp
// length bucket).
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "dd_internal.h"

namespace dd {

static std::mutex g_cache_mutex;

static std::string cache_key(const Plan *p, size_t nsamp_in) {
    cudaDeviceProp prop;
    char name[256] = "unknown";
    if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) snprintf(name, sizeof(name), "%s", prop.name);
    for (char *c = name; *c; ++c)
        if (*c == ' ') *c = '_';
    // bucket the gulp length by its power of two
    int b = 0;
    while ((size_t(1) << (b + 1)) <= nsamp_in) ++b;
    char key[512];
    snprintf(key, sizeof(key), "%s nchan=%d ndm=%d maxdelay=%d nsamp_log2=%d", name, p->nchan, p->ndm, p->maxdelay, b);
    return key;
}

bool cache_lookup(const Plan *p, size_t nsamp_in, TiledShape *out) {
    if (p->tune_cache.empty()) return false;
    std::lock_guard<std::mutex> g(g_cache_mutex);
    FILE *f = fopen(p->tune_cache.c_str(), "r");
    if (!f) return false;
    const std::string key = cache_key(p, nsamp_in);
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char *bar = strchr(line, '|');
        if (!bar) continue;
        *bar = 0;
        if (key == line) {
            TiledShape s;
            if (sscanf(bar + 1, "%d %d %d", &s.dms_per_warp, &s.words_per_lane, &s.chan_chunk) == 3 &&
                tiled_shape_supported(s)) {
                *out = s;
                found = true;
            }
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const Plan *p, size_t nsamp_in, const TiledShape &s) {
    if (p->tune_cache.empty()) return;
    std::lock_guard<std::mutex> g(g_cache_mutex);
    FILE *f = fopen(p->tune_cache.c_str(), "a");
    if (!f) return;
    fprintf(f, "%s|%d %d %d\n", cache_key(p, nsamp_in).c_str(), s.dms_per_warp, s.words_per_lane, s.chan_chunk);
    fclose(f);
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_plan_autotune(dd_plan *plan, size_t nsamp_in, void *stream, float *best_ms) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL plan");
    if (nsamp_in <= (size_t)p->maxdelay) return fail(DD_ERR_TOO_SHORT, "gulp shorter than the maximum delay");
    if (p->kernel == DD_KERNEL_SIMPLE) return fail(DD_ERR_INVALID_ARG, "plan uses the simple kernel");
    TiledShape cached;
    if (cache_lookup(p, nsamp_in, &cached) && ensure_shape_table(p, cached) == DD_OK) {
        p->shape = cached;
        if (best_ms) *best_ms = 0.0f;
        return DD_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ld_in = ((nsamp_in + 3) / 4 + 15) / 16 * 16;
    const size_t nout = nsamp_in - (size_t)p->maxdelay;
    const size_t ld_out = (nout + 3) / 4 * 4;
    uint8_t *in = nullptr;
    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    dd_status st = DD_OK;
    float best = 1e30f;
    TiledShape best_shape = p->shape;
    cudaError_t e = cudaMalloc(&in, (size_t)p->nchan * ld_in);
    if (e == cudaSuccess) e = cudaMalloc(&out, (size_t)p->ndm * ld_out * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(in, 0x6c, (size_t)p->nchan * ld_in, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) st = cuda_fail(e, "autotune setup");
    for (const TiledShape &cand : tiled_shape_candidates()) {
        if (st != DD_OK) break;
        if (ensure_shape_table(p, cand) != DD_OK) continue;  // shape does not fit this band
        st = launch_tiled(p, cand, in, ld_in, nsamp_in, out, ld_out, s);  // warm-up
        if (st != DD_OK) break;
        const int reps = 3;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(e, "event"); break; }
        for (int r = 0; r < reps && st == DD_OK; ++r) st = launch_tiled(p, cand, in, ld_in, nsamp_in, out, ld_out, s);
        if (st != DD_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
            st = cuda_fail(e, "event");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (ms < best) {
            best = ms;
            best_shape = cand;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (in) cudaFree(in);
    if (out) cudaFree(out);
    if (st != DD_OK) return st;
    p->shape = best_shape;
    // keep only the chosen shape's tables, unless a batch still points at some
    // of them (they are then freed with the plan)
    for (auto it = p->tables.begin(); it != p->tables.end() && p->live_batches == 0;) {
        if (it->first != shape_key(best_shape)) {
            cudaFree(it->second.tab);
            cudaFree(it->second.wsrel);
            it = p->tables.erase(it);
        } else {
            ++it;
        }
    }
    cache_store(p, nsamp_in, best_shape);
    if (best_ms) *best_ms = best;
    return DD_OK;
}
