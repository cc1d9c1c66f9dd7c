// Internal declarations shared by the library's translation units.
// Nothing here is part of the C ABI (include/dd.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/dd.h"

namespace dd {

// Record a failure message for dd_last_error() and return the status.
dd_status fail(dd_status s, const char *fmt, ...);
// Map a CUDA error to DD_ERR_CUDA (or DD_OK) with a message.
dd_status cuda_fail(cudaError_t e, const char *what);

#define DD_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return ::dd::cuda_fail(e__, #expr); \
    } while (0)

// Shape of the tiled dedispersion kernel.
struct TiledShape {
    int dms_per_warp = 2;   // DM trials per warp
    int words_per_lane = 3; // 16-sample words per lane along time
    int chan_chunk = 64;    // channels per shared-memory stage (one CSA group)
};

// Map key of a shape's tables in Plan::tables.
inline int shape_key(const TiledShape &s) { return s.chan_chunk * 10000 + s.dms_per_warp * 100 + s.words_per_lane; }

// Per-shape device tables of the tiled kernel, precomputed on the host.
struct ShapeTable {
    uint32_t *tab = nullptr;   // [n_dmb][nchan_pad][D] (slot word address << 5) | funnel shift
    int32_t *wsrel = nullptr;  // [n_dmb][nchan] first staged word, relative to the tile start
    int slot = 0;              // shared-memory words per staged channel
    int n_dmb = 0;
    int group = 64;            // channels per shared-memory stage
};

struct Plan {
    int nchan = 0;
    int ndm = 0;
    int maxdelay = 0;
    double tsamp = 0;
    std::vector<double> freqs;
    std::vector<double> dms;
    std::vector<int32_t> delays_host;   // [ndm][nchan]
    int32_t *delays_dev = nullptr;      // [ndm][nchan], device-resident for the plan's lifetime
    int device = 0;
    int kernel = DD_KERNEL_AUTO;
    TiledShape shape;
    std::map<int, ShapeTable> tables;   // keyed by shape_key()
    int live_batches = 0;               // batches whose descriptors point at these tables
    std::string tune_cache;
    // host-API staging (dd_execute_host), grown on demand
    uint8_t *stage_in = nullptr;
    size_t stage_in_bytes = 0;
    uint32_t *stage_out = nullptr;
    size_t stage_out_bytes = 0;
};

// Validation + delays (host, double precision).
dd_status compute_delays(int nchan, const double *freqs, double tsamp, int ndm, const double *dms,
                         int32_t *out, int *maxdelay);

// Layout checks shared by execute paths.
dd_status check_exec_args(const Plan *p, const void *d_in, size_t ld_in_bytes, size_t nsamp_in,
                          const void *d_out, size_t ld_out);

// Kernel launchers (asynchronous on stream).
dd_status launch_simple(const Plan *p, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                        uint32_t *d_out, size_t ld_out, cudaStream_t stream);
dd_status launch_tiled(const Plan *p, const TiledShape &shape, const uint8_t *d_in, size_t ld_in_bytes,
                       size_t nsamp_in, uint32_t *d_out, size_t ld_out, cudaStream_t stream);
// Per stage size (tiled_g32/64/128.cu): the launch of a shape with its tables,
// and the persistent multi-beam kernel of a shape (nullptr if not built).
namespace tiled {
struct BatchDesc;
}
using BatchKernelFn = void (*)(const tiled::BatchDesc *, unsigned long long *);
#define DD_DECLARE_GROUP(G)                                                                                      \
    dd_status launch_tiled_g##G(const Plan *p, const TiledShape &s, const ShapeTable &st, const uint8_t *d_in, \
                                size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out, size_t ld_out,          \
                                cudaStream_t stream);                                                          \
    BatchKernelFn batch_kernel_g##G(const TiledShape &s, bool big);
DD_DECLARE_GROUP(32)
DD_DECLARE_GROUP(64)
DD_DECLARE_GROUP(128)
#undef DD_DECLARE_GROUP
BatchKernelFn batch_kernel(const TiledShape &s, bool big);
bool tiled_shape_supported(const TiledShape &s);
dd_status ensure_shape_table(Plan *p, const TiledShape &s);
void free_shape_tables(Plan *p);
size_t tiled_smem_bytes(const Plan *p, const ShapeTable &st, int D);
// Device address of the tiled kernels' error word on the current device.
dd_status tile_error_word(unsigned **out);
std::vector<TiledShape> tiled_shape_candidates();
int tiled_max_nchan();

// Largest delay spread (delay[last][c] - delay[first][c], max over c) within
// any block of `dms_per_block` consecutive trials.
int max_block_spread(const Plan *p, int dms_per_block);

// Device address of the group count of a search context's last run.
const unsigned *search_dev_ngroups(const dd_search *search);

}  // namespace dd
