// Plan-free dedispersion that performs no memory allocation at call time.
//
// Who needs it: code that may not call cudaMalloc/cudaFree -- a telescope
// backend's real-time loop, where cudaFree can synchronise the whole device
// and cudaMalloc can stall for milliseconds; a host framework that owns all
// device memory through its own pool and forbids raw allocations; a plug-in
// running inside such a host.  These callers hand in their input and output
// buffers; the only other device memory the tiled kernel needs -- its
// per-(channel, trial) offset tables -- lives in a fixed, file-scope device
// array below instead of in a plan.
//
// Limits and sharing:
//  * The device array holds DD_NOALLOC_SCRATCH_BYTES (8 MiB) and is reserved
//    on every GPU that loads the library, until the process exits.  A band and
//    DM list whose tables do not fit are rejected with DD_ERR_INVALID_ARG.
//  * The host side builds the tables in fixed static host buffers of the same
//    size (a mutex serialises host threads) and copies them into the device
//    array on the caller's stream.  That copy is from pageable memory: it is
//    staged before cudaMemcpyAsync returns, which may wait for work already
//    queued on the stream.
//  * Every call overwrites the same device array.  Two calls whose kernels
//    overlap on the GPU (e.g. on two streams without ordering) race; order
//    them on one stream or with events.  Nothing in the array has to start at
//    zero: each call writes every table entry its kernel reads.
//  * The device address of the array is looked up (cudaGetSymbolAddress) by
//    the first call made on each device, with that device current, and cached;
//    make that first call before any stream capture.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "dd_internal.h"
#include "tiled_tile.cuh"

namespace dd {
namespace {

using namespace tiled;

constexpr size_t kScratchBytes = DD_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
// tile shape of this entry point: 16 trials per CTA, 2 words per lane
constexpr int kDT = 2;
constexpr int kW = 2;
constexpr int kD = kWarps * kDT;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// host-side staging for the tables and the delay table (fixed size, no heap)
static uint32_t g_host_tab[kScratchBytes / 4];
static int32_t g_host_delays[kScratchBytes / 4];
static std::mutex g_mutex;
static void *g_dev_ptr[kMaxDevices];

template <int NP>
__global__ void __launch_bounds__(kThreads, TileOcc<kDT, kW, NP>::value) dd_noalloc_kernel(const TiledArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int dmb = (int)(blockIdx.x % (unsigned)a.n_dmb);
    const long long tt = (long long)(blockIdx.x / (unsigned)a.n_dmb);
    tile_init_bars<kGroup>(smem);
    uint32_t phase = 0;
    dd_tile<kDT, kW, NP, kGroup>(a, dmb, tt, smem, phase);
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_execute_noalloc(int nchan, const double *freqs_mhz, double tsamp_s, int ndm,
                                        const double *dms, const uint8_t *d_in, size_t ld_in_bytes,
                                        size_t nsamp_in, uint32_t *d_out, size_t ld_out, void *stream) {
    using namespace dd::tiled;
    if (nchan <= 0 || ndm <= 0 || !freqs_mhz || !dms)
        return fail(DD_ERR_INVALID_ARG, "nchan/ndm must be positive and freqs/dms non-NULL");
    if (nchan > tiled_max_nchan()) return fail(DD_ERR_INVALID_ARG, "at most %d channels", tiled_max_nchan());
    const size_t n_dmb = ((size_t)ndm + kD - 1) / kD;
    const size_t nchan_pad = ((size_t)nchan + kGroup - 1) / kGroup * kGroup;
    const size_t tab_words = n_dmb * nchan_pad * kD;
    const size_t ws_words = n_dmb * (size_t)nchan;
    if ((size_t)ndm * nchan * 4 > kScratchBytes || (tab_words + ws_words) * 4 > kScratchBytes)
        return fail(DD_ERR_INVALID_ARG,
                    "band and DM list too large for the fixed %zu-byte scratch (%d channels x %d trials need %zu "
                    "bytes of tables)",
                    kScratchBytes, nchan, ndm, (tab_words + ws_words) * 4);

    std::lock_guard<std::mutex> lock(g_mutex);
    int maxdelay = 0;
    dd_status st = compute_delays(nchan, freqs_mhz, tsamp_s, ndm, dms, g_host_delays, &maxdelay);
    if (st != DD_OK) return st;
    if (!d_in || !d_out) return fail(DD_ERR_INVALID_ARG, "NULL input or output");
    if (nsamp_in <= (size_t)maxdelay)
        return fail(DD_ERR_TOO_SHORT, "nsamp_in (%zu) must exceed the maximum delay (%d)", nsamp_in, maxdelay);
    if (ld_in_bytes % 16 != 0 || ld_in_bytes < (nsamp_in + 3) / 4 || ((uintptr_t)d_in) % 16 != 0)
        return fail(DD_ERR_INVALID_ARG, "input layout: 16-byte aligned rows of ld_in_bytes >= ceil(nsamp_in/4)");
    const size_t nout = nsamp_in - (size_t)maxdelay;
    if (ld_out < nout || ld_out % 4 != 0 || ((uintptr_t)d_out) % 16 != 0)
        return fail(DD_ERR_INVALID_ARG, "output layout: 16-byte aligned rows of ld_out >= %zu, ld_out %% 4 == 0", nout);

    int dev = 0;
    DD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(DD_ERR_INVALID_ARG, "device index %d out of range", dev);
    if (!g_dev_ptr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                       "cudaGetSymbolAddress(scratch)");
        g_dev_ptr[dev] = ptr;
    }

    // tables: same layout as the plan's (see ensure_shape_table)
    int spread = 0;
    for (int d0 = 0; d0 < ndm; d0 += kD) {
        const int d1 = std::min(d0 + kD, ndm) - 1;
        for (int c = 0; c < nchan; ++c)
            spread = std::max(spread, (int)(g_host_delays[(size_t)d1 * nchan + c] - g_host_delays[(size_t)d0 * nchan + c]));
    }
    const int slot = tile_slot(kW, spread);
    const size_t smem = tile_smem_bytes(slot, kGroup, kD, nchan);
    if (smem > 227 * 1024) return fail(DD_ERR_INVALID_ARG, "delay spread too large for the tiled kernel");
    uint32_t *tab = g_host_tab;
    int32_t *wsrel = reinterpret_cast<int32_t *>(g_host_tab + tab_words);
    build_tile_tables(g_host_delays, ndm, nchan, kD, slot, tab, wsrel);
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *dev_tab = static_cast<uint32_t *>(g_dev_ptr[dev]);
    // pageable source: the copy is staged before cudaMemcpyAsync returns, so the
    // host buffers may be rebuilt by the next call right away
    DD_CUDA_TRY(cudaMemcpyAsync(dev_tab, g_host_tab, (tab_words + ws_words) * 4, cudaMemcpyHostToDevice, s));

    TiledArgs a;
    a.in = reinterpret_cast<const uint32_t *>(d_in);
    a.ld_w = (long long)(ld_in_bytes / 4);
    a.tab = dev_tab;
    a.wsrel = reinterpret_cast<const int32_t *>(dev_tab + tab_words);
    a.nchan = nchan;
    a.ndm = ndm;
    a.nout = (long long)nout;
    a.out = d_out;
    a.ld_out = (long long)ld_out;
    a.slot = slot;
    a.n_dmb = (int)n_dmb;
    st = tile_error_word(&a.err);
    if (st != DD_OK) return st;
    a.poll_limit = tiled::kStagePollLimit;
    const long long T = 16LL * 32 * kW;
    const long long nblocks = ((a.nout + T - 1) / T) * a.n_dmb;
    if (nblocks > 0x7fffffffLL) return fail(DD_ERR_INVALID_ARG, "gulp too long for one launch");
    auto kern = nchan >= 2048 ? dd_noalloc_kernel<15> : dd_noalloc_kernel<11>;
    if (smem > 48 * 1024) DD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)nblocks, kThreads, smem, s>>>(a);
    return cuda_fail(cudaGetLastError(), "dd_noalloc_kernel launch");
}
