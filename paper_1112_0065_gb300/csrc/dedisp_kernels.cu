// Direct dedispersion kernels for sm_103a (paper Section 2.2).
//
//   out[d][t] = sum_c x[c][t + delay[d][c]]     (exact uint32)
//
// Two kernels:
//  * dd_simple_kernel -- one thread per (DM, 4 consecutive samples), every
//    sample fetched from global memory.  Kept as a checking aid and for band
//    shapes the tiled kernel does not cover.
//  * dd_tiled_kernel  -- the production kernel.  A CTA owns D = 8*DT
//    consecutive DM trials and a tile of 512*W output samples.  For each stage
//    of G = 32, 64 or 128 channels the copy engine brings the packed 2-bit
//    window of every channel that the CTA's DMs need into shared memory (one
//    bulk copy per channel, completion on the stage's mbarrier; still packed:
//    16 samples per 32-bit word), where all D trials reuse it.  A lane owns W
//    words of 16 consecutive output samples for DT trials (W consecutive words
//    when W is odd, so that W+1 staged words serve them).  For every (trial,
//    channel) it realigns the staged window to the trial's delay with one
//    funnel shift, giving 16 samples as 2-bit lanes of one register, and adds
//    them into bit-sliced counters with a carry-save adder tree (Harley-Seal):
//    64 channels go into 6 bit-planes and a carry with 63 full adders, two
//    3-input logic ops each, i.e. about 2 logic ops per 16 sample-additions.
//    The stage's carry ripples into the upper planes, which stay in registers
//    across the whole band (11 planes for up to 2047 channels, 15 beyond);
//    after the last stage the planes become per-sample sums in 16-bit lanes.
//    There are no tensor cores here: the work is a gather-sum, not a dense
//    contraction.
#include <algorithm>
#include <mutex>

#include "dd_internal.h"
#include "tiled_tile.cuh"

namespace dd {

// ---------------------------------------------------------------------------
// simple kernel
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(128) dd_simple_kernel(const uint8_t *__restrict__ in, long long ld_in,
                                                         const int32_t *__restrict__ delays, int nchan,
                                                         uint32_t *__restrict__ out, long long ld_out,
                                                         long long nout) {
    const int d = blockIdx.y;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (t >= nout) return;
    const int32_t *drow = delays + (long long)d * nchan;
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    for (int c = 0; c < nchan; ++c) {
        const long long s = t + __ldg(drow + c);
        const uint8_t *row = in + (long long)c * ld_in;
        const long long b = s >> 2;
        const unsigned sh = (unsigned)(s & 3) * 2u;
        uint32_t w = __ldg(row + b);
        if (sh && b + 1 < ld_in) w |= (uint32_t)__ldg(row + b + 1) << 8;
        w >>= sh;
        a0 += w & 3u;
        a1 += (w >> 2) & 3u;
        a2 += (w >> 4) & 3u;
        a3 += (w >> 6) & 3u;
    }
    uint32_t *o = out + (long long)d * ld_out + t;
    o[0] = a0;
    if (t + 1 < nout) o[1] = a1;
    if (t + 2 < nout) o[2] = a2;
    if (t + 3 < nout) o[3] = a3;
}

dd_status launch_simple(const Plan *p, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out,
                        size_t ld_out, cudaStream_t stream) {
    const long long nout = (long long)nsamp_in - p->maxdelay;
    const int threads = 128;
    const long long nblk = (nout + 4LL * threads - 1) / (4LL * threads);
    if (nblk > 0x7fffffffLL || p->ndm > 65535) return fail(DD_ERR_INVALID_ARG, "gulp too long for the simple kernel");
    dim3 grid((unsigned)nblk, (unsigned)p->ndm);
    dd_simple_kernel<<<grid, threads, 0, stream>>>(d_in, (long long)ld_in_bytes, p->delays_dev, p->nchan, d_out,
                                                   (long long)ld_out, nout);
    return cuda_fail(cudaGetLastError(), "dd_simple_kernel launch");
}


// ---------------------------------------------------------------------------
// tiled kernel
// ---------------------------------------------------------------------------

size_t tiled_smem_bytes(const Plan *p, const ShapeTable &st, int D) {
    return tiled::tile_smem_bytes(st.slot, st.group, D, p->nchan);
}

// The tiled kernels' device error word (bit 0: a tile gave up waiting for its
// staged input), one per device, reached through its symbol address.
static __device__ unsigned g_tile_err;
static std::mutex g_tile_err_mutex;
static unsigned *g_tile_err_ptr[64];

dd_status tile_error_word(unsigned **out) {
    int dev = 0;
    DD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(DD_ERR_INVALID_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_tile_err_mutex);
    if (!g_tile_err_ptr[dev]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_tile_err);
        if (e != cudaSuccess || !ptr)
            return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress(tile error word)");
        g_tile_err_ptr[dev] = static_cast<unsigned *>(ptr);
    }
    *out = g_tile_err_ptr[dev];
    return DD_OK;
}

// (DMs per warp, words per lane) shapes; each is built with 32-, 64- and
// 128-channel stages (tiled_g32/64/128.cu).
static const int kShapes[][2] = {{1, 2}, {2, 1}, {2, 2}, {4, 1}, {1, 4}, {1, 3}, {2, 3}, {1, 5}};
static const int kGroups[] = {64, 32, 128};

bool tiled_shape_supported(const TiledShape &s) {
    bool group_ok = false;
    for (int g : kGroups) group_ok |= g == s.chan_chunk;
    if (!group_ok) return false;
    for (const auto &k : kShapes)
        if (k[0] == s.dms_per_warp && k[1] == s.words_per_lane) return true;
    return false;
}

std::vector<TiledShape> tiled_shape_candidates() {
    std::vector<TiledShape> v;
    for (int g : kGroups)
        for (const auto &k : kShapes) v.push_back(TiledShape{k[0], k[1], g});
    return v;
}

// bit-planes count up to 2^15-1 channels; the 16-bit sums hold 3*nchan <= 65535
int tiled_max_nchan() { return 21845; }

dd_status ensure_shape_table(Plan *p, const TiledShape &s) {
    using namespace tiled;
    if (!tiled_shape_supported(s)) return fail(DD_ERR_INVALID_ARG, "unsupported tiled kernel shape");
    const int key = shape_key(s);
    if (p->tables.count(key)) return DD_OK;
    if (s.chan_chunk != 64 && p->nchan >= 2048)
        return fail(DD_ERR_INVALID_ARG, "bands of 2048 channels or more use 64-channel stages");
    const int D = kWarps * s.dms_per_warp;
    const int G = s.chan_chunk;
    ShapeTable st;
    st.group = G;
    st.n_dmb = (p->ndm + D - 1) / D;
    const int spread = max_block_spread(p, D);
    st.slot = tile_slot(s.words_per_lane, spread);
    if (tiled_smem_bytes(p, st, D) > 227 * 1024)
        return fail(DD_ERR_INVALID_ARG, "delay spread too large for the tiled kernel's shared memory");
    const int nchan_pad = (p->nchan + G - 1) / G * G;
    std::vector<uint32_t> tab((size_t)st.n_dmb * nchan_pad * D);
    std::vector<int32_t> wsrel((size_t)st.n_dmb * p->nchan);
    build_tile_tables(p->delays_host.data(), p->ndm, p->nchan, D, st.slot, tab.data(), wsrel.data(), G);
    DD_CUDA_TRY(cudaMalloc(&st.tab, tab.size() * 4));
    cudaError_t e = cudaMalloc(&st.wsrel, wsrel.size() * 4);
    if (e == cudaSuccess) e = cudaMemcpy(st.tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st.wsrel, wsrel.data(), wsrel.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(st.tab);
        if (st.wsrel) cudaFree(st.wsrel);
        return cuda_fail(e, "uploading the tiled kernel tables");
    }
    p->tables[key] = st;
    return DD_OK;
}

void free_shape_tables(Plan *p) {
    for (auto &kv : p->tables) {
        cudaFree(kv.second.tab);
        cudaFree(kv.second.wsrel);
    }
    p->tables.clear();
}

dd_status launch_tiled(const Plan *p, const TiledShape &s, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                       uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
    auto it = p->tables.find(shape_key(s));
    if (it == p->tables.end()) return fail(DD_ERR_INTERNAL, "tiled kernel table missing for this shape");
    const ShapeTable &st = it->second;
    switch (s.chan_chunk) {
    case 32: return launch_tiled_g32(p, s, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    case 64: return launch_tiled_g64(p, s, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    case 128: return launch_tiled_g128(p, s, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    default: return fail(DD_ERR_INVALID_ARG, "unsupported channel stage %d", s.chan_chunk);
    }
}

BatchKernelFn batch_kernel(const TiledShape &s, bool big) {
    switch (s.chan_chunk) {
    case 32: return batch_kernel_g32(s, big);
    case 64: return batch_kernel_g64(s, big);
    case 128: return batch_kernel_g128(s, big);
    default: return nullptr;
    }
}

}  // namespace dd
