// Kernel templates of the tiled dedispersion path (single gulp and the
// persistent multi-beam launch) and the per-stage-size instantiation lists.
// Each tiled_g<G>.cu translation unit instantiates them for one channel-stage
// size G, so the instantiations compile in parallel.
#pragma once

#include "dd_internal.h"
#include "tiled_tile.cuh"

namespace dd {
namespace tiled {

template <int DT, int W, int NP, int G>
__global__ void __launch_bounds__(kThreads, TileOcc<DT, W, NP>::value) dd_tiled_kernel(const TiledArgs a) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int dmb = (int)(blockIdx.x % (unsigned)a.n_dmb);
    const long long tt = (long long)(blockIdx.x / (unsigned)a.n_dmb);
    tile_init_bars<G>(smem);
    uint32_t phase = 0;
    dd_tile<DT, W, NP, G>(a, dmb, tt, smem, phase);
}

// Persistent multi-beam kernel: one CTA per resident slot takes global tile
// indices from an atomic counter until the work list is exhausted (or a tile
// reports that its input never arrived).  The stage mbarriers sit at the
// start of shared memory for every beam, so their phases carry from tile to
// tile.
template <int DT, int W, int NP, int G>
__global__ void __launch_bounds__(kThreads, TileOcc<DT, W, NP>::value)
    dd_batch_kernel(const BatchDesc *__restrict__ desc, unsigned long long *__restrict__ counter) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ long long s_tile;
    const long long ntiles = desc->ntiles;
    tile_init_bars<G>(smem);
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = (long long)atomicAdd(counter, 1ULL);
        __syncthreads();
        const long long g = s_tile;
        __syncthreads();
        if (g >= ntiles) break;
        int b = 0;
        while (b + 1 < desc->nbeams && g >= desc->tile_start[b + 1]) ++b;
        const TiledArgs a = desc->beam[b];
        const long long local = g - desc->tile_start[b];
        if (!dd_tile<DT, W, NP, G>(a, (int)(local % a.n_dmb), local / a.n_dmb, smem, phase)) break;
        __syncthreads();
    }
}

template <int DT, int W, int NP, int G>
dd_status launch_tiled_t(const Plan *p, const ShapeTable &st, const uint8_t *d_in, size_t ld_in_bytes,
                         size_t nsamp_in, uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
    constexpr int D = kWarps * DT;
    constexpr long long T = 16LL * 32 * W;
    TiledArgs a;
    a.in = reinterpret_cast<const uint32_t *>(d_in);
    a.ld_w = (long long)(ld_in_bytes / 4);
    a.tab = st.tab;
    a.wsrel = st.wsrel;
    a.nchan = p->nchan;
    a.ndm = p->ndm;
    a.nout = (long long)nsamp_in - p->maxdelay;
    a.out = d_out;
    a.ld_out = (long long)ld_out;
    a.slot = st.slot;
    a.n_dmb = st.n_dmb;
    const dd_status es = tile_error_word(&a.err);
    if (es != DD_OK) return es;
    a.poll_limit = tiled::kStagePollLimit;
    const long long ntiles = (a.nout + T - 1) / T;
    const long long nblocks = ntiles * a.n_dmb;
    if (nblocks > 0x7fffffffLL) return fail(DD_ERR_INVALID_ARG, "gulp too long for one launch");
    const size_t smem = tiled_smem_bytes(p, st, D);
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        DD_CUDA_TRY(cudaFuncSetAttribute(dd_tiled_kernel<DT, W, NP, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        configured = smem;
    }
    dd_tiled_kernel<DT, W, NP, G><<<(unsigned)nblocks, kThreads, smem, stream>>>(a);
    return cuda_fail(cudaGetLastError(), "dd_tiled_kernel launch");
}

// The (DMs per warp, words per lane) shapes instantiated for every stage size.
#define DD_TILED_SHAPES(X) X(1, 2) X(2, 1) X(2, 2) X(4, 1) X(1, 4) X(1, 3) X(2, 3) X(1, 5)

// Launch of shape s with stage size G: 11 bit-planes, or 15 for bands of 2048
// channels or more when BIG (the stage sizes other than 64 serve narrower
// bands only).
template <int G, bool BIG>
dd_status launch_group(const Plan *p, const TiledShape &s, const ShapeTable &st, const uint8_t *d_in,
                       size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
    const bool big = p->nchan >= 2048;
    if (big && !BIG) return fail(DD_ERR_INVALID_ARG, "a %d-channel stage is instantiated for bands below 2048", G);
#define DD_ONE(dt, w)                                                                                           \
    if (s.dms_per_warp == dt && s.words_per_lane == w) {                                                        \
        if constexpr (BIG) {                                                                                    \
            if (big) return launch_tiled_t<dt, w, 15, G>(p, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream); \
        }                                                                                                       \
        return launch_tiled_t<dt, w, 11, G>(p, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);        \
    }
    DD_TILED_SHAPES(DD_ONE)
#undef DD_ONE
    return fail(DD_ERR_INVALID_ARG, "unsupported tiled kernel shape");
}

template <int G, bool BIG>
BatchKernelFn batch_group(const TiledShape &s, bool big) {
    if (big && !BIG) return nullptr;
#define DD_ONE(dt, w)                                                                                           \
    if (s.dms_per_warp == dt && s.words_per_lane == w) {                                                        \
        if constexpr (BIG) {                                                                                    \
            if (big) return dd_batch_kernel<dt, w, 15, G>;                                                      \
        }                                                                                                       \
        return dd_batch_kernel<dt, w, 11, G>;                                                                   \
    }
    DD_TILED_SHAPES(DD_ONE)
#undef DD_ONE
    return nullptr;
}

}  // namespace tiled
}  // namespace dd
