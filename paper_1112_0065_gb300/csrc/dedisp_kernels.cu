// Direct dedispersion kernels for sm_103a (paper Section 2.2).
//
//   out[d][t] = sum_c x[c][t + delay[d][c]]     (exact uint32)
//
// Two kernels:
//  * dd_simple_kernel -- one thread per (DM, 4 consecutive samples), every
//    sample fetched from global memory.  Kept as a checking aid and for band
//    shapes the tiled kernel does not cover.
//  * dd_tiled_kernel  -- the production kernel.  A CTA owns D = 8*DT
//    consecutive DM trials and a tile of 512*W output samples.  For each chunk
//    of 64 channels the packed 2-bit window of every channel that the CTA's
//    DMs need is staged once in shared memory (still packed: 16 samples per
//    32-bit word), and then reused by all D trials.  A lane owns W words of 16
//    consecutive output samples for DT trials.  For every (trial, channel) it
//    realigns the staged window to the trial's delay with one funnel shift,
//    giving 16 samples as 2-bit lanes of one register, and adds them into
//    bit-sliced counters with a carry-save adder tree (Harley-Seal): 64
//    channels go into 7 bit-planes with 63 full adders, two 3-input logic ops
//    each, i.e. about 2 logic ops per 16 sample-additions.  After each
//    64-channel group the planes are turned back into per-sample sums (byte
//    lanes, then 16-bit lanes) that stay in registers across the whole band.
//    There are no tensor cores here: the work is a gather-sum, not a dense
//    contraction.
#include <algorithm>

#include "dd_internal.h"

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

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kGroup = 64;  // channels per shared-memory stage (one carry-save tree)

struct TiledArgs {
    const uint32_t *in;     // packed input as 32-bit words (16 samples each)
    long long ld_w;         // words per channel row
    const uint32_t *tab;    // [n_dmb][nchan][D]: (slot word address << 5) | funnel shift, per (channel, trial)
    const int32_t *wsrel;   // [n_dmb][nchan]: first staged word of the channel, relative to the tile
    int nchan;
    int ndm;
    long long nout;
    uint32_t *out;
    long long ld_out;
    int slot;   // shared-memory words per staged channel
    int n_dmb;  // DM blocks
};

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Full adder on 32 independent bit positions: sum and carry of a+b+c.
__device__ __forceinline__ void full_add(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    sum = u ^ c;
    carry = (a & b) | (u & c);
}

template <int DT, int W>
struct Ctx {
    const uint32_t *win;  // staged windows of this stage
    const uint32_t *tab;  // [kGroup][D] packed (address, shift)
    int cn;               // channels present in this stage (<= kGroup)
    int lane;
    int jbase;            // first trial of this warp within the CTA
};

// 16 samples of channel c realigned to trial jj's delay, for each of the lane's
// W words (words lane, lane+32, ...): one funnel shift of two staged words.
template <int DT, int W>
__device__ __forceinline__ void fetch(const Ctx<DT, W> &x, int c, uint32_t (&v)[DT][W]) {
    if (c >= x.cn) {
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) v[jj][i] = 0u;
        return;
    }
    constexpr int D = kWarps * DT;
#pragma unroll
    for (int jj = 0; jj < DT; ++jj) {
        const uint32_t e = x.tab[c * D + x.jbase + jj];
        const uint32_t *p = x.win + (e >> 5) + x.lane;
        const unsigned sh = e & 31u;
#pragma unroll
        for (int i = 0; i < W; ++i) v[jj][i] = __funnelshift_r(p[32 * i], p[32 * i + 1], sh);
    }
}

// Harley-Seal carry-save tree: add channels [cb, cb + 2^L) into bit-planes
// P[0..L-1] (bit k of plane P[k] counts 2^k); returns the carry of weight 2^L.
template <int L, int DT, int W, int NP>
__device__ __forceinline__ void hs(const Ctx<DT, W> &x, uint32_t (&P)[DT][W][NP], uint32_t (&carry)[DT][W], int cb) {
    if constexpr (L == 1) {
        uint32_t a[DT][W], b[DT][W];
        fetch(x, cb, a);
        fetch(x, cb + 1, b);
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) full_add(carry[jj][i], P[jj][i][0], P[jj][i][0], a[jj][i], b[jj][i]);
    } else {
        uint32_t ca[DT][W], cc[DT][W];
        hs<L - 1>(x, P, ca, cb);
        hs<L - 1>(x, P, cc, cb + (1 << (L - 1)));
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i)
                full_add(carry[jj][i], P[jj][i][L - 1], P[jj][i][L - 1], ca[jj][i], cc[jj][i]);
    }
}

template <int DT, int W, int NP>
__global__ void __launch_bounds__(kThreads, (DT * W * NP > 48) ? 1 : 2) dd_tiled_kernel(const TiledArgs a) {
    constexpr int D = kWarps * DT;
    constexpr int TW = 32 * W;
    constexpr long long T = 16LL * TW;
    extern __shared__ __align__(16) uint32_t smem[];
    // two stages of [kGroup][slot] windows, then two of [kGroup][D] tables, then the channel bases
    uint32_t *const s_win0 = smem;
    uint32_t *const s_tab0 = smem + 2 * kGroup * a.slot;
    int32_t *s_ws = reinterpret_cast<int32_t *>(smem + 2 * kGroup * a.slot + 2 * kGroup * D);

    const int dmb = (int)(blockIdx.x % (unsigned)a.n_dmb);
    const long long tt = (long long)(blockIdx.x / (unsigned)a.n_dmb);
    const int d0 = dmb * D;
    const long long t0 = tt * T;
    const long long tw0 = t0 >> 4;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t *gtab = a.tab + (long long)dmb * a.nchan * D;
    const int32_t *gws = a.wsrel + (long long)dmb * a.nchan;
    const int nchunks = (a.nchan + kGroup - 1) / kGroup;

    for (int c = threadIdx.x; c < a.nchan; c += kThreads) s_ws[c] = __ldg(gws + c);
    __syncthreads();

    // copy one stage: every channel's packed window and its (address, shift) table rows
    auto stage = [&](int k, int b) {
        const int c0 = k * kGroup;
        const int cn = min(kGroup, a.nchan - c0);
        uint32_t *dst = s_win0 + b * (kGroup * a.slot);
        for (int cl = warp; cl < cn; cl += kWarps) {
            const int c = c0 + cl;
            const long long ws = tw0 + s_ws[c];
            const uint32_t *row = a.in + (long long)c * a.ld_w;
            for (int w = lane; w < a.slot; w += 32) {
                // words past the row end only ever feed outputs beyond nout: clamp the source
                const long long g = min(ws + w, a.ld_w - 1);
                cp_async4(dst + cl * a.slot + w, row + g);
            }
        }
        const uint32_t *src = gtab + (long long)c0 * D;
        uint32_t *tdst = s_tab0 + b * (kGroup * D);
        for (int i = threadIdx.x; i < cn * D / 4; i += kThreads) cp_async16(tdst + 4 * i, src + 4 * i);
        cp_async_commit();
    };

    uint32_t P[DT][W][NP];
#pragma unroll
    for (int jj = 0; jj < DT; ++jj)
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int k = 0; k < NP; ++k) P[jj][i][k] = 0u;

    stage(0, 0);
    for (int k = 0; k < nchunks; ++k) {
        if (k + 1 < nchunks) {
            stage(k + 1, (k + 1) & 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        Ctx<DT, W> x{s_win0 + (k & 1) * (kGroup * a.slot), s_tab0 + (k & 1) * (kGroup * D),
                     min(kGroup, a.nchan - k * kGroup), lane, warp * DT};
        uint32_t c64[DT][W];
        hs<6>(x, P, c64, 0);
        // ripple the weight-64 carry into the upper planes
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) {
                uint32_t c = c64[jj][i];
#pragma unroll
                for (int l = 6; l < NP; ++l) {
                    const uint32_t s = P[jj][i][l] ^ c;
                    c &= P[jj][i][l];
                    P[jj][i][l] = s;
                }
            }
        __syncthreads();
    }

    // bit-planes -> per-sample sums.  2-bit lane r of a plane holds (low bit,
    // high bit) of sample r; masking lanes r and r+8 into 16-bit halves gives
    // sum_k 2^k * lane = count(low) + 2*count(high) <= 3*nchan < 65536.
#pragma unroll
    for (int jj = 0; jj < DT; ++jj) {
        const int d = d0 + warp * DT + jj;
        if (d >= a.ndm) continue;
        uint32_t *orow = a.out + (long long)d * a.ld_out;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const long long t = t0 + 16LL * (lane + 32 * i);
            if (t >= a.nout) continue;
            uint32_t v[16];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                uint32_t h = 0u;
#pragma unroll
                for (int k = 0; k < NP; ++k) h += ((P[jj][i][k] >> (2 * r)) & 0x00030003u) << k;
                v[r] = h & 0xFFFFu;
                v[r + 8] = h >> 16;
            }
            if (t + 16 <= a.nout) {
                uint4 *o4 = reinterpret_cast<uint4 *>(orow + t);
#pragma unroll
                for (int q = 0; q < 4; ++q) o4[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else {
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    if (t + m < a.nout) orow[t + m] = v[m];
            }
        }
    }
}

template <int DT, int W, int NP>
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
    const long long ntiles = (a.nout + T - 1) / T;
    const long long nblocks = ntiles * a.n_dmb;
    if (nblocks > 0x7fffffffLL) return fail(DD_ERR_INVALID_ARG, "gulp too long for one launch");
    const size_t smem = tiled_smem_bytes(p, st, D);
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        DD_CUDA_TRY(cudaFuncSetAttribute(dd_tiled_kernel<DT, W, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        configured = smem;
    }
    dd_tiled_kernel<DT, W, NP><<<(unsigned)nblocks, kThreads, smem, stream>>>(a);
    return cuda_fail(cudaGetLastError(), "dd_tiled_kernel launch");
}

}  // namespace

size_t tiled_smem_bytes(const Plan *p, const ShapeTable &st, int D) {
    return (size_t)2 * kGroup * st.slot * 4 + (size_t)2 * kGroup * D * 4 + (size_t)p->nchan * 4;
}

static const TiledShape kShapes[] = {{1, 2, 64}, {2, 1, 64}, {2, 2, 64}, {4, 1, 64}, {1, 4, 64}};

bool tiled_shape_supported(const TiledShape &s) {
    for (const TiledShape &k : kShapes)
        if (k.dms_per_warp == s.dms_per_warp && k.words_per_lane == s.words_per_lane && k.chan_chunk == s.chan_chunk)
            return true;
    return false;
}

std::vector<TiledShape> tiled_shape_candidates() { return std::vector<TiledShape>(std::begin(kShapes), std::end(kShapes)); }

// bit-planes count up to 2^15-1 channels; the 16-bit sums hold 3*nchan <= 65535
int tiled_max_nchan() { return 21845; }

dd_status ensure_shape_table(Plan *p, const TiledShape &s) {
    const int key = s.dms_per_warp * 100 + s.words_per_lane;
    if (p->tables.count(key)) return DD_OK;
    const int D = kWarps * s.dms_per_warp;
    ShapeTable st;
    st.n_dmb = (p->ndm + D - 1) / D;
    const int spread = max_block_spread(p, D);
    st.slot = 32 * s.words_per_lane + 2 + (spread + 15) / 16;
    if (tiled_smem_bytes(p, st, D) > 227 * 1024)
        return fail(DD_ERR_INVALID_ARG, "delay spread too large for the tiled kernel's shared memory");
    std::vector<uint32_t> tab((size_t)st.n_dmb * p->nchan * D);
    std::vector<int32_t> wsrel((size_t)st.n_dmb * p->nchan);
    for (int b = 0; b < st.n_dmb; ++b) {
        const int d0 = b * D;
        for (int c = 0; c < p->nchan; ++c) {
            const int32_t dl0 = p->delays_host[(size_t)d0 * p->nchan + c];
            wsrel[(size_t)b * p->nchan + c] = dl0 >> 4;
            const int cl = c % kGroup;
            for (int j = 0; j < D; ++j) {
                const int d = std::min(d0 + j, p->ndm - 1);
                const int32_t o = (dl0 & 15) + p->delays_host[(size_t)d * p->nchan + c] - dl0;
                const uint32_t addr = (uint32_t)(cl * st.slot + (o >> 4));
                tab[((size_t)b * p->nchan + c) * D + j] = (addr << 5) | (uint32_t)(2 * (o & 15));
            }
        }
    }
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
    auto it = p->tables.find(s.dms_per_warp * 100 + s.words_per_lane);
    if (it == p->tables.end()) return fail(DD_ERR_INTERNAL, "tiled kernel table missing for this shape");
    const ShapeTable &st = it->second;
    const bool big = p->nchan >= 2048;
#define DD_SHAPE(dt, w)                                                                                          \
    if (s.dms_per_warp == dt && s.words_per_lane == w)                                                          \
        return big ? launch_tiled_t<dt, w, 15>(p, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream)      \
                   : launch_tiled_t<dt, w, 11>(p, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    DD_SHAPE(1, 2)
    DD_SHAPE(2, 1)
    DD_SHAPE(2, 2)
    DD_SHAPE(4, 1)
    DD_SHAPE(1, 4)
#undef DD_SHAPE
    return fail(DD_ERR_INVALID_ARG, "unsupported tiled kernel shape");
}

}  // namespace dd
