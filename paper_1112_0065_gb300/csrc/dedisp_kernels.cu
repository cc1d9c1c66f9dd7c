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
constexpr int kGroup = 64;  // channels per stage == one carry-save group
constexpr int kPlanes = 7;  // bit-planes for counts 0..64

struct TiledArgs {
    const uint32_t *in;  // packed input as 32-bit words (16 samples each)
    long long ld_w;      // words per channel row
    const int32_t *delays;
    int nchan;
    int ndm;
    long long nout;
    uint32_t *out;
    long long ld_out;
    int slot;  // shared-memory words per staged channel
    int n_dmb; // DM blocks
};

// Full adder on 32 independent bit positions: sum and carry of a+b+c.
__device__ __forceinline__ void full_add(uint32_t &carry, uint32_t &sum, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    sum = u ^ c;
    carry = (a & b) | (u & c);
}

template <int DT, int W>
struct Ctx {
    const uint32_t *win;  // staged windows, kGroup slots of `slot` words
    const int *off;       // [D][kGroup] sample offset of each trial into its channel slot
    int slot;
    int cn;               // channels present in this group (<= kGroup)
    int lane;
    int jbase;            // first trial of this warp within the CTA
};

// 16 samples of channel c realigned to trial jj's delay, for each of the lane's W words.
template <int DT, int W>
__device__ __forceinline__ void fetch(const Ctx<DT, W> &x, int c, uint32_t (&v)[DT][W]) {
    if (c >= x.cn) {
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i) v[jj][i] = 0u;
        return;
    }
#pragma unroll
    for (int jj = 0; jj < DT; ++jj) {
        const int o = x.off[(x.jbase + jj) * kGroup + c];
        const uint32_t *p = x.win + c * x.slot + (o >> 4) + x.lane;
        const unsigned sh = (unsigned)(o & 15) * 2u;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint32_t lo = p[32 * i];
            const uint32_t hi = p[32 * i + 1];
            v[jj][i] = __funnelshift_r(lo, hi, sh);
        }
    }
}

// Harley-Seal: fold channels [cb, cb + 2^L) into the bit-planes; returns the
// carry of weight 2^L.
template <int L, int DT, int W>
__device__ __forceinline__ void hs(const Ctx<DT, W> &x, uint32_t (&P)[DT][W][kPlanes], uint32_t (&carry)[DT][W],
                                   int cb) {
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

template <int DT, int W>
__global__ void __launch_bounds__(kThreads, (DT * W > 4) ? 1 : 2) dd_tiled_kernel(const TiledArgs a) {
    constexpr int D = kWarps * DT;
    constexpr int TW = 32 * W;
    constexpr long long T = 16LL * TW;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *s_win = smem;
    int *s_off = reinterpret_cast<int *>(smem + kGroup * a.slot);

    const int dmb = (int)(blockIdx.x % (unsigned)a.n_dmb);
    const long long tt = (long long)(blockIdx.x / (unsigned)a.n_dmb);
    const int d0 = dmb * D;
    const long long t0 = tt * T;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    // per-sample sums, two 16-bit lanes per register; see the store below for the order
    uint32_t acc[DT][W][8];
#pragma unroll
    for (int jj = 0; jj < DT; ++jj)
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[jj][i][k] = 0u;

    for (int c0 = 0; c0 < a.nchan; c0 += kGroup) {
        const int cn = min(kGroup, a.nchan - c0);
        __syncthreads();
        for (int cl = warp; cl < cn; cl += kWarps) {
            const int c = c0 + cl;
            const long long ws = (t0 + __ldg(a.delays + (long long)d0 * a.nchan + c)) >> 4;
            const uint32_t *row = a.in + (long long)c * a.ld_w;
            uint32_t *dst = s_win + cl * a.slot;
            for (int w = lane; w < a.slot; w += 32) {
                const long long gw = ws + w;
                dst[w] = gw < a.ld_w ? __ldg(row + gw) : 0u;
            }
            for (int j = lane; j < D; j += 32) {
                const int d = min(d0 + j, a.ndm - 1);
                s_off[j * kGroup + cl] = (int)(t0 + __ldg(a.delays + (long long)d * a.nchan + c) - (ws << 4));
            }
        }
        __syncthreads();

        Ctx<DT, W> x{s_win, s_off, a.slot, cn, lane, warp * DT};
        uint32_t P[DT][W][kPlanes];
#pragma unroll
        for (int jj = 0; jj < DT; ++jj)
#pragma unroll
            for (int i = 0; i < W; ++i)
#pragma unroll
                for (int k = 0; k < kPlanes; ++k) P[jj][i][k] = 0u;
        uint32_t top[DT][W];
        hs<6>(x, P, top, 0);

        // planes -> per-sample counts: byte lane m of B[r] is sample 4m+r (<= 192)
#pragma unroll
        for (int jj = 0; jj < DT; ++jj) {
#pragma unroll
            for (int i = 0; i < W; ++i) {
                P[jj][i][6] = top[jj][i];
                uint32_t B[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int k = 0; k < kPlanes; ++k)
#pragma unroll
                    for (int r = 0; r < 4; ++r) B[r] += ((P[jj][i][k] >> (2 * r)) & 0x03030303u) << k;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[jj][i][2 * r] += B[r] & 0x00FF00FFu;             // samples r, 8+r
                    acc[jj][i][2 * r + 1] += (B[r] >> 8) & 0x00FF00FFu;  // samples 4+r, 12+r
                }
            }
        }
    }

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
            for (int r = 0; r < 4; ++r) {
                v[r] = acc[jj][i][2 * r] & 0xFFFFu;
                v[4 + r] = acc[jj][i][2 * r + 1] & 0xFFFFu;
                v[8 + r] = acc[jj][i][2 * r] >> 16;
                v[12 + r] = acc[jj][i][2 * r + 1] >> 16;
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

template <int DT, int W>
dd_status launch_tiled_t(const Plan *p, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                         uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
    constexpr int D = kWarps * DT;
    constexpr long long T = 16LL * 32 * W;
    TiledArgs a;
    a.in = reinterpret_cast<const uint32_t *>(d_in);
    a.ld_w = (long long)(ld_in_bytes / 4);
    a.delays = p->delays_dev;
    a.nchan = p->nchan;
    a.ndm = p->ndm;
    a.nout = (long long)nsamp_in - p->maxdelay;
    a.out = d_out;
    a.ld_out = (long long)ld_out;
    const int spread = max_block_spread(p, D);
    a.slot = 32 * W + 2 + (spread + 15) / 16;
    a.n_dmb = (p->ndm + D - 1) / D;
    const long long ntiles = (a.nout + T - 1) / T;
    const long long nblocks = ntiles * a.n_dmb;
    if (nblocks > 0x7fffffffLL) return fail(DD_ERR_INVALID_ARG, "gulp too long for one launch");
    const size_t smem = (size_t)kGroup * a.slot * 4 + (size_t)D * kGroup * 4;
    if (smem > 227 * 1024) return launch_simple(p, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    static thread_local size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        DD_CUDA_TRY(cudaFuncSetAttribute(dd_tiled_kernel<DT, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        configured = smem;
    }
    dd_tiled_kernel<DT, W><<<(unsigned)nblocks, kThreads, smem, stream>>>(a);
    return cuda_fail(cudaGetLastError(), "dd_tiled_kernel launch");
}

}  // namespace

static const TiledShape kShapes[] = {{1, 2, 64}, {2, 1, 64}, {2, 2, 64}, {4, 1, 64}, {1, 4, 64}, {4, 2, 64}, {2, 4, 64}};

bool tiled_shape_supported(const TiledShape &s) {
    for (const TiledShape &k : kShapes)
        if (k.dms_per_warp == s.dms_per_warp && k.words_per_lane == s.words_per_lane && k.chan_chunk == s.chan_chunk)
            return true;
    return false;
}

std::vector<TiledShape> tiled_shape_candidates() { return std::vector<TiledShape>(std::begin(kShapes), std::end(kShapes)); }

// 16-bit lane sums hold up to 65535 = 3 * 21845 channels.
int tiled_max_nchan() { return 21845; }

dd_status launch_tiled(const Plan *p, const TiledShape &s, const uint8_t *d_in, size_t ld_in_bytes, size_t nsamp_in,
                       uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
#define DD_SHAPE(dt, w) \
    if (s.dms_per_warp == dt && s.words_per_lane == w) \
        return launch_tiled_t<dt, w>(p, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
    DD_SHAPE(1, 2)
    DD_SHAPE(2, 1)
    DD_SHAPE(2, 2)
    DD_SHAPE(4, 1)
    DD_SHAPE(1, 4)
    DD_SHAPE(4, 2)
    DD_SHAPE(2, 4)
#undef DD_SHAPE
    return fail(DD_ERR_INVALID_ARG, "unsupported tiled kernel shape");
}

}  // namespace dd
