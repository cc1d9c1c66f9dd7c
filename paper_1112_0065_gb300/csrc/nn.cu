// Candidate classifier: a small CNN over 64x64 DM-time snippets with bfloat16
// weights and activations and float accumulation, trained on the GPU by its
// own forward, backward and AdamW kernels.
//
// Network: four 3x3 convolutions (1->16->32->64->64 channels, zero padding,
// ReLU, 2x2 max pooling), fc 1024->128 (ReLU), fc 128->1 (logit); 191553
// parameters in one flat vector (order and flattening as in include/dd.h).
//
// Numerics: every sum starts from the bias and adds products in increasing
// (input channel, ky, kx) / input order, one thread per output, with fmaf --
// a product of two bfloat16 values is exact in float, so each step rounds
// once and the result equals a plain float sum in that order.  Activations
// after ReLU are rounded to bfloat16 (nearest even); pooling keeps the first
// maximum.  Gradients are float; each weight gradient is a two-stage sum
// (fixed chunks of the batch, then the chunks in order), so training is
// deterministic.  These are CUDA-core kernels (~12.5 M multiply-adds per
// snippet): the fixed summation order is what makes the logits reproducible
// bit for bit, which the tensor cores' internal accumulation order is not.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "dd_internal.h"
#include "tc.cuh"

namespace dd {
namespace {

constexpr int kConvLayers = 4;
constexpr int kCin[kConvLayers] = {1, 16, 32, 64};
constexpr int kCout[kConvLayers] = {16, 32, 64, 64};
constexpr int kHin[kConvLayers] = {64, 32, 16, 8};
constexpr int kFcIn = 1024, kFcHid = 128;
constexpr int kChunk = 16;  // samples per first-stage weight-gradient partial

struct Layout {
    long long cw[kConvLayers], cb[kConvLayers], f1w, f1b, f2w, f2b, total;
};

Layout make_layout() {
    Layout L;
    long long o = 0;
    for (int l = 0; l < kConvLayers; ++l) {
        L.cw[l] = o;
        o += (long long)kCout[l] * kCin[l] * 9;
        L.cb[l] = o;
        o += kCout[l];
    }
    L.f1w = o;
    o += (long long)kFcHid * kFcIn;
    L.f1b = o;
    o += kFcHid;
    L.f2w = o;
    o += kFcHid;
    L.f2b = o;
    o += 1;
    L.total = o;
    return L;
}

__device__ __forceinline__ float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
__device__ __forceinline__ uint16_t f2bf(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// ---- forward -------------------------------------------------------------------

// Forward convolution + ReLU + pooling, register-tiled and persistent.  A
// thread owns 8 output channels x a 2x4 block of convolution outputs (two
// pooled outputs side by side): per input channel it reads a 4x6 input patch
// and 9x8 weights from shared memory and issues 576 FMAs.  One 512-thread
// block per SM keeps the weights of its COB output channels resident
// ([ci][tap][co], float, copied from a per-call float image) and walks groups
// of SPB snippets; each group's inputs arrive in stages of CIC input channels
// by 4-byte cp.async copies into a ring of NBUF buffers, so the copies of
// the next NBUF - 1 stages overlap the FMAs of this one.
//
// Staged layout of a snippet (bfloat16, row stride RS >= H + 2, RS % 4 == 0):
// two leading zeros, then per channel one zero row followed by its H data rows
// (row data at offsets 0..H-1, zeros at H..RS-1), then one closing zero row.
// Padded coordinate (Y, X), 0 <= Y, X <= H + 1, of channel c sits at element
// 2 + (c(H+1) + Y) RS + X - 1: the left halo is the previous row's last zero,
// the right halo this row's first, the top and bottom halos are zero rows.  A
// thread reads a patch row with two 8-byte loads at offsets 4tx-2 and 4tx+2;
// RS is chosen so the half-warps' loads hit distinct banks.  Buffers are
// zeroed once; copies only ever write data elements.
//
// A halo tap adds w*0 to the sum, which leaves it unchanged (only the sign of
// an exact zero can differ, and the ReLU maps both zeros to +0), so every
// output equals the in-order sum from the bias over (ci, ky, kx) with the
// padded taps skipped.
constexpr int kConvThreads = 512;

template <int CI, int CO, int H, int COB, int SPB, int CIC, int RS, int NBUF>
struct ConvFwdCfg {
    static constexpr int HO = H / 2;
    static constexpr int PT = (H / 2) * (H / 4);  // 2x4 pixel tiles per snippet
    static constexpr int CTN = COB / 8;           // 8-channel tiles per block
    static constexpr int TILES = PT * CTN * SPB;  // thread tiles per block
    static constexpr int TPT = TILES / kConvThreads;  // tiles per thread
    static constexpr int NCB = CO / COB;          // output-channel blocks
    static constexpr int NK = CI / CIC;           // stages per snippet group
    static constexpr int CH = (H + 1) * RS;       // staged elements per channel
    static constexpr int SNIP = (2 + (CIC * (H + 1) + 1) * RS + 7) / 8 * 8;  // staged elements per snippet
    static constexpr int BUF = SPB * SNIP;        // elements per stage buffer
    static constexpr int W_FLOATS = CI * 9 * COB;
    static constexpr int CPS = SPB * CIC * H * H / 2;  // 4-byte copies per stage
    static constexpr size_t SMEM = (size_t)W_FLOATS * 4 + (size_t)NBUF * BUF * 2;
    static_assert(COB % 8 == 0 && CO % COB == 0 && H % 4 == 0 && CI % CIC == 0, "tile shape");
    static_assert(NBUF >= 2 && NBUF <= 4, "stage buffers");
    static_assert(TILES % kConvThreads == 0 && (TPT == 1 || CIC == CI), "whole tiles per thread");
    static_assert(RS % 4 == 0 && RS >= H + 2, "row stride");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Float image of a layer's weights in the staged order: dst[cb][ci][tap][co]
// = w[cb*COB + co][ci][tap] for every output-channel block cb.
struct WPrepLayer {
    const uint16_t *w;
    float *dst;
    int ci, cob, count;
};
struct WPrepArgs {
    WPrepLayer l[kConvLayers];
};

__global__ void conv_wprep_kernel(const WPrepArgs a) {
    const WPrepLayer L = a.l[blockIdx.y];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.count; i += gridDim.x * blockDim.x) {
        const int co = i % L.cob, k = (i / L.cob) % 9, ci = (i / (L.cob * 9)) % L.ci, cb = i / (L.cob * 9 * L.ci);
        L.dst[i] = bf2f(L.w[((cb * L.cob + co) * L.ci + ci) * 9 + k]);
    }
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
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

// Two float FMAs in one instruction (fma.rn.f32x2): each half is rounded to
// nearest exactly like fmaf, so pairing output channels changes no result;
// it halves the FMA instructions the schedulers issue.
__device__ __forceinline__ uint64_t pk2(float lo, float hi) {
    uint64_t d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float lo_f(uint64_t v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_f(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// acc += the taps of nci input channels: channel i's patch row r at
// xb + i*CH + r*RS (the 8-byte words holding padded columns 4tx-1 .. 4tx+4),
// its weights at wb + i*9*COB.  acc[cp][r][q] holds output channels 2cp (low
// half) and 2cp+1 (high half) of output (r, q) of the thread's 2x4 block.
template <int COB, int CH, int RS>
__device__ __forceinline__ void conv_accumulate(uint64_t (&acc)[4][2][4], const uint16_t *xb, const float *wb,
                                                int nci) {
#pragma unroll 1
    for (int ci = 0; ci < nci; ++ci) {
        uint64_t p[4][6];  // each input value in both halves
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const uint2 a = *reinterpret_cast<const uint2 *>(xb + ci * CH + r * RS);
            const uint2 c = *reinterpret_cast<const uint2 *>(xb + ci * CH + r * RS + 4);
            const float v[6] = {__uint_as_float(a.x & 0xffff0000u), __uint_as_float(a.y << 16),
                                __uint_as_float(a.y & 0xffff0000u), __uint_as_float(c.x << 16),
                                __uint_as_float(c.x & 0xffff0000u), __uint_as_float(c.y << 16)};
#pragma unroll
            for (int k = 0; k < 6; ++k) p[r][k] = pk2(v[k], v[k]);
        }
        const float *wk = wb + ci * 9 * COB;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const float4 wa = *reinterpret_cast<const float4 *>(wk + (ky * 3 + kx) * COB);
                const float4 wc = *reinterpret_cast<const float4 *>(wk + (ky * 3 + kx) * COB + 4);
                const uint64_t wv[4] = {pk2(wa.x, wa.y), pk2(wa.z, wa.w), pk2(wc.x, wc.y), pk2(wc.z, wc.w)};
#pragma unroll
                for (int cp = 0; cp < 4; ++cp)
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[cp][r][q] = ffma2(wv[cp], p[r + ky][q + kx], acc[cp][r][q]);
            }
    }
}

// ReLU, bfloat16 rounding and 2x2 max pooling (first maximum) of a thread's
// tile.  ARG: also record which of the four is the first maximum (training
// needs it).  Without ARG the window's float maximum is rounded once: ReLU and
// round-to-nearest are both non-decreasing, so the largest rounded value is
// the rounded largest value (a NaN counts as 0 either way), bit for bit.
template <int CO, int HO, bool ARG>
__device__ __forceinline__ void conv_epilogue(const uint64_t (&acc)[4][2][4], int n, int co_first, int ty, int tx,
                                              uint16_t *__restrict__ pooled, uint8_t *__restrict__ arg) {
    if constexpr (!ARG) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t packed = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                float m = -INFINITY;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t pr = acc[c / 2][q / 2][2 * j + q % 2];
                    m = fmaxf(m, (c & 1) ? hi_f(pr) : lo_f(pr));  // fmaxf drops NaNs
                }
                packed |= (uint32_t)f2bf(m > 0.0f ? m : 0.0f) << (16 * j);  // ReLU: +0 for -0, 0 and NaN
            }
            const long long o = (((long long)n * CO + co_first + c) * HO + ty) * HO + 2 * tx;
            *reinterpret_cast<uint32_t *>(pooled + o) = packed;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t packed = 0;
            uint32_t args = 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                // after the ReLU every value is a non-negative bfloat16 (+0 for
                // x <= 0 or NaN), whose bit patterns order like the values
                uint32_t best = 0;
                int a = 0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t pr = acc[c / 2][q / 2][2 * j + q % 2];
                    const float x = (c & 1) ? hi_f(pr) : lo_f(pr);
                    const uint32_t r = f2bf(x > 0.0f ? x : 0.0f);
                    if (q == 0 || r > best) {
                        best = r;
                        a = q;
                    }
                }
                packed |= best << (16 * j);
                args |= (uint32_t)a << (8 * j);
            }
            const long long o = (((long long)n * CO + co_first + c) * HO + ty) * HO + 2 * tx;
            *reinterpret_cast<uint32_t *>(pooled + o) = packed;
            *reinterpret_cast<uint16_t *>(arg + o) = (uint16_t)args;
        }
    }
}

template <int CI, int CO, int H, int COB, int SPB, int CIC, int RS, int NBUF, bool ARG>
__global__ void __launch_bounds__(kConvThreads, 1)
    conv_fwd_kernel(const uint16_t *__restrict__ in, const float *__restrict__ wprep, const uint16_t *__restrict__ b,
                    int N, uint16_t *__restrict__ pooled, uint8_t *__restrict__ arg) {
    using C = ConvFwdCfg<CI, CO, H, COB, SPB, CIC, RS, NBUF>;
    constexpr int HO = C::HO;
    extern __shared__ __align__(16) unsigned char smem[];
    float *ws = reinterpret_cast<float *>(smem);
    uint16_t *xs = reinterpret_cast<uint16_t *>(smem + (size_t)C::W_FLOATS * 4);
    const int tid = threadIdx.x;
    // the grid is a multiple of NCB: block i serves channel block i % NCB
    const int cb = blockIdx.x % C::NCB, cta = blockIdx.x / C::NCB, ncta = gridDim.x / C::NCB;
    const int ngroups = (N + SPB - 1) / SPB;
    const int nst = cta < ngroups ? (ngroups - cta + ncta - 1) / ncta * C::NK : 0;
    uint4 *z = reinterpret_cast<uint4 *>(xs);
    for (int i = tid; i < NBUF * C::BUF / 8; i += kConvThreads) z[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
    const float *wsrc = wprep + (size_t)cb * C::W_FLOATS;
    for (int i = tid; i < C::W_FLOATS / 4; i += kConvThreads) cp_async16(ws + 4 * i, wsrc + 4 * i);
    // stage s: group cta + ncta*(s / NK), input channels [k*CIC, (k+1)*CIC), k = s % NK
    auto issue = [&](int s) {
        const int g = cta + ncta * (s / C::NK), c0 = (s % C::NK) * CIC;
        uint16_t *dst = xs + (s % NBUF) * C::BUF;
#pragma unroll 4
        for (int i = tid; i < C::CPS; i += kConvThreads) {
            const int x2 = i % (H / 2), y = (i / (H / 2)) % H, cl = (i / (H * H / 2)) % CIC, j = i / (CIC * H * H / 2);
            const int n = g * SPB + j;
            if (n < N)
                cp_async4(dst + j * C::SNIP + 2 + (cl * (H + 1) + y + 1) * RS + 2 * x2,
                          in + (((long long)n * CI + c0 + cl) * H + y) * H + 2 * x2);
        }
    };
    // stages 0 .. NBUF-2 in flight (the weights travel with stage 0)
#pragma unroll
    for (int q = 0; q < NBUF - 1; ++q) {
        if (q < nst) issue(q);
        cp_async_commit();
    }
    uint64_t acc[4][2][4];
#pragma unroll 1
    for (int s = 0; s < nst; ++s) {
        // stage s + NBUF - 1 goes to the buffer stage s - 1 used (released by
        // the barrier that ended iteration s - 1)
        if (s + NBUF - 1 < nst) issue(s + NBUF - 1);
        cp_async_commit();
        cp_async_wait<NBUF - 1>();  // every group but the newest NBUF - 1: stage s is in
        __syncthreads();
        const int k = s % C::NK;
#pragma unroll 1
        for (int q = 0; q < C::TPT; ++q) {  // TPT > 1 only with one stage per group
            const int tile = tid + q * kConvThreads;
            const int pt = tile % C::PT, ct = (tile / C::PT) % C::CTN, sj = tile / (C::PT * C::CTN);
            const int ty = pt / (H / 4), tx = pt % (H / 4);
            const int cof = cb * COB + ct * 8;
            if (k == 0) {
#pragma unroll
                for (int cp = 0; cp < 4; ++cp) {
                    const uint64_t bias = pk2(bf2f(b[cof + 2 * cp]), bf2f(b[cof + 2 * cp + 1]));
#pragma unroll
                    for (int r = 0; r < 2; ++r)
#pragma unroll
                        for (int qq = 0; qq < 4; ++qq) acc[cp][r][qq] = bias;
                }
            }
            conv_accumulate<COB, C::CH, RS>(acc, xs + (s % NBUF) * C::BUF + sj * C::SNIP + 2 * ty * RS + 4 * tx,
                                            ws + k * CIC * 9 * COB + ct * 8, CIC);
            if (k == C::NK - 1) {
                const int n = (cta + ncta * (s / C::NK)) * SPB + sj;
                if (n < N) conv_epilogue<CO, HO, ARG>(acc, n, cof, ty, tx, pooled, arg);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

// fc1 (1024 -> 128, ReLU) of the tensor-core forward (channel-last
// features): a block computes 8 snippets x 128 outputs, a thread one output
// of 4 snippets; the snippets' features sit in shared memory (float) and each
// thread streams its weight row with 16-byte loads.  Every sum runs over the
// inputs in increasing order.
constexpr int kFc1Rows = 8;

// NHWC: the features are stored channel-last ([4][4][64]); feature f of the
// network's (channel, y, x) flattening then sits at (f % 16) * 64 + f / 16.
template <bool NHWC>
__global__ void __launch_bounds__(256) fc1_fwd_kernel(const uint16_t *__restrict__ feat,
                                                      const uint16_t *__restrict__ w,
                                                      const uint16_t *__restrict__ b, int N,
                                                      uint16_t *__restrict__ h1) {
    __shared__ __align__(16) float xs[kFc1Rows][kFcIn];
    const int o = threadIdx.x % kFcHid, sg = threadIdx.x / kFcHid;
    const int n0 = blockIdx.x * kFc1Rows;
#pragma unroll 4
    for (int e = threadIdx.x; e < kFc1Rows * kFcIn; e += 256) {
        const int r = e / kFcIn, i = e % kFcIn;
        const int src = NHWC ? (i % 16) * 64 + i / 16 : i;
        xs[r][i] = (n0 + r < N) ? bf2f(__ldg(feat + (long long)(n0 + r) * kFcIn + src)) : 0.0f;
    }
    __syncthreads();
    float acc[4];
    const float bias = bf2f(b[o]);
#pragma unroll
    for (int s = 0; s < 4; ++s) acc[s] = bias;
    const uint4 *wr = reinterpret_cast<const uint4 *>(w + (long long)o * kFcIn);  // 16-byte aligned rows
#pragma unroll 4
    for (int i8 = 0; i8 < kFcIn / 8; ++i8) {
        const uint4 wq = __ldg(wr + i8);
        const float wf[8] = {__uint_as_float(wq.x << 16), __uint_as_float(wq.x & 0xffff0000u),
                             __uint_as_float(wq.y << 16), __uint_as_float(wq.y & 0xffff0000u),
                             __uint_as_float(wq.z << 16), __uint_as_float(wq.z & 0xffff0000u),
                             __uint_as_float(wq.w << 16), __uint_as_float(wq.w & 0xffff0000u)};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float4 xa = *reinterpret_cast<const float4 *>(&xs[sg * 4 + s][i8 * 8]);
            const float4 xc = *reinterpret_cast<const float4 *>(&xs[sg * 4 + s][i8 * 8 + 4]);
            acc[s] = fmaf(wf[0], xa.x, acc[s]);
            acc[s] = fmaf(wf[1], xa.y, acc[s]);
            acc[s] = fmaf(wf[2], xa.z, acc[s]);
            acc[s] = fmaf(wf[3], xa.w, acc[s]);
            acc[s] = fmaf(wf[4], xc.x, acc[s]);
            acc[s] = fmaf(wf[5], xc.y, acc[s]);
            acc[s] = fmaf(wf[6], xc.z, acc[s]);
            acc[s] = fmaf(wf[7], xc.w, acc[s]);
        }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int n = n0 + sg * 4 + s;
        if (n < N) h1[(long long)n * kFcHid + o] = f2bf(acc[s] > 0.0f ? acc[s] : 0.0f);
    }
}

// fc1, persistent (the fixed-order forward's layout, features [n][64][4][4]):
// block b keeps the weights of outputs [64 (b % 2), +64) resident as
// bfloat16 in [i/8][o][8] order (a lane's 8 consecutive weights are one
// 16-byte load, the lanes of a warp consecutive outputs) and walks groups of
// kFc1Group snippets, whose features are staged as float with the next
// group's loads in flight in registers.  A thread owns one output of four
// snippets; every sum runs over the inputs in increasing order.
constexpr int kFc1Group = 16;
constexpr size_t kFc1Smem = (size_t)64 * kFcIn * 2 + (size_t)kFc1Group * kFcIn * 4;

__global__ void __launch_bounds__(256, 1) fc1_persist_kernel(const uint16_t *__restrict__ feat,
                                                             const uint16_t *__restrict__ w,
                                                             const uint16_t *__restrict__ b, int N,
                                                             uint16_t *__restrict__ h1) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint4 *ws = reinterpret_cast<uint4 *>(smem);                            // [128][64] x 8 bfloat16
    float *xs = reinterpret_cast<float *>(smem + (size_t)64 * kFcIn * 2);  // [kFc1Group][1024]
    const int tid = threadIdx.x;
    const int half = blockIdx.x & 1, cta = blockIdx.x >> 1, ncta = gridDim.x >> 1;
    const int o = tid & 63, sg = tid >> 6;
    for (int e = tid; e < 64 * (kFcIn / 8); e += 256) {
        const int oo = e & 63, i8 = e >> 6;
        ws[i8 * 64 + oo] = __ldg(reinterpret_cast<const uint4 *>(w + (long long)(64 * half + oo) * kFcIn) + i8);
    }
    const float bias = bf2f(b[64 * half + o]);
    const int ngroups = (N + kFc1Group - 1) / kFc1Group;
    // a group's features: kFc1Group x 128 uint4, 8 per thread
    uint4 nxt[kFc1Group * kFcIn / 8 / 256];
    auto fetch = [&](int g) {
#pragma unroll
        for (int k = 0; k < kFc1Group * kFcIn / 8 / 256; ++k) {
            const int e = tid + 256 * k, sn = e / (kFcIn / 8), i8 = e % (kFcIn / 8);
            const int n = g * kFc1Group + sn;
            nxt[k] = n < N ? __ldg(reinterpret_cast<const uint4 *>(feat + (long long)n * kFcIn) + i8)
                           : make_uint4(0, 0, 0, 0);
        }
    };
    if (cta < ngroups) fetch(cta);
#pragma unroll 1
    for (int g = cta; g < ngroups; g += ncta) {
        __syncthreads();  // the previous group's features are consumed
#pragma unroll
        for (int k = 0; k < kFc1Group * kFcIn / 8 / 256; ++k) {
            const int e = tid + 256 * k, sn = e / (kFcIn / 8), i8 = e % (kFcIn / 8);
            const uint4 q = nxt[k];
            float4 *dst = reinterpret_cast<float4 *>(xs + sn * kFcIn + 8 * i8);
            dst[0] = make_float4(__uint_as_float(q.x << 16), __uint_as_float(q.x & 0xffff0000u),
                                 __uint_as_float(q.y << 16), __uint_as_float(q.y & 0xffff0000u));
            dst[1] = make_float4(__uint_as_float(q.z << 16), __uint_as_float(q.z & 0xffff0000u),
                                 __uint_as_float(q.w << 16), __uint_as_float(q.w & 0xffff0000u));
        }
        __syncthreads();
        if (g + ncta < ngroups) fetch(g + ncta);
        float acc[4] = {bias, bias, bias, bias};
#pragma unroll 2
        for (int i8 = 0; i8 < kFcIn / 8; ++i8) {
            const uint4 wq = ws[i8 * 64 + o];
            const float wf[8] = {__uint_as_float(wq.x << 16), __uint_as_float(wq.x & 0xffff0000u),
                                 __uint_as_float(wq.y << 16), __uint_as_float(wq.y & 0xffff0000u),
                                 __uint_as_float(wq.z << 16), __uint_as_float(wq.z & 0xffff0000u),
                                 __uint_as_float(wq.w << 16), __uint_as_float(wq.w & 0xffff0000u)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 xa = *reinterpret_cast<const float4 *>(xs + (sg + 4 * k) * kFcIn + 8 * i8);
                const float4 xc = *reinterpret_cast<const float4 *>(xs + (sg + 4 * k) * kFcIn + 8 * i8 + 4);
                acc[k] = fmaf(wf[0], xa.x, acc[k]);
                acc[k] = fmaf(wf[1], xa.y, acc[k]);
                acc[k] = fmaf(wf[2], xa.z, acc[k]);
                acc[k] = fmaf(wf[3], xa.w, acc[k]);
                acc[k] = fmaf(wf[4], xc.x, acc[k]);
                acc[k] = fmaf(wf[5], xc.y, acc[k]);
                acc[k] = fmaf(wf[6], xc.z, acc[k]);
                acc[k] = fmaf(wf[7], xc.w, acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int n = g * kFc1Group + sg + 4 * k;
            if (n < N) h1[(long long)n * kFcHid + 64 * half + o] = f2bf(acc[k] > 0.0f ? acc[k] : 0.0f);
        }
    }
}

__global__ void fc2_fwd_kernel(const uint16_t *__restrict__ h1, const uint16_t *__restrict__ w,
                               const uint16_t *__restrict__ b, int N, float *__restrict__ z) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = bf2f(b[0]);
    for (int i = 0; i < kFcHid; ++i) acc = fmaf(bf2f(w[i]), bf2f(h1[n * kFcHid + i]), acc);
    z[n] = acc;
}

// ---- inference forward on the tensor cores -----------------------------------
//
// Implicit-GEMM convolution + ReLU + 2x2 max pooling with tcgen05.  A tile is
// M = 128 convolution outputs = 32 pooled outputs x their 2x2 windows (row m =
// 4 * pooled + position in the window), N = CO output channels, and K = the 9
// taps x CI input channels ordered (tap, channel), so that with activations
// stored channel-last (NHWC) 8 consecutive K values are one 16-byte load.
// The CTA keeps the weights (N x K, bfloat16) in shared memory, builds the
// im2col rows of its tiles K-chunk by K-chunk into two alternating buffers,
// one thread issues the MMAs of each chunk into a tensor-memory accumulator
// (two, alternating between tiles), and the epilogue of a tile -- bias,
// ReLU, bfloat16 rounding, max over the window -- runs while the tensor cores
// work on the next one.  Sums are fp32 in the tensor cores' own order, so the
// logits agree with the fixed-order forward to float round-off (the training
// path keeps the fixed-order kernels above).
// Polls of an MMA-completion mbarrier before a thread gives up (a poll that
// finds the phase incomplete suspends the thread for ~4 us on GB300: ~60 ms,
// against microseconds per tile); after a give-up a thread waits no more.
constexpr uint32_t kTcWaitPolls = 1u << 14;

template <int CI, int CO, int H, int TPC>
struct ConvTcCfg {
    static constexpr int HO = H / 2;
    static constexpr int K = CI == 1 ? 16 : 9 * CI;   // conv1: 9 taps padded to one MMA step
    static constexpr int KC = CI == 1 ? 16 : TPC * CI;  // K per chunk
    static constexpr int NCHUNK = K / KC;
    static constexpr int A_BYTES = 128 * KC * 2;
    static constexpr int B_BYTES = CO * K * 2;
    static constexpr size_t SMEM = (size_t)2 * A_BYTES + B_BYTES;
    static constexpr uint32_t TCOLS = 2 * CO <= 32 ? 32 : (2 * CO <= 64 ? 64 : (2 * CO <= 128 ? 128 : 256));
    static constexpr int MINB = SMEM <= 110 * 1024 ? 2 : 1;
    static_assert(K % KC == 0 && KC % 16 == 0 && (CI == 1 || CI % 8 == 0), "chunking");
    static_assert(CO % 16 == 0 && CO <= 128, "N of the MMA");
};

template <int CI, int CO, int H, int TPC>
__global__ void __launch_bounds__(256, (ConvTcCfg<CI, CO, H, TPC>::MINB))
    conv_tc_kernel(const uint16_t *__restrict__ in, const uint16_t *__restrict__ w, const uint16_t *__restrict__ b,
                   int N, uint16_t *__restrict__ out, unsigned *__restrict__ err) {
    using C = ConvTcCfg<CI, CO, H, TPC>;
    constexpr int HO = C::HO, HO2 = HO * HO, K = C::K, KC = C::KC;
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ float s_bias[CO];
    uint8_t *As = tsm;
    uint8_t *Bs = tsm + 2 * C::A_BYTES;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights as B = [co][k], k = tap * CI + ci (conv1: k = tap, taps 9..15 zero)
    for (int e = tid; e < CO * K; e += 256) {
        const int co = e / K, k = e % K;
        const int tap = CI == 1 ? k : k / CI, ci = CI == 1 ? 0 : k % CI;
        const uint16_t v = tap < 9 ? __ldg(w + ((long long)co * CI + ci) * 9 + tap) : (uint16_t)0;
        *reinterpret_cast<uint16_t *>(Bs + tc::kmajor_offset(co, k, K)) = v;
    }
    if (tid < CO) s_bias[tid] = bf2f(b[tid]);
    tc::fence_async_smem();
    if (warp == 0) tc::tmem_alloc(&s_tmem, C::TCOLS);
    if (tid == 0) {
        tc::mbar_init(&s_mbar[0], 1);
        tc::mbar_init(&s_mbar[1], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t a_addr = tc::smem_addr(As), b_addr = tc::smem_addr(Bs);
    const int ntiles = (N * HO2 + 31) / 32;
    const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int nst = my_tiles * C::NCHUNK;
    bool ok = true;

    // this thread's im2col row (fixed: 256 threads step over units of 128 rows)
    const int m = tid & 127;
    auto row_pos = [&](int tile, int &n, int &y, int &x) {
        const int P = tile * 32 + (m >> 2);
        n = P / HO2;
        const int pp = P % HO2;
        y = 2 * (pp / HO) + ((m >> 1) & 1);
        x = 2 * (pp % HO) + (m & 1);
    };
    auto fill = [&](uint8_t *A, int tile, int c) {
        int n, y, x;
        row_pos(tile, n, y, x);
        const bool live = n < N;
        if constexpr (CI == 1) {
            // one 16-byte group per thread: taps 8j .. 8j+7 of row m
            const int j = tid >> 7;
            uint32_t pk[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int t = 8 * j + i;
                const int yy = y + t / 3 - 1, xx = x + t % 3 - 1;
                uint16_t v = 0;
                if (live && t < 9 && yy >= 0 && yy < H && xx >= 0 && xx < H)
                    v = __ldg(in + ((long long)n * H + yy) * H + xx);
                pk[i >> 1] |= (uint32_t)v << (16 * (i & 1));
            }
            *reinterpret_cast<uint4 *>(A + tc::kmajor_offset(m, 8 * j, KC)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        } else {
            constexpr int G = CI / 8;                // 16-byte groups per pixel
            constexpr int UNITS = TPC * G;           // per row in this chunk
#pragma unroll 4
            for (int r = tid >> 7; r < UNITS; r += 2) {
                const int g = r % G, tl = r / G;
                const int tap = c * TPC + tl;
                const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (live && yy >= 0 && yy < H && xx >= 0 && xx < H)
                    v = __ldg(reinterpret_cast<const uint4 *>(in + (((long long)n * H + yy) * H + xx) * CI) + g);
                *reinterpret_cast<uint4 *>(A + tc::kmajor_offset(m, tl * CI + 8 * g, KC)) = v;
            }
        }
    };
    // bias, ReLU, bfloat16 rounding and 2x2 max of local tile lt (global tile `tile`)
    auto epilogue = [&](int lt, int tile, int stage) {
        if (ok) ok = tc::mbar_wait(&s_mbar[stage & 1], (uint32_t)(stage >> 1) & 1u, kTcWaitPolls);
        tc::fence_after_sync();
        constexpr int HALVES = CO >= 32 ? 2 : 1;  // column halves over the two warpgroups
        constexpr int CW = CO / HALVES;
        const int quad = warp & 3, half = warp >> 2;
        if (half < HALVES) {
            const int mm = 32 * quad + lane;
            const int P = tile * 32 + (mm >> 2);
            const int n = P / HO2, pp = P % HO2, q = mm & 3;
#pragma unroll
            for (int c0 = 0; c0 < CW; c0 += 16) {
                const int cb = half * CW + c0;
                float v[16];
                tc::tmem_ld16(tmem + (uint32_t)((lt & 1) * CO + cb) + ((uint32_t)(32 * quad) << 16), v);
                float mx[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float a = v[i] + s_bias[cb + i];
                    float r = bf2f(f2bf(a > 0.0f ? a : 0.0f));
                    r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, 1));
                    r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, 2));
                    mx[i] = r;
                }
                // lane q of the window writes channels cb + 4q .. cb + 4q + 3
                uint32_t w01 = 0, w23 = 0;
#pragma unroll
                for (int qq = 0; qq < 4; ++qq)
                    if (q == qq) {
                        w01 = (uint32_t)f2bf(mx[4 * qq]) | ((uint32_t)f2bf(mx[4 * qq + 1]) << 16);
                        w23 = (uint32_t)f2bf(mx[4 * qq + 2]) | ((uint32_t)f2bf(mx[4 * qq + 3]) << 16);
                    }
                if (n < N)
                    *reinterpret_cast<uint2 *>(out + ((long long)n * HO2 + pp) * CO + cb + 4 * q) = make_uint2(w01, w23);
            }
        }
    };

    for (int s = 0; s < nst; ++s) {
        const int lt = s / C::NCHUNK, c = s % C::NCHUNK;
        const int tile = (int)blockIdx.x + lt * (int)gridDim.x;
        const int buf = s & 1;
        if (s >= 2 && ok) ok = tc::mbar_wait(&s_mbar[buf], (uint32_t)((s - 2) >> 1) & 1u, kTcWaitPolls);
        fill(As + buf * C::A_BYTES, tile, c);
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t acc = tmem + (uint32_t)((lt & 1) * CO);
#pragma unroll 1
            for (int st = 0; st < KC / 16; ++st)
                tc::mma_bf16(acc, tc::smem_desc(a_addr + buf * C::A_BYTES + 256 * st, 128, KC / 8 * 128),
                             tc::smem_desc(b_addr + 256 * (c * (KC / 16) + st), 128, K / 8 * 128),
                             tc::idesc_bf16(128, CO), c > 0 || st > 0);
            tc::mma_commit(&s_mbar[buf]);
        }
        if (c == 0 && lt > 0) epilogue(lt - 1, tile - (int)gridDim.x, s - 1);
    }
    if (nst > 0) epilogue(my_tiles - 1, (int)blockIdx.x + (my_tiles - 1) * (int)gridDim.x, nst - 1);
    tc::fence_before_sync();
    if (__syncthreads_or(!ok)) {
        // some completion was not observed: give the last two commits one
        // more short bounded wait before the tensor memory is freed
        for (int k = 1; k <= 2 && nst - k >= 0; ++k) {
            const int sg = nst - k;
            tc::mbar_wait(&s_mbar[sg & 1], (uint32_t)(sg >> 1) & 1u, kTcWaitPolls / 64 + 1);
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, C::TCOLS);
    if (!ok && lane == 0) atomicOr(err, 1u);
}

// ---- backward ------------------------------------------------------------------

__global__ void __launch_bounds__(1024) bce_kernel(const float *__restrict__ z, const float *__restrict__ y, int N,
                                                   float *__restrict__ dz, float *__restrict__ loss) {
    __shared__ double s[1024];
    double acc = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const float zn = z[n];
        const float sg = 1.0f / (1.0f + expf(-zn));
        dz[n] = (sg - y[n]) / (float)N;
        const double zd = zn, yd = y[n];
        acc += (zd > 0 ? zd : 0) - zd * yd + log1p(exp(-fabs(zd)));
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(s[0] / N);
}

__global__ void fc2_bwd_kernel(const float *__restrict__ dz, const uint16_t *__restrict__ h1,
                               const uint16_t *__restrict__ w2, int N, float *__restrict__ g_w2,
                               float *__restrict__ g_b2, float *__restrict__ dh) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kFcHid) {
        float acc = 0.0f;
        for (int n = 0; n < N; ++n) acc += dz[n] * bf2f(h1[n * kFcHid + idx]);
        g_w2[idx] = acc;
    } else if (idx == kFcHid) {
        float acc = 0.0f;
        for (int n = 0; n < N; ++n) acc += dz[n];
        *g_b2 = acc;
    }
    for (int k = idx; k < N * kFcHid; k += gridDim.x * blockDim.x) {
        const int i = k % kFcHid, n = k / kFcHid;
        dh[k] = bf2f(h1[k]) > 0.0f ? dz[n] * bf2f(w2[i]) : 0.0f;
    }
}

__global__ void fc1_bwd_w_kernel(const float *__restrict__ dh, const uint16_t *__restrict__ feat, int N,
                                 float *__restrict__ g_w1, float *__restrict__ g_b1) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < kFcHid * kFcIn) {
        const int i = idx % kFcIn, o = idx / kFcIn;
        float acc = 0.0f;
        for (int n = 0; n < N; ++n) acc += dh[n * kFcHid + o] * bf2f(feat[(long long)n * kFcIn + i]);
        g_w1[idx] = acc;
    } else if (idx < kFcHid * kFcIn + kFcHid) {
        const int o = idx - kFcHid * kFcIn;
        float acc = 0.0f;
        for (int n = 0; n < N; ++n) acc += dh[n * kFcHid + o];
        g_b1[o] = acc;
    }
}

__global__ void fc1_bwd_x_kernel(const float *__restrict__ dh, const uint16_t *__restrict__ w1, int N,
                                 float *__restrict__ dfeat) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * kFcIn) return;
    const int i = idx % kFcIn, n = idx / kFcIn;
    float acc = 0.0f;
    for (int o = 0; o < kFcHid; ++o) acc += dh[n * kFcHid + o] * bf2f(w1[(long long)o * kFcIn + i]);
    dfeat[idx] = acc;
}

// gradient reaching pre-pool position (y, x) of channel co: only the pooled
// maximum receives it, and only when it passed the ReLU
template <int CO, int H>
__device__ __forceinline__ float routed(const float *dpool, const uint16_t *pooled, const uint8_t *arg, int n, int co,
                                        int y, int x) {
    constexpr int HO = H / 2;
    const long long o = (((long long)n * CO + co) * HO + (y >> 1)) * HO + (x >> 1);
    if (arg[o] != ((y & 1) << 1 | (x & 1))) return 0.0f;
    if (!(bf2f(pooled[o]) > 0.0f)) return 0.0f;
    return dpool[o];
}

// stage 1: partial[chunk][wi] over the samples of the chunk (wi < CO*CI*9 weights, then CO biases)
template <int CI, int CO, int H>
__global__ void conv_bwd_w_kernel(const float *__restrict__ dpool, const uint16_t *__restrict__ pooled,
                                  const uint8_t *__restrict__ arg, const uint16_t *__restrict__ in, int N,
                                  float *__restrict__ partial) {
    constexpr int HO = H / 2;
    constexpr int NW = CO * CI * 9 + CO;
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (wi >= NW) return;
    const int n0 = chunk * kChunk, n1 = min(N, n0 + kChunk);
    float acc = 0.0f;
    if (wi < CO * CI * 9) {
        const int kx = wi % 3, ky = (wi / 3) % 3, ci = (wi / 9) % CI, co = wi / (9 * CI);
        for (int n = n0; n < n1; ++n) {
            const uint16_t *src = in + ((long long)n * CI + ci) * H * H;
            for (int yo = 0; yo < HO; ++yo)
                for (int xo = 0; xo < HO; ++xo) {
                    const long long o = (((long long)n * CO + co) * HO + yo) * HO + xo;
                    if (!(bf2f(pooled[o]) > 0.0f)) continue;
                    const int q = arg[o];
                    const int yy = 2 * yo + (q >> 1) + ky - 1, xx = 2 * xo + (q & 1) + kx - 1;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= H) continue;
                    acc += dpool[o] * bf2f(src[yy * H + xx]);
                }
        }
    } else {
        const int co = wi - CO * CI * 9;
        for (int n = n0; n < n1; ++n)
            for (int k = 0; k < HO * HO; ++k) {
                const long long o = ((long long)n * CO + co) * HO * HO + k;
                if (bf2f(pooled[o]) > 0.0f) acc += dpool[o];
            }
    }
    partial[(long long)chunk * NW + wi] = acc;
}

// stage 2: sum the chunks in order into the weight and bias gradients
__global__ void conv_bwd_w_sum_kernel(const float *__restrict__ partial, int nchunks, int nw_weights, int nbias,
                                      float *__restrict__ g_w, float *__restrict__ g_b) {
    const int wi = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = nw_weights + nbias;
    if (wi >= nw) return;
    float acc = 0.0f;
    for (int c = 0; c < nchunks; ++c) acc += partial[(long long)c * nw + wi];
    if (wi < nw_weights) g_w[wi] = acc;
    else g_b[wi - nw_weights] = acc;
}

// gradient w.r.t. the layer input (the previous layer's pooled output)
template <int CI, int CO, int H>
__global__ void conv_bwd_x_kernel(const float *__restrict__ dpool, const uint16_t *__restrict__ pooled,
                                  const uint8_t *__restrict__ arg, const uint16_t *__restrict__ w, int N,
                                  float *__restrict__ din) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)N * CI * H * H) return;
    const int xx = (int)(idx % H), yy = (int)((idx / H) % H);
    const int ci = (int)((idx / (H * H)) % CI);
    const int n = (int)(idx / ((long long)H * H * CI));
    float acc = 0.0f;
    for (int co = 0; co < CO; ++co) {
        const uint16_t *wk = w + ((long long)co * CI + ci) * 9;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int y = yy - ky + 1, x = xx - kx + 1;
                if (y < 0 || y >= H || x < 0 || x >= H) continue;
                const float g = routed<CO, H>(dpool, pooled, arg, n, co, y, x);
                if (g != 0.0f) acc += g * bf2f(wk[ky * 3 + kx]);
            }
    }
    din[idx] = acc;
}

// ---- optimiser -------------------------------------------------------------------

__global__ void adamw_kernel(long long count, float *__restrict__ master, const float *__restrict__ g,
                             float *__restrict__ m, float *__restrict__ v, uint16_t *__restrict__ bf, float lr,
                             float beta1, float beta2, float eps, float wd, float c1, float c2) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    // written without fused multiply-adds so every step rounds like the plain formula
    const float gi = g[i];
    const float mi = __fadd_rn(__fmul_rn(beta1, m[i]), __fmul_rn(__fsub_rn(1.0f, beta1), gi));
    const float vi = __fadd_rn(__fmul_rn(beta2, v[i]), __fmul_rn(__fmul_rn(__fsub_rn(1.0f, beta2), gi), gi));
    m[i] = mi;
    v[i] = vi;
    const float mh = __fdiv_rn(mi, c1), vh = __fdiv_rn(vi, c2);
    const float upd = __fadd_rn(__fdiv_rn(mh, __fadd_rn(__fsqrt_rn(vh), eps)), __fmul_rn(wd, master[i]));
    const float w = __fsub_rn(master[i], __fmul_rn(lr, upd));
    master[i] = w;
    bf[i] = f2bf(w);
}

__global__ void to_bf16_kernel(long long count, const float *__restrict__ master, uint16_t *__restrict__ bf) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) bf[i] = f2bf(master[i]);
}

}  // namespace

struct NN {
    Layout L;
    int max_batch = 0;
    int step = 0;
    float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    uint16_t *bf = nullptr;
    uint16_t *pooled[kConvLayers] = {};
    uint8_t *arg[kConvLayers] = {};
    uint16_t *h1 = nullptr;
    float *z = nullptr, *dz = nullptr, *dh = nullptr, *loss = nullptr, *partial = nullptr;
    float *dpool[kConvLayers] = {};  // gradient w.r.t. each layer's pooled output
    unsigned *tc_err = nullptr;      // tensor-core forward: an MMA completion was not observed
    float *wprep = nullptr;          // float images of the convolution weights in staged order
    int wprep_off[kConvLayers] = {};
    int nsm = 0;
};

static void free_nn(NN *p) {
    if (!p) return;
    cudaFree(p->master);
    cudaFree(p->grad);
    cudaFree(p->m);
    cudaFree(p->v);
    cudaFree(p->bf);
    for (int l = 0; l < kConvLayers; ++l) {
        cudaFree(p->pooled[l]);
        cudaFree(p->arg[l]);
        cudaFree(p->dpool[l]);
    }
    cudaFree(p->h1);
    cudaFree(p->z);
    cudaFree(p->dz);
    cudaFree(p->dh);
    cudaFree(p->loss);
    cudaFree(p->partial);
    cudaFree(p->tc_err);
    cudaFree(p->wprep);
    delete p;
}

// Per layer: (CI, CO, H) and the tile parameters (COB, SPB, CIC, RS, NBUF).
#define DD_CONV_LAYERS(X)                \
    X(0, 1, 16, 64, 16, 1, 1, 68, 4)    \
    X(1, 16, 32, 32, 32, 1, 16, 48, 3)  \
    X(2, 32, 64, 16, 64, 2, 16, 24, 3)  \
    X(3, 64, 64, 8, 64, 8, 8, 12, 3)

// with_arg: record the pooling argmax of every layer (the backward pass needs it).
static dd_status nn_forward(NN *p, const uint16_t *x, int n, cudaStream_t s, bool with_arg) {
    const Layout &L = p->L;
    if (((uintptr_t)x) % 4 != 0) return fail(DD_ERR_INVALID_ARG, "snippets must be 4-byte aligned");
    WPrepArgs wa;
    int wmax = 0;
    for (int l = 0; l < kConvLayers; ++l) {
        wa.l[l].w = p->bf + L.cw[l];
        wa.l[l].dst = p->wprep + p->wprep_off[l];
        wa.l[l].ci = kCin[l];
        wa.l[l].count = kCin[l] * 9 * kCout[l];
        wmax = std::max(wmax, wa.l[l].count);
    }
#define DD_COB(LY, CI, CO, H, COB, SPB, CIC, RS, NBUF) wa.l[LY].cob = COB;
    DD_CONV_LAYERS(DD_COB)
#undef DD_COB
    conv_wprep_kernel<<<dim3((unsigned)((wmax + 255) / 256), kConvLayers), 256, 0, s>>>(wa);
    const uint16_t *in = x;
#define DD_CONV_FWD(l, CI, CO, H, COB, SPB, CIC, RS, NBUF)                                                    \
    {                                                                                                         \
        using C = ConvFwdCfg<CI, CO, H, COB, SPB, CIC, RS, NBUF>;                                             \
        auto kern = with_arg ? conv_fwd_kernel<CI, CO, H, COB, SPB, CIC, RS, NBUF, true>                     \
                             : conv_fwd_kernel<CI, CO, H, COB, SPB, CIC, RS, NBUF, false>;                   \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM); \
        if (e != cudaSuccess) return cuda_fail(e, "classifier forward");                                      \
        const int groups = (n + SPB - 1) / SPB;                                                               \
        int grid = p->nsm / C::NCB;                                                                           \
        if (grid > groups) grid = groups;                                                                     \
        if (grid < 1) grid = 1;                                                                               \
        kern<<<grid * C::NCB, kConvThreads, C::SMEM, s>>>(in, p->wprep + p->wprep_off[l], p->bf + L.cb[l], n, \
                                                           p->pooled[l], p->arg[l]);                          \
        in = p->pooled[l];                                                                                    \
    }
    DD_CONV_LAYERS(DD_CONV_FWD)
#undef DD_CONV_FWD
    {
        cudaError_t e = cudaFuncSetAttribute(fc1_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kFc1Smem);
        if (e != cudaSuccess) return cuda_fail(e, "classifier forward");
        const int groups = (n + kFc1Group - 1) / kFc1Group;
        int grid = p->nsm / 2;
        if (grid > groups) grid = groups;
        fc1_persist_kernel<<<2 * grid, 256, kFc1Smem, s>>>(p->pooled[3], p->bf + L.f1w, p->bf + L.f1b, n, p->h1);
    }
    fc2_fwd_kernel<<<(n + 127) / 128, 128, 0, s>>>(p->h1, p->bf + L.f2w, p->bf + L.f2b, n, p->z);
    return cuda_fail(cudaGetLastError(), "classifier forward");
}

// Inference forward: tensor-core convolutions with channel-last activations
// (stored in the pooled buffers), then the fully connected layers.
static dd_status nn_forward_tc(NN *p, const uint16_t *x, int n, cudaStream_t s) {
    const Layout &L = p->L;
    const uint16_t *in = x;
#define DD_CONV_TC(l, CI, CO, H, TPC)                                                                         \
    {                                                                                                         \
        using C = ConvTcCfg<CI, CO, H, TPC>;                                                                  \
        auto kern = conv_tc_kernel<CI, CO, H, TPC>;                                                           \
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM); \
        if (e != cudaSuccess) return cuda_fail(e, "classifier forward");                                      \
        const int ntiles = (n * C::HO * C::HO + 31) / 32;                                                     \
        const int grid = ntiles < p->nsm * C::MINB ? ntiles : p->nsm * C::MINB;                               \
        kern<<<grid, 256, C::SMEM, s>>>(in, p->bf + L.cw[l], p->bf + L.cb[l], n, p->pooled[l], p->tc_err);    \
        in = p->pooled[l];                                                                                    \
    }
    DD_CONV_TC(0, 1, 16, 64, 1)
    DD_CONV_TC(1, 16, 32, 32, 9)
    DD_CONV_TC(2, 32, 64, 16, 3)
    DD_CONV_TC(3, 64, 64, 8, 1)
#undef DD_CONV_TC
    fc1_fwd_kernel<true><<<(n + kFc1Rows - 1) / kFc1Rows, 256, 0, s>>>(p->pooled[3], p->bf + L.f1w, p->bf + L.f1b, n,
                                                                      p->h1);
    fc2_fwd_kernel<<<(n + 127) / 128, 128, 0, s>>>(p->h1, p->bf + L.f2w, p->bf + L.f2b, n, p->z);
    return cuda_fail(cudaGetLastError(), "classifier forward");
}

}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_nn_create(dd_nn **out, int max_batch) {
    if (!out || max_batch <= 0 || max_batch > (1 << 16)) return fail(DD_ERR_INVALID_ARG, "max_batch must be 1..65536");
    *out = nullptr;
    NN *p = new (std::nothrow) NN();
    if (!p) return fail(DD_ERR_NOMEM, "host allocation failed");
    p->L = make_layout();
    p->max_batch = max_batch;
    const size_t P = (size_t)p->L.total;
    const size_t nb = (size_t)max_batch;
    cudaError_t e = cudaMalloc(&p->master, P * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->grad, P * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->m, P * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->v, P * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->bf, P * 2);
    for (int l = 0; l < kConvLayers && e == cudaSuccess; ++l) {
        const size_t cells = nb * kCout[l] * (kHin[l] / 2) * (kHin[l] / 2);
        e = cudaMalloc(&p->pooled[l], cells * 2);
        if (e == cudaSuccess) e = cudaMalloc(&p->arg[l], cells);
        if (e == cudaSuccess) e = cudaMalloc(&p->dpool[l], cells * 4);
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->h1, nb * kFcHid * 2);
    if (e == cudaSuccess) e = cudaMalloc(&p->z, nb * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->dz, nb * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->dh, nb * kFcHid * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->loss, 4);
    size_t part = 0;
    for (int l = 0; l < kConvLayers; ++l) {
        const size_t nw = (size_t)kCout[l] * kCin[l] * 9 + kCout[l];
        part = std::max(part, nw * ((nb + kChunk - 1) / kChunk));
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->partial, part * 4);
    if (e == cudaSuccess) e = cudaMalloc(&p->tc_err, 4);
    int wtot = 0;
    for (int l = 0; l < kConvLayers; ++l) {
        p->wprep_off[l] = wtot;
        wtot += kCin[l] * 9 * kCout[l];
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->wprep, (size_t)wtot * 4);
    if (e == cudaSuccess) e = cudaMemset(p->tc_err, 0, 4);
    if (e == cudaSuccess) {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e == cudaSuccess) e = cudaMemset(p->master, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(p->m, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(p->v, 0, P * 4);
    if (e == cudaSuccess) e = cudaMemset(p->bf, 0, P * 2);
    if (e == cudaSuccess) e = cudaMemset(p->grad, 0, P * 4);
    if (e != cudaSuccess) {
        dd_status st = cuda_fail(e, "allocating classifier buffers");
        free_nn(p);
        return st;
    }
    *out = reinterpret_cast<dd_nn *>(p);
    return DD_OK;
}

dd_status dd_nn_set_params(dd_nn *nn, const float *h_master) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !h_master) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    const size_t P = (size_t)p->L.total;
    DD_CUDA_TRY(cudaMemcpy(p->master, h_master, P * 4, cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaMemset(p->m, 0, P * 4));
    DD_CUDA_TRY(cudaMemset(p->v, 0, P * 4));
    to_bf16_kernel<<<(unsigned)((P + 255) / 256), 256>>>((long long)P, p->master, p->bf);
    DD_CUDA_TRY(cudaGetLastError());
    DD_CUDA_TRY(cudaDeviceSynchronize());
    p->step = 0;
    return DD_OK;
}

dd_status dd_nn_get_params(const dd_nn *nn, float *h_master) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p || !h_master) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    DD_CUDA_TRY(cudaDeviceSynchronize());
    DD_CUDA_TRY(cudaMemcpy(h_master, p->master, (size_t)p->L.total * 4, cudaMemcpyDeviceToHost));
    return DD_OK;
}

dd_status dd_nn_forward(dd_nn *nn, const uint16_t *d_x, int n, float *d_logits, void *stream) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !d_x || n <= 0 || n > p->max_batch) return fail(DD_ERR_INVALID_ARG, "bad classifier forward arguments");
    cudaStream_t s = (cudaStream_t)stream;
    dd_status st = nn_forward(p, d_x, n, s, false);
    if (st != DD_OK) return st;
    if (d_logits) DD_CUDA_TRY(cudaMemcpyAsync(d_logits, p->z, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    return DD_OK;
}

dd_status dd_nn_forward_tc(dd_nn *nn, const uint16_t *d_x, int n, float *d_logits, void *stream) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !d_x || n <= 0 || n > p->max_batch) return fail(DD_ERR_INVALID_ARG, "bad classifier forward arguments");
    if (((uintptr_t)d_x) % 16 != 0) return fail(DD_ERR_INVALID_ARG, "snippets must be 16-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    dd_status st = nn_forward_tc(p, d_x, n, s);
    if (st != DD_OK) return st;
    if (d_logits) DD_CUDA_TRY(cudaMemcpyAsync(d_logits, p->z, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    return DD_OK;
}

dd_status dd_nn_status(const dd_nn *nn, unsigned *flags) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p || !flags) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    DD_CUDA_TRY(cudaMemcpy(flags, p->tc_err, 4, cudaMemcpyDeviceToHost));
    return DD_OK;
}

dd_status dd_nn_backward(dd_nn *nn, const uint16_t *d_x, const float *d_labels, int n, void *stream) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !d_x || !d_labels || n <= 0 || n > p->max_batch)
        return fail(DD_ERR_INVALID_ARG, "bad classifier backward arguments");
    cudaStream_t s = (cudaStream_t)stream;
    dd_status st = nn_forward(p, d_x, n, s, true);
    if (st != DD_OK) return st;
    const Layout &L = p->L;
    float *g = p->grad;
    bce_kernel<<<1, 1024, 0, s>>>(p->z, d_labels, n, p->dz, p->loss);
    fc2_bwd_kernel<<<(n * kFcHid + 255) / 256, 256, 0, s>>>(p->dz, p->h1, p->bf + L.f2w, n, g + L.f2w, g + L.f2b,
                                                            p->dh);
    fc1_bwd_w_kernel<<<(kFcHid * kFcIn + kFcHid + 255) / 256, 256, 0, s>>>(p->dh, p->pooled[3], n, g + L.f1w,
                                                                          g + L.f1b);
    fc1_bwd_x_kernel<<<(n * kFcIn + 255) / 256, 256, 0, s>>>(p->dh, p->bf + L.f1w, n, p->dpool[3]);
    const int nchunks = (n + kChunk - 1) / kChunk;
#define DD_CONV_BWD(l, CI, CO, H, INPTR)                                                                      \
    {                                                                                                         \
        constexpr int NW = CO * CI * 9 + CO;                                                                  \
        dim3 gw((NW + 127) / 128, nchunks);                                                                   \
        conv_bwd_w_kernel<CI, CO, H><<<gw, 128, 0, s>>>(p->dpool[l], p->pooled[l], p->arg[l], INPTR, n,       \
                                                         p->partial);                                         \
        conv_bwd_w_sum_kernel<<<(NW + 255) / 256, 256, 0, s>>>(p->partial, nchunks, CO * CI * 9, CO,          \
                                                               g + L.cw[l], g + L.cb[l]);                     \
        if (l > 0) {                                                                                          \
            const long long tot = (long long)n * CI * H * H;                                                  \
            conv_bwd_x_kernel<CI, CO, H><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(                      \
                p->dpool[l], p->pooled[l], p->arg[l], p->bf + L.cw[l], n, (l) > 0 ? p->dpool[(l) - 1] : nullptr); \
        }                                                                                                     \
    }
    DD_CONV_BWD(3, 64, 64, 8, p->pooled[2])
    DD_CONV_BWD(2, 32, 64, 16, p->pooled[1])
    DD_CONV_BWD(1, 16, 32, 32, p->pooled[0])
    DD_CONV_BWD(0, 1, 16, 64, d_x)
#undef DD_CONV_BWD
    return cuda_fail(cudaGetLastError(), "classifier backward");
}

dd_status dd_nn_get_grads(const dd_nn *nn, float *h_grads, void *stream) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p || !h_grads) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    DD_CUDA_TRY(cudaMemcpyAsync(h_grads, p->grad, (size_t)p->L.total * 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return DD_OK;
}

dd_status dd_nn_set_grads(dd_nn *nn, const float *h_grads) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !h_grads) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    DD_CUDA_TRY(cudaMemcpy(p->grad, h_grads, (size_t)p->L.total * 4, cudaMemcpyHostToDevice));
    return DD_OK;
}

dd_status dd_nn_get_loss(const dd_nn *nn, float *h_loss, void *stream) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p || !h_loss) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    DD_CUDA_TRY(cudaMemcpyAsync(h_loss, p->loss, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return DD_OK;
}

dd_status dd_nn_adamw(dd_nn *nn, float lr, float beta1, float beta2, float eps, float wd, void *stream) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL classifier");
    if (!(lr >= 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0) || !(wd >= 0))
        return fail(DD_ERR_INVALID_ARG, "bad AdamW hyper-parameters");
    p->step += 1;
    const float c1 = 1.0f - powf(beta1, (float)p->step);
    const float c2 = 1.0f - powf(beta2, (float)p->step);
    const long long P = p->L.total;
    adamw_kernel<<<(unsigned)((P + 255) / 256), 256, 0, (cudaStream_t)stream>>>(P, p->master, p->grad, p->m, p->v,
                                                                                  p->bf, lr, beta1, beta2, eps, wd,
                                                                                  c1, c2);
    return cuda_fail(cudaGetLastError(), "adamw_kernel launch");
}

dd_status dd_nn_get_state(const dd_nn *nn, float *h_m, float *h_v, uint16_t *h_bf16, int *step) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p) return fail(DD_ERR_INVALID_ARG, "NULL classifier");
    const size_t P = (size_t)p->L.total;
    DD_CUDA_TRY(cudaDeviceSynchronize());
    if (h_m) DD_CUDA_TRY(cudaMemcpy(h_m, p->m, P * 4, cudaMemcpyDeviceToHost));
    if (h_v) DD_CUDA_TRY(cudaMemcpy(h_v, p->v, P * 4, cudaMemcpyDeviceToHost));
    if (h_bf16) DD_CUDA_TRY(cudaMemcpy(h_bf16, p->bf, P * 2, cudaMemcpyDeviceToHost));
    if (step) *step = p->step;
    return DD_OK;
}

static const char kMagic[8] = {'D', 'D', 'N', 'N', 'C', 'K', 'P', '1'};

dd_status dd_nn_save(const dd_nn *nn, const char *path) {
    const NN *p = reinterpret_cast<const NN *>(nn);
    if (!p || !path) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    const size_t P = (size_t)p->L.total;
    std::vector<float> buf(3 * P);
    DD_CUDA_TRY(cudaDeviceSynchronize());
    DD_CUDA_TRY(cudaMemcpy(buf.data(), p->master, P * 4, cudaMemcpyDeviceToHost));
    DD_CUDA_TRY(cudaMemcpy(buf.data() + P, p->m, P * 4, cudaMemcpyDeviceToHost));
    DD_CUDA_TRY(cudaMemcpy(buf.data() + 2 * P, p->v, P * 4, cudaMemcpyDeviceToHost));
    FILE *f = fopen(path, "wb");
    if (!f) return fail(DD_ERR_INVALID_ARG, "cannot open %s for writing", path);
    const int64_t hdr[2] = {(int64_t)P, (int64_t)p->step};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, 8, 2, f) == 2 && fwrite(buf.data(), 4, 3 * P, f) == 3 * P;
    ok = (fclose(f) == 0) && ok;
    return ok ? DD_OK : fail(DD_ERR_INTERNAL, "short write to %s", path);
}

dd_status dd_nn_load(dd_nn *nn, const char *path) {
    NN *p = reinterpret_cast<NN *>(nn);
    if (!p || !path) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    const size_t P = (size_t)p->L.total;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(DD_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int64_t hdr[2];
    std::vector<float> buf(3 * P);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 && fread(hdr, 8, 2, f) == 2 &&
              hdr[0] == (int64_t)P && fread(buf.data(), 4, 3 * P, f) == 3 * P;
    fclose(f);
    if (!ok) return fail(DD_ERR_INVALID_ARG, "%s is not a classifier checkpoint of %zu parameters", path, P);
    DD_CUDA_TRY(cudaMemcpy(p->master, buf.data(), P * 4, cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaMemcpy(p->m, buf.data() + P, P * 4, cudaMemcpyHostToDevice));
    DD_CUDA_TRY(cudaMemcpy(p->v, buf.data() + 2 * P, P * 4, cudaMemcpyHostToDevice));
    to_bf16_kernel<<<(unsigned)((P + 255) / 256), 256>>>((long long)P, p->master, p->bf);
    DD_CUDA_TRY(cudaGetLastError());
    DD_CUDA_TRY(cudaDeviceSynchronize());
    p->step = (int)hdr[1];
    return DD_OK;
}

void dd_nn_destroy(dd_nn *nn) { free_nn(reinterpret_cast<NN *>(nn)); }

}  // extern "C"
