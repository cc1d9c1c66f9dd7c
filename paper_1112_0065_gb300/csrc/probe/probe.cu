// Measurement probes (a library of their own, libddprobe.so, loaded by the
// tests and by the benchmark's roofline figures only; not part of libdd.so):
//  - issue rates of the integer pipes of the current GPU, backing the INT32
//    roofline of the dedispersion kernel with a measurement: independent
//    chains of 3-input logic ops (LOP3), 32-bit adds, integer multiply-adds
//    and a LOP3 / multiply-add mix, timed with CUDA events on a full grid;
//  - float FMA issue rates (scalar and packed pairs);
//  - a tensor-core self-check of the classifier's tcgen05 building blocks;
//  - the give-up paths of the bounded mbarrier waits (here and in
//    tile_probe.cu), run without any fault.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include "dd_probe.h"

namespace dd {
namespace {

thread_local char g_probe_msg[256] = "";

dd_status fail(dd_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_probe_msg, sizeof g_probe_msg, fmt, ap);
    va_end(ap);
    return s;
}

dd_status cuda_fail(cudaError_t e, const char *what) {
    return fail(DD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define DD_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e__ = (expr);                           \
        if (e__ != cudaSuccess) return cuda_fail(e__, #expr); \
    } while (0)

}  // namespace
}  // namespace dd

extern "C" const char *dd_probe_last_error(void) { return dd::g_probe_msg; }

namespace dd {
namespace probe {
// Message of a failed probe call from another translation unit of the library.
dd_status report(dd_status s, const char *msg) { return fail(s, "%s", msg); }
}  // namespace probe
}  // namespace dd

namespace dd {
namespace {

__device__ __forceinline__ uint32_t p_lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t p_add(uint32_t a, uint32_t b) {
    uint32_t d;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t p_mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(uint32_t *out, int iters, uint32_t seed) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = seed * (k + 1) + threadIdx.x;
    uint32_t y = seed ^ threadIdx.x, z = seed + 77;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (OP == 0) x[k] = p_lop3(x[k], y, z);
                if (OP == 1) x[k] = p_add(x[k], y);
                if (OP == 2) x[k] = p_mad(x[k], y, z);
                if (OP == 3) x[k] = (k & 1) ? p_lop3(x[k], y, z) : p_mad(x[k], y, z);
            }
        y += 3;
        z ^= (uint32_t)it;
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k];
    out[blockIdx.x * 256 + threadIdx.x] = acc;
}

template <int OP>
dd_status time_op(uint32_t *buf, int blocks, cudaEvent_t e0, cudaEvent_t e1, double *tops) {
    const int iters = 4000;
    probe_kernel<OP><<<blocks, 256>>>(buf, 4, 1);
    DD_CUDA_TRY(cudaEventRecord(e0));
    probe_kernel<OP><<<blocks, 256>>>(buf, iters, 1);
    DD_CUDA_TRY(cudaEventRecord(e1));
    DD_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    DD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *tops = (double)blocks * 256 * iters * 16 * 8 / (ms * 1e-3) / 1e12;
    return DD_OK;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_probe_int_rates(double *tops) {
    if (!tops) return fail(DD_ERR_INVALID_ARG, "NULL output");
    int dev = 0, sms = 0;
    DD_CUDA_TRY(cudaGetDevice(&dev));
    DD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    uint32_t *buf = nullptr;
    DD_CUDA_TRY(cudaMalloc(&buf, (size_t)blocks * 256 * 4));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dd_status st = time_op<0>(buf, blocks, e0, e1, tops + 0);
    if (st == DD_OK) st = time_op<1>(buf, blocks, e0, e1, tops + 1);
    if (st == DD_OK) st = time_op<2>(buf, blocks, e0, e1, tops + 2);
    if (st == DD_OK) st = time_op<3>(buf, blocks, e0, e1, tops + 3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return st;
}

// ---------------------------------------------------------------------------
// Float FMA rates: scalar fma.rn.f32 against packed fma.rn.f32x2 (two
// independent single-precision FMAs per instruction, each rounded to nearest
// like fmaf), and a check that the packed form gives fmaf's results.
// ---------------------------------------------------------------------------

namespace dd {
namespace {

__device__ __forceinline__ unsigned long long p_ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float p_ffma(float a, float b, float c) {
    float d;
    asm volatile("fma.rn.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

template <int OP>
__global__ void __launch_bounds__(256) fp_probe_kernel(float *out, int iters, float seed) {
    float x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = seed * (k + 1) + (float)threadIdx.x * 1e-3f;
    const float y = 0.999f, z = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            if (OP == 0) {
#pragma unroll
                for (int k = 0; k < 16; ++k) x[k] = p_ffma(x[k], y, z);
            } else {
#pragma unroll
                for (int k = 0; k < 16; k += 2) {
                    const unsigned long long v = p_ffma2(pack2(x[k], x[k + 1]), pack2(y, y), pack2(z, z));
                    x[k] = __uint_as_float((uint32_t)v);
                    x[k + 1] = __uint_as_float((uint32_t)(v >> 32));
                }
            }
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) acc += x[k];
    out[blockIdx.x * 256 + threadIdx.x] = acc;
}

__global__ void fp_check_kernel(int n, unsigned long long *mismatch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    // reproducible pseudo-random operands over a wide exponent range
    uint32_t s = 2654435761u * (uint32_t)(i + 1);
    float v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        s ^= s << 13;
        s ^= s >> 17;
        s ^= s << 5;
        v[k] = __uint_as_float((s & 0x807FFFFFu) | ((100u + (s >> 27)) << 23));
    }
    const unsigned long long r = p_ffma2(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]));
    const float lo = __uint_as_float((uint32_t)r), hi = __uint_as_float((uint32_t)(r >> 32));
    if (__float_as_uint(lo) != __float_as_uint(fmaf(v[0], v[2], v[4])) ||
        __float_as_uint(hi) != __float_as_uint(fmaf(v[1], v[3], v[5])))
        atomicAdd(mismatch, 1ull);
}

template <int OP>
dd_status time_fp(float *buf, int blocks, cudaEvent_t e0, cudaEvent_t e1, double *tops) {
    const int iters = 4000;
    fp_probe_kernel<OP><<<blocks, 256>>>(buf, 4, 0.5f);
    DD_CUDA_TRY(cudaEventRecord(e0));
    fp_probe_kernel<OP><<<blocks, 256>>>(buf, iters, 0.5f);
    DD_CUDA_TRY(cudaEventRecord(e1));
    DD_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    DD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    *tops = (double)blocks * 256 * iters * 8 * 16 / (ms * 1e-3) / 1e12;
    return DD_OK;
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_probe_fp_rates(double *tops, unsigned long long *mismatches) {
    if (!tops || !mismatches) return fail(DD_ERR_INVALID_ARG, "NULL output");
    int dev = 0, sms = 0;
    DD_CUDA_TRY(cudaGetDevice(&dev));
    DD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8;
    float *buf = nullptr;
    unsigned long long *mm = nullptr;
    DD_CUDA_TRY(cudaMalloc(&buf, (size_t)blocks * 256 * 4));
    cudaError_t e = cudaMalloc(&mm, 8);
    if (e == cudaSuccess) e = cudaMemset(mm, 0, 8);
    if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "fp probe buffers");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dd_status st = time_fp<0>(buf, blocks, e0, e1, tops + 0);
    if (st == DD_OK) st = time_fp<1>(buf, blocks, e0, e1, tops + 1);
    if (st == DD_OK) {
        const int n = 1 << 24;
        fp_check_kernel<<<n / 256, 256>>>(n, mm);
        e = cudaMemcpy(mismatches, mm, 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_fail(e, "fp probe check");
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(mm);
    return st;
}

// ---------------------------------------------------------------------------
// Tensor-core self-check: one 128 x N x K bf16 GEMM through shared-memory
// descriptors, tensor memory and an mbarrier (the building blocks of the
// classifier's convolutions), so their layout can be checked against a host
// product on the GPU at hand.
// ---------------------------------------------------------------------------

#include "../tc.cuh"

namespace dd {
namespace {

__global__ void __launch_bounds__(128) tc_gemm_probe_kernel(const uint16_t *__restrict__ A,
                                                            const uint16_t *__restrict__ B, float *__restrict__ D,
                                                            int N, int K, unsigned *status) {
    extern __shared__ __align__(1024) uint8_t tsm[];
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    uint8_t *As = tsm;
    uint8_t *Bs = tsm + (size_t)128 * K * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kg = K / 8;
    for (int i = threadIdx.x; i < 128 * kg; i += 128) {
        const int r = i / kg, j = i % kg;
        *reinterpret_cast<uint4 *>(As + tc::kmajor_offset(r, 8 * j, K)) =
            *reinterpret_cast<const uint4 *>(A + (size_t)r * K + 8 * j);
    }
    for (int i = threadIdx.x; i < N * kg; i += 128) {
        const int r = i / kg, j = i % kg;
        *reinterpret_cast<uint4 *>(Bs + tc::kmajor_offset(r, 8 * j, K)) =
            *reinterpret_cast<const uint4 *>(B + (size_t)r * K + 8 * j);
    }
    tc::fence_async_smem();
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (warp == 0) tc::tmem_alloc(&s_tmem, ncols);
    if (threadIdx.x == 0) tc::mbar_init(&s_mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc::smem_addr(As), b0 = tc::smem_addr(Bs);
        const uint32_t sbo = (uint32_t)kg * 128;
        for (int s = 0; s < K / 16; ++s)
            tc::mma_bf16(tmem, tc::smem_desc(a0 + 256 * s, 128, sbo), tc::smem_desc(b0 + 256 * s, 128, sbo),
                         tc::idesc_bf16(128, N), s > 0);
        tc::mma_commit(&s_mbar);
    }
    const bool ok = tc::mbar_wait(&s_mbar, 0, 1u << 22);
    tc::fence_after_sync();
    if (!ok) {
        if (lane == 0) atomicOr(status, 1u);
    } else {
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) D[(size_t)(32 * warp + lane) * N + c0 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_probe_tc_gemm(const uint16_t *h_a, const uint16_t *h_b, float *h_d, int n, int k) {
    if (!h_a || !h_b || !h_d) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    if (n < 16 || n > 256 || n % 16 != 0 || k < 16 || k > 256 || k % 16 != 0)
        return fail(DD_ERR_INVALID_ARG, "n must be 16..256 and k 16..256, multiples of 16");
    uint16_t *a = nullptr, *b = nullptr;
    float *d = nullptr;
    unsigned *status = nullptr;
    const size_t smem = (size_t)(128 + n) * k * 2;
    cudaError_t e = cudaMalloc(&a, (size_t)128 * k * 2);
    if (e == cudaSuccess) e = cudaMalloc(&b, (size_t)n * k * 2);
    if (e == cudaSuccess) e = cudaMalloc(&d, (size_t)128 * n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&status, 4);
    if (e == cudaSuccess) e = cudaMemcpy(a, h_a, (size_t)128 * k * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b, h_b, (size_t)n * k * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(status, 0, 4);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        tc_gemm_probe_kernel<<<1, 128, smem>>>(a, b, d, n, k, status);
        e = cudaGetLastError();
    }
    unsigned st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(h_d, d, (size_t)128 * n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, 4, cudaMemcpyDeviceToHost);
    cudaFree(a);
    cudaFree(b);
    cudaFree(d);
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core probe");
    if (st) return fail(DD_ERR_TIMEOUT, "tensor-core probe: MMA completion not observed");
    return DD_OK;
}

// ---------------------------------------------------------------------------
// The give-up path of a bounded tensor-core wait, exercised without a fault:
// one CTA allocates tensor memory, arms an mbarrier that nothing ever
// arrives on, waits on it with the classifier's bounded poll (tc::mbar_wait),
// records the give-up in a status word, frees its tensor memory and returns.
// ---------------------------------------------------------------------------

namespace dd {
namespace {

__global__ void __launch_bounds__(128) wait_giveup_kernel(uint32_t limit, unsigned *status) {
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) tc::tmem_alloc(&s_tmem, 32);
    if (threadIdx.x == 0) tc::mbar_init(&s_mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // phase 0 never completes: no thread arrives and no MMA commits to it
    const bool ok = tc::mbar_wait(&s_mbar, 0u, limit);
    if (!ok && (threadIdx.x & 31) == 0) atomicOr(status, 1u << warp);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(s_tmem, 32);
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_probe_wait_giveup(unsigned poll_limit, unsigned *h_status) {
    if (!h_status || poll_limit == 0 || poll_limit > (1u << 20))
        return fail(DD_ERR_INVALID_ARG, "poll_limit must be 1..2^20 and h_status non-NULL");
    unsigned *status = nullptr;
    DD_CUDA_TRY(cudaMalloc(&status, 4));
    cudaError_t e = cudaMemset(status, 0, 4);
    if (e == cudaSuccess) {
        wait_giveup_kernel<<<1, 128>>>(poll_limit, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h_status, status, 4, cudaMemcpyDeviceToHost);
    cudaFree(status);
    if (e != cudaSuccess) return cuda_fail(e, "wait give-up probe");
    if (*h_status) return fail(DD_ERR_TIMEOUT, "bounded wait gave up after %u polls (warps 0x%x)", poll_limit, *h_status);
    return DD_OK;
}
