// Issue-rate probe for the integer pipes of the current GPU, used to back the
// INT32 roofline of the dedispersion kernel with a measurement: independent
// chains of 3-input logic ops (LOP3), 32-bit adds, integer multiply-adds and
// a LOP3 / multiply-add mix, timed with CUDA events on a full grid.
#include "dd_internal.h"

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
