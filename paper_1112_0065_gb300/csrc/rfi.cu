// Multibeam coincidence RFI mask (paper Section 2.1): the beams of the
// multibeam receiver act as reference antennas; a sample is interference when
// its total power exceeds k standard deviations in at least min_beams beams
// (the paper's example: 3 sigma in 4 or more of 13), decided independently
// for every sample and written as a boolean mask; masked samples can then be
// replaced, in every beam and channel, by the channel's mean level before
// dedispersion.
//
// Kernels:
//  * dd_zerodm_kernel  -- z_b[t] = sum_c x_b[c][t] for all beams in one
//    launch: 16-byte loads, 2-bit lanes added in byte lanes per 64-channel
//    slice, slices combined in shared memory; sum z and sum z^2 per beam.
//  * dd_rfi_mask_kernel -- per sample, the count of beams with
//    n z - S1 > 0 and (n z - S1)^2 > k^2 (n S2 - S1^2): the test
//    z > mean + k sigma done exactly in integers.
//  * dd_rfi_apply_kernel -- a thread owns one 16-sample word of a beam; when
//    any of its samples is masked it rewrites those 2-bit lanes of every
//    channel row with 1 + ((c + t) mod 2).
#include <new>

#include "dd_internal.h"

namespace dd {
namespace {

constexpr int kRfiMaxBeams = 64;

struct BeamPtrs {
    uint8_t *p[kRfiMaxBeams];
};

// A CTA takes 1024 samples of one beam (blockIdx.y).  Thread (slice s, group
// g) reads 64 samples (16 bytes) of each of up to 64 channels of its slice and
// adds them in byte lanes: acc[4*kw + i] byte j sums sample 16kw + 4j + i of
// the group.  The slices' byte sums meet in shared memory, where thread r
// (group r/16, word kw, lane i) adds its four samples over the slices in
// 16-bit lanes (at most 3 * 21844 < 2^16), then sum z and sum z^2.
constexpr int kZdSlices = 16;  // channel slices per pass (64 channels each)

__global__ void __launch_bounds__(256) dd_zerodm_kernel(const BeamPtrs beams, long long ld_bytes, int nchan,
                                                        long long nsamp, uint32_t *__restrict__ z, long long ldz,
                                                        unsigned long long *__restrict__ stats) {
    __shared__ uint32_t part[kZdSlices][16][16];  // [slice][group][4*kw + i]
    const int b = blockIdx.y;
    const uint8_t *in = beams.p[b];
    const int tid = threadIdx.x, g = tid & 15, sl = tid >> 4;
    const long long t_blk = (long long)blockIdx.x * 1024;
    const long long byte0 = t_blk / 4 + 16 * g;  // this thread's 16 bytes in every row
    const bool in_row = byte0 < ld_bytes;           // rows cover whole 16-byte groups
    // reducer role: samples t_blk + 64 rg + 16 rkw + 4 j + ri, j = 0..3
    const int rg = tid >> 4, rkw = (tid >> 2) & 3, ri = tid & 3;
    uint32_t lo = 0, hi = 0;  // 16-bit lanes: samples j = 0, 2 (lo) and 1, 3 (hi)
    for (int cs0 = 0; cs0 < nchan; cs0 += 64 * kZdSlices) {
        uint32_t acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0;
        const int c0 = cs0 + 64 * sl, c1 = min(nchan, c0 + 64);
        if (in_row) {
            const uint8_t *p = in + byte0;
#pragma unroll 4
            for (int c = c0; c < c1; ++c) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + (long long)c * ld_bytes));
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int kw = 0; kw < 4; ++kw)
#pragma unroll
                    for (int i = 0; i < 4; ++i) acc[4 * kw + i] += (wv[kw] >> (2 * i)) & 0x03030303u;
            }
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) part[sl][g][q] = acc[q];
        __syncthreads();
#pragma unroll
        for (int s2 = 0; s2 < kZdSlices; ++s2) {
            const uint32_t w = part[s2][rg][4 * rkw + ri];
            lo += w & 0x00FF00FFu;
            hi += (w >> 8) & 0x00FF00FFu;
        }
        __syncthreads();
    }
    const uint32_t v4[4] = {lo & 0xFFFFu, hi & 0xFFFFu, lo >> 16, hi >> 16};
    unsigned long long s1 = 0, s2 = 0;
    uint32_t *zr = z + (long long)b * ldz;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long t = t_blk + 64 * rg + 16 * rkw + 4 * j + ri;
        if (t < nsamp) {
            zr[t] = v4[j];
            s1 += v4[j];
            s2 += (unsigned long long)v4[j] * v4[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if ((tid & 31) == 0 && (s1 | s2)) {
        atomicAdd(stats + 2 * b, s1);
        atomicAdd(stats + 2 * b + 1, s2);
    }
}

__global__ void __launch_bounds__(256) dd_rfi_mask_kernel(const uint32_t *__restrict__ z, long long ldz, int nbeams,
                                                          long long nsamp, const unsigned long long *__restrict__ stats,
                                                          int k, int min_beams, uint8_t *__restrict__ mask,
                                                          unsigned long long *__restrict__ nmasked) {
    __shared__ long long s_s1[kRfiMaxBeams];
    __shared__ unsigned __int128 s_lim[kRfiMaxBeams];
    __shared__ unsigned s_cnt;
    const long long n = nsamp;
    if (threadIdx.x < nbeams) {
        const unsigned long long a = stats[2 * threadIdx.x], q = stats[2 * threadIdx.x + 1];
        // n S2 - S1^2 >= 0 (Cauchy-Schwarz)
        const unsigned __int128 var_n = (unsigned __int128)n * q - (unsigned __int128)a * a;
        s_s1[threadIdx.x] = (long long)a;
        s_lim[threadIdx.x] = (unsigned __int128)((long long)k * k) * var_n;
    }
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool m = false;
    if (t < nsamp) {
        int over = 0;
        for (int b = 0; b < nbeams; ++b) {
            const long long dev = n * (long long)z[(long long)b * ldz + t] - s_s1[b];
            over += dev > 0 && (unsigned __int128)dev * (unsigned long long)dev > s_lim[b];
        }
        m = over >= min_beams;
        mask[t] = (uint8_t)m;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && bal) atomicAdd(&s_cnt, (unsigned)__popc(bal));
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(nmasked, (unsigned long long)s_cnt);
}

__global__ void __launch_bounds__(256) dd_rfi_apply_kernel(const BeamPtrs beams, long long ld_bytes, int nchan,
                                                           long long nsamp, const uint8_t *__restrict__ mask) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // 16-sample word
    if (w >= (nsamp + 15) / 16) return;
    uint8_t *row0 = beams.p[blockIdx.y];
    const long long t0 = 16 * w;
    uint32_t M = 0;  // two bits per masked sample of the word
#pragma unroll
    for (int i = 0; i < 16; ++i)
        if (t0 + i < nsamp && mask[t0 + i]) M |= 3u << (2 * i);
    if (!M) return;
    // level 1 + ((c + t) mod 2) with t0 even: 01,10,01,... (even c) or 10,01,... (odd c)
    const uint32_t pat[2] = {0x99999999u, 0x66666666u};
    uint32_t *col = reinterpret_cast<uint32_t *>(row0) + w;
    const long long ldw = ld_bytes / 4;
    for (int c = 0; c < nchan; ++c) {
        uint32_t *p = col + (long long)c * ldw;
        *p = (*p & ~M) | (pat[c & 1] & M);
    }
}

struct Rfi {
    int nbeams_max = 0, nchan = 0;
    long long nsamp_max = 0, ldz = 0;
    uint32_t *z = nullptr;                // [nbeams_max][ldz] zero-DM series
    unsigned long long *stats = nullptr;  // [nbeams_max][2]: sum z, sum z^2; then the masked count
    uint8_t *mask = nullptr;              // [nsamp_max]
    long long nsamp = 0;
    int nbeams = 0;
};

void free_rfi(Rfi *r) {
    if (!r) return;
    cudaFree(r->z);
    cudaFree(r->stats);
    cudaFree(r->mask);
    delete r;
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" {

dd_status dd_rfi_create(dd_rfi **out, int nbeams_max, int nchan, size_t nsamp_max) {
    if (!out) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (nbeams_max <= 0 || nbeams_max > kRfiMaxBeams || nchan <= 0 || nchan > 21844 || nsamp_max == 0 ||
        nsamp_max > ((size_t)1 << 31))
        return fail(DD_ERR_INVALID_ARG, "nbeams_max 1..%d, nchan 1..21844, nsamp_max 1..2^31", kRfiMaxBeams);
    Rfi *r = new (std::nothrow) Rfi();
    if (!r) return fail(DD_ERR_NOMEM, "host allocation failed");
    r->nbeams_max = nbeams_max;
    r->nchan = nchan;
    r->nsamp_max = (long long)nsamp_max;
    r->ldz = ((long long)nsamp_max + 15) / 16 * 16;
    cudaError_t e = cudaMalloc(&r->z, (size_t)nbeams_max * r->ldz * 4);
    if (e == cudaSuccess) e = cudaMalloc(&r->stats, ((size_t)2 * nbeams_max + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc(&r->mask, (size_t)r->ldz);
    if (e != cudaSuccess) {
        dd_status st = cuda_fail(e, "allocating RFI buffers");
        free_rfi(r);
        return st;
    }
    *out = reinterpret_cast<dd_rfi *>(r);
    return DD_OK;
}

dd_status dd_rfi_run(dd_rfi *rfi, uint8_t *const *d_in, int nbeams, size_t ld_in_bytes, size_t nsamp, int k_sigma,
                     int min_beams, int apply, void *stream) {
    Rfi *r = reinterpret_cast<Rfi *>(rfi);
    if (!r || !d_in) return fail(DD_ERR_INVALID_ARG, "NULL RFI context or beam list");
    if (nbeams <= 0 || nbeams > r->nbeams_max || nsamp == 0 || (long long)nsamp > r->nsamp_max)
        return fail(DD_ERR_INVALID_ARG, "nbeams or nsamp beyond the RFI context's capacity");
    if (ld_in_bytes % 16 != 0 || ld_in_bytes < (nsamp + 3) / 4)
        return fail(DD_ERR_INVALID_ARG, "ld_in_bytes must be a multiple of 16 covering nsamp samples");
    if (k_sigma < 0 || k_sigma > 1000 || min_beams <= 0)
        return fail(DD_ERR_INVALID_ARG, "k_sigma must be 0..1000 and min_beams >= 1");
    BeamPtrs bp{};
    for (int b = 0; b < nbeams; ++b) {
        if (!d_in[b] || ((uintptr_t)d_in[b]) % 16 != 0)
            return fail(DD_ERR_INVALID_ARG, "beam %d input NULL or not 16-byte aligned", b);
        bp.p[b] = d_in[b];
    }
    cudaStream_t st = (cudaStream_t)stream;
    r->nsamp = (long long)nsamp;
    r->nbeams = nbeams;
    DD_CUDA_TRY(cudaMemsetAsync(r->stats, 0, ((size_t)2 * nbeams + 1) * 8, st));
    const long long nw = ((long long)nsamp + 15) / 16;
    const unsigned gw = (unsigned)((nw + 255) / 256);
    dd_zerodm_kernel<<<dim3((unsigned)(((long long)nsamp + 1023) / 1024), (unsigned)nbeams), 256, 0, st>>>(
        bp, (long long)ld_in_bytes, r->nchan, (long long)nsamp, r->z, r->ldz, r->stats);
    dd_rfi_mask_kernel<<<(unsigned)(((long long)nsamp + 255) / 256), 256, 0, st>>>(
        r->z, r->ldz, nbeams, (long long)nsamp, r->stats, k_sigma, min_beams, r->mask, r->stats + 2 * nbeams);
    if (apply)
        dd_rfi_apply_kernel<<<dim3(gw, (unsigned)nbeams), 256, 0, st>>>(bp, (long long)ld_in_bytes, r->nchan,
                                                                        (long long)nsamp, r->mask);
    return cuda_fail(cudaGetLastError(), "RFI kernels");
}

dd_status dd_rfi_result(const dd_rfi *rfi, long long *nmasked, void *stream) {
    const Rfi *r = reinterpret_cast<const Rfi *>(rfi);
    if (!r || !nmasked) return fail(DD_ERR_INVALID_ARG, "NULL argument");
    unsigned long long v = 0;
    DD_CUDA_TRY(cudaMemcpyAsync(&v, r->stats + 2 * r->nbeams, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    DD_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *nmasked = (long long)v;
    return DD_OK;
}

dd_status dd_rfi_buffers(const dd_rfi *rfi, const uint32_t **d_zerodm, size_t *ld_zerodm, const uint8_t **d_mask) {
    const Rfi *r = reinterpret_cast<const Rfi *>(rfi);
    if (!r) return fail(DD_ERR_INVALID_ARG, "NULL RFI context");
    if (d_zerodm) *d_zerodm = r->z;
    if (ld_zerodm) *ld_zerodm = (size_t)r->ldz;
    if (d_mask) *d_mask = r->mask;
    return DD_OK;
}

void dd_rfi_destroy(dd_rfi *rfi) { free_rfi(reinterpret_cast<Rfi *>(rfi)); }

}  // extern "C"
