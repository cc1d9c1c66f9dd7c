// Input layouts: time-major (SIGPROC-style) 2-bit filterbank data, where each
// time sample's channels follow one another (4 per byte, channel c in bits
// 2(c%4) of byte c/4), turned into the channel-major rows the dedispersion
// kernels read (4 time samples per byte, sample t in bits 2(t%4) of byte
// t/4).  Paper Section 1 describes the 2-bit data; the corner turn only
// moves 2-bit values.
//
// dd_corner_turn_kernel: a CTA moves a tile of 64 samples x 64 channels
// through shared memory.  Thread (group g, quad q) packs the 4 bytes of
// samples 4q..4q+3 for channels 4g..4g+3 into one word, transposes that 4x4
// matrix of 2-bit cells with two masked swaps (cells 6 bits apart inside the
// 2x2 blocks, then blocks 12 bits apart), and so obtains the byte of each of
// the 4 channels holding those 4 samples.
#include "dd_internal.h"

namespace dd {
namespace {

__device__ __forceinline__ uint32_t transpose4x4_2bit(uint32_t w) {
    // cell (s, c) at bit 8s + 2c moves to bit 8c + 2s
    uint32_t t = ((w >> 6) ^ w) & 0x00CC00CCu;
    w ^= t ^ (t << 6);
    t = ((w >> 12) ^ w) & 0x0000F0F0u;
    w ^= t ^ (t << 12);
    return w;
}

__global__ void __launch_bounds__(256) dd_corner_turn_kernel(const uint8_t *__restrict__ tm, long long ld_tm,
                                                             int nchan, long long nsamp, uint8_t *__restrict__ cm,
                                                             long long ld_cm) {
    __shared__ uint8_t in_t[64][17];   // [sample][channel byte], padded
    __shared__ uint8_t out_t[64][17];  // [channel][sample byte], padded
    const long long t0 = (long long)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const int cb = (nchan + 3) / 4;  // bytes per time sample
    const int tid = threadIdx.x;
    for (int i = tid; i < 64 * 16; i += 256) {
        const int s = i >> 4, b = i & 15;
        const long long t = t0 + s;
        const int byte = c0 / 4 + b;
        in_t[s][b] = (t < nsamp && byte < cb) ? tm[t * ld_tm + byte] : (uint8_t)0;
    }
    __syncthreads();
    {
        const int g = tid & 15, q = tid >> 4;  // channel group (4 channels), sample quad (4 samples)
        const uint32_t w = (uint32_t)in_t[4 * q][g] | ((uint32_t)in_t[4 * q + 1][g] << 8) |
                           ((uint32_t)in_t[4 * q + 2][g] << 16) | ((uint32_t)in_t[4 * q + 3][g] << 24);
        const uint32_t o = transpose4x4_2bit(w);
#pragma unroll
        for (int c = 0; c < 4; ++c) out_t[4 * g + c][q] = (uint8_t)(o >> (8 * c));
    }
    __syncthreads();
    for (int i = tid; i < 64 * 16; i += 256) {
        const int ch = i >> 4, b = i & 15;
        const int c = c0 + ch;
        const long long byte = t0 / 4 + b;
        if (c < nchan && byte < ld_cm) {
            // channels past the band's end were read as zero; samples past nsamp likewise
            cm[(long long)c * ld_cm + byte] = out_t[ch][b];
        }
    }
}

}  // namespace
}  // namespace dd

using namespace dd;

extern "C" dd_status dd_corner_turn(const uint8_t *d_tm, size_t ld_tm_bytes, int nchan, size_t nsamp, uint8_t *d_cm,
                                    size_t ld_cm_bytes, void *stream) {
    if (!d_tm || !d_cm || nchan <= 0 || nsamp == 0) return fail(DD_ERR_INVALID_ARG, "NULL buffer or empty shape");
    if (ld_tm_bytes < (size_t)(nchan + 3) / 4 || ld_cm_bytes < (nsamp + 3) / 4)
        return fail(DD_ERR_INVALID_ARG, "row strides too short for nchan / nsamp");
    const long long ntile_t = ((long long)nsamp + 63) / 64;
    // output rows are written in whole tiles: cover the padding of the last tile too
    const long long ntile_t_out = ((long long)ld_cm_bytes * 4 + 63) / 64;
    const long long nt = ntile_t > ntile_t_out ? ntile_t : ntile_t_out;
    if (nt > 0x7fffffffLL) return fail(DD_ERR_INVALID_ARG, "gulp too long");
    dim3 grid((unsigned)nt, (unsigned)((nchan + 63) / 64));
    dd_corner_turn_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(d_tm, (long long)ld_tm_bytes, nchan,
                                                                  (long long)nsamp, d_cm, (long long)ld_cm_bytes);
    return cuda_fail(cudaGetLastError(), "dd_corner_turn_kernel launch");
}
