// Probe of the dedispersion tile's give-up path: the tile routine of the
// product library (tiled_tile.cuh), run on a tiny band with stage mbarriers
// that can never complete, so every bounded wait runs out.  No fault and no
// endless wait is involved: the stage copies themselves land normally.
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../tiled_tile.cuh"
#include "dd_probe.h"

namespace dd {
namespace probe {
dd_status report(dd_status s, const char *msg);
}  // namespace probe

namespace {

constexpr int kProbeChan = 64, kProbeDT = 2, kProbeW = 3, kProbeG = 64;
constexpr int kProbeD = tiled::kWarps * kProbeDT;
constexpr int kProbeSamples = 16 * 32 * kProbeW;  // one time tile

__global__ void __launch_bounds__(tiled::kThreads) tile_giveup_kernel(const tiled::TiledArgs a, int *ret) {
    extern __shared__ __align__(16) uint32_t smem[];
    if (threadIdx.x == 0) {
        // one arrival more than the G window copies and the table copy make
        uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
        tc::mbar_init(&bars[0], kProbeG + 2);
        tc::mbar_init(&bars[1], kProbeG + 2);
        tc::fence_mbar_init();
    }
    uint32_t phase = 0;
    const bool ok = tiled::dd_tile<kProbeDT, kProbeW, 11, kProbeG>(a, 0, 0, smem, phase);
    if (threadIdx.x == 0) *ret = ok ? 1 : 0;
}

dd_status cuda_check(cudaError_t e, const char *what) {
    return e == cudaSuccess ? DD_OK : probe::report(DD_ERR_CUDA, what);
}

}  // namespace
}  // namespace dd

extern "C" dd_status dd_probe_tile_giveup(unsigned poll_limit, unsigned *h_err, long long *h_written) {
    using namespace dd;
    using namespace dd::tiled;
    if (!h_err || !h_written || poll_limit == 0 || poll_limit > (1u << 20))
        return probe::report(DD_ERR_INVALID_ARG, "poll_limit must be 1..2^20 and outputs non-NULL");
    // all delays 0: one DM block, one time tile, one stage
    const std::vector<int32_t> delays((size_t)kProbeD * kProbeChan, 0);
    const int slot = tile_slot(kProbeW, 0);
    std::vector<uint32_t> tab((size_t)kProbeChan * kProbeD);
    std::vector<int32_t> wsrel(kProbeChan);
    build_tile_tables(delays.data(), kProbeD, kProbeChan, kProbeD, slot, tab.data(), wsrel.data(), kProbeG);
    const long long ld_w = kProbeSamples / 16, ld_out = kProbeSamples;
    const size_t in_bytes = (size_t)kProbeChan * ld_w * 4, out_words = (size_t)kProbeD * ld_out;
    const size_t tab_bytes = tab.size() * 4, ws_bytes = wsrel.size() * 4;
    unsigned char *buf = nullptr;
    const size_t total = in_bytes + out_words * 4 + tab_bytes + ws_bytes + 16;
    dd_status st = cuda_check(cudaMalloc(&buf, total), "cudaMalloc");
    if (st != DD_OK) return st;
    uint32_t *d_in = reinterpret_cast<uint32_t *>(buf);
    uint32_t *d_out = reinterpret_cast<uint32_t *>(buf + in_bytes);
    uint32_t *d_tab = reinterpret_cast<uint32_t *>(buf + in_bytes + out_words * 4);
    int32_t *d_ws = reinterpret_cast<int32_t *>(buf + in_bytes + out_words * 4 + tab_bytes);
    unsigned *d_err = reinterpret_cast<unsigned *>(buf + total - 16);
    int *d_ret = reinterpret_cast<int *>(buf + total - 8);
    cudaError_t e = cudaMemset(buf, 0, in_bytes);
    if (e == cudaSuccess) e = cudaMemset(d_out, 0xFF, out_words * 4);
    if (e == cudaSuccess) e = cudaMemset(d_err, 0, 16);
    if (e == cudaSuccess) e = cudaMemcpy(d_tab, tab.data(), tab_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ws, wsrel.data(), ws_bytes, cudaMemcpyHostToDevice);
    TiledArgs a;
    a.in = d_in;
    a.ld_w = ld_w;
    a.tab = d_tab;
    a.wsrel = d_ws;
    a.nchan = kProbeChan;
    a.ndm = kProbeD;
    a.nout = kProbeSamples;
    a.out = d_out;
    a.ld_out = ld_out;
    a.slot = slot;
    a.n_dmb = 1;
    a.err = d_err;
    a.poll_limit = poll_limit;
    const size_t smem = tile_smem_bytes(slot, kProbeG, kProbeD, kProbeChan);
    if (e == cudaSuccess && smem > 48 * 1024)
        e = cudaFuncSetAttribute(tile_giveup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        tile_giveup_kernel<<<1, kThreads, smem>>>(a, d_ret);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    std::vector<uint32_t> out(out_words);
    int ret = -1;
    if (e == cudaSuccess) e = cudaMemcpy(h_err, d_err, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&ret, d_ret, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out.data(), d_out, out_words * 4, cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_check(e, "tile give-up probe");
    long long written = 0;
    for (uint32_t v : out) written += v != 0xFFFFFFFFu;
    *h_written = written;
    if (ret != 0 && ret != 1) return probe::report(DD_ERR_INTERNAL, "tile give-up probe: no return value");
    if (*h_err & 1u) return probe::report(DD_ERR_TIMEOUT, "the tile gave up waiting for its stages");
    return DD_OK;
}
