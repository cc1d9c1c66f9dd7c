// Instantiations of the tiled dedispersion kernels with 32-channel
// shared-memory stages (a 32-channel carry-save tree per stage).
#include "tiled_launch.cuh"

namespace dd {

dd_status launch_tiled_g32(const Plan *p, const TiledShape &s, const ShapeTable &st, const uint8_t *d_in,
                           size_t ld_in_bytes, size_t nsamp_in, uint32_t *d_out, size_t ld_out, cudaStream_t stream) {
    return tiled::launch_group<32, false>(p, s, st, d_in, ld_in_bytes, nsamp_in, d_out, ld_out, stream);
}

BatchKernelFn batch_kernel_g32(const TiledShape &s, bool big) { return tiled::batch_group<32, false>(s, big); }

}  // namespace dd
