// Backward blend kernels for 32x32-pixel tiles (see lp_blend_bwd.cuh).
#include "lp_blend_bwd.cuh"

namespace lp {

cudaError_t launch_blend_bwd_t32(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return launch_bwd_tile<32>(V, batch, pix, a, st);
}

int blend_bwd_occupancy_t32(int V, int batch, int pix) { return occ_bwd_tile<32>(V, batch, pix); }

}  // namespace lp
