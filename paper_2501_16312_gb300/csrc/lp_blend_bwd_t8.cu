// Backward blend kernels for 8x8-pixel tiles (see lp_blend_bwd.cuh).
#include "lp_blend_bwd.cuh"

namespace lp {

cudaError_t launch_blend_bwd_t8(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return launch_bwd_tile<8>(V, batch, pix, a, st);
}

int blend_bwd_occupancy_t8(int V, int batch, int pix) { return occ_bwd_tile<8>(V, batch, pix); }

}  // namespace lp
