// Forward blend kernels for 8x8-pixel tiles (see lp_blend_fwd.cuh).
#include "lp_blend_fwd.cuh"

namespace lp {

cudaError_t launch_blend_fwd_t8(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return launch_fwd_tile<8>(V, batch, pix, a, st);
}

int blend_fwd_occupancy_t8(int V, int batch, int pix) { return occ_fwd_tile<8>(V, batch, pix); }

}  // namespace lp
