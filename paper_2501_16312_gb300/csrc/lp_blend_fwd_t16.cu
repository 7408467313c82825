// Forward blend kernels for 16x16-pixel tiles (see lp_blend_fwd.cuh).
#include "lp_blend_fwd.cuh"

namespace lp {

cudaError_t launch_blend_fwd_t16(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return launch_fwd_tile<16>(V, batch, pix, a, st);
}

int blend_fwd_occupancy_t16(int V, int batch, int pix) { return occ_fwd_tile<16>(V, batch, pix); }

}  // namespace lp
