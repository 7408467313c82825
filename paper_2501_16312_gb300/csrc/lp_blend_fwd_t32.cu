// Forward blend kernels for 32x32-pixel tiles (see lp_blend_fwd.cuh).
#include "lp_blend_fwd.cuh"

namespace lp {

cudaError_t launch_blend_fwd_t32(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return launch_fwd_tile<32>(V, batch, pix, a, st);
}

int blend_fwd_occupancy_t32(int V, int batch, int pix) { return occ_fwd_tile<32>(V, batch, pix); }

}  // namespace lp
