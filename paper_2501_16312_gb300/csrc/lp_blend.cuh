// Shared pieces of the forward and backward blend kernels (sm_103a).
//
// A tile of TILE x TILE pixels (TILE = 8, 16 or 32, a tuning choice; 16 is
// the paper's patch size) is processed by TILE^2 / PIX threads; each thread
// owns a strip of PIX horizontally adjacent pixels, so that one 128-bit
// shared-memory load of a face plane feeds PIX pixels, and each warp a
// rectangle of the tile (WarpGrid: 8 x 8 pixels, or 8 x 16 with four pixels
// per thread), the unit of the per-warp skips.  Blocks are persistent and
// pull tiles of all cameras from one atomic queue.
#pragma once

#include "lp_device.cuh"
#include "lp_internal.h"

namespace lp {


__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sums of N values (N a power of two, 2..32) over the warp by recursive
// halving: at each step a lane keeps one half of its values and adds the
// partner's copy of that half.  Returns, in every lane, the total of value
// warp_sum_index<N>(lane); N values cost about 4N instructions instead of
// 10N for N separate warp_sum calls.
template <int N>
__device__ __forceinline__ float warp_sum_multi(float (&v)[N], int lane) {
#pragma unroll
    for (int m = N, o = 16; m > 1; m >>= 1, o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < m / 2; ++k) {
            const float send = up ? v[k] : v[k + m / 2];
            const float keep = up ? v[k + m / 2] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float t = v[0];
#pragma unroll
    for (int o = 16 / N; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

template <int N>
__device__ __forceinline__ int warp_sum_index(int lane) {
    return (lane >> (5 - (N >= 32 ? 5 : N >= 16 ? 4 : N >= 8 ? 3 : N >= 4 ? 2 : 1))) & (N - 1);
}

struct TileGeom {
    int tile;
    int tx0, ty0;         // first pixel of the tile
    int width, height;
    int pix_base;
};

template <int TILE>
__device__ __forceinline__ TileGeom tile_geom(const CamsParam& cams, int tile) {
    const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
    const int lt = tile - cm.tile_base;
    const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
    return TileGeom{tile, tx * TILE, ty * TILE, cm.width, cm.height, cm.pix_base};
}

}  // namespace lp
