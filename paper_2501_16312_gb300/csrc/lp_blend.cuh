// Shared pieces of the forward and backward blend kernels (sm_103a).
//
// A tile of 16x16 pixels is processed by 256 / PIX threads; thread t owns the
// strip of PIX horizontally adjacent pixels starting at
// (lx0, ly) = ((t % (16 / PIX)) * PIX, t / (16 / PIX)), so that one 128-bit
// shared-memory load of a face plane feeds PIX pixels.  Blocks are
// persistent and pull tiles of all cameras from one atomic queue.
#pragma once

#include "lp_device.cuh"
#include "lp_internal.h"

namespace lp {

constexpr int kTile = 16;
constexpr int kTilePixels = kTile * kTile;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

struct TileGeom {
    int tile;
    int tx0, ty0;         // first pixel of the tile
    int width, height;
    int pix_base;
};

__device__ __forceinline__ TileGeom tile_geom(const CamsParam& cams, int tile) {
    const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
    const int lt = tile - cm.tile_base;
    const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
    return TileGeom{tile, tx * kTile, ty * kTile, cm.width, cm.height, cm.pix_base};
}

}  // namespace lp
