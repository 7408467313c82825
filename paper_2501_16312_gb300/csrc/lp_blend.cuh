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


// Lane groups of a blend warp (lane_groups(TILE, PIX) of them: 1, 2 or 4).
// The forward writes one contributor-mask row per group and the backward's
// groups walk
// their own rows independently, so that a group visits only the entries that
// its own pixels blended.  Four groups are the quadrants of the warp's pixel
// rectangle, two its upper and lower halves.  A warp rectangle has WR rows
// of TPR threads (WR * TPR = 32): lanes 16..31 hold its lower half (lane bit
// 4), and lane bit log2(TPR) - 1 marks a thread in the right half of a row.
template <int TILE, int PIX> struct LaneGroups {
    using WG = WarpGrid<TILE, PIX>;
    static constexpr int G = lane_groups(TILE, PIX);
    static_assert(G == 1 || G == 2 || G == 4, "1, 2 or 4 lane groups");
    static_assert(WG::TPR * WG::WR == 32 && WG::TPR >= 2 && WG::TPR <= 16, "rows of whole threads");
    static constexpr int kColBit = WG::TPR == 2 ? 0 : WG::TPR == 4 ? 1 : WG::TPR == 8 ? 2 : 3;
    // the lane bits that name a group
    static constexpr uint32_t kGroupBits = G == 1 ? 0u : G == 2 ? 16u : (16u | (1u << kColBit));
    __device__ __forceinline__ static int group(int lane) {
        return G == 1 ? 0 : G == 2 ? lane >> 4 : ((lane >> 4) << 1) | ((lane >> kColBit) & 1);
    }
    // the group's first lane (every other lane bit clear) writes its mask row
    __device__ __forceinline__ static bool leader(int lane) { return (lane & ~(int)kGroupBits) == 0; }
    // OR of x over the lanes of each lane's group
    __device__ __forceinline__ static uint32_t reduce_or(uint32_t x) {
        if (G == 1) return __reduce_or_sync(0xffffffffu, x);
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if (!((kGroupBits >> b) & 1u)) x |= __shfl_xor_sync(0xffffffffu, x, 1 << b);
        return x;
    }
};

// Word w of lane group g's contributor-mask row for warp `warp` of a tile.
// The G rows of a warp are interleaved word by word (a warp's block holds
// cstride words per group), so that the groups' words of one chunk of
// entries share a 32-byte sector.
template <int G>
__device__ __forceinline__ uint32_t* mask_word(uint32_t* contrib, uint32_t cstride, int warp, int g, uint32_t w) {
    return contrib + (size_t)warp * G * cstride + (size_t)w * G + g;
}
template <int G>
__device__ __forceinline__ const uint32_t* mask_word(const uint32_t* contrib, uint32_t cstride, int warp, int g,
                                                     uint32_t w) {
    return contrib + (size_t)warp * G * cstride + (size_t)w * G + g;
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
