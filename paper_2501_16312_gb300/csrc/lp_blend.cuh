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
    __host__ __device__ __forceinline__ static int group(int lane) {
        return G == 1 ? 0 : G == 2 ? lane >> 4 : ((lane >> 4) << 1) | ((lane >> kColBit) & 1);
    }
    // the group's first lane (every other lane bit clear) writes its mask row
    __host__ __device__ __forceinline__ static bool leader(int lane) { return (lane & ~(int)kGroupBits) == 0; }
    // OR of x over the lanes of each lane's group
    __device__ __forceinline__ static uint32_t reduce_or(uint32_t x) {
        if (G == 1) return __reduce_or_sync(0xffffffffu, x);
#pragma unroll
        for (int b = 0; b < 5; ++b)
            if (!((kGroupBits >> b) & 1u)) x |= __shfl_xor_sync(0xffffffffu, x, 1 << b);
        return x;
    }
};

// The pixel rectangle of lane group g of warp w in its tile: columns
// [x0, x0 + GW), rows [y0, y0 + GH).
template <int TILE, int PIX> struct GroupRect {
    using WG = WarpGrid<TILE, PIX>;
    static constexpr int G = LaneGroups<TILE, PIX>::G;
    static constexpr int GX = G == 4 ? 2 : 1, GY = G == 1 ? 1 : 2;
    static constexpr int GW = WG::WC / GX, GH = WG::WR / GY;
    static constexpr int x0(int w, int g) { return (w % WG::NWX) * WG::WC + (G == 4 ? (g & 1) : 0) * GW; }
    static constexpr int y0(int w, int g) { return (w / WG::NWX) * WG::WR + (G == 4 ? g >> 1 : G == 2 ? g : 0) * GH; }
};

// Band bits of a staged record for its tile (Staged::bands): bit w G + g is
// clear when the ray through every pixel of lane group g's rectangle in warp
// w provably misses the primitive.  The ray meets the primitive at pixel p
// only if every entry face lies below every exit face there, d_f(p) < d_b(p);
// each pair's difference is linear in p, so its largest value over a
// rectangle is at a corner, and a rectangle where some pair stays below
// -margin (a bound on the rounding of the planes' evaluation) holds no
// covered pixel.
//
// Only pairs of faces that share an edge are tried.  The covered pixels of a
// convex primitive form its silhouette polygon, the intersection of the
// half-planes d_f < d_b of its silhouette edges, and every silhouette edge
// joins an entry face to an exit face.  Every two faces of a tetrahedron
// share an edge (at most 4 entry/exit pairs); two faces of an octahedron
// share one when their indices differ in one vertex choice (one bit), which
// leaves its 4 or 6 silhouette edges of the 16 entry/exit pairs.  Trying
// fewer pairs can only keep more rectangles, never drop a covered one,
// whatever the shape.
template <int V, int TILE, int PIX>
__device__ __forceinline__ uint64_t band_mask(const Staged<V>& s, uint32_t meta) {
    using R = GroupRect<TILE, PIX>;
    constexpr int F = Kind<V>::F;
    constexpr int NR = WarpGrid<TILE, PIX>::NW * R::G;   // rectangles
    static_assert(NR >= 1 && NR <= 64, "one bit per rectangle");
    constexpr float XM = (float)(TILE - 1);
    const int nf = meta_nf(meta);
    if (nf <= 0 || nf >= F) return 0ull;
    uint64_t mask = NR == 64 ? ~0ull : (1ull << NR) - 1ull;
    // the margin bounds the rounding of every term of a plane's evaluation at
    // a pixel of the tile (offsets up to |dx0| + TILE - 1 from the anchor)
    const float ox = fabsf(s.dx0) + XM, oy = fabsf(s.dy0) + XM;
    auto pair = [&](int f, int b) {
        const float4 pf = s.pl[f], pb = s.pl[b];
        const float ef = __fmaf_rn(pf.x, s.dx0, __fmaf_rn(pf.y, s.dy0, pf.z));   // at the tile origin
        const float eb = __fmaf_rn(pb.x, s.dx0, __fmaf_rn(pb.y, s.dy0, pb.z));
        const float da = pb.x - pf.x, db = pb.y - pf.y, de = eb - ef;
        const float margin = 1e-5f * (fabsf(pb.z) + fabsf(pf.z) + fabsf(eb) + fabsf(ef) +
                                      ox * (fabsf(pb.x) + fabsf(pf.x)) + oy * (fabsf(pb.y) + fabsf(pf.y))) +
                             1e-30f;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            const int w = r / R::G, g = r % R::G;
            const float x0 = (float)R::x0(w, g), x1 = x0 + (float)(R::GW - 1);
            const float y0 = (float)R::y0(w, g), y1 = y0 + (float)(R::GH - 1);
            const float m = de + fmaxf(da * x0, da * x1) + fmaxf(db * y0, db * y1);
            if (m < -margin) mask &= ~(1ull << r);
        }
    };
    if (V == 6) {
        // face index -> slot (3 bits each), and the entry faces as a set
        uint32_t slot_of = 0u, E = 0u;
#pragma unroll
        for (int q = 0; q < F; ++q) {
            const int fc = meta_face(meta, q);
            slot_of |= (uint32_t)q << (3 * fc);
            if (q < nf) E |= 1u << fc;
        }
        // entry faces whose neighbour across bit k (k = 1, 2, 4) is an exit
        // face: bit i of byte log2(k) of sil
        const uint32_t n1 = ((E & 0x55u) << 1) | ((E >> 1) & 0x55u);
        const uint32_t n2 = ((E & 0x33u) << 2) | ((E >> 2) & 0x33u);
        const uint32_t n4 = ((E & 0x0Fu) << 4) | ((E >> 4) & 0x0Fu);
        uint32_t sil = (E & ~n1) | ((E & ~n2) << 8) | ((E & ~n4) << 16);
        while (sil) {
            const int bit = __ffs(sil) - 1;
            sil &= sil - 1u;
            const int i = bit & 7, k = 1 << (bit >> 3);
            pair((int)((slot_of >> (3 * i)) & 7u), (int)((slot_of >> (3 * (i ^ k))) & 7u));
        }
    } else {
        for (int f = 0; f < nf; ++f)
            for (int b = nf; b < F; ++b) pair(f, b);
    }
    return mask;
}

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
