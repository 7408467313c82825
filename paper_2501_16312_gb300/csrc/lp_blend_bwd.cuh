// Backward per-tile rasterization (sm_103a).
//
// A lane group of a warp (LaneGroups) skips the entries the forward blended
// at none of its pixels (the forward's mask row of that group) without
// evaluating their spans; the groups of a warp walk their rows independently.
//
// Sec. 3.4 "Rasterization Backpropagation": each tile walks its list back to
// front from the furthest last contributor of its pixels, recomputes every
// span bit-identically to the forward (same staging, same span routine),
// recovers T_i = T_{i+1} / tau_i from the stored transmittance before the
// last contributor (never dividing by the last primitive's tau, which may be
// ~0), keeps the suffix colour B_i = o_i c_i + tau_i B_{i+1} (B = background
// behind the last contributor) and forms
//   dL/dc_i = T_i o_i g,   dL/do_i = T_i (c_i - B_{i+1}) . g,
//   dL/ds = dL/do sigma tau,   dL/dsigma = dL/do s tau,
// and, since s = exit(x, y) - entry(x, y) with plane depth a x + b y + e, the
// plane gradients -+ dL/ds (x, y, 1) of the arg-max entry and arg-min exit
// faces -- the plane form of the paper's MTIA barycentric derivatives.  A
// thread sums its strip of pixels: the colour and sigma terms into one
// 16-byte row, each face's (x, y, 1) terms into one row per run of pixels
// sharing the face; it adds each row to the record's accumulator with one
// vector atomic (sm_90 and later).
//
// The kernels are templates over the tile edge; each of lp_blend_bwd_t8.cu,
// _t16.cu and _t32.cu instantiates one edge.
#pragma once

#include "lp_blend.cuh"

namespace lp {

namespace {

// Resident threads per SM the backward is compiled for, which sets its
// register budget.  Measured best on the 500k-octahedron, 8-view and
// 1M-tetrahedron, 16-view workloads: 1536 on 8x8 tiles (42 registers; 4-9%
// faster than 768), 1024 on 16x16 tiles with two pixels per thread (64
// registers; 8% faster, where 1280 was 35% slower), 768 otherwise (80
// registers; four pixels per thread spill heavily below that).
template <int TILE, int PIX> constexpr int bwd_resident_threads() {
    return TILE == 8 ? 1536 : (TILE == 16 && PIX == 2 ? 1024 : 768);
}
template <int TILE, int PIX> constexpr int bwd_min_blocks() {
    constexpr int nt = TILE * TILE / PIX;
    return bwd_resident_threads<TILE, PIX>() / nt > 0 ? bwd_resident_threads<TILE, PIX>() / nt : 1;
}

template <int V, int BATCH, int PIX, int TILE>
__global__ void __launch_bounds__(TILE * TILE / PIX, bwd_min_blocks<TILE, PIX>()) k_blend_bwd(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, const float* __restrict__ dimage,
    const uint32_t* __restrict__ last_in, const float* __restrict__ tl_in, float* __restrict__ acc,
    float* __restrict__ acc_col,
    int* __restrict__ tile_counter, const uint32_t* __restrict__ contrib, uint32_t cstride,
    const uint32_t* __restrict__ order) {
    constexpr int ACC = Acc<V>::kPlane;
    constexpr int NT = TILE * TILE / PIX;
    constexpr int MW = BATCH / 32;   // contributor-mask words per batch
    static_assert(NT % 32 == 0, "whole warps");
    static_assert(BATCH % 32 == 0, "whole mask words per batch");
    __shared__ Staged<V> sm[BATCH];
    __shared__ int s_tile;
    __shared__ int s_max;
    // entries of the batch that some lane group of the block visits (bit j:
    // entry lo + j), two sets used by alternate batches
    __shared__ uint32_t s_need[2][MW];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    int ly, lx0;   // the forward's pixel layout, so that warp w's mask bits are its own
    WarpGrid<TILE, PIX>::pixel(tid, ly, lx0);
    using LG = LaneGroups<TILE, PIX>;
    if (tid < 2 * MW) s_need[tid / MW][tid % MW] = 0u;
    int kb = 0;   // batches walked by this block, over all its tiles
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(tile_counter, 1);
            s_tile = order && q < cams.total_tiles ? (int)order[q] : q;
            s_max = 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= cams.total_tiles) break;
        const TileGeom tg = tile_geom<TILE>(cams, tile);
        const int py = tg.ty0 + ly;
        const uint2 rg = ranges[tile];
        const int plane = tg.width * tg.height;
        const float* gi = dimage + 3 * (size_t)tg.pix_base;
        float g0[PIX], g1[PIX], g2[PIX], Tcur[PIX], B0[PIX], B1[PIX], B2[PIX];
        uint32_t last[PIX];
        bool first[PIX];
        uint32_t lmax = 0;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            const int px = tg.tx0 + lx0 + i;
            g0[i] = g1[i] = g2[i] = 0.f; Tcur[i] = 1.f; last[i] = 0;
            if (px < tg.width && py < tg.height) {
                const int idx = py * tg.width + px;
                g0[i] = gi[idx]; g1[i] = gi[plane + idx]; g2[i] = gi[2 * plane + idx];
                last[i] = last_in[tg.pix_base + idx];
                Tcur[i] = tl_in[tg.pix_base + idx];
            }
            B0[i] = bg0; B1[i] = bg1; B2[i] = bg2;
            first[i] = true;
            lmax = max(lmax, last[i]);
        }
        if (lmax > 0) atomicMax(&s_max, (int)lmax);
        __syncthreads();
        const int hi_all = s_max;
        for (int hi = hi_all; hi > 0; hi -= BATCH) {
            const int lo = max(0, hi - BATCH);
            const int nb = hi - lo;
            // This lane group's bits of the forward's contributor mask for
            // entries lo .. hi - 1 (bit j of bm: entry lo + j), loaded once
            // per batch: lane g (MW + 1) + q fetches word q of group g's run,
            // each lane shifts its own group's words into place, and the walk
            // below visits the set bits only.
            const int grp = LG::group(lane);
            uint32_t bm[MW];
            {
                const uint32_t e0 = rg.x + (uint32_t)lo;
                const uint32_t w0 = e0 >> 5, sh = e0 & 31u;
                const uint32_t w_last = (e0 + (uint32_t)nb - 1u) >> 5;   // last word of the run
                const int lg = lane / (MW + 1), lq = lane - lg * (MW + 1);
                uint32_t src = 0u;
                if (lg < LG::G && w0 + (uint32_t)lq <= w_last)
                    src = contrib ? __ldg(mask_word<LG::G>(contrib, cstride, tid >> 5, lg, w0 + (uint32_t)lq))
                                  : 0xffffffffu;
#pragma unroll
                for (int q = 0; q < MW; ++q) {
                    const uint32_t lo_w = __shfl_sync(0xffffffffu, src, grp * (MW + 1) + q);
                    const uint32_t hi_w = __shfl_sync(0xffffffffu, src, grp * (MW + 1) + q + 1);
                    uint32_t m = sh ? (lo_w >> sh) | (hi_w << (32u - sh)) : lo_w;
                    const int valid = nb - 32 * q;   // entries of this word inside the batch
                    if (valid < 32) m &= valid > 0 ? (1u << valid) - 1u : 0u;
                    bm[q] = m;
                }
            }
            // Only the entries some lane group of the block visits are staged.
            uint32_t* need = s_need[kb & 1];
#pragma unroll
            for (int q = 0; q < MW; ++q) {
                const uint32_t u = __reduce_or_sync(0xffffffffu, bm[q]);
                if (lane == 0 && u) atomicOr(need + q, u);
            }
            __syncthreads();   // the sets are complete, and the last batch's walk is over
            for (int j = tid; j < nb; j += NT)
                if ((need[j >> 5] >> (j & 31)) & 1u) stage_record<V>(rec, vals[rg.x + lo + j], tg.tx0, tg.ty0, sm[j]);
            if (tid < MW) s_need[(kb + 1) & 1][tid] = 0u;   // for the next batch
            ++kb;
            __syncthreads();
            // Each lane group walks its own set bits, back to front, one mask
            // word at a time; the warp steps while some group has a bit left
            // in the word, and a group without one idles.  Entries the forward
            // blended at none of a group's pixels are never visited by that
            // group.
#pragma unroll 1
            for (int q = MW - 1; q >= 0; --q)
            for (uint32_t mq = bm[q];;) {
                const bool have = mq != 0u;
                if (!__any_sync(0xffffffffu, have)) break;
                int j = 0;
                if (have) {
                    const int bit = 31 - __clz(mq);
                    mq ^= 1u << bit;
                    j = 32 * q + bit;
                }
                const uint32_t idx = (uint32_t)(lo + j);
                const Staged<V>& p = sm[j];
                bool any = false;
#pragma unroll
                for (int i = 0; i < PIX; ++i) any |= have && idx < last[i];
                float sp[PIX];
                int sf[PIX], sb[PIX];
                bool c[PIX];
                bool anyc = false;
#pragma unroll
                for (int i = 0; i < PIX; ++i) c[i] = false;
                if (any) {
                    // one pass with the entry/exit slots: with the entries this
                    // warp blended nowhere skipped, most warps contribute
                    spans<V, PIX, true>(p, (float)lx0 + p.dx0, (float)ly + p.dy0, sp, sf, sb);
#pragma unroll
                    for (int i = 0; i < PIX; ++i) {
                        c[i] = idx < last[i] && sp[i] > 0.f;
                        anyc |= c[i];
                    }
                }
                if (!__any_sync(0xffffffffu, anyc)) continue;
                float gr0 = 0.f, gr1 = 0.f, gr2 = 0.f, gsig = 0.f;
                float gsp[PIX];
#pragma unroll
                for (int i = 0; i < PIX; ++i) gsp[i] = 0.f;
                if (anyc) {
#pragma unroll
                    for (int i = 0; i < PIX; ++i) {
                        if (c[i]) {
                            const float xs = span_x(p.sigma, sp[i]);
                            const float tau = span_tau(xs);
                            const float o = span_opacity(xs, tau);
                            // tau >= 1e-3 wherever we divide (T stayed >= 1e-3 before
                            // the last contributor), so the fast division is safe
                            const float Ti = first[i] ? Tcur[i] : __fdividef(Tcur[i], tau);
                            first[i] = false;
                            Tcur[i] = Ti;
                            const float w = Ti * o;
                            gr0 = fmaf(w, g0[i], gr0);
                            gr1 = fmaf(w, g1[i], gr1);
                            gr2 = fmaf(w, g2[i], gr2);
                            const float dLdo = Ti * ((p.r - B0[i]) * g0[i] + (p.g - B1[i]) * g1[i] +
                                                     (p.b - B2[i]) * g2[i]);
                            B0[i] = fmaf(o, p.r, tau * B0[i]);
                            B1[i] = fmaf(o, p.g, tau * B1[i]);
                            B2[i] = fmaf(o, p.b, tau * B2[i]);
                            gsp[i] = dLdo * p.sigma * tau;        // dL/d span
                            gsig = fmaf(dLdo * sp[i], tau, gsig);  // dL/d sigma
                        }
                    }
                }
                float* A = acc + (size_t)p.rec * ACC;        // plane moments
                float* Ac = acc_col + (size_t)p.rec * 4;     // colour and density
                if (!anyc) continue;
                // Colour and density: each contributing lane adds its own row
                // with one 16-byte vector atomic (measured faster than summing
                // over the lane group with shuffles first, at every threshold
                // of contributing lanes tried).
                atomicAdd(reinterpret_cast<float4*>(Ac), make_float4(gr0, gr1, gr2, gsig));
                // Planes: each contributing lane adds the (x, y, 1) row of an
                // entry or exit face once per run of its pixels that share
                // that face, one 16-byte vector atomic each (measured faster
                // than warp butterflies over the faces, however many lanes
                // contribute).  Offsets (px - X0, py - Y0) are from the anchor.
                const float lyc = (float)ly + p.dy0;
                float4 re = make_float4(0.f, 0.f, 0.f, 0.f), rb = re;
                int fe = -1, fb = -1;
#pragma unroll
                for (int i = 0; i < PIX; ++i) {
                    if (!c[i]) continue;
                    const float lxc = (float)(lx0 + i) + p.dx0;
                    const float gx = gsp[i] * lxc, gy = gsp[i] * lyc, g1 = gsp[i];
                    if (sf[i] != fe) {
                        if (fe >= 0) atomicAdd(reinterpret_cast<float4*>(A + 4 * fe), re);
                        fe = sf[i];
                        re = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    if (sb[i] != fb) {
                        if (fb >= 0) atomicAdd(reinterpret_cast<float4*>(A + 4 * fb), rb);
                        fb = sb[i];
                        rb = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    re.x -= gx; re.y -= gy; re.z -= g1;
                    rb.x += gx; rb.y += gy; rb.z += g1;
                }
                atomicAdd(reinterpret_cast<float4*>(A + 4 * fe), re);
                atomicAdd(reinterpret_cast<float4*>(A + 4 * fb), rb);
            }
        }
        __syncthreads();
    }
}

template <int V, int BATCH, int PIX, int TILE>
cudaError_t bwd_t(const BlendArgs& a, cudaStream_t st) {
    k_blend_bwd<V, BATCH, PIX, TILE><<<a.grid, TILE * TILE / PIX, 0, st>>>(
        a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.dimage, a.last, a.tl, a.acc,
        a.acc_col, a.tile_counter, a.contrib, a.contrib_stride, a.order);
    return cudaGetLastError();
}

template <int V, int BATCH, int PIX, int TILE>
int bwd_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blend_bwd<V, BATCH, PIX, TILE>, TILE * TILE / PIX, 0);
    return nb;
}

#define LP_PIX_CASES_B(FN, V, B, T, ...)                                                     \
    if constexpr (tile_pix_ok(T, 1)) { if (pix == 1) return FN<V, B, 1, T>(__VA_ARGS__); }   \
    if constexpr (tile_pix_ok(T, 2)) { if (pix == 2) return FN<V, B, 2, T>(__VA_ARGS__); }   \
    if constexpr (tile_pix_ok(T, 4)) { if (pix == 4) return FN<V, B, 4, T>(__VA_ARGS__); }
#define LP_BLEND_DISPATCH_B(FN, T, BAD, ...)                                                 \
    if (V == 6) {                                                                            \
        if (batch == 32) { LP_PIX_CASES_B(FN, 6, 32, T, __VA_ARGS__) }                       \
        else if (batch == 128) { LP_PIX_CASES_B(FN, 6, 128, T, __VA_ARGS__) }                \
        else { LP_PIX_CASES_B(FN, 6, 64, T, __VA_ARGS__) }                                   \
    } else {                                                                                 \
        if (batch == 32) { LP_PIX_CASES_B(FN, 4, 32, T, __VA_ARGS__) }                       \
        else if (batch == 128) { LP_PIX_CASES_B(FN, 4, 128, T, __VA_ARGS__) }                \
        else { LP_PIX_CASES_B(FN, 4, 64, T, __VA_ARGS__) }                                   \
    }                                                                                        \
    return BAD;

template <int TILE>
cudaError_t launch_bwd_tile(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    LP_BLEND_DISPATCH_B(bwd_t, TILE, cudaErrorInvalidValue, a, st)
}

template <int TILE>
int occ_bwd_tile(int V, int batch, int pix) {
    LP_BLEND_DISPATCH_B(bwd_occ, TILE, 0)
}

}  // namespace

}  // namespace lp
