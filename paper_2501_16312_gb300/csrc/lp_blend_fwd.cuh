// Forward per-tile rasterization and compositing (sm_103a).
//
// Sec. 3.2 "Rasterization" and "Compositing": each 16x16 tile walks its
// depth-sorted list front to back, staging batches of projected records in
// shared memory; each pixel ray is clipped against the primitive's face
// half-spaces, the span s gives the opacity o = 1 - exp(-sigma s) (App.
// "Gradient Computation"), colours are blended front to back, and a pixel
// stops once its transmittance falls below 1e-3 (cumulative opacity 0.999),
// after blending the primitive that crossed it.  A tile stops when all of its
// pixels have.  Per pixel the kernel keeps, for the backward, the number of
// list entries up to the last contributor and the transmittance before it,
// and per lane group of a warp (LaneGroups) one bit per list entry its
// pixels blended.  A warp skips the records that the staging test proves
// cover none of its pixels.
//
// MODE 1 also counts (pixel, primitive) pairs.  MODE 2 is the depth pass
// (App. "Depth and Surface Reconstruction"): the same walk, stopping each
// pixel at the first primitive that takes the cumulative opacity above 0.5
// and writing the depth where the ray enters that primitive (0 if none).
//
// The kernels are templates over the tile edge; each of lp_blend_fwd_t8.cu,
// _t16.cu and _t32.cu instantiates one edge (one translation unit each, so
// they compile in parallel).
#pragma once

#include "lp_blend.cuh"

namespace lp {

namespace {

// Word w of a contributor-mask row, at p: a plain store when the word holds
// entries of this tile only (no other block writes it, and it is written
// once), an atomic OR when it may share bits with a neighbouring tile's list.
__device__ __forceinline__ void put_mask_word(uint32_t* p, uint32_t w, uint32_t v, uint2 rg) {
    if (32ull * w >= rg.x && 32ull * w + 32ull <= rg.y) *p = v;
    else atomicOr(p, v);
}

template <int V, int BATCH, int PIX, int MODE, int TILE>
__global__ void __launch_bounds__(TILE * TILE / PIX) k_blend_fwd(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, float* __restrict__ image,
    uint32_t* __restrict__ last_out, float* __restrict__ tl_out, int* __restrict__ tile_counter,
    unsigned long long* __restrict__ pair_counts, float* __restrict__ depth_out,
    uint32_t* __restrict__ contrib, uint32_t cstride, const uint32_t* __restrict__ order) {
    constexpr bool COUNT = MODE == 1;
    constexpr bool DEPTH = MODE == 2;
    constexpr float kStop = DEPTH ? 0.5f : kStopT;
    constexpr int NT = TILE * TILE / PIX;
    __shared__ Staged<V> sm[BATCH];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    int ly, lx0;
    WarpGrid<TILE, PIX>::pixel(tid, ly, lx0);
    using LG = LaneGroups<TILE, PIX>;
    const int grp = LG::group(lane);
    const uint32_t group_lanes = __match_any_sync(0xffffffffu, grp);   // the lanes of this lane's group
    const bool write_mask = !DEPTH && contrib != nullptr;
    unsigned long long n_iter = 0, n_eval = 0, n_hit = 0, n_iter_last = 0;
    for (;;) {
        if (tid == 0) {
            const int q = atomicAdd(tile_counter, 1);
            s_tile = order && q < cams.total_tiles ? (int)order[q] : q;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= cams.total_tiles) break;
        const TileGeom tg = tile_geom<TILE>(cams, tile);
        const int py = tg.ty0 + ly;
        const uint2 rg = ranges[tile];
        const int n = (int)(rg.y - rg.x);
        float T[PIX], c0[PIX], c1[PIX], c2[PIX], tl[PIX];
        uint32_t last[PIX];
        float dep[PIX];              // depth pass only
        bool done[PIX];
        bool tdone = true;
        // mask bits of this lane group waiting for the next chunk to complete
        // their word (group leaders only)
        uint32_t pend = 0u;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            T[i] = 1.f; c0[i] = c1[i] = c2[i] = 0.f; tl[i] = 1.f; last[i] = 0;
            dep[i] = 0.f;
            done[i] = !(tg.tx0 + lx0 + i < tg.width && py < tg.height);
            tdone &= done[i];
        }
        for (int b0 = 0; b0 < n; b0 += BATCH) {
            if (__syncthreads_count(!tdone) == 0) break;
            const int nb = min(BATCH, n - b0);
            for (int j = tid; j < nb; j += NT) {
                const uint32_t meta = stage_record<V>(rec, vals[rg.x + b0 + j], tg.tx0, tg.ty0, sm[j]);
                sm[j].bands = band_mask<V, TILE, PIX>(sm[j], meta);
            }
            __syncthreads();
            if (__any_sync(0xffffffffu, !tdone)) {   // warp-uniform, as the exit below
                for (int jw = 0; jw < nb; jw += 32) {
                    // Entries b0 + jw .. b0 + jw + 31: the ones the staging
                    // test leaves possibly covered in this lane group's
                    // rectangle (bit j - jw), one ballot per group.
                    uint32_t mq = 0u;
                    {
                        const int jl = jw + lane;
                        const uint64_t bl = jl < nb ? sm[jl].bands >> ((tid >> 5) * LG::G) : 0ull;
#pragma unroll
                        for (int g = 0; g < LG::G; ++g) {
                            const uint32_t bal = __ballot_sync(0xffffffffu, (uint32_t)(bl >> g) & 1u);
                            mq = grp == g ? bal : mq;
                        }
                    }
                    uint32_t bm = 0;   // bit j - jw: this thread blended entry b0 + j
                    // Each lane group walks its own entries front to back, and
                    // stops taking them once all of its pixels have stopped;
                    // the warp steps while some group has one left.
                    for (;;) {
                        if (!(__ballot_sync(0xffffffffu, !tdone) & group_lanes)) mq = 0u;
                        const bool have = mq != 0u;
                        if (!__any_sync(0xffffffffu, have)) break;
                        if (have) {
                            const int bit = __ffs(mq) - 1;
                            mq &= mq - 1u;
                            const int j = jw + bit;
                            const Staged<V>& p = sm[j];
                            float sp[PIX];
                            spans<V, PIX, false>(p, (float)lx0 + p.dx0, (float)ly + p.dy0, sp, nullptr, nullptr);
                            tdone = true;
                            bool blended = false;
#pragma unroll
                            for (int i = 0; i < PIX; ++i) {
                                const bool in = !done[i];   // visited and not proven uncovered: evaluated
                                if (COUNT) n_eval += in;
                                if (in && sp[i] > 0.f) {
                                    blended = true;
                                    if (COUNT) ++n_hit;
                                    const float xs = span_x(p.sigma, sp[i]);
                                    const float tau = span_tau(xs);
                                    const float w = T[i] * span_opacity(xs, tau);
                                    c0[i] = fmaf(w, p.r, c0[i]);
                                    c1[i] = fmaf(w, p.g, c1[i]);
                                    c2[i] = fmaf(w, p.b, c2[i]);
                                    tl[i] = T[i];
                                    T[i] *= tau;
                                    last[i] = (uint32_t)(b0 + j + 1);
                                    done[i] = T[i] < kStop;
                                    if (DEPTH && done[i]) {
                                        // entry depth: centre depth + max over the entry faces
                                        float e = -CUDART_INF_F;
                                        for (int f = 0; f < p.nf; ++f)
                                            e = fmaxf(e, __fmaf_rn(p.pl[f].x, (float)(lx0 + i) + p.dx0,
                                                                   __fmaf_rn(p.pl[f].y, (float)ly + p.dy0, p.pl[f].z)));
                                        dep[i] = __fadd_rn(p.pl[0].w, e);
                                    }
                                }
                                tdone &= done[i];
                            }
                            if (write_mask && blended) bm |= 1u << bit;
                        }
                    }
                    // the warp stops once all of its pixels have
                    const bool stop = !__any_sync(0xffffffffu, !tdone);
                    if (write_mask) {
                        // entries b0 + jw .. b0 + jw + 31 of the tile's list,
                        // blended at some pixel of this lane's group.  Words
                        // follow each other without gaps until the warp stops,
                        // so word w is complete once this word's low part
                        // joins the previous one's high part.
                        bm = LG::reduce_or(bm);
                        if (LG::leader(lane)) {
                            const uint32_t e0 = rg.x + (uint32_t)(b0 + jw);
                            const uint32_t w = e0 >> 5, sh = e0 & 31u;
                            const uint32_t v = pend | (bm << sh);
                            if (v) put_mask_word(mask_word<LG::G>(contrib, cstride, tid >> 5, grp, w), w, v, rg);
                            pend = sh ? bm >> (32u - sh) : 0u;
                            // no word follows after the tile's last one or once
                            // the warp stops: the next word is complete as well
                            if (pend && (stop || b0 + jw + 32 >= n)) {
                                put_mask_word(mask_word<LG::G>(contrib, cstride, tid >> 5, grp, w + 1u), w + 1u,
                                              pend, rg);
                                pend = 0u;
                            }
                        }
                    }
                    if (stop) break;
                }
            }
        }
        if (COUNT) {
            // entries a pixel walked: up to the one that stopped it, else the
            // whole list (the tile walks on while any pixel is active); and
            // up to its last contributor
#pragma unroll
            for (int i = 0; i < PIX; ++i) {
                n_iter_last += last[i];
                n_iter += done[i] ? last[i] : (uint32_t)n;
            }
        }
        const int plane = tg.width * tg.height;
        float* img = image + 3 * (size_t)tg.pix_base;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            const int px = tg.tx0 + lx0 + i;
            if (DEPTH) {
                if (px < tg.width && py < tg.height) depth_out[tg.pix_base + py * tg.width + px] = dep[i];
                continue;
            }
            if (px < tg.width && py < tg.height) {
                const int idx = py * tg.width + px;
                img[idx] = fmaf(T[i], bg0, c0[i]);
                img[plane + idx] = fmaf(T[i], bg1, c1[i]);
                img[2 * plane + idx] = fmaf(T[i], bg2, c2[i]);
                last_out[tg.pix_base + idx] = last[i];
                tl_out[tg.pix_base + idx] = tl[i];
            }
        }
        __syncthreads();
    }
    if (COUNT) {
        unsigned long long a = n_iter, b = n_eval, c = n_hit, d = n_iter_last;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        if ((tid & 31) == 0) {
            atomicAdd(pair_counts, a);
            atomicAdd(pair_counts + 1, b);
            atomicAdd(pair_counts + 2, c);
            atomicAdd(pair_counts + 3, d);
        }
    }
}

template <int V, int BATCH, int PIX, int TILE>
cudaError_t fwd_t(const BlendArgs& a, cudaStream_t st) {
    constexpr int NT = TILE * TILE / PIX;
    if (a.depth)
        k_blend_fwd<V, BATCH, PIX, 2, TILE><<<a.grid, NT, 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl,
            a.tile_counter, a.pair_counts, a.depth, nullptr, 0u, a.order);
    else if (a.count)
        k_blend_fwd<V, BATCH, PIX, 1, TILE><<<a.grid, NT, 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl,
            a.tile_counter, a.pair_counts, nullptr, a.contrib, a.contrib_stride, a.order);
    else
        k_blend_fwd<V, BATCH, PIX, 0, TILE><<<a.grid, NT, 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl,
            a.tile_counter, a.pair_counts, nullptr, a.contrib, a.contrib_stride, a.order);
    return cudaGetLastError();
}

template <int V, int BATCH, int PIX, int TILE>
int fwd_occ() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_blend_fwd<V, BATCH, PIX, 0, TILE>,
                                                  TILE * TILE / PIX, 0);
    return nb;
}

// Dispatch over (V, BATCH, PIX) for one tile edge; a (tile, pix) pair the
// kernels are not built for is rejected (lp_set_tuning checks it first).
#define LP_PIX_CASES(FN, V, B, T, ...)                                                       \
    if constexpr (tile_pix_ok(T, 1)) { if (pix == 1) return FN<V, B, 1, T>(__VA_ARGS__); }   \
    if constexpr (tile_pix_ok(T, 2)) { if (pix == 2) return FN<V, B, 2, T>(__VA_ARGS__); }   \
    if constexpr (tile_pix_ok(T, 4)) { if (pix == 4) return FN<V, B, 4, T>(__VA_ARGS__); }
#define LP_BLEND_DISPATCH(FN, T, BAD, ...)                                                   \
    if (V == 6) {                                                                            \
        if (batch == 32) { LP_PIX_CASES(FN, 6, 32, T, __VA_ARGS__) }                         \
        else if (batch == 128) { LP_PIX_CASES(FN, 6, 128, T, __VA_ARGS__) }                  \
        else { LP_PIX_CASES(FN, 6, 64, T, __VA_ARGS__) }                                     \
    } else {                                                                                 \
        if (batch == 32) { LP_PIX_CASES(FN, 4, 32, T, __VA_ARGS__) }                         \
        else if (batch == 128) { LP_PIX_CASES(FN, 4, 128, T, __VA_ARGS__) }                  \
        else { LP_PIX_CASES(FN, 4, 64, T, __VA_ARGS__) }                                     \
    }                                                                                        \
    return BAD;

template <int TILE>
cudaError_t launch_fwd_tile(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    LP_BLEND_DISPATCH(fwd_t, TILE, cudaErrorInvalidValue, a, st)
}

template <int TILE>
int occ_fwd_tile(int V, int batch, int pix) {
    LP_BLEND_DISPATCH(fwd_occ, TILE, 0)
}

}  // namespace

}  // namespace lp
