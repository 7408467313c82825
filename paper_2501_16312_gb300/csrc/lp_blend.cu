// Per-tile rasterization and compositing (sm_103a).
//
// Forward, Sec. 3.2 "Rasterization" and "Compositing": each 16x16 tile walks
// its depth-sorted list front to back, staging batches of projected records
// in shared memory; each pixel ray is clipped against the primitive's face
// half-spaces, the span gives the opacity o = 1 - exp(-sigma s) (App.
// "Gradient Computation"), colours are blended front to back, and a pixel
// stops once its transmittance falls below 1e-3 (cumulative opacity 0.999),
// after blending the primitive that crossed it.  A tile stops when all of its
// pixels have.
//
// Backward, Sec. 3.4 "Rasterization Backpropagation": the tile walks its list
// back to front from the furthest last contributor of its pixels, recomputes
// each span bit-identically, recovers T_i = T_{i+1} / tau_i from the stored
// transmittance before the last contributor, keeps the suffix colour
// B_i = o_i c_i + tau_i B_{i+1}, and accumulates dL/d(colour, sigma) and
// dL/d(plane coefficients) of the entry and exit faces.  Per-warp sums are
// formed with shuffles before one atomic add per value.
//
// Both kernels are persistent: blocks pull tiles of all cameras from one
// atomic queue.
#include "lp_device.cuh"
#include "lp_internal.h"

namespace lp {

namespace {

constexpr int kTile = 16;
constexpr int kThreads = kTile * kTile;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

template <int V, int BATCH, bool COUNT>
__global__ void __launch_bounds__(kThreads) k_blend_fwd(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, float* __restrict__ image,
    uint32_t* __restrict__ last_out, float* __restrict__ tl_out, int* __restrict__ tile_counter,
    unsigned long long* __restrict__ pair_counts) {
    __shared__ Staged<V> sm[BATCH];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const int lx = tid % kTile, ly = tid / kTile;
    unsigned long long n_iter = 0, n_hit = 0;
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(tile_counter, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= cams.total_tiles) break;
        const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
        const int lt = tile - cm.tile_base;
        const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        const bool inside = px < cm.width && py < cm.height;
        const int tx0 = tx * kTile, ty0 = ty * kTile;
        const uint2 rg = ranges[tile];
        const int n = (int)(rg.y - rg.x);
        float T = 1.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, tl = 1.f;
        uint32_t last = 0;
        bool done = !inside;
        for (int b0 = 0; b0 < n; b0 += BATCH) {
            if (__syncthreads_count(!done) == 0) break;
            const int nb = min(BATCH, n - b0);
            for (int j = tid; j < nb; j += kThreads) stage_record<V>(rec, vals[rg.x + b0 + j], tx0, ty0, sm[j]);
            __syncthreads();
            if (!done) {
                for (int j = 0; j < nb; ++j) {
                    const float s = span_at<V>(sm[j], (float)lx, (float)ly);
                    if (COUNT) ++n_iter;
                    if (s > 0.f) {
                        if (COUNT) ++n_hit;
                        const float tau = span_tau(sm[j].sigma, s);
                        const float w = T * (1.f - tau);
                        c0 = fmaf(w, sm[j].rgb[0], c0);
                        c1 = fmaf(w, sm[j].rgb[1], c1);
                        c2 = fmaf(w, sm[j].rgb[2], c2);
                        tl = T;
                        T *= tau;
                        last = (uint32_t)(b0 + j + 1);
                        if (T < kStopT) { done = true; break; }
                    }
                }
            }
        }
        if (inside) {
            const int plane = cm.width * cm.height;
            const int idx = py * cm.width + px;
            float* img = image + 3 * (size_t)cm.pix_base;
            img[idx] = fmaf(T, bg0, c0);
            img[plane + idx] = fmaf(T, bg1, c1);
            img[2 * plane + idx] = fmaf(T, bg2, c2);
            last_out[cm.pix_base + idx] = last;
            tl_out[cm.pix_base + idx] = tl;
        }
        __syncthreads();
    }
    if (COUNT) {
        unsigned long long a = n_iter, b = n_hit;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if ((tid & 31) == 0) {
            atomicAdd(pair_counts, a);
            atomicAdd(pair_counts + 1, b);
        }
    }
}

template <int V, int BATCH>
__global__ void __launch_bounds__(kThreads) k_blend_bwd(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, const float* __restrict__ dimage,
    const uint32_t* __restrict__ last_in, const float* __restrict__ tl_in, float* __restrict__ acc,
    int* __restrict__ tile_counter) {
    constexpr int F = Kind<V>::F;
    constexpr int ACC = Acc<V>::kFloats;
    __shared__ Staged<V> sm[BATCH];
    __shared__ int s_tile;
    __shared__ int s_max;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int lx = tid % kTile, ly = tid / kTile;
    for (;;) {
        if (tid == 0) {
            s_tile = atomicAdd(tile_counter, 1);
            s_max = 0;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= cams.total_tiles) break;
        const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
        const int lt = tile - cm.tile_base;
        const int ty = lt / cm.tiles_x, tx = lt - ty * cm.tiles_x;
        const int px = tx * kTile + lx, py = ty * kTile + ly;
        const bool inside = px < cm.width && py < cm.height;
        const int tx0 = tx * kTile, ty0 = ty * kTile;
        const uint2 rg = ranges[tile];
        float g0 = 0.f, g1 = 0.f, g2 = 0.f, tl = 1.f;
        uint32_t last = 0;
        if (inside) {
            const int plane = cm.width * cm.height;
            const int idx = py * cm.width + px;
            const float* gi = dimage + 3 * (size_t)cm.pix_base;
            g0 = gi[idx]; g1 = gi[plane + idx]; g2 = gi[2 * plane + idx];
            last = last_in[cm.pix_base + idx];
            tl = tl_in[cm.pix_base + idx];
        }
        if (last > 0) atomicMax(&s_max, (int)last);
        __syncthreads();
        const int hi_all = s_max;
        float Tcur = tl, B0 = bg0, B1 = bg1, B2 = bg2;
        bool first = true;
        for (int hi = hi_all; hi > 0; hi -= BATCH) {
            const int lo = max(0, hi - BATCH);
            const int nb = hi - lo;
            __syncthreads();
            for (int j = tid; j < nb; j += kThreads) stage_record<V>(rec, vals[rg.x + lo + j], tx0, ty0, sm[j]);
            __syncthreads();
            for (int j = nb - 1; j >= 0; --j) {
                const Staged<V>& p = sm[j];
                float s = 0.f;
                int sf = 0, sb = 0;
                bool c = false;
                if ((uint32_t)(lo + j) < last) {
                    s = span_arg<V>(p, (float)lx, (float)ly, sf, sb);
                    c = s > 0.f;
                }
                if (__ballot_sync(0xffffffffu, c) == 0u) continue;
                float gr0 = 0.f, gr1 = 0.f, gr2 = 0.f, gsig = 0.f, gs = 0.f;
                if (c) {
                    const float tau = span_tau(p.sigma, s);
                    const float o = 1.f - tau;
                    const float Ti = first ? tl : Tcur / tau;
                    first = false;
                    Tcur = Ti;
                    const float w = Ti * o;
                    gr0 = w * g0; gr1 = w * g1; gr2 = w * g2;
                    const float dLdo = Ti * ((p.rgb[0] - B0) * g0 + (p.rgb[1] - B1) * g1 + (p.rgb[2] - B2) * g2);
                    B0 = fmaf(o, p.rgb[0], tau * B0);
                    B1 = fmaf(o, p.rgb[1], tau * B1);
                    B2 = fmaf(o, p.rgb[2], tau * B2);
                    gs = dLdo * p.sigma * tau;      // dL/d span
                    gsig = dLdo * s * tau;          // dL/d sigma
                }
                // integer pixel offsets from the record's anchor (X0, Y0)
                const float lxc = (float)lx + p.dx0, lyc = (float)ly + p.dy0;
                float* A = acc + (size_t)p.rec * ACC;
                gr0 = warp_sum(gr0); gr1 = warp_sum(gr1); gr2 = warp_sum(gr2); gsig = warp_sum(gsig);
                if (lane == 0) {
                    atomicAdd(A + 3 * F + 0, gr0);
                    atomicAdd(A + 3 * F + 1, gr1);
                    atomicAdd(A + 3 * F + 2, gr2);
                    atomicAdd(A + 3 * F + 3, gsig);
                }
                // span = exit - entry; plane depth = a lxc + b lyc + e0
                unsigned used = __reduce_or_sync(0xffffffffu, c ? ((1u << sf) | (1u << sb)) : 0u);
                while (used) {
                    const int f = __ffs(used) - 1;
                    used &= used - 1;
                    const float v = c ? (f == sf ? -gs : (f == sb ? gs : 0.f)) : 0.f;
                    const float ga = warp_sum(v * lxc), gb = warp_sum(v * lyc), ge = warp_sum(v);
                    if (lane == 0) {
                        atomicAdd(A + 3 * f + 0, ga);
                        atomicAdd(A + 3 * f + 1, gb);
                        atomicAdd(A + 3 * f + 2, ge);
                    }
                }
            }
        }
        __syncthreads();
    }
}

template <int V, int BATCH>
cudaError_t fwd_t(const BlendArgs& a, cudaStream_t st) {
    if (a.count)
        k_blend_fwd<V, BATCH, true><<<a.grid, kThreads, 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl,
            a.tile_counter, a.pair_counts);
    else
        k_blend_fwd<V, BATCH, false><<<a.grid, kThreads, 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl,
            a.tile_counter, a.pair_counts);
    return cudaGetLastError();
}

template <int V, int BATCH>
cudaError_t bwd_t(const BlendArgs& a, cudaStream_t st) {
    k_blend_bwd<V, BATCH><<<a.grid, kThreads, 0, st>>>(a.rec, a.vals, a.ranges, *a.cams, a.bg[0],
                                                       a.bg[1], a.bg[2], a.dimage, a.last, a.tl,
                                                       a.acc, a.tile_counter);
    return cudaGetLastError();
}

}  // namespace

#define LP_BATCH_DISPATCH(FN, V, B, A, ST)                                   \
    switch (B) {                                                             \
        case 32: return V == 6 ? FN<6, 32>(A, ST) : FN<4, 32>(A, ST);         \
        case 128: return V == 6 ? FN<6, 128>(A, ST) : FN<4, 128>(A, ST);      \
        case 256: return V == 6 ? FN<6, 256>(A, ST) : FN<4, 256>(A, ST);      \
        default: return V == 6 ? FN<6, 64>(A, ST) : FN<4, 64>(A, ST);         \
    }

cudaError_t launch_blend_fwd(int V, int batch, const BlendArgs& a, cudaStream_t st) {
    LP_BATCH_DISPATCH(fwd_t, V, batch, a, st)
}

cudaError_t launch_blend_bwd(int V, int batch, const BlendArgs& a, cudaStream_t st) {
    LP_BATCH_DISPATCH(bwd_t, V, batch, a, st)
}

}  // namespace lp
