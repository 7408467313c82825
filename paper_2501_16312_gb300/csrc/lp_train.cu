// Optimisation-step kernels (sm_103a): the paper's primitive parameter layer,
// the L1 image-loss gradient and a fused Adam update.
//
// Sec. 3.1: a primitive is stored as its centre c, a rotation quaternion
// q = (w, x, y, z), per-corner distances and an opacity logit; its vertices
// are c +- d_i R(q) e_i (octahedron, opposite vertices share a distance) or
// c + d_k R(q) b_k over the four regular-tetrahedron directions b_k, and
// alpha = sigmoid(logit).  Distances are used as given (linear), as the paper
// scales their learning rate by the scene extent (App. "Experimental
// Setting").  Sec. 3.4: gradients flow back through the rotation into the
// quaternion and distances ("the gradient flow w.r.t. the corners splits when
// undoing the rotation"); for an octahedron the two vertices of an axis enter
// with opposite signs.  Sec. 3.4 uses Adam.
#include <cuda_runtime.h>

#include <cstdint>

#include <cmath>

#include "linprim.h"
#include "lp_device.cuh"
#include "lp_internal.h"

namespace lp {

namespace {

__device__ __forceinline__ void quat_rot(const float q[4], float R[3][3], float& norm) {
    norm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float in = 1.f / norm;
    const float w = q[0] * in, x = q[1] * in, y = q[2] * in, z = q[3] * in;
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// Local direction of vertex k, the distance it uses and its sign.
template <int V>
__device__ __forceinline__ void local_dir(int k, float e[3], int& di, float& sgn) {
    if (V == 6) {
        e[0] = e[1] = e[2] = 0.f;
        e[k / 2] = 1.f;
        di = k / 2;
        sgn = (k & 1) ? -1.f : 1.f;
    } else {
        const float r = 0.57735026918962576f;   // 1 / sqrt(3)
        e[0] = (k == 0 || k == 1) ? r : -r;
        e[1] = (k == 0 || k == 2) ? r : -r;
        e[2] = (k == 0 || k == 3) ? r : -r;
        di = k;
        sgn = 1.f;
    }
}

template <int V>
__global__ void __launch_bounds__(256) k_params_fwd(int n, const float* __restrict__ centre,
                                                    const float* __restrict__ quat,
                                                    const float* __restrict__ dist,
                                                    const float* __restrict__ logit,
                                                    float* __restrict__ verts, float* __restrict__ opacity) {
    constexpr int ND = V == 6 ? 3 : 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float q[4], R[3][3], nrm, d[ND], c[3];
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] = quat[4 * (size_t)i + a];
#pragma unroll
    for (int a = 0; a < ND; ++a) d[a] = dist[(size_t)i * ND + a];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = centre[3 * (size_t)i + a];
    quat_rot(q, R, nrm);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        float e[3], sgn;
        int di;
        local_dir<V>(k, e, di, sgn);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float r = R[a][0] * e[0] + R[a][1] * e[1] + R[a][2] * e[2];
            verts[((size_t)i * V + k) * 3 + a] = fmaf(sgn * d[di], r, c[a]);
        }
    }
    opacity[i] = 1.f / (1.f + __expf(-logit[i]));
}

template <int V>
__global__ void __launch_bounds__(256) k_params_bwd(int n, const float* __restrict__ quat,
                                                    const float* __restrict__ dist,
                                                    const float* __restrict__ logit,
                                                    const float* __restrict__ dverts,
                                                    const float* __restrict__ dopacity,
                                                    float* __restrict__ dcentre, float* __restrict__ dquat,
                                                    float* __restrict__ ddist, float* __restrict__ dlogit) {
    constexpr int ND = V == 6 ? 3 : 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float q[4], R[3][3], nrm, d[ND], gd[ND], dR[3][3], gc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 4; ++a) q[a] = quat[4 * (size_t)i + a];
#pragma unroll
    for (int a = 0; a < ND; ++a) { d[a] = dist[(size_t)i * ND + a]; gd[a] = 0.f; }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dR[a][b] = 0.f;
    quat_rot(q, R, nrm);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        float e[3], sgn, g[3];
        int di;
        local_dir<V>(k, e, di, sgn);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g[a] = dverts[((size_t)i * V + k) * 3 + a];
            gc[a] += g[a];
        }
        float r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) r[a] = R[a][0] * e[0] + R[a][1] * e[1] + R[a][2] * e[2];
        gd[di] += sgn * (r[0] * g[0] + r[1] * g[1] + r[2] * g[2]);
        const float s = sgn * d[di];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) dR[a][b] = fmaf(s * g[a], e[b], dR[a][b]);
    }
    // d R(q_hat) / d q_hat, then the normalisation q_hat = q / |q|
    const float in = 1.f / nrm;
    const float w = q[0] * in, x = q[1] * in, y = q[2] * in, z = q[3] * in;
    float g[4];
    g[0] = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    g[1] = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                  z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    g[2] = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                  w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    g[3] = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                  y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float dot = g[0] * w + g[1] * x + g[2] * y + g[3] * z;
    dquat[4 * (size_t)i + 0] = (g[0] - dot * w) * in;
    dquat[4 * (size_t)i + 1] = (g[1] - dot * x) * in;
    dquat[4 * (size_t)i + 2] = (g[2] - dot * y) * in;
    dquat[4 * (size_t)i + 3] = (g[3] - dot * z) * in;
#pragma unroll
    for (int a = 0; a < ND; ++a) ddist[(size_t)i * ND + a] = gd[a];
#pragma unroll
    for (int a = 0; a < 3; ++a) dcentre[3 * (size_t)i + a] += gc[a];
    const float al = 1.f / (1.f + __expf(-logit[i]));
    dlogit[i] = dopacity[i] * al * (1.f - al);
}

// L = mean |image - target|; dL/dimage = sign(image - target) / count.
__global__ void __launch_bounds__(256) k_l1(const float* __restrict__ img, const float* __restrict__ tgt,
                                            long long count, float* __restrict__ grad,
                                            double* __restrict__ loss) {
    const float inv = 1.f / (float)count;
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = img[i] - tgt[i];
        grad[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
        s += fabsf(d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        if (loss) atomicAdd(loss, t / (double)count);
    }
}

struct AdamGroups {
    int n;
    long long offset[LP_ADAM_MAX_GROUPS];
    long long count[LP_ADAM_MAX_GROUPS];
    float lr[LP_ADAM_MAX_GROUPS];
    float lr_final[LP_ADAM_MAX_GROUPS];
    int decay_steps[LP_ADAM_MAX_GROUPS];
    int period[LP_ADAM_MAX_GROUPS];
    int head[LP_ADAM_MAX_GROUPS];
    float lr_tail[LP_ADAM_MAX_GROUPS];
};

// Adam (Kingma & Ba) over every group in one launch.  The step counter lives
// in device memory so that replays of a captured step advance it.
__device__ __forceinline__ float adam_lr(const AdamGroups& G, int k, uint32_t j, int t) {
    if (G.period[k] > 0 && j % (uint32_t)G.period[k] >= (uint32_t)G.head[k]) return G.lr_tail[k];
    if (G.decay_steps[k] > 0) {
        const float f = fminf((float)t / (float)G.decay_steps[k], 1.f);
        return expf((1.f - f) * logf(G.lr[k]) + f * logf(G.lr_final[k]));
    }
    return G.lr[k];
}

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float c1, float c2) {
    m = fmaf(b1, m, (1.f - b1) * g);
    v = fmaf(b2, v, (1.f - b2) * g * g);
    p -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

__device__ __forceinline__ int adam_group_of(const AdamGroups& G, long long i) {
    int k = 0;
    while (k + 1 < G.n && i >= G.offset[k] + G.count[k]) ++k;
    return (i < G.offset[k] || i >= G.offset[k] + G.count[k]) ? -1 : k;   // -1: gap between groups
}

__global__ void __launch_bounds__(256) k_adam(float* __restrict__ p, const float* __restrict__ g,
                                              float* __restrict__ m, float* __restrict__ v, AdamGroups G,
                                              long long total, float b1, float b2, float eps,
                                              const int* __restrict__ step) {
    const int t = *step + 1;
    const float c1 = 1.f / (1.f - powf(b1, (float)t));
    const float c2 = 1.f / (1.f - powf(b2, (float)t));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = adam_group_of(G, i);
        if (k < 0) continue;
        const float lr = adam_lr(G, k, (uint32_t)(i - G.offset[k]), t);
        float pi = p[i], mi = m[i], vi = v[i];
        adam_one(pi, g[i], mi, vi, lr, b1, b2, eps, c1, c2);
        p[i] = pi;
        m[i] = mi;
        v[i] = vi;
    }
}

// Same update, four elements per thread with 16-byte accesses; used when the
// arrays are 16-byte aligned and every group's offset and count are
// multiples of 4 (so a vector never straddles two groups).
__global__ void __launch_bounds__(256) k_adam4(float4* __restrict__ p, const float4* __restrict__ g,
                                               float4* __restrict__ m, float4* __restrict__ v, AdamGroups G,
                                               long long total4, float b1, float b2, float eps,
                                               const int* __restrict__ step) {
    const int t = *step + 1;
    const float c1 = 1.f / (1.f - powf(b1, (float)t));
    const float c2 = 1.f / (1.f - powf(b2, (float)t));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total4;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = adam_group_of(G, 4 * i);
        if (k < 0) continue;
        const uint32_t j = (uint32_t)(4 * i - G.offset[k]);
        float4 pp = p[i], mm = m[i], vv = v[i];
        const float4 gg = g[i];
        adam_one(pp.x, gg.x, mm.x, vv.x, adam_lr(G, k, j, t), b1, b2, eps, c1, c2);
        adam_one(pp.y, gg.y, mm.y, vv.y, adam_lr(G, k, j + 1, t), b1, b2, eps, c1, c2);
        adam_one(pp.z, gg.z, mm.z, vv.z, adam_lr(G, k, j + 2, t), b1, b2, eps, c1, c2);
        adam_one(pp.w, gg.w, mm.w, vv.w, adam_lr(G, k, j + 3, t), b1, b2, eps, c1, c2);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

__global__ void k_increment(int* step) { *step += 1; }

// ---------------------------------------------------------------- population
// Sec. 3.4 "Adaptive Population Control" with App. "Experimental Setting"'s
// thresholds.  A decision pass writes each primitive's action and output
// count, an exclusive scan turns the counts into destination rows, and an
// apply pass compacts every array set into the new population.

constexpr uint8_t kPrune = LP_POP_PRUNE, kKeep = LP_POP_KEEP, kClone = LP_POP_CLONE, kSplit = LP_POP_SPLIT;

struct PopRules {
    float logit_min, max_scene_frac, clone_scene_frac, extent, thr;
    uint32_t max_px;
};

// Sec. 3.4's size: an octahedron's longest axis, twice its largest distance;
// a tetrahedron's sqrt(2) times the distance to its furthest corner.
template <int V>
__global__ void __launch_bounds__(256) k_pop_decide(int n, const float* __restrict__ dist,
                                                    const float* __restrict__ logit,
                                                    const float* __restrict__ gsum,
                                                    const uint32_t* __restrict__ gcount,
                                                    const uint32_t* __restrict__ pxmax, PopRules R,
                                                    uint8_t* __restrict__ action, uint32_t* __restrict__ outc) {
    constexpr int ND = V == 6 ? 3 : 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float m = 0.f;
#pragma unroll
    for (int a = 0; a < ND; ++a) m = fmaxf(m, fabsf(dist[(size_t)i * ND + a]));
    const float size = __fmul_rn(V == 6 ? 2.f : 1.41421356f, m);
    uint8_t act;
    if (logit[i] < R.logit_min || size > __fmul_rn(R.max_scene_frac, R.extent) || pxmax[i] > R.max_px) {
        act = kPrune;
    } else {
        const uint32_t c = gcount[i];
        const float g = c > 0 ? __fdiv_rn(gsum[i], (float)c) : 0.f;
        act = g > R.thr ? (size < __fmul_rn(R.clone_scene_frac, R.extent) ? kClone : kSplit) : kKeep;
    }
    action[i] = act;
    outc[i] = act == kPrune ? 0u : (act == kKeep ? 1u : 2u);
}

// One (array set, field) pair of the apply pass: `width` floats per row.
// kind 0: parameters copied to both children; 1: distances, divided by 1.2
// for split children; 2: optimiser state, zero for new rows; 3: the centre
// parameter (written by k_pop_centre instead).
struct PopJob {
    const float* src;
    float* dst;
    int width;
    int kind;
};
constexpr int kPopMaxJobs = 20;   // 4 sets x 5 fields
struct PopJobs {
    PopJob job[kPopMaxJobs];
};

// Each thread takes kPopUnroll elements a block apart and issues all their
// loads before any store, so that enough bytes are in flight to cover HBM
// latency (one dependent load chain per thread measured 1-2 TB/s).
constexpr int kPopUnroll = 8;

template <int W, typename I>
__device__ __forceinline__ void pop_job(I total, const uint8_t* __restrict__ action,
                                        const uint32_t* __restrict__ dest, const PopJob& jb) {
    const float* __restrict__ src = jb.src;
    float* __restrict__ dst = jb.dst;
    const I step = (I)blockDim.x;
    const I stride = (I)gridDim.x * blockDim.x * kPopUnroll;
    for (I base = (I)blockIdx.x * blockDim.x * kPopUnroll + threadIdx.x; base < total; base += stride) {
        uint8_t act[kPopUnroll];
        size_t o[kPopUnroll];
        float v[kPopUnroll];
#pragma unroll
        for (int u = 0; u < kPopUnroll; ++u) {
            const I e = base + (I)u * step;
            act[u] = kPrune;
            o[u] = 0;
            if (e < total) {
                const I i = e / W;   // a division by a constant
                act[u] = action[i];
                o[u] = (size_t)dest[i] * W + (size_t)(e - i * W);
            }
        }
#pragma unroll
        for (int u = 0; u < kPopUnroll; ++u) v[u] = act[u] != kPrune ? src[base + (I)u * step] : 0.f;
#pragma unroll
        for (int u = 0; u < kPopUnroll; ++u) {
            if (act[u] == kPrune) continue;
            if (act[u] == kKeep) {
                dst[o[u]] = v[u];
            } else if (act[u] == kClone) {
                dst[o[u]] = v[u];
                dst[o[u] + W] = jb.kind == 2 ? 0.f : v[u];
            } else {
                const float c = jb.kind == 2 ? 0.f : (jb.kind == 1 ? __fdiv_rn(v[u], 1.2f) : v[u]);
                dst[o[u]] = c;
                dst[o[u] + W] = c;
            }
        }
    }
}

template <int W>
__device__ __forceinline__ void pop_job_any(int n, const uint8_t* __restrict__ action,
                                            const uint32_t* __restrict__ dest, const PopJob& jb) {
    const unsigned long long total = (unsigned long long)n * W;
    // 32-bit indexing whenever the padded index range fits
    if (total + (unsigned long long)gridDim.x * blockDim.x * kPopUnroll < 0xffffffffull)
        pop_job<W, uint32_t>((uint32_t)total, action, dest, jb);
    else
        pop_job<W, unsigned long long>(total, action, dest, jb);
}

__global__ void __launch_bounds__(256) k_pop_apply(int n, const uint8_t* __restrict__ action,
                                                   const uint32_t* __restrict__ dest, PopJobs J) {
    const PopJob jb = J.job[blockIdx.y];
    if (jb.kind == 3) return;
    switch (jb.width) {   // the widths of the parameter arrays: 1, 3, 4 and 3 K
        case 1: pop_job_any<1>(n, action, dest, jb); break;
        case 3: pop_job_any<3>(n, action, dest, jb); break;
        case 4: pop_job_any<4>(n, action, dest, jb); break;
        case 12: pop_job_any<12>(n, action, dest, jb); break;
        case 27: pop_job_any<27>(n, action, dest, jb); break;
        default: pop_job_any<48>(n, action, dest, jb); break;
    }
}

// Split children's centres: c + R(q) (|d| * z) for an octahedron (standard
// deviations equal to the distances along the rotated axes), c + (max|d| / 2) z
// for a tetrahedron; kept and cloned rows copy the centre.
template <int V>
__global__ void __launch_bounds__(256) k_pop_centre(int n, const uint8_t* __restrict__ action,
                                                    const uint32_t* __restrict__ dest,
                                                    const float* __restrict__ centre,
                                                    const float* __restrict__ quat,
                                                    const float* __restrict__ dist,
                                                    const float* __restrict__ normals,
                                                    float* __restrict__ out) {
    constexpr int ND = V == 6 ? 3 : 4;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t act = action[i];
    if (act == kPrune) return;
    const size_t o = dest[i];
    float c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = centre[3 * (size_t)i + a];
    if (act != kSplit) {
#pragma unroll
        for (int r = 0; r < (act == kClone ? 2 : 1); ++r)
#pragma unroll
            for (int a = 0; a < 3; ++a) out[3 * (o + r) + a] = c[a];
        return;
    }
    float d[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) d[a] = fabsf(dist[(size_t)i * ND + a]);
    float R[3][3], nrm;
    if (V == 6) {
        float q[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) q[a] = quat[4 * (size_t)i + a];
        quat_rot(q, R, nrm);
    }
#pragma unroll
    for (int ch = 0; ch < 2; ++ch) {
        const float* z = normals + ((size_t)i * 2 + ch) * 3;
        float off[3];
        if (V == 6) {
            const float s0 = d[0] * z[0], s1 = d[1] * z[1], s2 = d[2] * z[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) off[a] = R[a][0] * s0 + R[a][1] * s1 + R[a][2] * s2;
        } else {
            float m = 0.f;
#pragma unroll
            for (int a = 0; a < ND; ++a) m = fmaxf(m, d[a]);
#pragma unroll
            for (int a = 0; a < 3; ++a) off[a] = 0.5f * m * z[a];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) out[3 * (o + ch) + a] = c[a] + off[a];
    }
}

int grid_for(long long n, int bs, int cap) {
    const long long g = (n + bs - 1) / bs;
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

}  // namespace

}  // namespace lp

extern "C" {

lp_status lp_params_forward(int kind, int n, const float* centre, const float* quat, const float* dist,
                            const float* logit, float* verts, float* opacity, void* stream) {
    if ((kind != LP_OCTAHEDRON && kind != LP_TETRAHEDRON) || n < 0) return LP_ERR_INVALID;
    if (n == 0) return LP_OK;
    if (!centre || !quat || !dist || !logit || !verts || !opacity) return LP_ERR_INVALID;
    const int grid = (n + 255) / 256;
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == LP_OCTAHEDRON)
        lp::k_params_fwd<6><<<grid, 256, 0, st>>>(n, centre, quat, dist, logit, verts, opacity);
    else
        lp::k_params_fwd<4><<<grid, 256, 0, st>>>(n, centre, quat, dist, logit, verts, opacity);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_params_backward(int kind, int n, const float* quat, const float* dist, const float* logit,
                             const float* dverts, const float* dopacity, float* dcentre, float* dquat,
                             float* ddist, float* dlogit, void* stream) {
    if ((kind != LP_OCTAHEDRON && kind != LP_TETRAHEDRON) || n < 0) return LP_ERR_INVALID;
    if (n == 0) return LP_OK;
    if (!quat || !dist || !logit || !dverts || !dopacity || !dcentre || !dquat || !ddist || !dlogit)
        return LP_ERR_INVALID;
    const int grid = (n + 255) / 256;
    cudaStream_t st = (cudaStream_t)stream;
    if (kind == LP_OCTAHEDRON)
        lp::k_params_bwd<6><<<grid, 256, 0, st>>>(n, quat, dist, logit, dverts, dopacity, dcentre, dquat,
                                                  ddist, dlogit);
    else
        lp::k_params_bwd<4><<<grid, 256, 0, st>>>(n, quat, dist, logit, dverts, dopacity, dcentre, dquat,
                                                  ddist, dlogit);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_l1_loss_grad(const float* image, const float* target, long long count, float* grad,
                          double* loss, void* stream) {
    if (count < 0 || (count > 0 && (!image || !target || !grad))) return LP_ERR_INVALID;
    if (count == 0) return LP_OK;
    lp::k_l1<<<lp::grid_for(count, 256, 4096), 256, 0, (cudaStream_t)stream>>>(image, target, count, grad,
                                                                               loss);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_adam_step(float* params, const float* grads, float* m, float* v, const lp_adam_group* groups,
                       int n_groups, float beta1, float beta2, float eps, int* step, void* stream) {
    if (!params || !grads || !m || !v || !groups || !step) return LP_ERR_INVALID;
    if (n_groups < 1 || n_groups > LP_ADAM_MAX_GROUPS) return LP_ERR_INVALID;
    lp::AdamGroups G;
    G.n = n_groups;
    long long total = 0;
    for (int k = 0; k < n_groups; ++k) {
        if (groups[k].offset < 0 || groups[k].count < 0 || groups[k].count > 0xffffffffll) return LP_ERR_INVALID;
        if (k > 0 && groups[k].offset < groups[k - 1].offset + groups[k - 1].count) return LP_ERR_INVALID;
        G.offset[k] = groups[k].offset;
        G.count[k] = groups[k].count;
        G.lr[k] = groups[k].lr;
        if (groups[k].period < 0 || groups[k].head < 0 || groups[k].decay_steps < 0) return LP_ERR_INVALID;
        if (groups[k].decay_steps > 0 && !(groups[k].lr > 0.f && groups[k].lr_final > 0.f)) return LP_ERR_INVALID;
        G.lr_final[k] = groups[k].lr_final;
        G.decay_steps[k] = groups[k].decay_steps;
        G.period[k] = groups[k].period;
        G.head[k] = groups[k].head;
        G.lr_tail[k] = groups[k].lr_tail;
        total = groups[k].offset + groups[k].count;
    }
    cudaStream_t st = (cudaStream_t)stream;
    bool vec = ((uintptr_t)params | (uintptr_t)grads | (uintptr_t)m | (uintptr_t)v) % 16 == 0;
    for (int k = 0; k < n_groups; ++k) vec = vec && groups[k].offset % 4 == 0 && groups[k].count % 4 == 0;
    if (total > 0 && vec)
        lp::k_adam4<<<lp::grid_for(total / 4, 256, 152 * 8), 256, 0, st>>>(
            reinterpret_cast<float4*>(params), reinterpret_cast<const float4*>(grads), reinterpret_cast<float4*>(m),
            reinterpret_cast<float4*>(v), G, total / 4, beta1, beta2, eps, step);
    else if (total > 0)
        lp::k_adam<<<lp::grid_for(total, 256, 152 * 16), 256, 0, st>>>(params, grads, m, v, G, total, beta1,
                                                                      beta2, eps, step);
    lp::k_increment<<<1, 1, 0, st>>>(step);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

long long lp_population_scratch(long long n) {
    if (n < 0) return 0;
    return ((n + 3) / 4) * 4 + lp::scan_blocks(n) + 4;
}

lp_status lp_population_decide(int kind, int n, const float* dist, const float* logit, const float* grad_sum,
                               const unsigned int* grad_count, const unsigned int* px_max,
                               const lp_population_rules* rules, unsigned char* action, unsigned int* dest,
                               unsigned int* n_out, unsigned int* scratch, void* stream) {
    if ((kind != LP_OCTAHEDRON && kind != LP_TETRAHEDRON) || n < 0 || !rules || !n_out) return LP_ERR_INVALID;
    const lp_population_rules& r = *rules;
    auto pos = [](float x) { return x > 0.f && std::isfinite(x); };
    if (!pos(r.scene_extent) || !(r.min_opacity > 0.f && r.min_opacity < 1.f) || !pos(r.max_scene_frac) ||
        !pos(r.grad_threshold) || !pos(r.clone_scene_frac))
        return LP_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(n_out, 0, sizeof(unsigned int), st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
    if (!dist || !logit || !grad_sum || !grad_count || !px_max || !action || !dest || !scratch)
        return LP_ERR_INVALID;
    lp::PopRules R;
    const double p = r.min_opacity;
    R.logit_min = (float)std::log(p / (1.0 - p));   // sigmoid(logit) < p
    R.max_scene_frac = r.max_scene_frac;
    R.clone_scene_frac = r.clone_scene_frac;
    R.extent = r.scene_extent;
    R.thr = r.grad_threshold;
    R.max_px = r.max_pixels;
    uint32_t* outc = scratch;
    uint32_t* sums = scratch + ((n + 3) / 4) * 4;
    const int grid = (n + 255) / 256;
    if (kind == LP_OCTAHEDRON)
        lp::k_pop_decide<6><<<grid, 256, 0, st>>>(n, dist, logit, grad_sum, grad_count, px_max, R, action, outc);
    else
        lp::k_pop_decide<4><<<grid, 256, 0, st>>>(n, dist, logit, grad_sum, grad_count, px_max, R, action, outc);
    if (cudaGetLastError() != cudaSuccess) return LP_ERR_CUDA;
    return lp::launch_scan(outc, n, dest, sums, n_out, st) == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

lp_status lp_population_apply(int kind, int sh_coeffs, int n, const unsigned char* action,
                              const unsigned int* dest, const float* normals, const lp_param_arrays* src,
                              const lp_param_arrays* dst, int n_sets, void* stream) {
    if ((kind != LP_OCTAHEDRON && kind != LP_TETRAHEDRON) || n < 0) return LP_ERR_INVALID;
    if (!(sh_coeffs == 1 || sh_coeffs == 4 || sh_coeffs == 9 || sh_coeffs == 16)) return LP_ERR_INVALID;
    if (n_sets < 1 || n_sets > 4 || !src || !dst) return LP_ERR_INVALID;
    if (n == 0) return LP_OK;
    if (!action || !dest || !normals) return LP_ERR_INVALID;
    const int D = kind == LP_OCTAHEDRON ? 3 : 4;
    lp::PopJobs J;
    int nj = 0;
    for (int s = 0; s < n_sets; ++s) {
        const float* sp[5] = {src[s].centre, src[s].quat, src[s].dist, src[s].logit, src[s].sh};
        float* dp[5] = {dst[s].centre, dst[s].quat, dst[s].dist, dst[s].logit, dst[s].sh};
        const int w[5] = {3, 4, D, 1, 3 * sh_coeffs};
        for (int f = 0; f < 5; ++f) {
            if (!sp[f] || !dp[f]) return LP_ERR_INVALID;
            J.job[nj].src = sp[f];
            J.job[nj].dst = dp[f];
            J.job[nj].width = w[f];
            J.job[nj].kind = s > 0 ? 2 : (f == 0 ? 3 : (f == 2 ? 1 : 0));
            ++nj;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const long long widest = (long long)n * 3 * sh_coeffs > 4ll * n ? (long long)n * 3 * sh_coeffs : 4ll * n;
    dim3 grid(lp::grid_for((widest + lp::kPopUnroll - 1) / lp::kPopUnroll, 256, 152 * 8), nj);
    lp::k_pop_apply<<<grid, 256, 0, st>>>(n, action, dest, J);
    const int g1 = (n + 255) / 256;
    if (kind == LP_OCTAHEDRON)
        lp::k_pop_centre<6><<<g1, 256, 0, st>>>(n, action, dest, src[0].centre, src[0].quat, src[0].dist, normals,
                                                dst[0].centre);
    else
        lp::k_pop_centre<4><<<g1, 256, 0, st>>>(n, action, dest, src[0].centre, src[0].quat, src[0].dist, normals,
                                                dst[0].centre);
    return cudaGetLastError() == cudaSuccess ? LP_OK : LP_ERR_CUDA;
}

}  // extern "C"
