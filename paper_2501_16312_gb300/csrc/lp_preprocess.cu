// Per-primitive preprocess (forward) and its backward chain (sm_103a).
//
// Forward, Sec. 3.2 "Preprocessing": transform the centre and vertices to
// camera space, map the vertices into the EWA 3D affine ray space linearised
// at the centre (App. "Ray Space Approximation"), build the faces' ray-space
// planes, evaluate Eq. 1's density and the view-dependent SH colour, and
// bound the projection by a pixel/tile rectangle.
//
// Backward, Sec. 3.4 "Preprocessing Backpropagation": chain the per-face
// plane, colour and density gradients collected by the backward blend through
// the plane construction, the ray-space map and the view transform to the
// world-space centre and vertices, the SH coefficients and the opacity.
//
// One thread per primitive; the thread loops over the cameras so that each
// primitive's inputs are read from HBM once per call.
#include "lp_device.cuh"
#include "lp_geom.cuh"
#include "lp_internal.h"

namespace lp {

namespace {

// A 16-byte load the compiler keeps where it is written (inside a camera
// loop), so that a loop-invariant input is re-read from L1 instead of held in
// registers across the loop.
__device__ __forceinline__ float4 ld4_each(const float* p) {
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_each(const float* p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

template <int V, int DEG>
__global__ void __launch_bounds__(128, 4) k_preprocess(PrimsDev P, CamsParam cams, float* __restrict__ rec,
                                                    uint32_t* __restrict__ counts,
                                                    int4* __restrict__ trect,
                                                    uint32_t* __restrict__ zbits,
                                                    uint32_t* __restrict__ meta_out) {
    constexpr int F = Kind<V>::F;
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;

    float c[3], v[V][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = __ldg(P.centre + 3 * (size_t)i + a);
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) v[k][a] = __ldg(P.verts + ((size_t)i * V + k) * 3 + a);
    const float alpha = __ldg(P.opacity + i);
    float sh[K * 3];
#pragma unroll
    for (int q = 0; q < K * 3; ++q) sh[q] = __ldg(P.sh + (size_t)i * K * 3 + q);

    // Eq. 1: sigma = -log(1 - 0.99 alpha) / (2 d_min), d_min the smallest
    // centre-vertex distance (for an octahedron min(d_x, d_y, d_z)).
    float dmin = CUDART_INF_F;
    bool degenerate = false;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float dx = v[k][0] - c[0], dy = v[k][1] - c[1], dz = v[k][2] - c[2];
        dmin = fminf(dmin, sqrtf(dx * dx + dy * dy + dz * dz));
        degenerate |= dx == 0.f && dy == 0.f && dz == 0.f;
    }
    const float sigma = -log1pf(-kAlphaScale * alpha) / (2.f * dmin);
    // A vertex on the centre leaves Eq. 1 without a density: not visible.  The
    // second test only catches offsets so small (below ~1e-19) that d_min
    // underflows in binary32, and a non-finite opacity.
    degenerate |= !(sigma < CUDART_INF_F);
    uint32_t px_side = 0;   // largest pixel-rectangle side over the views
    // The record is assembled in shared memory, where the face planes go to
    // their slots by computed address, then copied out in 16-byte stores.  A
    // thread's row is padded by 16 bytes so that rows start on distinct banks.
    constexpr int kRow = Rec<V>::kVec4 + 1;
    __shared__ float4 srec[128 * kRow];
    float* o = reinterpret_cast<float*>(srec + threadIdx.x * kRow);

    for (int cv = 0; cv < cams.n; ++cv) {
        const CamDev& cm = cams.cam[cv];
        const size_t r = (size_t)cv * P.n + i;
        Geom g;
        const bool vis = centre_geom(cm, c, g) && !degenerate;
        zbits[r] = __float_as_uint(g.tc[2]);
        if (!vis) {
            counts[r] = 0;
            trect[r] = make_int4(0, 0, 0, 0);
            continue;
        }
        float q[V][3];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float d[3];
            vertex_local(cm, g, v[k], c, q[k], d);
        }
        aa_widen<V>(cams, q);
        float qxmin = CUDART_INF_F, qxmax = -CUDART_INF_F, qymin = CUDART_INF_F, qymax = -CUDART_INF_F;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            qxmin = fminf(qxmin, q[k][0]); qxmax = fmaxf(qxmax, q[k][0]);
            qymin = fminf(qymin, q[k][1]); qymax = fmaxf(qymax, q[k][1]);
        }
        // Pixel p is covered when its centre p + 0.5 lies in the projected box.
        float fx0 = ceilf(__fsub_rn(__fadd_rn(g.xc, qxmin), 0.5f));
        float fx1 = floorf(__fsub_rn(__fadd_rn(g.xc, qxmax), 0.5f));
        float fy0 = ceilf(__fsub_rn(__fadd_rn(g.yc, qymin), 0.5f));
        float fy1 = floorf(__fsub_rn(__fadd_rn(g.yc, qymax), 0.5f));
        fx0 = fmaxf(fx0, 0.f); fx1 = fminf(fx1, (float)(cm.width - 1));
        fy0 = fmaxf(fy0, 0.f); fy1 = fminf(fy1, (float)(cm.height - 1));
        if (fx0 > fx1 || fy0 > fy1) {
            counts[r] = 0;
            trect[r] = make_int4(0, 0, 0, 0);
            continue;
        }
        const int T = cams.tile;
        const int tx0 = (int)fx0 / T, tx1 = (int)fx1 / T, ty0 = (int)fy0 / T, ty1 = (int)fy1 / T;
        px_side = max(px_side, (uint32_t)max((int)fx1 - (int)fx0 + 1, (int)fy1 - (int)fy0 + 1));
        counts[r] = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
        // global id of the rectangle's first tile, row stride, width, height
        trect[r] = make_int4(cm.tile_base + ty0 * cm.tiles_x + tx0, cm.tiles_x, tx1 - tx0 + 1, ty1 - ty0 + 1);

        // Face planes in the local frame (origin at the ray-space centre,
        // which lies inside the primitive): outward normal n, entry face iff
        // n_z < 0; depth - z_c = a x + b y + e with a = -n_x/n_z, b = -n_y/n_z,
        // e = (n . q0) / n_z.
        int nf = 0;
        float pl[F][3];
        bool front[F];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            int i0, i1, i2;
            face_vertices<V>(f, i0, i1, i2);
            float n[3];
            face_normal(q[i0], q[i1], q[i2], n);
            const float h = n[0] * q[i0][0] + n[1] * q[i0][1] + n[2] * q[i0][2];
            const float sgn = h < 0.f ? -1.f : 1.f;
            n[0] *= sgn; n[1] *= sgn; n[2] *= sgn;
            float nz = n[2];
            if (plane_degenerate(n)) {
                const float m = kEdgeOn * (fabsf(n[0]) + fabsf(n[1]));
                nz = (n[2] < 0.f) ? -fmaxf(m, 1e-37f) : fmaxf(m, 1e-37f);
            }
            const float inz = 1.f / nz;
            pl[f][0] = -n[0] * inz;
            pl[f][1] = -n[1] * inz;
            pl[f][2] = (n[0] * q[i0][0] + n[1] * q[i0][1] + n[2] * q[i0][2]) * inz;
            front[f] = nz < 0.f;
            nf += front[f] ? 1 : 0;
        }
        // re-anchor to pixel (X0, Y0): e0 = e - a fxo - b fyo
        uint32_t meta = (uint32_t)nf;
        int sf = 0, sb = nf;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int s = front[f] ? sf++ : sb++;
            meta |= (uint32_t)f << (4 + 3 * s);
            o[8 + 3 * s] = pl[f][0];
            o[9 + 3 * s] = pl[f][1];
            o[10 + 3 * s] = __fmaf_rn(-pl[f][0], g.fxo, __fmaf_rn(-pl[f][1], g.fyo, pl[f][2]));
        }

        // Colour: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5), dir from the camera
        // to the centre (3DGS convention, Sec. 3.1).
        float dir[3] = {c[0] - cm.campos[0], c[1] - cm.campos[1], c[2] - cm.campos[2]};
        const float idl = rsqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        dir[0] *= idl; dir[1] *= idl; dir[2] *= idl;
        float Y[16];
        sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
        float rgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], sh[3 * k + ch], s);
            rgb[ch] = fmaxf(s, 0.f);
        }
        srec[threadIdx.x * kRow] = make_float4(__int_as_float(g.X0), __int_as_float(g.Y0), sigma,
                                               __uint_as_float(meta));
        if (meta_out) meta_out[r] = meta;   // the chain reads the face order densely
        // rgb, then the ray-space depth of the centre (the planes are relative to it)
        srec[threadIdx.x * kRow + 1] = make_float4(rgb[0], rgb[1], rgb[2], g.len);
        float4* dst = reinterpret_cast<float4*>(rec + r * Rec<V>::kFloats);
#pragma unroll
        for (int k = 0; k < Rec<V>::kVec4; ++k) dst[k] = srec[threadIdx.x * kRow + k];
    }
    if (P.px_max && px_side > P.px_max[i]) P.px_max[i] = px_side;   // one thread per primitive
}

// ------------------------------------------------------------------ backward
// PART 0: the geometry (planes -> vertices, centre anchor, density); PART 1:
// the colour (SH coefficients and the view direction's centre term); PART 2:
// both in one pass (always used when the view-space statistics are
// gathered, which need both parts per view).  The split form lowers the
// registers a thread holds (the SH coefficients and their gradients live
// only in PART 1), which pays where many cameras make the loop long.  The
// geometry pass is held to four resident blocks per SM (128 registers), the
// colour pass, which holds 48 SH gradients, to four for octahedra (a few
// spills, measured faster) and three for tetrahedra: the loop waits on
// memory once per camera, and the resident warps hide it.
template <int V, int DEG, int PART>
__global__ void __launch_bounds__(128, PART == 2 ? 1 : (PART == 1 ? (V == 6 ? 4 : 3) : 4))
k_chain(PrimsDev P, CamsParam cams, const uint32_t* __restrict__ meta_in, const uint32_t* __restrict__ counts,
        const float* __restrict__ acc, float* __restrict__ dcentre, float* __restrict__ dverts,
        float* __restrict__ dopacity, float* __restrict__ dsh, int accumulate) {
    constexpr int F = Kind<V>::F;
    constexpr int K = (DEG + 1) * (DEG + 1);
    constexpr int KP = Acc<V>::kPlane;
    const float* acc_col = acc + (size_t)cams.n * P.n * KP;   // the colour block follows the planes
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n) return;

    float c[3], v[V][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) c[a] = __ldg(P.centre + 3 * (size_t)i + a);
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) v[k][a] = __ldg(P.verts + ((size_t)i * V + k) * 3 + a);
    const float alpha = __ldg(P.opacity + i);
    // The colour passes re-read the SH coefficients per camera (L1 hits;
    // 16-byte loads when a row is a multiple of 16 bytes and the array is
    // 16-byte aligned), which leaves the registers to the gradients; other
    // rows are held in registers, loaded once.  PART 1 stores its gradients
    // 16 bytes at a time on the same condition.
    constexpr bool kVecSH = PART != 0 && (K * 3) % 4 == 0;
    constexpr bool kRow4 = (K * 3) % 4 == 0;
    const bool sh_aligned = ((uintptr_t)P.sh & 15u) == 0;
    const bool dsh_aligned = ((uintptr_t)dsh & 15u) == 0;
    constexpr int kRegSH = PART != 0 && !kVecSH ? K * 3 : 1;
    float sh_reg[kRegSH];
    if constexpr (kRegSH > 1) {
        if (kRow4 && sh_aligned) {
            const float4* s4 = reinterpret_cast<const float4*>(P.sh + (size_t)i * K * 3);
#pragma unroll
            for (int q = 0; q < (kRow4 ? K * 3 / 4 : 1); ++q) {
                const float4 t = __ldg(s4 + q);
                sh_reg[4 * q] = t.x; sh_reg[4 * q + 1] = t.y; sh_reg[4 * q + 2] = t.z; sh_reg[4 * q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < K * 3; ++q) sh_reg[q] = __ldg(P.sh + (size_t)i * K * 3 + q);
        }
    }
    const float* shp = P.sh + (size_t)i * K * 3;
    float dmin = CUDART_INF_F;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float dx = v[k][0] - c[0], dy = v[k][1] - c[1], dz = v[k][2] - c[2];
        dmin = fminf(dmin, sqrtf(dx * dx + dy * dy + dz * dz));
    }

    float gc[3] = {0.f, 0.f, 0.f};
    float gv[V][3];
#pragma unroll
    for (int k = 0; k < V; ++k) gv[k][0] = gv[k][1] = gv[k][2] = 0.f;
    float gsh[PART != 0 ? K * 3 : 1];
    if constexpr (PART != 0) {
#pragma unroll
        for (int q = 0; q < K * 3; ++q) gsh[q] = 0.f;
    }
    float gsigma = 0.f;
    float vg_sum = 0.f;     // view-space position-gradient norms of the visible views

    // The cameras that see the primitive: all tile counts are read up front
    // (independent loads, in flight together), so a visible camera then costs
    // one dependent memory round trip, for its accumulator row.
    uint32_t vis = 0;
#pragma unroll 8
    for (int cv = 0; cv < cams.n; ++cv) vis |= (counts[(size_t)cv * P.n + i] != 0u ? 1u : 0u) << cv;
    const uint32_t vg_count = __popc(vis);

    while (vis) {
        const int cv = __ffs(vis) - 1;
        vis &= vis - 1;
        const size_t r = (size_t)cv * P.n + i;
        const CamDev& cm = cams.cam[cv];
        const float* A = acc + r * KP;
        // The geometry reads the record's face order (dense array) with its
        // plane row; its top four bits are always zero, and testing them
        // keeps the load ahead of the branch on the row.  The colour pass
        // reads one 16-byte row.
        const uint32_t meta = PART != 1 ? meta_in[r] : 0u;
        bool any = (meta >> 28) != 0u;
        float4 col = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (PART != 0) {
            col = __ldg(reinterpret_cast<const float4*>(acc_col) + r);
            any |= col.x != 0.f || col.y != 0.f || col.z != 0.f || col.w != 0.f;
        }
        if constexpr (PART != 1) {
#pragma unroll
            for (int q = 0; q < F; ++q) {
                const float4 a = __ldg(reinterpret_cast<const float4*>(A) + q);
                any |= a.x != 0.f || a.y != 0.f || a.z != 0.f;
            }
        }
        if (!any) continue;   // no pixel produced a gradient for this record
        float ga_rgb[3], ga_sig;
        ga_rgb[0] = col.x; ga_rgb[1] = col.y; ga_rgb[2] = col.z;
        ga_sig = col.w;

        Geom g;
        float gtc[3] = {0.f, 0.f, 0.f};
        if constexpr (PART != 1) {
        centre_geom(cm, c, g);
        float q[V][3], d[V][3];
#pragma unroll
        for (int k = 0; k < V; ++k) vertex_local(cm, g, v[k], c, q[k], d[k]);
        aa_widen<V>(cams, q);   // the planes were built on the moved vertices (constant move)

        // planes -> local ray-space vertices q, and the projected centre.
        // Faces are visited in a fixed order; the record's permutation gives
        // the slot whose accumulator holds each face's gradient.
        float gq[V][3];
#pragma unroll
        for (int k = 0; k < V; ++k) gq[k][0] = gq[k][1] = gq[k][2] = 0.f;
        float gxc = 0.f, gyc = 0.f;
        uint32_t slot_of = 0;   // inverse of the record's permutation, 3 bits per face
#pragma unroll
        for (int t = 0; t < F; ++t) slot_of |= (uint32_t)t << (3 * meta_face(meta, t));
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int s = (int)((slot_of >> (3 * f)) & 7u);
            // accumulators hold sums over g (px - X0, py - Y0, 1); the pixel's
            // offset from the projected centre is (px - X0 - fxo, py - Y0 - fyo)
            const float4 a4 = __ldg(reinterpret_cast<const float4*>(A) + s);
            const float Ge = a4.z;
            const float Ga = __fmaf_rn(-g.fxo, Ge, a4.x), Gb = __fmaf_rn(-g.fyo, Ge, a4.y);
            // (a face without gradient is not skipped: its terms are exact
            // zeros, and lanes of a warp then stay together)
            int iv[3];
            face_vertices<V>(f, iv[0], iv[1], iv[2]);
            float n[3];
            face_normal(q[iv[0]], q[iv[1]], q[iv[2]], n);
            if (plane_degenerate(n)) continue;
            const float inz = 1.f / n[2];
            const float a = -n[0] * inz, b = -n[1] * inz;
            // moving the projected centre moves every plane with it
            gxc -= a * Ge;
            gyc -= b * Ge;
            // The plane's depth at pixel p is sum_k lambda_k(p) q_k.z with
            // lambda the face's 2D barycentric coordinates, and moving vertex k
            // by (dx, dy) changes it by -lambda_k (a dx + b dy).  So with
            // G_k = sum_p g lambda_k(p), dL/dq_k = G_k (-a, -b, 1).  lambda_k(p)
            // = cross(q_l - q_j, p - q_j) / n_z for the next two vertices j, l
            // in the face's order, hence G_k = cross(q_l - q_j, (Ga, Gb) -
            // q_j Ge) / n_z: no term is multiplied by the (possibly large)
            // slopes before the cross product, which keeps nearly edge-on
            // faces as accurate as the others.
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                const float* qj = q[iv[(kk + 1) % 3]];
                const float* ql = q[iv[(kk + 2) % 3]];
                const float ex = ql[0] - qj[0], ey = ql[1] - qj[1];
                const float mx = __fmaf_rn(-qj[0], Ge, Ga), my = __fmaf_rn(-qj[1], Ge, Gb);
                const float Gk = (ex * my - ey * mx) * inz;
                float* gk = gq[iv[kk]];
                gk[0] = fmaf(-a, Gk, gk[0]);
                gk[1] = fmaf(-b, Gk, gk[1]);
                gk[2] += Gk;
            }
        }

        // q_k = J (t_k - tc); x_c = phi_x(tc), y_c = phi_y(tc).  The planes
        // depend on tc through the projected centre plus q_k, whose sum
        // phi(tc) + J (t_k - tc) has derivative dJ/dtc (t_k - tc) in tc: the
        // anchor's J and the vertices' -J cancel exactly and are left out of
        // the centre gradient (their binary32 residue would be all error).
        // The densification statistic, a translation of the whole primitive,
        // takes the anchor terms alone.
        float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f, gJ2[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const float gd0 = g.j00 * gq[k][0] + g.j2[0] * gq[k][2];
            const float gd1 = g.j11 * gq[k][1] + g.j2[1] * gq[k][2];
            const float gd2 = g.j02 * gq[k][0] + g.j12 * gq[k][1] + g.j2[2] * gq[k][2];
            gJ00 += gq[k][0] * d[k][0];
            gJ02 += gq[k][0] * d[k][2];
            gJ11 += gq[k][1] * d[k][1];
            gJ12 += gq[k][1] * d[k][2];
            gJ2[0] += gq[k][2] * d[k][0];
            gJ2[1] += gq[k][2] * d[k][1];
            gJ2[2] += gq[k][2] * d[k][2];
            // world vertex: t = R v + T
#pragma unroll
            for (int a = 0; a < 3; ++a)
                gv[k][a] += cm.R[a] * gd0 + cm.R[3 + a] * gd1 + cm.R[6 + a] * gd2;
        }
        const float tx = g.tc[0], ty = g.tc[1], tz = g.tc[2];
        const float itz = 1.f / tz, itz2 = itz * itz;
        // d phi_xy / d tc = J rows 0, 1 (the anchor; statistic only)
        gtc[0] += g.j00 * gxc;
        gtc[1] += g.j11 * gyc;
        gtc[2] += g.j02 * gxc + g.j12 * gyc;
        // d J / d tc
        float gjt[3] = {0.f, 0.f, 0.f};
        gjt[2] += gJ00 * (-cm.fx * itz2);
        gjt[0] += gJ02 * (-cm.fx * itz2);
        gjt[2] += gJ02 * (2.f * cm.fx * tx * itz2 * itz);
        gjt[2] += gJ11 * (-cm.fy * itz2);
        gjt[1] += gJ12 * (-cm.fy * itz2);
        gjt[2] += gJ12 * (2.f * cm.fy * ty * itz2 * itz);
        {
            const float il = 1.f / g.len;
            const float dot = gJ2[0] * g.j2[0] + gJ2[1] * g.j2[1] + gJ2[2] * g.j2[2];
#pragma unroll
            for (int a = 0; a < 3; ++a) gjt[a] += (gJ2[a] - g.j2[a] * dot) * il;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) gtc[a] += gjt[a];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            gc[a] += cm.R[a] * gjt[0] + cm.R[3 + a] * gjt[1] + cm.R[6 + a] * gjt[2];
        }

        if constexpr (PART != 0) {
        // colour -> SH coefficients and view direction
        float dir[3] = {c[0] - cm.campos[0], c[1] - cm.campos[1], c[2] - cm.campos[2]};
        const float dist = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        const float idl = 1.f / dist;
        dir[0] *= idl; dir[1] *= idl; dir[2] *= idl;
        float Y[16];
        sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
        float sh[K * 3];
        if constexpr (kVecSH) {
            if (sh_aligned) {
#pragma unroll
                for (int q = 0; q < K * 3 / 4; ++q) {
                    const float4 t = ld4_each(shp + 4 * q);
                    sh[4 * q] = t.x; sh[4 * q + 1] = t.y; sh[4 * q + 2] = t.z; sh[4 * q + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < K * 3; ++q) sh[q] = ld_each(shp + q);
            }
        } else {
#pragma unroll
            for (int q = 0; q < K * 3; ++q) sh[q] = sh_reg[kRegSH > 1 ? q : 0];
        }
        float grgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], sh[3 * k + ch], s);
            grgb[ch] = s > 0.f ? ga_rgb[ch] : 0.f;
        }
        float w[16];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            w[k] = sh[3 * k] * grgb[0] + sh[3 * k + 1] * grgb[1] + sh[3 * k + 2] * grgb[2];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gsh[3 * k + ch] += Y[k] * grgb[ch];
        }
        float gdir[3];
        sh_basis_vjp<DEG>(dir[0], dir[1], dir[2], w, gdir);
        const float dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        float gw[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gw[a] = (gdir[a] - dir[a] * dd) * idl;
            gc[a] += gw[a];
        }
        if constexpr (PART == 2) {
            if (P.grad_sum) {
                // translating the whole primitive leaves t_k - tc unchanged:
                // its camera-space gradient is the anchor terms plus the colour's
                float gt[3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    gt[a] = gtc[a] + cm.R[3 * a] * gw[0] + cm.R[3 * a + 1] * gw[1] + cm.R[3 * a + 2] * gw[2];
                vg_sum += ndc_grad_norm(cm, gt, g.tc[2]);
            }
        }
        }

        if constexpr (PART != 0) gsigma += ga_sig;
    }
    if (P.grad_sum) {
        P.grad_sum[i] += vg_sum;
        P.grad_count[i] += vg_count;
    }

    // Eq. 1 with d_min frozen: d sigma / d alpha = 0.99 / ((1 - 0.99 alpha) 2 d_min)
    const float galpha = gsigma != 0.f ? gsigma * kAlphaScale / ((1.f - kAlphaScale * alpha) * 2.f * dmin) : 0.f;
    if constexpr (PART == 1) {
        // after PART 0, which wrote (or added) the geometric terms
#pragma unroll
        for (int a = 0; a < 3; ++a) dcentre[3 * (size_t)i + a] += gc[a];
        dopacity[i] = accumulate ? dopacity[i] + galpha : galpha;
        if (kRow4 && dsh_aligned) {
            float4* d4 = reinterpret_cast<float4*>(dsh + (size_t)i * K * 3);
#pragma unroll
            for (int q = 0; q < (kRow4 ? K * 3 / 4 : 1); ++q) {
                float4 o = make_float4(gsh[4 * q], gsh[4 * q + 1], gsh[4 * q + 2], gsh[4 * q + 3]);
                if (accumulate) {
                    const float4 t = d4[q];
                    o.x += t.x; o.y += t.y; o.z += t.z; o.w += t.w;
                }
                d4[q] = o;
            }
        } else {
#pragma unroll
            for (int q = 0; q < K * 3; ++q) {
                float& o = dsh[(size_t)i * K * 3 + q];
                o = accumulate ? o + gsh[q] : gsh[q];
            }
        }
        return;
    }
    if (accumulate) {
#pragma unroll
        for (int a = 0; a < 3; ++a) dcentre[3 * (size_t)i + a] += gc[a];
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) dverts[((size_t)i * V + k) * 3 + a] += gv[k][a];
        if constexpr (PART == 2) dopacity[i] += galpha;
        if constexpr (PART == 2) {
#pragma unroll
            for (int q = 0; q < K * 3; ++q) dsh[(size_t)i * K * 3 + q] += gsh[q];
        }
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) dcentre[3 * (size_t)i + a] = gc[a];
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) dverts[((size_t)i * V + k) * 3 + a] = gv[k][a];
        if constexpr (PART == 2) dopacity[i] = galpha;
        if constexpr (PART == 2) {
#pragma unroll
            for (int q = 0; q < K * 3; ++q) dsh[(size_t)i * K * 3 + q] = gsh[q];
        }
    }
}

template <int V, int DEG>
cudaError_t launch_pre_t(const PrimsDev& P, const CamsParam& cams, float* rec, uint32_t* counts,
                         int4* trect, uint32_t* zbits, uint32_t* meta, cudaStream_t st) {
    const int bs = 128;
    const int grid = (P.n + bs - 1) / bs;
    if (grid > 0) k_preprocess<V, DEG><<<grid, bs, 0, st>>>(P, cams, rec, counts, trect, zbits, meta);
    return cudaGetLastError();
}

template <int V, int DEG>
cudaError_t launch_chain_t(const PrimsDev& P, const CamsParam& cams, const uint32_t* meta,
                           const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop,
                           float* dsh, int accumulate, int split, cudaStream_t st) {
    const int bs = 128;
    const int grid = (P.n + bs - 1) / bs;
    if (grid > 0) {
        if (P.grad_sum || !split) {
            k_chain<V, DEG, 2><<<grid, bs, 0, st>>>(P, cams, meta, counts, acc, dc, dv, dop, dsh, accumulate);
        } else {
            k_chain<V, DEG, 0><<<grid, bs, 0, st>>>(P, cams, meta, counts, acc, dc, dv, dop, dsh, accumulate);
            k_chain<V, DEG, 1><<<grid, bs, 0, st>>>(P, cams, meta, counts, acc, dc, dv, dop, dsh, accumulate);
        }
    }
    return cudaGetLastError();
}

}  // namespace

#define LP_DISPATCH(V, DEG, CALL)                                        \
    switch (DEG) {                                                       \
        case 0: return (V == 6) ? CALL(6, 0) : CALL(4, 0);               \
        case 1: return (V == 6) ? CALL(6, 1) : CALL(4, 1);               \
        case 2: return (V == 6) ? CALL(6, 2) : CALL(4, 2);               \
        default: return (V == 6) ? CALL(6, 3) : CALL(4, 3);              \
    }

cudaError_t launch_preprocess(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                              uint32_t* counts, int4* trect, uint32_t* zbits, uint32_t* meta, cudaStream_t st) {
#define CALL(v, d) launch_pre_t<v, d>(P, cams, rec, counts, trect, zbits, meta, st)
    LP_DISPATCH(V, deg, CALL)
#undef CALL
}

cudaError_t launch_chain(int V, int deg, const PrimsDev& P, const CamsParam& cams, const uint32_t* meta,
                         const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop,
                         float* dsh, int accumulate, int split, cudaStream_t st) {
#define CALL(v, d) launch_chain_t<v, d>(P, cams, meta, counts, acc, dc, dv, dop, dsh, accumulate, split, st)
    LP_DISPATCH(V, deg, CALL)
#undef CALL
}

}  // namespace lp
