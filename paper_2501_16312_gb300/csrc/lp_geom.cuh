// Geometry shared by the preprocess and chain kernels of both span modes
// (sm_103a): the camera-space centre, its accurate projection and the plane
// anchor, vertex offsets, face normals and the 2D filter's vertex move.
#pragma once

#include "lp_device.cuh"

namespace lp {

struct Geom {
    float tc[3];       // camera-space centre (binary32 key-field sequence)
    float xc, yc;      // projected centre (binary32 key-field sequence)
    float j00, j02, j11, j12;   // rows 0,1 of the EWA Jacobian
    float j2[3];       // row 2: tc / |tc|
    float len;         // |tc|
    int X0, Y0;        // integer pixel anchoring the record's planes
    float fxo, fyo;    // accurate projected centre minus (X0 + 0.5, Y0 + 0.5)
};

// Camera-space centre t = R c + T as unevaluated pairs hi + lo.
__device__ __forceinline__ void xform_df(const CamDev& cm, const float c[3], float hi[3], float lo[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float s = cm.T[i], l = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float p, pe, s2, se;
            two_prod(cm.R[3 * i + j], c[j], p, pe);
            two_sum(s, p, s2, se);
            s = s2;
            l = __fadd_rn(l, __fadd_rn(se, pe));
        }
        fast_two_sum(s, l, hi[i], lo[i]);
    }
}

// x = f (t / z) + cc with t, z given as pairs; result as a pair.  The
// remainder th - u zh of the correctly rounded quotient is exact.
__device__ __forceinline__ void project_df(float f, float cc, float th, float tl, float zh, float zl,
                                           float& xh, float& xl) {
    const float u = __fdiv_rn(th, zh);
    float r = __fmaf_rn(-u, zh, th);
    r = __fadd_rn(r, tl);
    r = __fmaf_rn(-u, zl, r);
    const float ul = __fdiv_rn(r, zh);
    float p, pe, sum, se;
    two_prod(f, u, p, pe);
    pe = __fmaf_rn(f, ul, pe);
    two_sum(p, cc, sum, se);
    fast_two_sum(sum, __fadd_rn(se, pe), xh, xl);
}

__device__ __forceinline__ void anchor(float xh, float xl, int& X0, float& fo) {
    xh = fminf(fmaxf(xh, -16777216.f), 16777216.f);
    const float f0 = floorf(xh);
    X0 = (int)f0;
    fo = __fadd_rn(__fsub_rn(__fsub_rn(xh, f0), 0.5f), xl);
}

// Camera-space centre, projected centre and the EWA Jacobian at the centre,
// J = d phi / d t with phi(t) = (fx tx/tz + cx, fy ty/tz + cy, |t|).
__device__ __forceinline__ bool centre_geom(const CamDev& cm, const float c[3], Geom& g) {
    xform_rn(cm, c[0], c[1], c[2], g.tc);
    if (!(g.tc[2] > kNearZ)) return false;
    const float u = __fdiv_rn(g.tc[0], g.tc[2]);
    const float w = __fdiv_rn(g.tc[1], g.tc[2]);
    g.xc = __fadd_rn(__fmul_rn(cm.fx, u), cm.cx);
    g.yc = __fadd_rn(__fmul_rn(cm.fy, w), cm.cy);
    // the view frustum: the projected centre within 1.3 times the image
    // (|x_ndc|, |y_ndc| <= 1.3).  Off-axis primitives near the camera plane
    // would otherwise get linearised boxes covering the whole image.
    const float W = (float)cm.width, H = (float)cm.height;
    if (!(g.xc >= __fmul_rn(kFrustumLo, W) && g.xc <= __fmul_rn(kFrustumHi, W) &&
          g.yc >= __fmul_rn(kFrustumLo, H) && g.yc <= __fmul_rn(kFrustumHi, H)))
        return false;
    g.j00 = __fdiv_rn(cm.fx, g.tc[2]);
    g.j02 = -__fmul_rn(g.j00, u);
    g.j11 = __fdiv_rn(cm.fy, g.tc[2]);
    g.j12 = -__fmul_rn(g.j11, w);
    g.len = sqrtf(g.tc[0] * g.tc[0] + g.tc[1] * g.tc[1] + g.tc[2] * g.tc[2]);
    const float il = 1.f / g.len;
    g.j2[0] = g.tc[0] * il; g.j2[1] = g.tc[1] * il; g.j2[2] = g.tc[2] * il;
    // accurate projected centre for the plane anchor
    float th[3], tl[3], xh, xl, yh, yl;
    xform_df(cm, c, th, tl);
    project_df(cm.fx, cm.cx, th[0], tl[0], th[2], tl[2], xh, xl);
    project_df(cm.fy, cm.cy, th[1], tl[1], th[2], tl[2], yh, yl);
    anchor(xh, xl, g.X0, g.fxo);
    anchor(yh, yl, g.Y0, g.fyo);
    return true;
}

// Local ray-space offset q = J d of one vertex, d = R (v - c) its offset
// from the centre rotated into the camera frame (binary32 key-field
// sequence; rotating the small offset keeps its relative accuracy).
__device__ __forceinline__ void vertex_local(const CamDev& cm, const Geom& g, const float v[3],
                                             const float c[3], float q[3], float d[3]) {
    const float w0 = __fsub_rn(v[0], c[0]), w1 = __fsub_rn(v[1], c[1]), w2 = __fsub_rn(v[2], c[2]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
        d[m] = __fadd_rn(__fadd_rn(__fmul_rn(cm.R[3 * m], w0), __fmul_rn(cm.R[3 * m + 1], w1)),
                         __fmul_rn(cm.R[3 * m + 2], w2));
    q[0] = __fadd_rn(__fmul_rn(g.j00, d[0]), __fmul_rn(g.j02, d[2]));
    q[1] = __fadd_rn(__fmul_rn(g.j11, d[1]), __fmul_rn(g.j12, d[2]));
    q[2] = g.j2[0] * d[0] + g.j2[1] * d[1] + g.j2[2] * d[2];
}

// Unnormalised face normal n = (q1 - q0) x (q2 - q0).
__device__ __forceinline__ void face_normal(const float* q0, const float* q1, const float* q2,
                                            float n[3]) {
    const float e1[3] = {q1[0] - q0[0], q1[1] - q0[1], q1[2] - q0[2]};
    const float e2[3] = {q2[0] - q0[0], q2[1] - q0[1], q2[2] - q0[2]};
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
}

// A face is treated as seen exactly edge-on (no depth plane) when its normal
// has |n_z| below this fraction of |n_x| + |n_y|; its plane is then clamped.
constexpr float kEdgeOn = 1e-30f;

__device__ __forceinline__ bool plane_degenerate(const float n[3]) {
    return !(fabsf(n[2]) >= kEdgeOn * (fabsf(n[0]) + fabsf(n[1]))) || n[2] == 0.f;
}

// Sec. 3.3 2D filter: the vertices on the projected bounding box move
// outward, parallel to the screen (a vertex on the maximum moves up, else one
// on the minimum moves down), by half the filter size for an octahedron,
// whose opposite vertices mirror the move, and the whole size for a
// tetrahedron.  Decided and applied in binary32 on the key-field values.
template <int V>
__device__ __forceinline__ void aa_widen(const CamsParam& cams, float (&q)[V][3]) {
    const float s = V == 6 ? cams.aa_half : cams.aa_full;
    if (!(s > 0.f)) return;
    float xmin = q[0][0], xmax = q[0][0], ymin = q[0][1], ymax = q[0][1];
#pragma unroll
    for (int k = 1; k < V; ++k) {
        xmin = fminf(xmin, q[k][0]); xmax = fmaxf(xmax, q[k][0]);
        ymin = fminf(ymin, q[k][1]); ymax = fmaxf(ymax, q[k][1]);
    }
#pragma unroll
    for (int k = 0; k < V; ++k) {
        if (q[k][0] == xmax) q[k][0] = __fadd_rn(q[k][0], s);
        else if (q[k][0] == xmin) q[k][0] = __fsub_rn(q[k][0], s);
        if (q[k][1] == ymax) q[k][1] = __fadd_rn(q[k][1], s);
        else if (q[k][1] == ymin) q[k][1] = __fsub_rn(q[k][1], s);
    }
}

}  // namespace lp
