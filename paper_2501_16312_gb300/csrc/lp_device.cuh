// Device-side definitions shared by the LinPrim kernels (sm_103a).
//
// Paper: "LinPrim: Linear Primitives for Differentiable Volumetric Rendering"
// (arXiv 2501.16312).  Section references below are to that paper.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

namespace lp {

constexpr int kMaxCams = 32;
constexpr float kNearZ = 0.2f;      // centres at camera depth <= 0.2 are culled
// View frustum in pixels: a centre projecting outside [lo W, hi W] x [lo H, hi H]
// (normalised device coordinates beyond +-1.3) is culled.
constexpr float kFrustumLo = -0.15f;
constexpr float kFrustumHi = 1.15f;
constexpr float kStopT = 1e-3f;     // Sec. 3.2: stop at cumulative opacity 0.999
constexpr float kAlphaScale = 0.99f;  // Eq. 1
constexpr int kStatusCapacity = 1;
constexpr int kStatusTimeout = 2;

// Tile-list length the scan writes when the 64-bit total of the tile counts
// reaches 2^32 - 1: 32-bit list offsets cannot address such a list, so every
// stage treats it as empty (and the scan latches kStatusCapacity).
constexpr uint32_t kListOverflow = 0xffffffffu;

// The list length to process: E from the device, capped by the host's bound,
// or 0 after an overflowed scan.
__device__ __forceinline__ long long list_len(const uint32_t* n_dev, long long bound) {
    const uint32_t e = *n_dev;
    return e == kListOverflow ? 0ll : min((long long)e, bound);
}

// One camera, pre-digested on the host.  R, T: rows of the world->camera
// matrix; campos = -R^T T.  Tiles of this camera occupy global tile ids
// [tile_base, tile_base + tiles_x * tiles_y); its pixels start at pix_base in
// the packed image (3 planes of width*height floats at 3 * pix_base).
struct CamDev {
    float R[9];
    float T[3];
    float fx, fy, cx, cy;
    float campos[3];
    int width, height, tiles_x, tiles_y, tile_base, pix_base;
};

// Passed by value as a kernel parameter (captured into CUDA graphs with it).
struct CamsParam {
    int n;
    int total_tiles;
    int tile;
    int total_pixels;
    // Sec. 3.3 2D filter: outward move of the bounding-box vertices in
    // pixels, for octahedra (half the filter) and tetrahedra; 0 = off
    float aa_half, aa_full;
    CamDev cam[kMaxCams];
};

struct PrimsDev {
    int n;
    const float* centre;
    const float* verts;
    const float* opacity;
    const float* sh;
    // Densification statistics (App. "Experimental Setting"), null when not
    // gathered: the forward raises px_max to the largest pixel-rectangle side
    // of each view, the backward adds each visible view's view-space position
    // gradient norm to grad_sum and counts the view in grad_count.
    uint32_t* px_max = nullptr;
    float* grad_sum = nullptr;
    uint32_t* grad_count = nullptr;
};

// NDC norm of a camera-space translation gradient g (the primitive moved
// parallel to the image plane at depth z): d x_ndc = 2 f_x / (W z) d t_x.
__device__ __forceinline__ float ndc_grad_norm(const CamDev& cm, const float g[3], float z) {
    const float gx = g[0] * (float)cm.width * z / (2.f * cm.fx);
    const float gy = g[1] * (float)cm.height * z / (2.f * cm.fy);
    return sqrtf(gx * gx + gy * gy);
}

template <int V> struct Kind;
template <> struct Kind<6> { static constexpr int F = 8; };   // octahedron
template <> struct Kind<4> { static constexpr int F = 4; };   // tetrahedron

// Face f's three vertex indices.  Octahedron vertices come in +/- pairs per
// axis, (0,1), (2,3), (4,5); each face takes one vertex of each pair.  A
// tetrahedron's face k is the triangle opposite vertex k.
template <int V>
__device__ __forceinline__ void face_vertices(int f, int& i0, int& i1, int& i2) {
    if (V == 6) {
        i0 = (f >> 2) & 1;
        i1 = 2 + ((f >> 1) & 1);
        i2 = 4 + (f & 1);
    } else {
        i0 = (f == 0) ? 1 : 0;
        i1 = (f <= 1) ? 2 : 1;
        i2 = (f <= 2) ? 3 : 2;
    }
}

// Projected record of one (camera, primitive) pair, written by the
// preprocess and read by both blend kernels.  Layout in 32-bit words:
//   [0] X0  [1] Y0        integer pixel near the projected centre (int bits)
//   [2] sigma             density, Eq. 1
//   [3] meta              bits 0-3: nf, the number of entry faces; then 3 bits
//                         per slot: the face index held by that slot
//   [4..6] rgb            view-dependent colour
//   [7]                   unused
//   [8 + 3s .. 10 + 3s]   plane of slot s: depth - z_c = a (px - X0)
//                         + b (py - Y0) + e0 at the centre of pixel (px, py);
//                         slots [0, nf) are entry faces, [nf, F) exit faces.
// Anchoring the planes to an integer pixel keeps every pixel offset an exact
// integer in binary32, so steep faces lose no accuracy to the offset.
template <int V> struct Rec {
    static constexpr int F = Kind<V>::F;
    static constexpr int kFloats = 8 + 3 * F;   // 32 (octahedron), 20 (tetrahedron)
    static constexpr int kVec4 = kFloats / 4;
};

__device__ __forceinline__ int meta_nf(uint32_t meta) { return (int)(meta & 15u); }
__device__ __forceinline__ int meta_face(uint32_t meta, int slot) {
    return (int)((meta >> (4 + 3 * slot)) & 7u);
}

// Per-record gradient accumulators written by the backward blend, in two
// blocks of one array (records R):
//   planes, [R][F][4] at the start: [4s .. 4s+2] sums of g * (px - X0,
//          py - Y0, 1) over the pixels where slot s bounds the span, g =
//          dL/d(plane depth); [4s + 3] stays zero.  Each slot is one 16-byte
//          row, so one vector atomic adds a pixel's three terms;
//   colour, [R][4] after the planes: dL/d rgb, dL/d sigma (one 16-byte row).
// The chain's geometry and colour passes each read only their own block.
template <int V> struct Acc {
    static constexpr int F = Kind<V>::F;
    static constexpr int kPlane = 4 * F;           // 32, 16
    static constexpr int kFloats = kPlane + 4;     // per record over both blocks
};

// -------------------------------------------------------------------------
// Error-free transformations (Knuth's TwoSum, FMA-based TwoProduct) used to
// carry the projected centre as an unevaluated sum hi + lo of two floats.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// -------------------------------------------------------------------------
// Binary32 key-field arithmetic.  Culling, the depth key and the pixel
// rectangle are integers decided by floating point, so they are computed
// with a fixed order of single-rounding operations (no contraction).

__device__ __forceinline__ void xform_rn(const CamDev& c, float x, float y, float z, float t[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float a = __fmul_rn(c.R[3 * i + 0], x);
        float b = __fmul_rn(c.R[3 * i + 1], y);
        float d = __fmul_rn(c.R[3 * i + 2], z);
        t[i] = __fadd_rn(__fadd_rn(__fadd_rn(a, b), d), c.T[i]);
    }
}

// -------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3, in the 3DGS order and signs
// (Sec. 3.1: colours follow 3DGS).  Y[k] for unit direction (x, y, z).
struct ShC {
    static constexpr float c0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
    static constexpr float c1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
    static constexpr float c2a = 1.0925484305920792f;   // sqrt(15/pi)/2
    static constexpr float c2b = 0.31539156525252005f;  // sqrt(5/pi)/4
    static constexpr float c2c = 0.5462742152960396f;   // sqrt(15/pi)/4
    static constexpr float c3a = 0.5900435899266435f;   // sqrt(35/(2 pi))/4
    static constexpr float c3b = 2.890611442640554f;    // sqrt(105/pi)/2
    static constexpr float c3c = 0.4570457994644658f;   // sqrt(21/(2 pi))/4
    static constexpr float c3d = 0.3731763325901154f;   // sqrt(7/pi)/4
    static constexpr float c3e = 1.445305721320277f;    // sqrt(105/pi)/4
};

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = ShC::c0;
    if (DEG < 1) return;
    Y[1] = -ShC::c1 * y;
    Y[2] = ShC::c1 * z;
    Y[3] = -ShC::c1 * x;
    if (DEG < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = ShC::c2a * x * y;
    Y[5] = -ShC::c2a * y * z;
    Y[6] = ShC::c2b * (2.f * zz - xx - yy);
    Y[7] = -ShC::c2a * x * z;
    Y[8] = ShC::c2c * (xx - yy);
    if (DEG < 3) return;
    Y[9] = -ShC::c3a * y * (3.f * xx - yy);
    Y[10] = ShC::c3b * x * y * z;
    Y[11] = -ShC::c3c * y * (4.f * zz - xx - yy);
    Y[12] = ShC::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -ShC::c3c * x * (4.f * zz - xx - yy);
    Y[14] = ShC::c3e * z * (xx - yy);
    Y[15] = -ShC::c3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k Y_k(d) w_k with respect to the (unit) direction d.
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float* w, float g[3]) {
    g[0] = g[1] = g[2] = 0.f;
    if (DEG < 1) return;
    g[0] += -ShC::c1 * w[3];
    g[1] += -ShC::c1 * w[1];
    g[2] += ShC::c1 * w[2];
    if (DEG < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] += ShC::c2a * y * w[4] - ShC::c2a * z * w[7] - 2.f * ShC::c2b * x * w[6] +
            2.f * ShC::c2c * x * w[8];
    g[1] += ShC::c2a * x * w[4] - ShC::c2a * z * w[5] - 2.f * ShC::c2b * y * w[6] -
            2.f * ShC::c2c * y * w[8];
    g[2] += -ShC::c2a * y * w[5] + 4.f * ShC::c2b * z * w[6] - ShC::c2a * x * w[7];
    if (DEG < 3) return;
    g[0] += -ShC::c3a * 6.f * x * y * w[9] + ShC::c3b * y * z * w[10] +
            ShC::c3c * 2.f * x * y * w[11] - ShC::c3d * 6.f * x * z * w[12] -
            ShC::c3c * (4.f * zz - 3.f * xx - yy) * w[13] + ShC::c3e * 2.f * x * z * w[14] -
            ShC::c3a * (3.f * xx - 3.f * yy) * w[15];
    g[1] += -ShC::c3a * (3.f * xx - 3.f * yy) * w[9] + ShC::c3b * x * z * w[10] -
            ShC::c3c * (4.f * zz - xx - 3.f * yy) * w[11] - ShC::c3d * 6.f * y * z * w[12] +
            ShC::c3c * 2.f * x * y * w[13] - ShC::c3e * 2.f * y * z * w[14] +
            ShC::c3a * 6.f * x * y * w[15];
    g[2] += ShC::c3b * x * y * w[10] - ShC::c3c * 8.f * y * z * w[11] +
            ShC::c3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12] - ShC::c3c * 8.f * x * z * w[13] +
            ShC::c3e * (xx - yy) * w[14];
}

// -------------------------------------------------------------------------
// 3-input FP32 min/max (Blackwell), as inline PTX; exact like fminf/fmaxf.
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// -------------------------------------------------------------------------
// A record staged in shared memory for one tile.  Planes are float4
// (a, b, e0, 0) for 128-bit shared loads, anchored at the record's integer
// pixel (X0, Y0): pixel (tx0 + lx, ty0 + ly) of the tile evaluates depth =
// a X + b Y + e0 at the exact integer offsets X = lx + dx0, Y = ly + dy0 from
// the anchor, with (dx0, dy0) = (tx0 - X0, ty0 - Y0).  The arithmetic of a
// pixel is then the same whatever tile holds it, and near the primitive
// (where its spans matter) the terms are no larger than its own depth
// extent.  The forward and backward blends both stage through
// stage_record() and evaluate through the same span routines, so they
// compute bit-identical spans.  pl[0].w carries the ray-space depth of the
// centre, to which the planes' depths are relative (used by the depth pass
// only).
template <int V> struct alignas(16) Staged {
    static constexpr int F = Kind<V>::F;
    float4 pl[F];
    float sigma, r, g, b;
    float dx0, dy0;    // tx0 - X0, ty0 - Y0 (integers)
    int nf;
    int rec;           // record index (camera * n + primitive)
    // bit w G + g: the pixel rectangle of lane group g of warp w (WarpGrid,
    // LaneGroups) may hold a pixel whose ray meets the primitive; clear only
    // when some entry/exit face pair proves it cannot, with a margin above
    // binary32 rounding (forward only)
    uint64_t bands;
};

// Which pixels of a TILE x TILE tile a thread of a blend block owns, with
// PIX horizontally adjacent pixels per thread.  Each warp covers one
// rectangle of WR rows by WC columns: 8 x 8 pixels with one or two pixels
// per thread (4 x 8 with one), 8 x 16 with four.  Warps tile the tile row by
// row; inside a warp, TPR threads make one row.
template <int TILE, int PIX> struct WarpGrid {
    static constexpr int WC0 = PIX >= 4 ? 16 : 8;
    static constexpr int WC = WC0 < TILE ? WC0 : TILE;   // warp width in pixels
    static constexpr int WR = 32 * PIX / WC;             // warp height in rows
    static constexpr int NWX = TILE / WC;                // warps across the tile
    static constexpr int TPR = WC / PIX;                 // threads per warp row
    static constexpr int NW = TILE * TILE / PIX / 32;    // warps per tile
    static_assert(WC % PIX == 0 && TILE % WC == 0 && TILE % WR == 0 && NW * 32 * PIX == TILE * TILE,
                  "warps of whole rectangles");
    __host__ __device__ __forceinline__ static void pixel(int tid, int& ly, int& lx0) {
        const int w = tid >> 5, lane = tid & 31;
        ly = (w / NWX) * WR + lane / TPR;
        lx0 = (w % NWX) * WC + (lane % TPR) * PIX;
    }
};

// Stages record r for the tile at (tx0, ty0); returns the record's meta word.
template <int V>
__device__ __forceinline__ uint32_t stage_record(const float* __restrict__ rec, int r, int tx0, int ty0,
                                                 Staged<V>& s) {
    constexpr int F = Kind<V>::F;
    const float4* src = reinterpret_cast<const float4*>(rec + (size_t)r * Rec<V>::kFloats);
    float buf[Rec<V>::kFloats];
#pragma unroll
    for (int q = 0; q < Rec<V>::kVec4; ++q) {
        float4 v = __ldg(src + q);
        buf[4 * q + 0] = v.x; buf[4 * q + 1] = v.y; buf[4 * q + 2] = v.z; buf[4 * q + 3] = v.w;
    }
    const float dx0 = (float)(tx0 - __float_as_int(buf[0]));
    const float dy0 = (float)(ty0 - __float_as_int(buf[1]));
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const float a = buf[8 + 3 * f], b = buf[9 + 3 * f], e = buf[10 + 3 * f];
        s.pl[f] = make_float4(a, b, e, 0.f);
    }
    s.pl[0].w = buf[7];
    s.sigma = buf[2];
    s.r = buf[4]; s.g = buf[5]; s.b = buf[6];
    s.dx0 = dx0; s.dy0 = dy0;
    const uint32_t meta = __float_as_uint(buf[3]);
    s.nf = meta_nf(meta);
    s.rec = r;
    return meta;
}

// Ray/primitive spans of a strip of PIX pixels at anchor offsets (X0 + i, Y),
// i < PIX (X0 = lx0 + dx0, Y = ly + dy0, exact integers), by
// half-space clipping of each pixel ray against the convex primitive: entry
// = max over the NF entry faces, exit = min over the others.  This equals the
// distance between the two MTIA hits of Sec. 3.2 "Rasterization".  NF is a
// template argument so the entry/exit split costs nothing per face; with ARG
// the arg-max entry slot and arg-min exit slot are returned too.
template <int V, int PIX, int NF, bool ARG>
__device__ __forceinline__ void spans_nf(const Staged<V>& s, float lx0, float ly, float* sp, int* sf,
                                         int* sb) {
    constexpr int F = Kind<V>::F;
    if constexpr (NF <= 0 || NF >= F) {   // no entry or no exit face: not a closed convex primitive
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            sp[i] = 0.f;
            if (ARG) { sf[i] = 0; sb[i] = F - 1; }
        }
    } else if constexpr (ARG) {
        float tf[PIX], tb[PIX];
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            tf[i] = -CUDART_INF_F;
            tb[i] = CUDART_INF_F;
            sf[i] = 0; sb[i] = F - 1;
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const float4 p = s.pl[f];
            const float t = __fmaf_rn(p.y, ly, p.z);
#pragma unroll
            for (int i = 0; i < PIX; ++i) {
                const float d = __fmaf_rn(p.x, lx0 + (float)i, t);
                if (f < NF) { if (d > tf[i]) { tf[i] = d; sf[i] = f; } }
                else        { if (d < tb[i]) { tb[i] = d; sb[i] = f; } }
            }
        }
#pragma unroll
        for (int i = 0; i < PIX; ++i) sp[i] = __fsub_rn(tb[i], tf[i]);
    } else {
        // depths of all faces, then entry max / exit min two faces per 3-input op
        float d[F][PIX];
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const float4 p = s.pl[f];
            const float t = __fmaf_rn(p.y, ly, p.z);
#pragma unroll
            for (int i = 0; i < PIX; ++i) d[f][i] = __fmaf_rn(p.x, lx0 + (float)i, t);
        }
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            float tf = d[0][i];
#pragma unroll
            for (int f = 1; f + 1 < NF; f += 2) tf = max3f(tf, d[f][i], d[f + 1][i]);
            if ((NF - 1) % 2 == 1) tf = fmaxf(tf, d[NF - 1][i]);
            float tb = d[NF][i];
#pragma unroll
            for (int f = NF + 1; f + 1 < F; f += 2) tb = min3f(tb, d[f][i], d[f + 1][i]);
            if ((F - NF - 1) % 2 == 1) tb = fminf(tb, d[F - 1][i]);
            sp[i] = __fsub_rn(tb, tf);
        }
    }
}

template <int V, int PIX, bool ARG>
__device__ __forceinline__ void spans(const Staged<V>& s, float lx0, float ly, float* sp, int* sf,
                                      int* sb) {
    if (V == 6) {
        switch (s.nf) {
            case 1: spans_nf<V, PIX, 1, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 2: spans_nf<V, PIX, 2, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 3: spans_nf<V, PIX, 3, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 4: spans_nf<V, PIX, 4, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 5: spans_nf<V, PIX, 5, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 6: spans_nf<V, PIX, 6, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 7: spans_nf<V, PIX, 7, ARG>(s, lx0, ly, sp, sf, sb); break;
            default: spans_nf<V, PIX, 0, ARG>(s, lx0, ly, sp, sf, sb); break;
        }
    } else {
        switch (s.nf) {
            case 1: spans_nf<V, PIX, 1, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 2: spans_nf<V, PIX, 2, ARG>(s, lx0, ly, sp, sf, sb); break;
            case 3: spans_nf<V, PIX, 3, ARG>(s, lx0, ly, sp, sf, sb); break;
            default: spans_nf<V, PIX, 0, ARG>(s, lx0, ly, sp, sf, sb); break;
        }
    }
}

// Transmittance and opacity of a span, App. "Gradient Computation":
// tau = exp(-sigma s), o = 1 - tau.  For a faint span (x = sigma s small)
// 1 - tau keeps few correct digits, which would carry into the colour and
// opacity gradients; there o comes from the Taylor polynomial of 1 - exp(-x),
// five terms, whose truncation error below x = 1/16 is under 2e-9 relative.
// Above it 1 - tau is accurate to about 1e-6 relative.
__device__ __forceinline__ float span_x(float sigma, float s) { return __fmul_rn(sigma, s); }
__device__ __forceinline__ float span_tau(float x) { return __expf(-x); }
__device__ __forceinline__ float span_opacity(float x, float tau) {
    const float p = x * __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, __fmaf_rn(x, 1.f / 120.f, -1.f / 24.f), 1.f / 6.f),
                                               -0.5f), 1.f);
    return x < 0.0625f ? p : 1.f - tau;
}

__device__ __forceinline__ int camera_of_tile(const CamsParam& cams, int tile) {
    int c = 0;
    while (c + 1 < cams.n && tile >= cams.cam[c + 1].tile_base) ++c;
    return c;
}

}  // namespace lp
