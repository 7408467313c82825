// Exact spans, without the ray-space approximation (sm_103a).
//
// App. "Ray Space Approximation" evaluates a variant that renders with the
// true perspective ray of each pixel instead of the EWA affine ray space, at
// about twice the rasterization cost.  The ray of pixel centre (x, y) is
// lambda d with d = ((x - cx)/fx, (y - cy)/fy, 1) in camera space; it enters
// a convex primitive at the largest entry-face hit and leaves at the smallest
// exit-face hit, and the span is the distance between them, (lam_out - lam_in)
// |d| (world units).  Which faces enter depends on the pixel, so each face is
// classified per pixel by the sign of n . d.
//
// Which faces a ray can enter through does not depend on the pixel: the
// camera lies outside exactly those faces' half-spaces (for the others a
// ray can only leave), so the faces are split once per record, entry faces
// first, as in the ray-space mode.
//
// Each face is stored as the camera-space half-space n' . (t - c) <= 1 around
// the primitive's centre c (outward normal n scaled so the right side is 1),
// evaluated relative to the centre depth: with L = n'_x (x - x_c)/fx +
// n'_y (y - y_c)/fy (x_c, y_c the projected centre), D = n' . d = L + D0 and
// D0 = n' . c / c_z, the hit is lambda = c_z + (1 - c_z L)/D.  The stored
// quantities are small offsets, so the span does not cancel between two large
// depths.  Per face a record keeps float4 (p, q, L0, D0) with p = n'_x/fx,
// q = n'_y/fy and L0 = L at the anchor pixel (X0, Y0).
//
// The tile rectangle is the box of the perspectively projected vertices,
// which needs every vertex in front: a primitive with a vertex at depth
// <= 0.2 is not drawn in this mode.  The 2D filter does not apply.  One
// schedule is built (32 records per batch, 4 pixels per thread).
#include "lp_blend.cuh"
#include "lp_geom.cuh"

namespace lp {

namespace {

constexpr int kBatchX = 32;
// pixels per thread and threads per block of the exact-span blends for a
// TILE x TILE tile: strips of 4 pixels, of 2 on 8x8 tiles (one whole warp)
template <int TILE> constexpr int pix_x() { return TILE == 8 ? 2 : 4; }
template <int TILE> constexpr int threads_x() { return TILE * TILE / pix_x<TILE>(); }

template <int V> struct RecX {
    static constexpr int F = Kind<V>::F;
    static constexpr int kFloats = 8 + 4 * F;   // 40 (octahedron), 24 (tetrahedron)
};

// per face slot (= face) dL/d(p, q, L0, D0); then rgb, sigma, c_z (the last
// is collected by the backward but not needed by the chain, see k_chain_x),
// padded to whole 16-byte rows so that each row takes one vector atomic
template <int V> struct AccX {
    static constexpr int F = Kind<V>::F;
    static constexpr int kFloats = 4 * F + 8;   // 40, 24
};

// Camera-space offsets d = R (v - c) of a vertex (the key-field sequence).
__device__ __forceinline__ void vertex_offset(const CamDev& cm, const float v[3], const float c[3], float d[3]) {
    const float w0 = __fsub_rn(v[0], c[0]), w1 = __fsub_rn(v[1], c[1]), w2 = __fsub_rn(v[2], c[2]);
#pragma unroll
    for (int m = 0; m < 3; ++m)
        d[m] = __fadd_rn(__fadd_rn(__fmul_rn(cm.R[3 * m], w0), __fmul_rn(cm.R[3 * m + 1], w1)),
                         __fmul_rn(cm.R[3 * m + 2], w2));
}

// Face f as n' = n / h with n the normal of the offsets' triangle and
// h = n . d0 (the centre is inside, so h != 0 for a proper primitive; a face
// through the centre gets n' = 0, a constraint every ray meets).
template <int V>
__device__ __forceinline__ void face_plane_x(const float d[V][3], int f, float np[3], float& h) {
    int i0, i1, i2;
    face_vertices<V>(f, i0, i1, i2);
    float n[3];
    face_normal(d[i0], d[i1], d[i2], n);
    h = n[0] * d[i0][0] + n[1] * d[i0][1] + n[2] * d[i0][2];
    const float ih = h != 0.f ? 1.f / h : 0.f;
    np[0] = n[0] * ih; np[1] = n[1] * ih; np[2] = n[2] * ih;
}

template <int V, int DEG>
__global__ void __launch_bounds__(128) k_preprocess_x(PrimsDev P, CamsParam cams, float* __restrict__ rec,
                                                      uint32_t* __restrict__ counts, int4* __restrict__ trect,
                                                      uint32_t* __restrict__ zbits) {
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
    // Eq. 1 (d_min from the world-space vertices) and the degenerate case, as
    // in the ray-space mode
    float dmin = CUDART_INF_F;
    bool degenerate = false;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float dx = v[k][0] - c[0], dy = v[k][1] - c[1], dz = v[k][2] - c[2];
        dmin = fminf(dmin, sqrtf(dx * dx + dy * dy + dz * dz));
        degenerate |= dx == 0.f && dy == 0.f && dz == 0.f;
    }
    const float sigma = -log1pf(-kAlphaScale * alpha) / (2.f * dmin);
    degenerate |= !(sigma < CUDART_INF_F);
    uint32_t px_side = 0;   // largest pixel-rectangle side over the views

    for (int cv = 0; cv < cams.n; ++cv) {
        const CamDev& cm = cams.cam[cv];
        const size_t r = (size_t)cv * P.n + i;
        Geom g;
        bool vis = centre_geom(cm, c, g) && !degenerate;
        zbits[r] = __float_as_uint(g.tc[2]);
        float d[V][3];
        float qxmin = CUDART_INF_F, qxmax = -CUDART_INF_F, qymin = CUDART_INF_F, qymax = -CUDART_INF_F;
        if (vis) {
#pragma unroll
            for (int k = 0; k < V; ++k) {
                vertex_offset(cm, v[k], c, d[k]);
                // the vertex's perspective projection, as an offset from the
                // projected centre (binary32 key-field sequence)
                const float X = __fadd_rn(g.tc[0], d[k][0]), Y = __fadd_rn(g.tc[1], d[k][1]);
                const float Z = __fadd_rn(g.tc[2], d[k][2]);
                vis = vis && Z > kNearZ;
                const float uu = __fdiv_rn(X, Z), ww = __fdiv_rn(Y, Z);
                const float qx = __fsub_rn(__fadd_rn(__fmul_rn(cm.fx, uu), cm.cx), g.xc);
                const float qy = __fsub_rn(__fadd_rn(__fmul_rn(cm.fy, ww), cm.cy), g.yc);
                qxmin = fminf(qxmin, qx); qxmax = fmaxf(qxmax, qx);
                qymin = fminf(qymin, qy); qymax = fmaxf(qymax, qy);
            }
        }
        if (!vis) {
            counts[r] = 0;
            trect[r] = make_int4(0, 0, 0, 0);
            continue;
        }
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
        trect[r] = make_int4(cm.tile_base + ty0 * cm.tiles_x + tx0, cm.tiles_x, tx1 - tx0 + 1, ty1 - ty0 + 1);

        float out[8];   // header: anchor, sigma, meta, rgb, centre depth
        const float icz = 1.f / g.tc[2];
        float pl[F][4];
        bool front[F];
        int nf = 0;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            float np[3], h;
            face_plane_x<V>(d, f, np, h);
            const float p = np[0] / cm.fx, q = np[1] / cm.fy;
            pl[f][0] = p;
            pl[f][1] = q;
            pl[f][2] = -__fmaf_rn(p, g.fxo, __fmul_rn(q, g.fyo));
            pl[f][3] = (np[0] * g.tc[0] + np[1] * g.tc[1] + np[2] * g.tc[2]) * icz;
            // the camera (the origin) lies outside the face's half-space
            // n' . t <= 1 + n' . c: every ray can only enter through it
            front[f] = 1.f + np[0] * g.tc[0] + np[1] * g.tc[1] + np[2] * g.tc[2] < 0.f;
            nf += front[f] ? 1 : 0;
        }
        // slots: faces the camera sees from outside first (entry faces); a
        // slot is one float4, stored at its computed address
        float4* dst = reinterpret_cast<float4*>(rec + r * RecX<V>::kFloats);
        uint32_t meta = (uint32_t)nf;
        int sf = 0, sb = nf;
#pragma unroll
        for (int f = 0; f < F; ++f) {
            const int s = front[f] ? sf++ : sb++;
            meta |= (uint32_t)f << (4 + 3 * s);
            dst[2 + s] = make_float4(pl[f][0], pl[f][1], pl[f][2], pl[f][3]);
        }
        float dir[3] = {c[0] - cm.campos[0], c[1] - cm.campos[1], c[2] - cm.campos[2]};
        const float idl = rsqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        dir[0] *= idl; dir[1] *= idl; dir[2] *= idl;
        float Y[16];
        sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], sh[3 * k + ch], s);
            out[4 + ch] = fmaxf(s, 0.f);
        }
        dst[0] = make_float4(__int_as_float(g.X0), __int_as_float(g.Y0), sigma, __uint_as_float(meta));
        dst[1] = make_float4(out[4], out[5], out[6], g.tc[2]);
    }
    if (P.px_max && px_side > P.px_max[i]) P.px_max[i] = px_side;   // one thread per primitive
}

// ------------------------------------------------------------------- blend
template <int V> struct alignas(16) StagedX {
    static constexpr int F = Kind<V>::F;
    float4 pl[F];      // (p, q, L0, D0): L = p X + q Y + L0 at the anchor offset (X, Y)
    float sigma, r, g, b;
    float cz, dx0, dy0;
    int nf;            // entry faces (slots 0 .. nf - 1)
    int rec;
};

template <int V>
__device__ __forceinline__ void stage_record_x(const float* __restrict__ rec, int r, int tx0, int ty0,
                                               StagedX<V>& s) {
    constexpr int F = Kind<V>::F;
    const float4* src = reinterpret_cast<const float4*>(rec + (size_t)r * RecX<V>::kFloats);
    const float4 h0 = __ldg(src), h1 = __ldg(src + 1);
    const float dx0 = (float)(tx0 - __float_as_int(h0.x));
    const float dy0 = (float)(ty0 - __float_as_int(h0.y));
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const float4 pl = __ldg(src + 2 + f);
        s.pl[f] = pl;   // evaluated at anchor offsets, whatever the tile
    }
    s.sigma = h0.z;
    s.r = h1.x; s.g = h1.y; s.b = h1.z;
    s.cz = h1.w;
    s.dx0 = dx0; s.dy0 = dy0;
    s.nf = meta_nf(__float_as_uint(h0.w));
    s.rec = r;
}

// Spans of a strip of PIX pixels.  rn[i] = |d| of pixel i.  Slots < NF are
// entry faces: a ray meets the primitive only if it crosses each of them
// inward (D < 0), and then enters no earlier than its hit; the other faces
// bound the exit where the ray leaves them (D > 0).  With ARG the entry /
// exit slots are returned too; ent[i] = entry hit minus c_z.
template <int V, int PIX, int NF, bool ARG>
__device__ __forceinline__ void spans_x_nf(const StagedX<V>& s, float lx0, float ly, const float* rn, float* sp,
                                           int* sf, int* sb, float* ent_out) {
    constexpr int F = Kind<V>::F;
    if constexpr (NF <= 0 || NF >= F) {   // no entry or no exit face: not a closed primitive seen from outside
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            sp[i] = -1.f;
            if (ARG) { sf[i] = 0; sb[i] = F - 1; }
            if (ent_out) ent_out[i] = 0.f;
        }
    } else {
    float en[PIX], ex[PIX];
#pragma unroll
    for (int i = 0; i < PIX; ++i) {
        en[i] = -s.cz;   // lambda > 0: the hit must lie in front of the camera
        ex[i] = CUDART_INF_F;
        if (ARG) { sf[i] = 0; sb[i] = NF; }
    }
#pragma unroll
    for (int f = 0; f < F; ++f) {
        const float4 p = s.pl[f];
        const float t = __fmaf_rn(p.y, ly, p.z);
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            const float L = __fmaf_rn(p.x, lx0 + (float)i, t);
            const float D = __fadd_rn(L, p.w);
            const float dl = __fdividef(__fmaf_rn(-s.cz, L, 1.f), D);
            if (f < NF) {
                const float e = D < 0.f ? dl : CUDART_INF_F;   // not crossed inward: no hit
                if (ARG) { if (e > en[i]) { en[i] = e; sf[i] = f; } }
                else en[i] = fmaxf(en[i], e);
            } else {
                const float x = D > 0.f ? dl : CUDART_INF_F;   // never left: no bound
                if (ARG) { if (x < ex[i]) { ex[i] = x; sb[i] = f; } }
                else ex[i] = fminf(ex[i], x);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < PIX; ++i) {
        sp[i] = __fmul_rn(__fsub_rn(ex[i], en[i]), rn[i]);   // +inf - inf, -inf: no hit
        if (!(sp[i] < CUDART_INF_F)) sp[i] = -1.f;
        if (ent_out) ent_out[i] = en[i];
    }
    }
}

template <int V, int PIX, bool ARG>
__device__ __forceinline__ void spans_x(const StagedX<V>& s, float lx0, float ly, const float* rn, float* sp,
                                        int* sf, int* sb, float* ent_out) {
    if (V == 6) {
        switch (s.nf) {
            case 1: spans_x_nf<V, PIX, 1, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 2: spans_x_nf<V, PIX, 2, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 3: spans_x_nf<V, PIX, 3, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 4: spans_x_nf<V, PIX, 4, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 5: spans_x_nf<V, PIX, 5, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 6: spans_x_nf<V, PIX, 6, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 7: spans_x_nf<V, PIX, 7, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            default: spans_x_nf<V, PIX, 0, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
        }
    } else {
        switch (s.nf) {
            case 1: spans_x_nf<V, PIX, 1, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 2: spans_x_nf<V, PIX, 2, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            case 3: spans_x_nf<V, PIX, 3, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
            default: spans_x_nf<V, PIX, 0, ARG>(s, lx0, ly, rn, sp, sf, sb, ent_out); break;
        }
    }
}

__device__ __forceinline__ float ray_norm(const CamDev& cm, int px, int py) {
    const float rx = ((float)px + 0.5f - cm.cx) / cm.fx;
    const float ry = ((float)py + 0.5f - cm.cy) / cm.fy;
    return sqrtf(1.f + rx * rx + ry * ry);
}

// MODE 0: image; 1: also the pair counters; 2: depth pass.
template <int V, int MODE, int TILE>
__global__ void __launch_bounds__(threads_x<TILE>()) k_blend_fwd_x(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, float* __restrict__ image,
    uint32_t* __restrict__ last_out, float* __restrict__ tl_out, int* __restrict__ tile_counter,
    unsigned long long* __restrict__ pair_counts, float* __restrict__ depth_out,
    uint32_t* __restrict__ contrib, uint32_t cstride, const uint32_t* __restrict__ order) {
    constexpr int PIX = pix_x<TILE>(), NT = threads_x<TILE>(), RW = TILE / PIX, BATCH = kBatchX;
    constexpr bool COUNT = MODE == 1, DEPTH = MODE == 2;
    constexpr float kStop = DEPTH ? 0.5f : kStopT;
    __shared__ StagedX<V> sm[BATCH];
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int ly = tid / RW, lx0 = (tid % RW) * PIX;
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
        const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
        const int py = tg.ty0 + ly;
        const uint2 rg = ranges[tile];
        const int n = (int)(rg.y - rg.x);
        float T[PIX], c0[PIX], c1[PIX], c2[PIX], tl[PIX], rn[PIX], dep[PIX];
        uint32_t last[PIX];
        bool done[PIX];
        bool tdone = true;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            T[i] = 1.f; c0[i] = c1[i] = c2[i] = 0.f; tl[i] = 1.f; last[i] = 0; dep[i] = 0.f;
            rn[i] = ray_norm(cm, tg.tx0 + lx0 + i, py);
            done[i] = !(tg.tx0 + lx0 + i < tg.width && py < tg.height);
            tdone &= done[i];
        }
        for (int b0 = 0; b0 < n; b0 += BATCH) {
            if (__syncthreads_count(!tdone) == 0) break;
            const int nb = min(BATCH, n - b0);
            for (int j = tid; j < nb; j += NT) stage_record_x<V>(rec, vals[rg.x + b0 + j], tg.tx0, tg.ty0, sm[j]);
            __syncthreads();
            if (__any_sync(0xffffffffu, !tdone)) {   // warp-uniform, as the exit below
                bool stop = false;
                for (int jw = 0; jw < nb && !stop; jw += 32) {
                  uint32_t bm = 0;   // bit j - jw: this thread blended entry b0 + j
                  const int je = min(nb, jw + 32);
                  for (int j = jw; j < je; ++j) {
                    const StagedX<V>& p = sm[j];
                    if (COUNT) {
#pragma unroll
                        for (int i = 0; i < PIX; ++i) n_iter += !done[i];
                    }
                    float sp[PIX], en[PIX];
                    spans_x<V, PIX, false>(p, (float)lx0 + p.dx0, (float)ly + p.dy0, rn, sp, nullptr, nullptr,
                                           DEPTH ? en : nullptr);
                    tdone = true;
                    bool blended = false;
#pragma unroll
                    for (int i = 0; i < PIX; ++i) {
                        const bool in = !done[i];
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
                            if (DEPTH && done[i]) dep[i] = __fmul_rn(__fadd_rn(p.cz, en[i]), rn[i]);
                        }
                        tdone &= done[i];
                    }
                    if (write_mask && blended) bm |= 1u << (j - jw);
                    // warp-uniform exit (the mask reduction below needs every lane)
                    if (__all_sync(0xffffffffu, tdone)) { stop = true; break; }
                  }
                  if (write_mask) {
                      // this warp's bits for entries b0 + jw .. b0 + jw + 31 of the list
                      bm = __reduce_or_sync(0xffffffffu, bm);
                      if (lane == 0 && bm) {
                          const uint32_t e0 = rg.x + (uint32_t)(b0 + jw);
                          const uint32_t w = e0 >> 5, sh = e0 & 31u;
                          uint32_t* cw = contrib + (size_t)(tid >> 5) * cstride;
                          atomicOr(cw + w, bm << sh);
                          if (sh) atomicOr(cw + w + 1, bm >> (32u - sh));
                      }
                  }
                }
            }
        }
        if (COUNT) {
#pragma unroll
            for (int i = 0; i < PIX; ++i) n_iter_last += last[i];
        }
        const int plane = tg.width * tg.height;
        float* img = image + 3 * (size_t)tg.pix_base;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            const int px = tg.tx0 + lx0 + i;
            if (!(px < tg.width && py < tg.height)) continue;
            const int idx = py * tg.width + px;
            if (DEPTH) {
                depth_out[tg.pix_base + idx] = dep[i];
                continue;
            }
            img[idx] = fmaf(T[i], bg0, c0[i]);
            img[plane + idx] = fmaf(T[i], bg1, c1[i]);
            img[2 * plane + idx] = fmaf(T[i], bg2, c2[i]);
            last_out[tg.pix_base + idx] = last[i];
            tl_out[tg.pix_base + idx] = tl[i];
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

// Backward: the blend recurrences are those of the ray-space mode; the span
// s = (delta_out - delta_in) |d| of a face f with delta = N / D, N = 1 - c_z L,
// D = L + D0, L = p X + q Y + L0 (X, Y the pixel offsets from the anchor) has
//   d delta/dL = -(c_z + delta)/D,  d delta/dD0 = -delta/D,  d delta/dc_z = -L/D.
template <int V, int TILE>
__global__ void __launch_bounds__(threads_x<TILE>()) k_blend_bwd_x(
    const float* __restrict__ rec, const uint32_t* __restrict__ vals, const uint2* __restrict__ ranges,
    CamsParam cams, float bg0, float bg1, float bg2, const float* __restrict__ dimage,
    const uint32_t* __restrict__ last_in, const float* __restrict__ tl_in, float* __restrict__ acc,
    int* __restrict__ tile_counter, const uint32_t* __restrict__ contrib, uint32_t cstride,
    const uint32_t* __restrict__ order) {
    constexpr int F = Kind<V>::F;
    constexpr int ACC = AccX<V>::kFloats;
    constexpr int PIX = pix_x<TILE>(), NT = threads_x<TILE>(), RW = TILE / PIX, BATCH = kBatchX;
    __shared__ StagedX<V> sm[BATCH];
    __shared__ int s_tile;
    __shared__ int s_max;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int ly = tid / RW, lx0 = (tid % RW) * PIX;
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
        const CamDev& cm = cams.cam[camera_of_tile(cams, tile)];
        const int py = tg.ty0 + ly;
        const uint2 rg = ranges[tile];
        const int plane = tg.width * tg.height;
        const float* gi = dimage + 3 * (size_t)tg.pix_base;
        float g0[PIX], g1[PIX], g2[PIX], Tcur[PIX], B0[PIX], B1[PIX], B2[PIX], rn[PIX];
        uint32_t last[PIX];
        bool first[PIX];
        uint32_t lmax = 0;
#pragma unroll
        for (int i = 0; i < PIX; ++i) {
            const int px = tg.tx0 + lx0 + i;
            g0[i] = g1[i] = g2[i] = 0.f; Tcur[i] = 1.f; last[i] = 0;
            rn[i] = ray_norm(cm, px, py);
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
            __syncthreads();
            for (int j = tid; j < nb; j += NT) stage_record_x<V>(rec, vals[rg.x + lo + j], tg.tx0, tg.ty0, sm[j]);
            __syncthreads();
            for (int j = nb - 1; j >= 0; --j) {
                const StagedX<V>& p = sm[j];
                const uint32_t idx = (uint32_t)(lo + j);
                if (contrib) {
                    // the forward blended this entry at none of this warp's pixels
                    const uint32_t e = rg.x + idx;
                    const uint32_t* cw = contrib + (size_t)(tid >> 5) * cstride;
                    if (!((__ldg(cw + (e >> 5)) >> (e & 31u)) & 1u)) continue;
                }
                bool any = false;
#pragma unroll
                for (int i = 0; i < PIX; ++i) any |= idx < last[i];
                if (__ballot_sync(0xffffffffu, any) == 0u) continue;
                float sp[PIX];
                int sf[PIX], sb[PIX];
                bool c[PIX];
                bool anyc = false;
                spans_x<V, PIX, true>(p, (float)lx0 + p.dx0, (float)ly + p.dy0, rn, sp, sf, sb, nullptr);
#pragma unroll
                for (int i = 0; i < PIX; ++i) {
                    c[i] = idx < last[i] && sp[i] > 0.f;
                    anyc |= c[i];
                }
                if (__ballot_sync(0xffffffffu, anyc) == 0u) continue;
                // per contributing pixel: the entry and exit faces' terms
                // dL/d(p, q, L0, D0); per thread: rgb, sigma, c_z sums
                float ge[PIX][4], gx[PIX][4];
                float h0 = 0.f, h1 = 0.f, h2 = 0.f, hs = 0.f, hz = 0.f;
#pragma unroll
                for (int i = 0; i < PIX; ++i) {
#pragma unroll
                    for (int m = 0; m < 4; ++m) ge[i][m] = gx[i][m] = 0.f;
                    if (!c[i]) continue;
                    const float xs = span_x(p.sigma, sp[i]);
                    const float tau = span_tau(xs);
                    const float o = span_opacity(xs, tau);
                    const float Ti = first[i] ? Tcur[i] : __fdividef(Tcur[i], tau);
                    first[i] = false;
                    Tcur[i] = Ti;
                    const float w = Ti * o;
                    h0 = fmaf(w, g0[i], h0);
                    h1 = fmaf(w, g1[i], h1);
                    h2 = fmaf(w, g2[i], h2);
                    const float dLdo = Ti * ((p.r - B0[i]) * g0[i] + (p.g - B1[i]) * g1[i] + (p.b - B2[i]) * g2[i]);
                    B0[i] = fmaf(o, p.r, tau * B0[i]);
                    B1[i] = fmaf(o, p.g, tau * B1[i]);
                    B2[i] = fmaf(o, p.b, tau * B2[i]);
                    hs = fmaf(dLdo * sp[i], tau, hs);                     // dL/dsigma
                    const float gs = dLdo * p.sigma * tau * rn[i];        // dL/d(delta_out - delta_in)
                    const float X = (float)(lx0 + i) + p.dx0, Y = (float)ly + p.dy0;
#pragma unroll
                    for (int side = 0; side < 2; ++side) {
                        const int f = side ? sb[i] : sf[i];
                        const float gd = side ? gs : -gs;
                        float4 pl = p.pl[0];
#pragma unroll
                        for (int ff = 1; ff < F; ++ff)
                            if (ff == f) pl = p.pl[ff];
                        const float L = __fmaf_rn(pl.x, X, __fmaf_rn(pl.y, Y, pl.z));
                        const float D = __fadd_rn(L, pl.w);
                        const float iD = 1.f / D;
                        const float dl = __fmaf_rn(-p.cz, L, 1.f) * iD;
                        const float gL = -gd * (p.cz + dl) * iD;
                        float* t = side ? gx[i] : ge[i];
                        t[0] = gL * X;
                        t[1] = gL * Y;
                        t[2] = gL;
                        t[3] = -gd * dl * iD;
                        hz = fmaf(-gd * L, iD, hz);                       // dL/dc_z
                    }
                }
                if (!anyc) continue;
                // each contributing lane adds its own rows, one 16-byte vector
                // atomic each: colour and density, c_z, and a face's four
                // terms once per run of the lane's pixels sharing that face
                float* Ag = acc + (size_t)p.rec * ACC;
                atomicAdd(reinterpret_cast<float4*>(Ag + 4 * F), make_float4(h0, h1, h2, hs));
                atomicAdd(Ag + 4 * F + 4, hz);
                float4 re = make_float4(0.f, 0.f, 0.f, 0.f), rb = re;
                int fe = -1, fb = -1;
#pragma unroll
                for (int i = 0; i < PIX; ++i) {
                    if (!c[i]) continue;
                    if (sf[i] != fe) {
                        if (fe >= 0) atomicAdd(reinterpret_cast<float4*>(Ag + 4 * fe), re);
                        fe = sf[i];
                        re = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    if (sb[i] != fb) {
                        if (fb >= 0) atomicAdd(reinterpret_cast<float4*>(Ag + 4 * fb), rb);
                        fb = sb[i];
                        rb = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    re.x += ge[i][0]; re.y += ge[i][1]; re.z += ge[i][2]; re.w += ge[i][3];
                    rb.x += gx[i][0]; rb.y += gx[i][1]; rb.z += gx[i][2]; rb.w += gx[i][3];
                }
                atomicAdd(reinterpret_cast<float4*>(Ag + 4 * fe), re);
                atomicAdd(reinterpret_cast<float4*>(Ag + 4 * fb), rb);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- chain
template <int V, int DEG>
__global__ void __launch_bounds__(128) k_chain_x(PrimsDev P, CamsParam cams, const float* __restrict__ rec,
                                                 const uint32_t* __restrict__ counts,
                                                 const float* __restrict__ acc, float* __restrict__ dcentre,
                                                 float* __restrict__ dverts, float* __restrict__ dopacity,
                                                 float* __restrict__ dsh, int accumulate) {
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
    float dmin = CUDART_INF_F;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float dx = v[k][0] - c[0], dy = v[k][1] - c[1], dz = v[k][2] - c[2];
        dmin = fminf(dmin, sqrtf(dx * dx + dy * dy + dz * dz));
    }
    float gc[3] = {0.f, 0.f, 0.f}, gv[V][3], gsh[K * 3], gsigma = 0.f;
#pragma unroll
    for (int k = 0; k < V; ++k) gv[k][0] = gv[k][1] = gv[k][2] = 0.f;
#pragma unroll
    for (int q = 0; q < K * 3; ++q) gsh[q] = 0.f;
    float vg_sum = 0.f;     // view-space position-gradient norms of the visible views

    // the cameras that see the primitive, from tile counts read up front
    uint32_t vis = 0;
#pragma unroll 8
    for (int cv = 0; cv < cams.n; ++cv) vis |= (counts[(size_t)cv * P.n + i] != 0u ? 1u : 0u) << cv;
    const uint32_t vg_count = __popc(vis);

    while (vis) {
        const int cv = __ffs(vis) - 1;
        vis &= vis - 1;
        const size_t r = (size_t)cv * P.n + i;
        const float* A = acc + r * AccX<V>::kFloats;
        // face order read with the row (top four bits always zero; the test
        // keeps the load ahead of the branch)
        const uint32_t meta = __float_as_uint(rec[r * RecX<V>::kFloats + 3]);
        bool any = (meta >> 28) != 0u;
#pragma unroll
        for (int q = 0; q < AccX<V>::kFloats; ++q) any |= A[q] != 0.f;
        if (!any) continue;
        const CamDev& cm = cams.cam[cv];
        Geom g;
        centre_geom(cm, c, g);
        float d[V][3];
#pragma unroll
        for (int k = 0; k < V; ++k) vertex_offset(cm, v[k], c, d[k]);
        float gd[V][3];
#pragma unroll
        for (int k = 0; k < V; ++k) gd[k][0] = gd[k][1] = gd[k][2] = 0.f;
        // The hit lambda = h / (n . d) of a face does not depend on the centre:
        // the centre-relative form only serves precision, and its centre terms
        // (through D0, c_z and the anchor) cancel exactly.  Only the partial
        // derivatives with the centre held fixed are taken, which are the
        // vertices' total derivatives; the centre gets the colour's gradient.
        const float cx = g.tc[0], cy = g.tc[1], icz = 1.f / g.tc[2];
#pragma unroll
        for (int s = 0; s < F; ++s) {
            const float Gp = A[4 * s], Gq = A[4 * s + 1], GL0 = A[4 * s + 2], GD0 = A[4 * s + 3];
            if (Gp == 0.f && Gq == 0.f && GL0 == 0.f && GD0 == 0.f) continue;
            const int f = meta_face(meta, s);
            int i0, i1, i2;
            face_vertices<V>(f, i0, i1, i2);
            float n[3];
            face_normal(d[i0], d[i1], d[i2], n);
            const float h = n[0] * d[i0][0] + n[1] * d[i0][1] + n[2] * d[i0][2];
            if (h == 0.f) continue;
            const float ih = 1.f / h;
            const float np[3] = {n[0] * ih, n[1] * ih, n[2] * ih};
            // L0 = -(p fxo + q fyo); p = n'_x / fx, q = n'_y / fy, D0 = n' . c / c_z
            const float Gpt = Gp - g.fxo * GL0, Gqt = Gq - g.fyo * GL0;
            float G[3] = {Gpt / cm.fx + GD0 * cx * icz, Gqt / cm.fy + GD0 * cy * icz, GD0};
            // n' = n / h with h = n . d0
            const float Gn = G[0] * np[0] + G[1] * np[1] + G[2] * np[2];
            float gn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gn[a] = (G[a] - Gn * d[i0][a]) * ih;
                gd[i0][a] -= Gn * np[a];
            }
            // n = e1 x e2
            const float e1[3] = {d[i1][0] - d[i0][0], d[i1][1] - d[i0][1], d[i1][2] - d[i0][2]};
            const float e2[3] = {d[i2][0] - d[i0][0], d[i2][1] - d[i0][1], d[i2][2] - d[i0][2]};
            const float g1[3] = {e2[1] * gn[2] - e2[2] * gn[1], e2[2] * gn[0] - e2[0] * gn[2],
                                 e2[0] * gn[1] - e2[1] * gn[0]};
            const float g2[3] = {gn[1] * e1[2] - gn[2] * e1[1], gn[2] * e1[0] - gn[0] * e1[2],
                                 gn[0] * e1[1] - gn[1] * e1[0]};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gd[i1][a] += g1[a];
                gd[i2][a] += g2[a];
                gd[i0][a] -= g1[a] + g2[a];
            }
        }
        // d_k = R (v_k - c)
#pragma unroll
        for (int k = 0; k < V; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                gv[k][a] += cm.R[a] * gd[k][0] + cm.R[3 + a] * gd[k][1] + cm.R[6 + a] * gd[k][2];

        // colour -> SH coefficients and view direction (as in the ray-space mode)
        float dir[3] = {c[0] - cm.campos[0], c[1] - cm.campos[1], c[2] - cm.campos[2]};
        const float dist = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
        const float idl = 1.f / dist;
        dir[0] *= idl; dir[1] *= idl; dir[2] *= idl;
        float Y[16];
        sh_basis<DEG>(dir[0], dir[1], dir[2], Y);
        float grgb[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float s = 0.5f;
#pragma unroll
            for (int k = 0; k < K; ++k) s = fmaf(Y[k], sh[3 * k + ch], s);
            grgb[ch] = s > 0.f ? A[4 * F + ch] : 0.f;
        }
        float wk[16];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            wk[k] = sh[3 * k] * grgb[0] + sh[3 * k + 1] * grgb[1] + sh[3 * k + 2] * grgb[2];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) gsh[3 * k + ch] += Y[k] * grgb[ch];
        }
        float gdir[3];
        sh_basis_vjp<DEG>(dir[0], dir[1], dir[2], wk, gdir);
        const float dd = gdir[0] * dir[0] + gdir[1] * dir[1] + gdir[2] * dir[2];
        float gw[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gw[a] = (gdir[a] - dir[a] * dd) * idl;
            gc[a] += gw[a];
        }
        if (P.grad_sum) {
            // a translation moves every vertex: camera-space gradient sum_k gd_k
            // plus the colour's
            float gt[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gt[a] = cm.R[3 * a] * gw[0] + cm.R[3 * a + 1] * gw[1] + cm.R[3 * a + 2] * gw[2];
#pragma unroll
                for (int k = 0; k < V; ++k) gt[a] += gd[k][a];
            }
            vg_sum += ndc_grad_norm(cm, gt, g.tc[2]);
        }
        gsigma += A[4 * F + 3];
    }
    if (P.grad_sum) {
        P.grad_sum[i] += vg_sum;
        P.grad_count[i] += vg_count;
    }
    const float galpha = gsigma != 0.f ? gsigma * kAlphaScale / ((1.f - kAlphaScale * alpha) * 2.f * dmin) : 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float& o = dcentre[3 * (size_t)i + a];
        o = accumulate ? o + gc[a] : gc[a];
    }
#pragma unroll
    for (int k = 0; k < V; ++k)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float& o = dverts[((size_t)i * V + k) * 3 + a];
            o = accumulate ? o + gv[k][a] : gv[k][a];
        }
    dopacity[i] = accumulate ? dopacity[i] + galpha : galpha;
#pragma unroll
    for (int q = 0; q < K * 3; ++q) {
        float& o = dsh[(size_t)i * K * 3 + q];
        o = accumulate ? o + gsh[q] : gsh[q];
    }
}

template <int V, int DEG>
cudaError_t pre_x_t(const PrimsDev& P, const CamsParam& cams, float* rec, uint32_t* counts, int4* trect,
                    uint32_t* zbits, cudaStream_t st) {
    const int grid = (P.n + 127) / 128;
    if (grid > 0) k_preprocess_x<V, DEG><<<grid, 128, 0, st>>>(P, cams, rec, counts, trect, zbits);
    return cudaGetLastError();
}

template <int V, int DEG>
cudaError_t chain_x_t(const PrimsDev& P, const CamsParam& cams, const float* rec, const uint32_t* counts,
                      const float* acc,
                      float* dc, float* dv, float* dop, float* dsh, int accumulate, cudaStream_t st) {
    const int grid = (P.n + 127) / 128;
    if (grid > 0) k_chain_x<V, DEG><<<grid, 128, 0, st>>>(P, cams, rec, counts, acc, dc, dv, dop, dsh, accumulate);
    return cudaGetLastError();
}

}  // namespace

int rec_floats_x(int V) { return V == 6 ? RecX<6>::kFloats : RecX<4>::kFloats; }
int acc_floats_x(int V) { return V == 6 ? AccX<6>::kFloats : AccX<4>::kFloats; }

#define LP_X_DISPATCH(V, DEG, CALL)                                      \
    switch (DEG) {                                                       \
        case 0: return (V == 6) ? CALL(6, 0) : CALL(4, 0);               \
        case 1: return (V == 6) ? CALL(6, 1) : CALL(4, 1);               \
        case 2: return (V == 6) ? CALL(6, 2) : CALL(4, 2);               \
        default: return (V == 6) ? CALL(6, 3) : CALL(4, 3);              \
    }

cudaError_t launch_preprocess_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                                uint32_t* counts, int4* trect, uint32_t* zbits, cudaStream_t st) {
#define CALL(v, d) pre_x_t<v, d>(P, cams, rec, counts, trect, zbits, st)
    LP_X_DISPATCH(V, deg, CALL)
#undef CALL
}

cudaError_t launch_chain_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, const float* rec,
                           const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop, float* dsh,
                           int accumulate, cudaStream_t st) {
#define CALL(v, d) chain_x_t<v, d>(P, cams, rec, counts, acc, dc, dv, dop, dsh, accumulate, st)
    LP_X_DISPATCH(V, deg, CALL)
#undef CALL
}

namespace {

template <int TILE>
cudaError_t fwd_x_t(int V, const BlendArgs& a, cudaStream_t st) {
#define FWD(v, m)                                                                                        \
    k_blend_fwd_x<v, m, TILE><<<a.grid, threads_x<TILE>(), 0, st>>>(                                    \
        a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.image, a.last, a.tl, a.tile_counter, \
        a.pair_counts, a.depth, m == 2 ? nullptr : a.contrib, a.contrib_stride, a.order)
    const int m = a.depth ? 2 : (a.count ? 1 : 0);
    if (V == 6) {
        if (m == 2) FWD(6, 2); else if (m == 1) FWD(6, 1); else FWD(6, 0);
    } else {
        if (m == 2) FWD(4, 2); else if (m == 1) FWD(4, 1); else FWD(4, 0);
    }
#undef FWD
    return cudaGetLastError();
}

template <int TILE>
cudaError_t bwd_x_t(int V, const BlendArgs& a, cudaStream_t st) {
    if (V == 6)
        k_blend_bwd_x<6, TILE><<<a.grid, threads_x<TILE>(), 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.dimage, a.last, a.tl, a.acc,
            a.tile_counter, a.contrib, a.contrib_stride, a.order);
    else
        k_blend_bwd_x<4, TILE><<<a.grid, threads_x<TILE>(), 0, st>>>(
            a.rec, a.vals, a.ranges, *a.cams, a.bg[0], a.bg[1], a.bg[2], a.dimage, a.last, a.tl, a.acc,
            a.tile_counter, a.contrib, a.contrib_stride, a.order);
    return cudaGetLastError();
}

template <int TILE>
int occ_x_t(int V, bool fwd) {
    int nb = 0;
    if (V == 6)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd ? (const void*)k_blend_fwd_x<6, 0, TILE>
                                                               : (const void*)k_blend_bwd_x<6, TILE>,
                                                      threads_x<TILE>(), 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd ? (const void*)k_blend_fwd_x<4, 0, TILE>
                                                               : (const void*)k_blend_bwd_x<4, TILE>,
                                                      threads_x<TILE>(), 0);
    return nb;
}

}  // namespace

cudaError_t launch_blend_fwd_x(int tile, int V, const BlendArgs& a, cudaStream_t st) {
    return tile == 8 ? fwd_x_t<8>(V, a, st) : tile == 32 ? fwd_x_t<32>(V, a, st) : fwd_x_t<16>(V, a, st);
}

cudaError_t launch_blend_bwd_x(int tile, int V, const BlendArgs& a, cudaStream_t st) {
    return tile == 8 ? bwd_x_t<8>(V, a, st) : tile == 32 ? bwd_x_t<32>(V, a, st) : bwd_x_t<16>(V, a, st);
}

int blend_x_occupancy(int tile, int V, bool fwd) {
    return tile == 8 ? occ_x_t<8>(V, fwd) : tile == 32 ? occ_x_t<32>(V, fwd) : occ_x_t<16>(V, fwd);
}

}  // namespace lp
