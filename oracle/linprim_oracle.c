/*
 * FP64 CPU oracle for the LinPrim rasterizer (arXiv 2501.16312).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use this file.  It shares no code, header,
 * constant or helper with the CUDA rasterizer package.
 *
 * It is a plain, slow, brute-force restatement of the paper's forward and
 * backward pass, in the order the paper gives them:
 *
 *   Sec. 3.2 "Preprocessing"  view transform; EWA 3D affine ray-space map
 *                             around the centre (App. "Ray Space
 *                             Approximation"); view-dependent SH colour as in
 *                             3DGS (Sec. 3.1 "Memory Requirements");
 *                             screen-space bounding box.
 *   Sec. 3.2 "Global Sorting and Tiling"  per-tile keys (tile, depth),
 *                             approximate front-to-back order by centre depth.
 *   Sec. 3.2 "Rasterization"  per pixel ray: Moeller-Trumbore intersection
 *                             (MTIA) with every triangular face in ray space
 *                             (ray direction +z); 0 or 2 hits; density Eq. 1.
 *   App. "Gradient Computation", opacity o = 1 - exp(-sigma (i2 - i1)).
 *   Sec. 3.2 "Compositing"    front-to-back alpha blending, stop once the
 *                             cumulative opacity reaches 0.999.
 *   Sec. 3.4 + App. "Gradient Computation"  backward: blending -> (alpha,
 *                             colour) -> intersection depths -> ray-space
 *                             corners through the MTIA barycentric
 *                             derivatives -> world space; the density
 *                             normalisation d_min carries no gradient
 *                             (App. "Experimental Setting").
 *
 * Readings where the paper is silent (pixel centres at x+0.5, principal point,
 * OpenCV axes, culling at centre depth <= 0.2, key layout, tie order, stop
 * rule inclusive of the primitive that crosses the threshold, colour clamp at
 * zero) are each marked "reading" where they apply below.
 *
 * Integers decided by floating point (culling, depth key, pixel/tile
 * rectangle) are computed in IEEE binary32 with a fixed operation order and no
 * contraction (compile with -ffp-contract=off); everything else is binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_V 6
#define ORC_MAX_F 8
#define ORC_STOP_T 1e-3      /* Sec. 3.2: stop at cumulative opacity 0.999 */
#define ORC_NEAR 0.2f        /* reading: cull when centre depth <= 0.2 */

typedef struct {
    int nv;                  /* vertices per primitive: 6 octahedron, 4 tetrahedron */
    int n;                   /* number of primitives */
    int sh_degree;           /* 0..3 */
    const double* centre;    /* [n][3] world */
    const double* verts;     /* [n][nv][3] world */
    const double* opacity;   /* [n], alpha in [0,1) */
    const double* sh;        /* [n][(deg+1)^2][3] */
    const double* dmin;      /* optional [n] frozen density normaliser, or NULL */
    double aa_kernel;        /* 2D anti-aliasing filter size in pixels (Sec. 3.3), 0 = off */
    int exact;               /* 1: no ray-space approximation (App. "Ray Space Approximation") */
} orc_prims;

typedef struct {
    double viewmat[16];      /* world -> camera, row-major, OpenCV axes */
    double fx, fy, cx, cy;
    int width, height;
} orc_camera;

/* Face topology.  Octahedron vertices are (+a0,-a0,+a1,-a1,+a2,-a2); each face
 * takes one vertex per axis (Sec. 3.1).  A tetrahedron face omits one vertex. */
static const int OCTA_FACES[8][3] = {
    {0, 2, 4}, {0, 2, 5}, {0, 3, 4}, {0, 3, 5},
    {1, 2, 4}, {1, 2, 5}, {1, 3, 4}, {1, 3, 5}};
static const int TETRA_FACES[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

static int n_faces(int nv) { return nv == 6 ? 8 : 4; }
static const int* face_vertices(int nv, int f) {
    return nv == 6 ? OCTA_FACES[f] : TETRA_FACES[f];
}

/* ------------------------------------------------------------------ SH basis
 * Real spherical harmonics up to degree 3 in the 3DGS ordering and sign
 * convention (Sec. 3.1: colours "following the same approach described in
 * 3DGS"): index l*l + l + m, basis = (-1)^m times the standard real SH.  The
 * normalisation constants are written as their closed forms. */
static void sh_basis(int degree, const double d[3], double Y[16], double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    const double c0 = 0.5 / sqrt(pi);
    const double c1 = sqrt(3.0 / (4.0 * pi));
    const double c2a = 0.5 * sqrt(15.0 / pi);
    const double c2b = 0.25 * sqrt(5.0 / pi);
    const double c2c = 0.25 * sqrt(15.0 / pi);
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double c3b = 0.5 * sqrt(105.0 / pi);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c3d = 0.25 * sqrt(7.0 / pi);
    const double c3e = 0.25 * sqrt(105.0 / pi);
    double x = d[0], y = d[1], z = d[2];
    int k;
    for (k = 0; k < 16; ++k) {
        Y[k] = 0.0;
        if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    }
#define SETD(k, a, b, c) do { if (dY) { dY[k][0] = (a); dY[k][1] = (b); dY[k][2] = (c); } } while (0)
    Y[0] = c0;
    if (degree < 1) return;
    Y[1] = -c1 * y;            SETD(1, 0.0, -c1, 0.0);
    Y[2] = c1 * z;             SETD(2, 0.0, 0.0, c1);
    Y[3] = -c1 * x;            SETD(3, -c1, 0.0, 0.0);
    if (degree < 2) return;
    Y[4] = c2a * x * y;        SETD(4, c2a * y, c2a * x, 0.0);
    Y[5] = -c2a * y * z;       SETD(5, 0.0, -c2a * z, -c2a * y);
    Y[6] = c2b * (2 * z * z - x * x - y * y);
                               SETD(6, -2 * c2b * x, -2 * c2b * y, 4 * c2b * z);
    Y[7] = -c2a * x * z;       SETD(7, -c2a * z, 0.0, -c2a * x);
    Y[8] = c2c * (x * x - y * y);
                               SETD(8, 2 * c2c * x, -2 * c2c * y, 0.0);
    if (degree < 3) return;
    Y[9] = -c3a * y * (3 * x * x - y * y);
                               SETD(9, -c3a * 6 * x * y, -c3a * (3 * x * x - 3 * y * y), 0.0);
    Y[10] = c3b * x * y * z;   SETD(10, c3b * y * z, c3b * x * z, c3b * x * y);
    Y[11] = -c3c * y * (4 * z * z - x * x - y * y);
                               SETD(11, -c3c * (-2 * x * y), -c3c * (4 * z * z - x * x - 3 * y * y),
                                    -c3c * (8 * y * z));
    Y[12] = c3d * z * (2 * z * z - 3 * x * x - 3 * y * y);
                               SETD(12, c3d * (-6 * x * z), c3d * (-6 * y * z),
                                    c3d * (6 * z * z - 3 * x * x - 3 * y * y));
    Y[13] = -c3c * x * (4 * z * z - x * x - y * y);
                               SETD(13, -c3c * (4 * z * z - 3 * x * x - y * y), -c3c * (-2 * x * y),
                                    -c3c * (8 * x * z));
    Y[14] = c3e * z * (x * x - y * y);
                               SETD(14, c3e * 2 * x * z, -c3e * 2 * y * z, c3e * (x * x - y * y));
    Y[15] = -c3a * x * (x * x - 3 * y * y);
                               SETD(15, -c3a * (3 * x * x - 3 * y * y), -c3a * (-6 * x * y), 0.0);
#undef SETD
}

/* Threads of the OpenMP loops over pixels (n <= 0: all processors); returns
 * the count in effect, 1 when built without OpenMP.  Timing only. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_sh_basis(int degree, const double dir[3], double* Y, double* dY) {
    double y[16], dy[16][3];
    int k;
    sh_basis(degree, dir, y, dY ? dy : NULL);
    for (k = 0; k < 16; ++k) {
        Y[k] = y[k];
        if (dY) { dY[3 * k] = dy[k][0]; dY[3 * k + 1] = dy[k][1]; dY[3 * k + 2] = dy[k][2]; }
    }
    return 0;
}

/* -------------------------------------------------- FP32 key-field replay
 * The integers the rasterizer derives from floating point -- culling, the
 * centre-depth key and the pixel rectangle of the projected bounding box
 * (Sec. 3.2 "Preprocessing", last step) -- are taken in binary32 with this
 * exact operation order, each operation rounded once. */
typedef struct {
    int visible;
    uint32_t zbits;
    int px0, px1, py0, py1;     /* inclusive pixel rectangle; empty if px0 > px1 */
    int shx[ORC_MAX_V], shy[ORC_MAX_V];   /* 2D filter: outward shift direction of each vertex */
    float shift;                /* 2D filter: shift in pixels */
} orc_keyfields;

/* Sec. 3.3 2D filter: vertices on the bounding box move outward by this many
 * pixels, parallel to the screen.  Reading: an octahedron's opposite vertices
 * mirror the move, so each moves by half the kernel size; a tetrahedron
 * vertex moves by the full kernel size.  Rounded once to binary32. */
static float aa_shift_f32(const orc_prims* P) {
    return (float)(P->nv == 6 ? 0.5 * P->aa_kernel : P->aa_kernel);
}

static void f32_transform(const float M[12], const float x[3], float t[3]) {
    int i;
    for (i = 0; i < 3; ++i) {
        float a = M[4 * i + 0] * x[0];
        float b = M[4 * i + 1] * x[1];
        float c = M[4 * i + 2] * x[2];
        float s = a + b;
        s = s + c;
        t[i] = s + M[4 * i + 3];
    }
}

static float f32_max(const float* q, int n) {
    float m = -INFINITY;
    int k;
    for (k = 0; k < n; ++k) if (q[k] > m) m = q[k];
    return m;
}

static float f32_min(const float* q, int n) {
    float m = INFINITY;
    int k;
    for (k = 0; k < n; ++k) if (q[k] < m) m = q[k];
    return m;
}

static void keyfields_f32(const orc_prims* P, const orc_camera* cam, int i, orc_keyfields* kf) {
    float M[12], c[3], tc[3];
    float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    float u, w, xc, yc, j00, j02, j11, j12;
    float qxmin = INFINITY, qxmax = -INFINITY, qymin = INFINITY, qymax = -INFINITY;
    float xmin, xmax, ymin, ymax, fx0, fx1, fy0, fy1;
    float qxs[ORC_MAX_V], qys[ORC_MAX_V];
    int k;
    for (k = 0; k < 12; ++k) M[k] = (float)cam->viewmat[k];
    for (k = 0; k < 3; ++k) c[k] = (float)P->centre[3 * i + k];
    f32_transform(M, c, tc);
    kf->visible = 0;
    kf->zbits = 0;
    kf->px0 = 1; kf->px1 = 0; kf->py0 = 1; kf->py1 = 0;
    kf->shift = 0.0f;
    for (k = 0; k < ORC_MAX_V; ++k) kf->shx[k] = kf->shy[k] = 0;
    memcpy(&kf->zbits, &tc[2], 4);
    if (!(tc[2] > ORC_NEAR)) return;
    /* reading: Eq. 1 divides by the smallest centre-vertex distance, so a
     * primitive with a vertex on its centre has no density; it is not visible */
    for (k = 0; k < P->nv; ++k) {
        const double* v = P->verts + (size_t)(i * P->nv + k) * 3;
        if ((float)v[0] == c[0] && (float)v[1] == c[1] && (float)v[2] == c[2]) return;
    }
    u = tc[0] / tc[2];
    w = tc[1] / tc[2];
    xc = fx * u; xc = xc + cx;
    yc = fy * w; yc = yc + cy;
    /* reading: only primitives in the view frustum are drawn (the "Frustum"
     * count of App. Table 7); the frustum is taken as the projected centre
     * within 1.3 times the image, normalised device coordinates in [-1.3, 1.3],
     * decided in binary32 on the key-field values */
    {
        const float W = (float)cam->width, H = (float)cam->height;
        const float lox = -0.15f * W, hix = 1.15f * W, loy = -0.15f * H, hiy = 1.15f * H;
        if (!(xc >= lox && xc <= hix && yc >= loy && yc <= hiy)) return;
    }
    kf->visible = 1;
    j00 = fx / tc[2]; j02 = -(j00 * u);
    j11 = fy / tc[2]; j12 = -(j11 * w);
    for (k = 0; k < P->nv; ++k) {
        float v[3], w[3], dd[3], d0, d2, d1, qx, qy, a, b;
        int m;
        /* vertex offset from the centre, rotated into the camera frame */
        for (m = 0; m < 3; ++m) v[m] = (float)P->verts[(size_t)(i * P->nv + k) * 3 + m];
        for (m = 0; m < 3; ++m) w[m] = v[m] - c[m];
        for (m = 0; m < 3; ++m) {
            float r0 = M[4 * m + 0] * w[0];
            float r1 = M[4 * m + 1] * w[1];
            float r2 = M[4 * m + 2] * w[2];
            float s = r0 + r1;
            dd[m] = s + r2;
        }
        d0 = dd[0]; d1 = dd[1]; d2 = dd[2];
        if (P->exact) {
            /* exact mode: the vertex's camera-space position tc + d and its
             * perspective projection, as offsets from the projected centre */
            float X = tc[0] + d0, Y = tc[1] + d1, Z = tc[2] + d2, uu, ww;
            if (!(Z > ORC_NEAR)) { kf->visible = 0; return; }   /* reading: every vertex in front */
            uu = X / Z; ww = Y / Z;
            qx = fx * uu; qx = qx + cx; qx = qx - xc;
            qy = fy * ww; qy = qy + cy; qy = qy - yc;
        } else {
        a = j00 * d0; b = j02 * d2; qx = a + b;
        a = j11 * d1; b = j12 * d2; qy = a + b;
        }
        qxs[k] = qx;
        qys[k] = qy;
        if (qx < qxmin) qxmin = qx;
        if (qx > qxmax) qxmax = qx;
        if (qy < qymin) qymin = qy;
        if (qy > qymax) qymax = qy;
    }
    if (P->aa_kernel > 0.0 && !P->exact) {
        /* Sec. 3.3 2D filter: the vertices on the box move outward (a vertex
         * on the maximum moves up; otherwise one on the minimum moves down),
         * and the box is taken again over the moved vertices */
        const float sh = aa_shift_f32(P);
        kf->shift = sh;
        qxmin = INFINITY; qxmax = -INFINITY; qymin = INFINITY; qymax = -INFINITY;
        for (k = 0; k < P->nv; ++k) {
            float qx = qxs[k], qy = qys[k];
            kf->shx[k] = qx == f32_max(qxs, P->nv) ? 1 : (qx == f32_min(qxs, P->nv) ? -1 : 0);
            kf->shy[k] = qy == f32_max(qys, P->nv) ? 1 : (qy == f32_min(qys, P->nv) ? -1 : 0);
            if (kf->shx[k] > 0) qx = qx + sh;
            else if (kf->shx[k] < 0) qx = qx - sh;
            if (kf->shy[k] > 0) qy = qy + sh;
            else if (kf->shy[k] < 0) qy = qy - sh;
            if (qx < qxmin) qxmin = qx;
            if (qx > qxmax) qxmax = qx;
            if (qy < qymin) qymin = qy;
            if (qy > qymax) qymax = qy;
        }
    }
    xmin = xc + qxmin; xmax = xc + qxmax;
    ymin = yc + qymin; ymax = yc + qymax;
    /* reading: pixel p is covered when its centre p + 0.5 lies in [min, max] */
    fx0 = ceilf(xmin - 0.5f);  fx1 = floorf(xmax - 0.5f);
    fy0 = ceilf(ymin - 0.5f);  fy1 = floorf(ymax - 0.5f);
    fx0 = fmaxf(fx0, 0.0f);    fx1 = fminf(fx1, (float)(cam->width - 1));
    fy0 = fmaxf(fy0, 0.0f);    fy1 = fminf(fy1, (float)(cam->height - 1));
    if (fx0 > fx1 || fy0 > fy1) return;     /* rectangle stays empty */
    kf->px0 = (int)fx0; kf->px1 = (int)fx1;
    kf->py0 = (int)fy0; kf->py1 = (int)fy1;
}

/* --------------------------------------------------------- FP64 preprocess */
typedef struct {
    orc_keyfields kf;
    double tc[3];               /* camera-space centre */
    double tv[ORC_MAX_V][3];    /* camera-space vertices */
    double J[3][3];             /* EWA Jacobian of the ray-space map at tc */
    double pc[3];               /* ray-space centre phi(tc) */
    double p[ORC_MAX_V][3];     /* ray-space vertices phi(tc) + J (tv - tc) */
    double dmin, sigma;
    double dir[3], dist;        /* unit world view direction, |c - campos| */
    int exact;                  /* spans by the true perspective ray (p = tv) */
    double fx, fy, cx, cy;      /* intrinsics, for the exact ray direction */
    double rgb_raw[3], rgb[3];
} orc_pp;

static void cam_rotation(const orc_camera* cam, double R[3][3], double T[3]) {
    int i, j;
    for (i = 0; i < 3; ++i) {
        for (j = 0; j < 3; ++j) R[i][j] = cam->viewmat[4 * i + j];
        T[i] = cam->viewmat[4 * i + 3];
    }
}

static void transform64(const double R[3][3], const double T[3], const double* x, double t[3]) {
    int i;
    for (i = 0; i < 3; ++i) t[i] = R[i][0] * x[0] + R[i][1] * x[1] + R[i][2] * x[2] + T[i];
}

/* EWA ray-space map (App. "Ray Space Approximation"):
 *   phi(t) = (fx tx/tz + cx, fy ty/tz + cy, |t|),
 * linearised around the camera-space centre: J = d phi / d t at tc. */
static void ewa_jacobian(const orc_camera* cam, const double t[3], double J[3][3]) {
    double tz = t[2], len = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    J[0][0] = cam->fx / tz; J[0][1] = 0.0;          J[0][2] = -cam->fx * t[0] / (tz * tz);
    J[1][0] = 0.0;          J[1][1] = cam->fy / tz; J[1][2] = -cam->fy * t[1] / (tz * tz);
    J[2][0] = t[0] / len;   J[2][1] = t[1] / len;   J[2][2] = t[2] / len;
}

static int sh_count(int degree) { return (degree + 1) * (degree + 1); }

static void preprocess(const orc_prims* P, const orc_camera* cam, int i, orc_pp* pp) {
    double R[3][3], T[3], campos[3], d[3], Y[16];
    int k, m, ch, K = sh_count(P->sh_degree);
    const double* c = P->centre + 3 * i;
    keyfields_f32(P, cam, i, &pp->kf);
    cam_rotation(cam, R, T);
    transform64(R, T, c, pp->tc);
    ewa_jacobian(cam, pp->tc, pp->J);
    pp->pc[0] = cam->fx * pp->tc[0] / pp->tc[2] + cam->cx;
    pp->pc[1] = cam->fy * pp->tc[1] / pp->tc[2] + cam->cy;
    pp->pc[2] = sqrt(pp->tc[0] * pp->tc[0] + pp->tc[1] * pp->tc[1] + pp->tc[2] * pp->tc[2]);
    pp->dmin = INFINITY;
    for (k = 0; k < P->nv; ++k) {
        const double* v = P->verts + (size_t)(i * P->nv + k) * 3;
        double dv[3], r;
        transform64(R, T, v, pp->tv[k]);
        for (m = 0; m < 3; ++m) dv[m] = pp->tv[k][m] - pp->tc[m];
        for (m = 0; m < 3; ++m)
            pp->p[k][m] = pp->pc[m] + pp->J[m][0] * dv[0] + pp->J[m][1] * dv[1] + pp->J[m][2] * dv[2];
        r = sqrt((v[0] - c[0]) * (v[0] - c[0]) + (v[1] - c[1]) * (v[1] - c[1]) +
                 (v[2] - c[2]) * (v[2] - c[2]));
        if (r < pp->dmin) pp->dmin = r;
    }
    pp->exact = P->exact;
    pp->fx = cam->fx; pp->fy = cam->fy; pp->cx = cam->cx; pp->cy = cam->cy;
    if (P->exact) {
        /* no ray-space map: the primitive stays in camera space */
        for (k = 0; k < P->nv; ++k)
            for (m = 0; m < 3; ++m) pp->p[k][m] = pp->tv[k][m];
        for (m = 0; m < 3; ++m) pp->pc[m] = pp->tc[m];
    }
    /* Sec. 3.3 2D filter: move the vertices the binary32 box chose outward,
     * parallel to the screen (no-op when the filter is off) */
    for (k = 0; k < P->nv; ++k) {
        pp->p[k][0] += pp->kf.shx[k] * (double)pp->kf.shift;
        pp->p[k][1] += pp->kf.shy[k] * (double)pp->kf.shift;
    }
    /* Eq. 1 generalised to both kinds: d_min is the smallest centre-vertex
     * distance (for an octahedron this is min(d_x, d_y, d_z)). */
    if (P->dmin) pp->dmin = P->dmin[i];
    pp->sigma = -log1p(-0.99 * P->opacity[i]) / (2.0 * pp->dmin);
    /* camera position in world: -R^T T */
    for (m = 0; m < 3; ++m) campos[m] = -(R[0][m] * T[0] + R[1][m] * T[1] + R[2][m] * T[2]);
    for (m = 0; m < 3; ++m) d[m] = c[m] - campos[m];
    pp->dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (m = 0; m < 3; ++m) pp->dir[m] = d[m] / pp->dist;
    sh_basis(P->sh_degree, pp->dir, Y, NULL);
    for (ch = 0; ch < 3; ++ch) {
        double s = 0.0;
        for (k = 0; k < K; ++k) s += Y[k] * P->sh[((size_t)i * K + k) * 3 + ch];
        pp->rgb_raw[ch] = s + 0.5;
        pp->rgb[ch] = pp->rgb_raw[ch] > 0.0 ? pp->rgb_raw[ch] : 0.0;
    }
}

/* ------------------------------------------------------------------- MTIA
 * Moeller-Trumbore with ray origin r = (rx, ry, 0) and direction (0, 0, 1) in
 * ray space.  With e1 = p1 - p0, e2 = p2 - p0 and s = r - p0:
 *   det = -(e1 x e2)_z,  u = (s . (D x e2)) / det,  v = (D . (s x e1)) / det,
 * and the hit depth is the barycentric interpolation
 *   i = (1 - u - v) p0z + u p1z + v p2z.
 * Returns 1 on a hit (u, v >= 0, u + v <= 1, det != 0). */
static int mtia(const double p0[3], const double p1[3], const double p2[3], double rx, double ry,
                double* u_out, double* v_out, double* det_out, double* depth) {
    double e1x = p1[0] - p0[0], e1y = p1[1] - p0[1];
    double e2x = p2[0] - p0[0], e2y = p2[1] - p0[1];
    double sx = rx - p0[0], sy = ry - p0[1];
    double det = -e1x * e2y + e1y * e2x;
    double u, v;
    if (det == 0.0) return 0;
    u = (-sx * e2y + sy * e2x) / det;
    v = (sx * e1y - sy * e1x) / det;
    *u_out = u; *v_out = v; *det_out = det;
    *depth = (1.0 - u - v) * p0[2] + u * p1[2] + v * p2[2];
    return u >= 0.0 && v >= 0.0 && u + v <= 1.0;
}

/* Gradient of the hit depth w.r.t. the three corners (App. "Gradient
 * Computation"): the z-components are the barycentrics (1-u-v, u, v); the
 * x/y-components chain through du/dp and dv/dp, which follow from
 * u = Nu/det, v = Nv/det as  du/dq = (dNu/dq - u ddet/dq)/det  (same for v).
 * For corner 0 this is the printed formula; corners 1, 2 are the analogues. */
static void mtia_grad(const double p0[3], const double p1[3], const double p2[3], double rx,
                      double ry, double di[3][3]) {
    double u, v, det, depth;
    double dNu[3][2], dNv[3][2], dD[3][2];
    int k, a;
    mtia(p0, p1, p2, rx, ry, &u, &v, &det, &depth);
    /* corner 0 */
    dD[0][0] = p2[1] - p1[1];   dD[0][1] = p1[0] - p2[0];
    dNu[0][0] = p2[1] - ry;     dNu[0][1] = rx - p2[0];
    dNv[0][0] = ry - p1[1];     dNv[0][1] = p1[0] - rx;
    /* corner 1 */
    dD[1][0] = -(p2[1] - p0[1]); dD[1][1] = p2[0] - p0[0];
    dNu[1][0] = 0.0;             dNu[1][1] = 0.0;
    dNv[1][0] = -(ry - p0[1]);   dNv[1][1] = rx - p0[0];
    /* corner 2 */
    dD[2][0] = p1[1] - p0[1];    dD[2][1] = -(p1[0] - p0[0]);
    dNu[2][0] = ry - p0[1];      dNu[2][1] = -(rx - p0[0]);
    dNv[2][0] = 0.0;             dNv[2][1] = 0.0;
    for (k = 0; k < 3; ++k) {
        for (a = 0; a < 2; ++a) {
            double du = (dNu[k][a] - u * dD[k][a]) / det;
            double dv = (dNv[k][a] - v * dD[k][a]) / det;
            di[k][a] = -(du + dv) * p0[2] + du * p1[2] + dv * p2[2];
        }
    }
    di[0][2] = 1.0 - u - v;
    di[1][2] = u;
    di[2][2] = v;
}

/* Test hook: one triangle / ray.  out = {hit, u, v, det, depth},
 * grad = d depth / d (p0, p1, p2), row-major [3][3]. */
int orc_mtia(const double* p0, const double* p1, const double* p2, double rx, double ry,
             double* out, double* grad) {
    double u = 0, v = 0, det = 0, depth = 0, di[3][3];
    int hit = mtia(p0, p1, p2, rx, ry, &u, &v, &det, &depth), k, a;
    out[0] = hit; out[1] = u; out[2] = v; out[3] = det; out[4] = depth;
    if (grad && det != 0.0) {
        mtia_grad(p0, p1, p2, rx, ry, di);
        for (k = 0; k < 3; ++k)
            for (a = 0; a < 3; ++a) grad[3 * k + a] = di[k][a];
    }
    return hit;
}

/* Exact mode (App. "Ray Space Approximation", the variant without it): the
 * pixel ray from the camera centre (the camera-space origin) along
 * d = ((rx - cx)/fx, (ry - cy)/fy, 1), intersected with the camera-space
 * triangle by Moller-Trumbore; lam is the ray parameter (the hit is lam d). */
static int mtia_ray(const double p0[3], const double p1[3], const double p2[3], const double d[3],
                    double* lam) {
    double e1[3], e2[3], pv[3], tv[3], qv[3], det, u, v;
    int m;
    for (m = 0; m < 3; ++m) { e1[m] = p1[m] - p0[m]; e2[m] = p2[m] - p0[m]; tv[m] = -p0[m]; }
    pv[0] = d[1] * e2[2] - d[2] * e2[1];
    pv[1] = d[2] * e2[0] - d[0] * e2[2];
    pv[2] = d[0] * e2[1] - d[1] * e2[0];
    det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
    if (det == 0.0) return 0;
    u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) / det;
    qv[0] = tv[1] * e1[2] - tv[2] * e1[1];
    qv[1] = tv[2] * e1[0] - tv[0] * e1[2];
    qv[2] = tv[0] * e1[1] - tv[1] * e1[0];
    v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) / det;
    *lam = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) / det;
    return u >= 0.0 && v >= 0.0 && u + v <= 1.0 && *lam > 0.0;
}

/* d lam / d (p0, p1, p2) of the ray's hit with the triangle's plane: with
 * n = (p1 - p0) x (p2 - p0), lam = (p0 . n) / (d . n), so
 * d lam = [dp0 . n + (p0 - lam d) . dn] / (d . n), and with a = (p0 - lam d)/(d . n),
 * a . dn = de1 . (e2 x a) + de2 . (a x e1). */
static void mtia_ray_grad(const double p0[3], const double p1[3], const double p2[3], const double d[3],
                          double lam, double g[3][3]) {
    double e1[3], e2[3], n[3], a[3], dn;
    int m;
    for (m = 0; m < 3; ++m) { e1[m] = p1[m] - p0[m]; e2[m] = p2[m] - p0[m]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    dn = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    for (m = 0; m < 3; ++m) a[m] = (p0[m] - lam * d[m]) / dn;
    g[1][0] = e2[1] * a[2] - e2[2] * a[1];
    g[1][1] = e2[2] * a[0] - e2[0] * a[2];
    g[1][2] = e2[0] * a[1] - e2[1] * a[0];
    g[2][0] = a[1] * e1[2] - a[2] * e1[1];
    g[2][1] = a[2] * e1[0] - a[0] * e1[2];
    g[2][2] = a[0] * e1[1] - a[1] * e1[0];
    for (m = 0; m < 3; ++m) g[0][m] = n[m] / dn - g[1][m] - g[2][m];
}

static double exact_dir(const orc_pp* pp, double rx, double ry, double d[3]) {
    d[0] = (rx - pp->cx) / pp->fx;
    d[1] = (ry - pp->cy) / pp->fy;
    d[2] = 1.0;
    return sqrt(d[0] * d[0] + d[1] * d[1] + 1.0);
}

/* Span of the pixel ray through a primitive by MTIA over all faces (Sec. 3.2
 * "Rasterization"): i1 = nearest hit, i2 = farthest hit.  Returns 1 when the
 * ray crosses the primitive (two hits with i2 > i1). */
static int span_mtia(const orc_pp* pp, int nv, double rx, double ry, double* i1, double* i2,
                     int* f1, int* f2) {
    int f, F = n_faces(nv), nhit = 0;
    double lo = INFINITY, hi = -INFINITY, d[3], dl = 0.0;
    if (pp->exact) dl = exact_dir(pp, rx, ry, d);
    for (f = 0; f < F; ++f) {
        const int* fv = face_vertices(nv, f);
        double u, v, det, depth, lam;
        int hit;
        if (pp->exact) {
            hit = mtia_ray(pp->p[fv[0]], pp->p[fv[1]], pp->p[fv[2]], d, &lam);
            depth = lam * dl;   /* distance along the ray */
        } else {
            hit = mtia(pp->p[fv[0]], pp->p[fv[1]], pp->p[fv[2]], rx, ry, &u, &v, &det, &depth);
        }
        if (hit) {
            ++nhit;
            if (depth < lo) { lo = depth; *f1 = f; }
            if (depth > hi) { hi = depth; *f2 = f; }
        }
    }
    *i1 = lo; *i2 = hi;
    return nhit >= 2 && hi > lo;
}

/* Independent second formulation: clip the ray against the face half-spaces
 * of the convex primitive (entry = max over faces whose outward normal faces
 * the camera, exit = min over the others).  Used to cross-check MTIA and to
 * flag rays that graze the primitive.  lo2 / hi2 (may be NULL) receive the
 * second largest entry depth and the second smallest exit depth. */
static int span_clip2(const orc_pp* pp, int nv, double rx, double ry, double* i1, double* i2, double* lo2_out,
                      double* hi2_out) {
    int f, F = n_faces(nv);
    double lo = -INFINITY, hi = INFINITY, lo2 = -INFINITY, hi2 = INFINITY;
    if (pp->exact) {
        /* the ray lam d against each face's half-space n . t <= h (outward n) */
        double d[3], dl = exact_dir(pp, rx, ry, d);
        for (f = 0; f < F; ++f) {
            const int* fv = face_vertices(nv, f);
            const double *a = pp->p[fv[0]], *b = pp->p[fv[1]], *c = pp->p[fv[2]];
            double e1[3], e2[3], n[3], h, den;
            int m;
            for (m = 0; m < 3; ++m) { e1[m] = b[m] - a[m]; e2[m] = c[m] - a[m]; }
            n[0] = e1[1] * e2[2] - e1[2] * e2[1];
            n[1] = e1[2] * e2[0] - e1[0] * e2[2];
            n[2] = e1[0] * e2[1] - e1[1] * e2[0];
            if (n[0] * (a[0] - pp->pc[0]) + n[1] * (a[1] - pp->pc[1]) + n[2] * (a[2] - pp->pc[2]) < 0)
                for (m = 0; m < 3; ++m) n[m] = -n[m];
            h = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
            den = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
            if (den == 0.0) {
                if (h < 0.0) { *i1 = INFINITY; *i2 = -INFINITY; return 0; }
                continue;
            }
            if (den < 0) {
                const double t = h / den * dl;
                if (t > lo) { lo2 = lo; lo = t; } else if (t > lo2) lo2 = t;
            } else {
                const double t = h / den * dl;
                if (t < hi) { hi2 = hi; hi = t; } else if (t < hi2) hi2 = t;
            }
        }
        *i1 = lo; *i2 = hi;
        if (lo2_out) *lo2_out = lo2;
        if (hi2_out) *hi2_out = hi2;
        return hi > lo && lo > 0.0;
    }
    for (f = 0; f < F; ++f) {
        const int* fv = face_vertices(nv, f);
        const double *a = pp->p[fv[0]], *b = pp->p[fv[1]], *c = pp->p[fv[2]];
        double e1[3], e2[3], n[3], h, z;
        int m;
        for (m = 0; m < 3; ++m) { e1[m] = b[m] - a[m]; e2[m] = c[m] - a[m]; }
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        /* orient outward: the ray-space centre lies inside */
        if (n[0] * (a[0] - pp->pc[0]) + n[1] * (a[1] - pp->pc[1]) + n[2] * (a[2] - pp->pc[2]) < 0)
            for (m = 0; m < 3; ++m) n[m] = -n[m];
        h = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
        if (n[2] == 0.0) {
            if (n[0] * rx + n[1] * ry > h) { *i1 = INFINITY; *i2 = -INFINITY; return 0; }
            continue;
        }
        z = (h - n[0] * rx - n[1] * ry) / n[2];
        if (n[2] < 0) { if (z > lo) { lo2 = lo; lo = z; } else if (z > lo2) lo2 = z; }
        else          { if (z < hi) { hi2 = hi; hi = z; } else if (z < hi2) hi2 = z; }
    }
    *i1 = lo; *i2 = hi;
    if (lo2_out) *lo2_out = lo2;
    if (hi2_out) *hi2_out = hi2;
    return hi > lo;
}

static int span_clip(const orc_pp* pp, int nv, double rx, double ry, double* i1, double* i2) {
    return span_clip2(pp, nv, rx, ry, i1, i2, NULL, NULL);
}

/* ----------------------------------------------------------- per-camera set */
typedef struct {
    int n;
    orc_pp* pp;
    int* order;         /* visible primitives in ascending (depth bits, index) */
    int n_order;
    /* Sec. 3.2 "Global Sorting and Tiling": the primitives whose rectangle
     * meets each 16x16 tile of the image, in the order above.  A pixel's
     * candidates are those of its tile; the rectangle test in blend_pixel
     * rejects the rest of them exactly as it rejects every primitive outside
     * the tile, so each pixel visits the same primitives in the same order
     * as a walk over the whole sorted list would. */
    int tiles_x, tiles_y;
    long long* tile_start;   /* [tiles + 1] */
    int* tile_list;
} orc_view;

#define ORC_BIN 16

static const orc_pp* g_sort_pp;
static int cmp_depth(const void* a, const void* b) {
    int i = *(const int*)a, j = *(const int*)b;
    uint32_t zi = g_sort_pp[i].kf.zbits, zj = g_sort_pp[j].kf.zbits;
    if (zi != zj) return zi < zj ? -1 : 1;
    return (i > j) - (i < j);
}

static int view_build(const orc_prims* P, const orc_camera* cam, orc_view* V) {
    int i;
    V->n = P->n;
    V->tile_start = NULL;
    V->tile_list = NULL;
    V->pp = (orc_pp*)calloc((size_t)(P->n > 0 ? P->n : 1), sizeof(orc_pp));
    V->order = (int*)malloc(sizeof(int) * (size_t)(P->n > 0 ? P->n : 1));
    if (!V->pp || !V->order) return -1;
    V->n_order = 0;
    for (i = 0; i < P->n; ++i) {
        preprocess(P, cam, i, &V->pp[i]);
        if (V->pp[i].kf.visible) V->order[V->n_order++] = i;
    }
    /* Sec. 3.2 "Global Sorting and Tiling": approximate front-to-back order
     * by centre depth; reading: ties by primitive index. */
    g_sort_pp = V->pp;
    qsort(V->order, (size_t)V->n_order, sizeof(int), cmp_depth);
    /* per-tile candidate lists: count, prefix, fill in sorted order */
    {
        long long nt, t, total = 0;
        int pass, j, tx, ty;
        V->tiles_x = (cam->width + ORC_BIN - 1) / ORC_BIN;
        V->tiles_y = (cam->height + ORC_BIN - 1) / ORC_BIN;
        nt = (long long)V->tiles_x * V->tiles_y;
        V->tile_start = (long long*)calloc((size_t)(nt + 1), sizeof(long long));
        if (!V->tile_start) return -1;
        for (pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
                long long run = 0;
                for (t = 0; t < nt; ++t) {
                    long long c = V->tile_start[t];
                    V->tile_start[t] = run;
                    run += c;
                }
                V->tile_start[nt] = total = run;
                V->tile_list = (int*)malloc(sizeof(int) * (size_t)(total > 0 ? total : 1));
                if (!V->tile_list) return -1;
            }
            for (j = 0; j < V->n_order; ++j) {
                const orc_keyfields* kf = &V->pp[V->order[j]].kf;
                if (kf->px0 > kf->px1 || kf->py0 > kf->py1) continue;
                for (ty = kf->py0 / ORC_BIN; ty <= kf->py1 / ORC_BIN; ++ty)
                    for (tx = kf->px0 / ORC_BIN; tx <= kf->px1 / ORC_BIN; ++tx) {
                        t = (long long)ty * V->tiles_x + tx;
                        if (pass == 0) ++V->tile_start[t];
                        else V->tile_list[V->tile_start[t]++] = V->order[j];
                    }
            }
        }
        /* the fill advanced every start to the next tile's start */
        for (t = nt; t > 0; --t) V->tile_start[t] = V->tile_start[t - 1];
        V->tile_start[0] = 0;
    }
    return 0;
}

static void view_free(orc_view* V) {
    free(V->pp);
    free(V->order);
    free(V->tile_start);
    free(V->tile_list);
}

/* --------------------------------------------------------- per-pixel blend */
typedef struct {
    int prim, f1, f2;
    double i1, i2, s, tau, o, T;
} orc_contrib;

typedef struct {
    double rgb[3];
    int n_contrib;
    double T_final;
    int borderline;     /* bit 0: stop decision within 1e-3 (relative) of the threshold;
                           bit 1: the ray grazes a primitive's silhouette;
                           bit 2: the depth decision (T crossing 0.5) within 1e-4 of 0.5 */
    double min_span;    /* smallest span among contributors (diagnostic) */
    double depth;       /* App. "Depth and Surface Reconstruction": ray entry depth of the
                           first primitive after which the cumulative opacity exceeds 0.5;
                           0 when it never does */
} orc_pixel;

/* Forward for one pixel; fills `list` (capacity cap) with the contributors
 * in blend order.  Returns the number of contributors. */
static int blend_pixel(const orc_prims* P, const orc_view* V, const double bg[3], int x, int y,
                       orc_contrib* list, int cap, orc_pixel* out) {
    double rx = x + 0.5, ry = y + 0.5;   /* reading: sample at the pixel centre */
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int nc = 0, ch;
    out->borderline = 0;
    out->min_span = INFINITY;
    out->depth = 0.0;
    /* a pixel outside the image lies in no rectangle: no candidates */
    const int inside = x >= 0 && y >= 0 && x / ORC_BIN < V->tiles_x && y / ORC_BIN < V->tiles_y;
    const long long t = inside ? (long long)(y / ORC_BIN) * V->tiles_x + x / ORC_BIN : 0;
    const long long j_end = inside ? V->tile_start[t + 1] : 0;
    long long jj;
    for (jj = inside ? V->tile_start[t] : 0; jj < j_end; ++jj) {
        int i = V->tile_list[jj];
        const orc_pp* pp = &V->pp[i];
        double i1, i2, s, tau, o, Tn;
        int f1 = -1, f2 = -1;
        if (x < pp->kf.px0 || x > pp->kf.px1 || y < pp->kf.py0 || y > pp->kf.py1) continue;
        /* the colour is continuous across a silhouette but its derivative
         * with respect to the vertices is not (the span's derivative is
         * finite just inside and zero outside), so a ray passing within
         * rounding of a silhouette may take either side in binary32: flag
         * spans within 1e-5 of the primitive's depth extent of zero.  The
         * same holds across an edge between two entry faces or two exit
         * faces of a primitive the ray crosses: the span is continuous there
         * but its derivative follows whichever face bounds it, so a ray
         * whose two nearest entry (or exit) depths agree to within 1e-5 of
         * the depth extent is flagged too. */
        {
            double c1, c2, lo2, hi2, zlo = INFINITY, zhi = -INFINITY;
            int k;
            for (k = 0; k < P->nv; ++k) {
                if (pp->p[k][2] < zlo) zlo = pp->p[k][2];
                if (pp->p[k][2] > zhi) zhi = pp->p[k][2];
            }
            span_clip2(pp, P->nv, rx, ry, &c1, &c2, &lo2, &hi2);
            if (fabs(c2 - c1) <= 1e-5 * (zhi - zlo)) out->borderline |= 2;
            if (c2 > c1 && (c1 - lo2 <= 1e-5 * (zhi - zlo) || hi2 - c2 <= 1e-5 * (zhi - zlo)))
                out->borderline |= 2;
        }
        if (!span_mtia(pp, P->nv, rx, ry, &i1, &i2, &f1, &f2)) continue;
        s = i2 - i1;
        tau = exp(-pp->sigma * s);
        o = -expm1(-pp->sigma * s);            /* o = 1 - exp(-sigma s) */
        for (ch = 0; ch < 3; ++ch) C[ch] += T * o * pp->rgb[ch];
        Tn = T * tau;
        if (nc < cap) {
            orc_contrib* c = &list[nc];
            c->prim = i; c->f1 = f1; c->f2 = f2;
            c->i1 = i1; c->i2 = i2; c->s = s; c->tau = tau; c->o = o; c->T = T;
        }
        ++nc;
        if (s < out->min_span) out->min_span = s;
        /* the stop test is ambiguous in binary32 when T lands within 1e-3
         * (relative) of the threshold: the product of tens of binary32
         * transmittance factors, some from near-camera primitives whose
         * planes are evaluated far from their anchor, carries relative
         * errors of that order */
        if (fabs(Tn - ORC_STOP_T) <= 1e-3 * ORC_STOP_T) out->borderline |= 1;
        /* depth: the first primitive that takes the cumulative opacity 1 - T
         * above 0.5; reading: its distance is where the ray enters it */
        if (out->depth == 0.0 && T >= 0.5 && Tn < 0.5) out->depth = i1;
        if (fabs(Tn - 0.5) <= 1e-4 * 0.5) out->borderline |= 4;
        T = Tn;
        /* reading: the primitive that takes T below 1e-3 is blended, then stop */
        if (T < ORC_STOP_T) break;
    }
    for (ch = 0; ch < 3; ++ch) out->rgb[ch] = C[ch] + T * bg[ch];
    out->n_contrib = nc;
    out->T_final = T;
    return nc;
}

/* --------------------------------------------------------------- backward */
typedef struct {
    double dp[ORC_MAX_V][3];   /* dL / d ray-space vertex */
    double drgb[3];
    double dsigma;
    int touched;
} orc_pgrad;

static void blend_pixel_backward(const orc_prims* P, const orc_view* V, const double bg[3], int x,
                                 int y, const orc_contrib* list, int nc, const double g[3],
                                 orc_pgrad* G) {
    double rx = x + 0.5, ry = y + 0.5, B[3];
    int j, ch, k, a;
    for (ch = 0; ch < 3; ++ch) B[ch] = bg[ch];
    for (j = nc - 1; j >= 0; --j) {
        const orc_contrib* c = &list[j];
        const orc_pp* pp = &V->pp[c->prim];
        orc_pgrad* pg = &G[c->prim];
        double dL_do = 0.0, dL_ds, di1[3][3], di2[3][3];
        const int* fv1 = face_vertices(P->nv, c->f1);
        const int* fv2 = face_vertices(P->nv, c->f2);
        /* C = sum_i T_i o_i c_i + T_end bg, with T_{i+1} = T_i (1 - o_i):
         * dC/dc_i = T_i o_i;  dC/do_i = T_i (c_i - B_{i+1}),
         * B_i = o_i c_i + (1 - o_i) B_{i+1},  B_{end} = bg. */
        for (ch = 0; ch < 3; ++ch) {
            pg->drgb[ch] += c->T * c->o * g[ch];
            dL_do += c->T * (pp->rgb[ch] - B[ch]) * g[ch];
        }
        for (ch = 0; ch < 3; ++ch) B[ch] = c->o * pp->rgb[ch] + c->tau * B[ch];
        /* o = 1 - exp(-sigma s): do/ds = sigma tau, do/dsigma = s tau */
        dL_ds = dL_do * pp->sigma * c->tau;
        pg->dsigma += dL_do * c->s * c->tau;
        /* s = i2 - i1 */
        if (pp->exact) {
            /* i = lam |d|: d i / dp = |d| d lam / dp */
            double d[3], dl = exact_dir(pp, rx, ry, d);
            mtia_ray_grad(pp->p[fv1[0]], pp->p[fv1[1]], pp->p[fv1[2]], d, c->i1 / dl, di1);
            mtia_ray_grad(pp->p[fv2[0]], pp->p[fv2[1]], pp->p[fv2[2]], d, c->i2 / dl, di2);
            for (k = 0; k < 3; ++k)
                for (a = 0; a < 3; ++a) { di1[k][a] *= dl; di2[k][a] *= dl; }
        } else {
            mtia_grad(pp->p[fv1[0]], pp->p[fv1[1]], pp->p[fv1[2]], rx, ry, di1);
            mtia_grad(pp->p[fv2[0]], pp->p[fv2[1]], pp->p[fv2[2]], rx, ry, di2);
        }
        for (k = 0; k < 3; ++k)
            for (a = 0; a < 3; ++a) {
                pg->dp[fv1[k]][a] += -dL_ds * di1[k][a];
                pg->dp[fv2[k]][a] += dL_ds * di2[k][a];
            }
        pg->touched = 1;
    }
}

/* Chain one primitive's ray-space / colour / density gradients back to the
 * world-space features (Sec. 3.4 "Preprocessing Backpropagation"). */
static void chain_primitive(const orc_prims* P, const orc_camera* cam, int i, const orc_pp* pp,
                            const orc_pgrad* pg, double* dcentre, double* dverts, double* dopacity,
                            double* dsh) {
    double R[3][3], T[3], dtc[3] = {0, 0, 0}, dtv[ORC_MAX_V][3], dpc[3] = {0, 0, 0};
    double dJ[3][3] = {{0}}, Y[16], dY[16][3], ddir[3] = {0, 0, 0};
    int k, a, b, m, ch, K = sh_count(P->sh_degree);
    double tx = pp->tc[0], ty = pp->tc[1], tz = pp->tc[2];
    double len = pp->pc[2];
    cam_rotation(cam, R, T);
    if (pp->exact) {
        /* p_k = tv_k: the gradients are camera-space already; the centre
         * enters only through the colour (below) */
        for (k = 0; k < P->nv; ++k)
            for (a = 0; a < 3; ++a) dtv[k][a] = pg->dp[k][a];
    } else {
    /* p_k = phi(tc) + J(tc) (tv_k - tc) */
    for (k = 0; k < P->nv; ++k) {
        for (a = 0; a < 3; ++a) dtv[k][a] = 0.0;
        for (m = 0; m < 3; ++m) {
            double gm = pg->dp[k][m];
            dpc[m] += gm;
            for (a = 0; a < 3; ++a) {
                dtv[k][a] += pp->J[m][a] * gm;                    /* d/d tv_k */
                dtc[a] -= pp->J[m][a] * gm;                       /* -J part of d/d tc */
                dJ[m][a] += gm * (pp->tv[k][a] - pp->tc[a]);      /* d/dJ */
            }
        }
    }
    /* d phi / d tc = J */
    for (m = 0; m < 3; ++m)
        for (a = 0; a < 3; ++a) dtc[a] += pp->J[m][a] * dpc[m];
    /* dJ/dtc: J row 0 = (fx/tz, 0, -fx tx/tz^2), row 1 likewise, row 2 = t/|t| */
    dtc[2] += dJ[0][0] * (-cam->fx / (tz * tz));
    dtc[0] += dJ[0][2] * (-cam->fx / (tz * tz));
    dtc[2] += dJ[0][2] * (2.0 * cam->fx * tx / (tz * tz * tz));
    dtc[2] += dJ[1][1] * (-cam->fy / (tz * tz));
    dtc[1] += dJ[1][2] * (-cam->fy / (tz * tz));
    dtc[2] += dJ[1][2] * (2.0 * cam->fy * ty / (tz * tz * tz));
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            double d_ab = (a == b ? 1.0 : 0.0) - pp->tc[a] * pp->tc[b] / (len * len);
            dtc[b] += dJ[2][a] * d_ab / len;
        }
    }
    /* camera space -> world: t = R x + T */
    for (a = 0; a < 3; ++a) {
        double s = 0.0;
        for (m = 0; m < 3; ++m) s += R[m][a] * dtc[m];
        dcentre[3 * i + a] += s;
    }
    for (k = 0; k < P->nv; ++k)
        for (a = 0; a < 3; ++a) {
            double s = 0.0;
            for (m = 0; m < 3; ++m) s += R[m][a] * dtv[k][m];
            dverts[(size_t)(i * P->nv + k) * 3 + a] += s;
        }
    /* colour: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5), dir = (c - campos)/|c - campos| */
    sh_basis(P->sh_degree, pp->dir, Y, dY);
    for (ch = 0; ch < 3; ++ch) {
        double gc = pp->rgb_raw[ch] > 0.0 ? pg->drgb[ch] : 0.0;
        for (k = 0; k < K; ++k) {
            dsh[((size_t)i * K + k) * 3 + ch] += Y[k] * gc;
            for (a = 0; a < 3; ++a) ddir[a] += dY[k][a] * P->sh[((size_t)i * K + k) * 3 + ch] * gc;
        }
    }
    for (a = 0; a < 3; ++a) {
        double s = 0.0;
        for (b = 0; b < 3; ++b)
            s += ((a == b ? 1.0 : 0.0) - pp->dir[a] * pp->dir[b]) * ddir[b];
        dcentre[3 * i + a] += s / pp->dist;
    }
    /* density, Eq. 1, d_min frozen: d sigma / d alpha = 0.99 / ((1 - 0.99 alpha) 2 d_min) */
    dopacity[i] += pg->dsigma * 0.99 / ((1.0 - 0.99 * P->opacity[i]) * 2.0 * pp->dmin);
}

/* ------------------------------------------------------------ public entry */
#define ORC_LIST_CAP 65536

/* Render the listed pixels of one camera.  rgb_out [npix][3] (may be NULL),
 * info_out [npix][4] = {n_contrib, T_final, borderline, min_span} (may be
 * NULL).  If dL_dC [npix][3] is given, the gradients of L = sum dL_dC . rgb
 * are ADDED into dcentre/dverts/dopacity/dsh. */
int orc_render_pixels(const orc_prims* P, const orc_camera* cam, const double* bg, long long npix,
                      const int* px, const int* py, double* rgb_out, double* info_out,
                      const double* dL_dC, double* dcentre, double* dverts, double* dopacity,
                      double* dsh) {
    orc_view V;
    orc_pgrad* G = NULL;
    long long q;
    int i, rc = 0;
    if (view_build(P, cam, &V)) return -1;
    if (dL_dC) {
        G = (orc_pgrad*)calloc((size_t)(P->n > 0 ? P->n : 1), sizeof(orc_pgrad));
        if (!G) { view_free(&V); return -1; }
    }
#pragma omp parallel
    {
        orc_contrib* list = (orc_contrib*)malloc(sizeof(orc_contrib) * ORC_LIST_CAP);
        orc_pgrad* Gl = NULL;
        if (G) Gl = (orc_pgrad*)calloc((size_t)(P->n > 0 ? P->n : 1), sizeof(orc_pgrad));
        if (!list || (G && !Gl)) {
#pragma omp atomic write
            rc = -1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (q = 0; q < npix; ++q) {
                orc_pixel o;
                int nc = blend_pixel(P, &V, bg, px[q], py[q], list, ORC_LIST_CAP, &o);
                if (nc > ORC_LIST_CAP) {
#pragma omp atomic write
                    rc = -2;
                }
                if (rgb_out) { rgb_out[3 * q] = o.rgb[0]; rgb_out[3 * q + 1] = o.rgb[1]; rgb_out[3 * q + 2] = o.rgb[2]; }
                if (info_out) {
                    info_out[4 * q] = o.n_contrib; info_out[4 * q + 1] = o.T_final;
                    info_out[4 * q + 2] = o.borderline; info_out[4 * q + 3] = o.min_span;
                }
                if (G && nc <= ORC_LIST_CAP)
                    blend_pixel_backward(P, &V, bg, px[q], py[q], list, nc, dL_dC + 3 * q, Gl);
            }
            if (G) {
#pragma omp critical
                {
                    int p2, k, a;
                    for (p2 = 0; p2 < P->n; ++p2) {
                        if (!Gl[p2].touched) continue;
                        G[p2].touched = 1;
                        G[p2].dsigma += Gl[p2].dsigma;
                        for (a = 0; a < 3; ++a) G[p2].drgb[a] += Gl[p2].drgb[a];
                        for (k = 0; k < P->nv; ++k)
                            for (a = 0; a < 3; ++a) G[p2].dp[k][a] += Gl[p2].dp[k][a];
                    }
                }
            }
        }
        free(list);
        free(Gl);
    }
    if (G && rc == 0)
        for (i = 0; i < P->n; ++i)
            if (G[i].touched) chain_primitive(P, cam, i, &V.pp[i], &G[i], dcentre, dverts, dopacity, dsh);
    free(G);
    view_free(&V);
    return rc;
}

/* Whole images, packed [cam][3][H][W]; info [cam][H][W][4] as above (may be
 * NULL).  With dL_dimage (same layout as image) the gradients are ADDED. */
int orc_render(const orc_prims* P, const orc_camera* cams, int ncams, const double* bg,
               double* image, double* info, const double* dL_dimage, double* dcentre,
               double* dverts, double* dopacity, double* dsh) {
    long long off = 0;
    int c;
    for (c = 0; c < ncams; ++c) {
        long long W = cams[c].width, H = cams[c].height, npix = W * H, q;
        int* px = (int*)malloc(sizeof(int) * (size_t)(npix > 0 ? npix : 1));
        int* py = (int*)malloc(sizeof(int) * (size_t)(npix > 0 ? npix : 1));
        double* rgb = (double*)malloc(sizeof(double) * 3 * (size_t)(npix > 0 ? npix : 1));
        double* g = dL_dimage ? (double*)malloc(sizeof(double) * 3 * (size_t)(npix > 0 ? npix : 1)) : NULL;
        int rc, ch;
        if (!px || !py || !rgb || (dL_dimage && !g)) return -1;
        for (q = 0; q < npix; ++q) {
            px[q] = (int)(q % W);
            py[q] = (int)(q / W);
            if (g)
                for (ch = 0; ch < 3; ++ch) g[3 * q + ch] = dL_dimage[3 * off + ch * npix + q];
        }
        rc = orc_render_pixels(P, &cams[c], bg, npix, px, py, rgb, info ? info + 4 * off : NULL, g,
                               dcentre, dverts, dopacity, dsh);
        if (rc) return rc;
        if (image)
            for (q = 0; q < npix; ++q)
                for (ch = 0; ch < 3; ++ch) image[3 * off + ch * npix + q] = rgb[3 * q + ch];
        free(px); free(py); free(rgb); free(g);
        off += npix;
    }
    return 0;
}

/* Depth map of the listed pixels of one camera: depth_out[q] as defined in
 * orc_pixel, flags_out[q] the pixel's borderline word. */
int orc_depth_pixels(const orc_prims* P, const orc_camera* cam, long long npix, const int* px,
                     const int* py, double* depth_out, int* flags_out) {
    orc_view V;
    long long q;
    int rc = 0;
    if (view_build(P, cam, &V)) return -1;
#pragma omp parallel
    {
        orc_contrib* list = (orc_contrib*)malloc(sizeof(orc_contrib) * ORC_LIST_CAP);
        if (!list) {
#pragma omp atomic write
            rc = -1;
        } else {
#pragma omp for schedule(dynamic, 64)
            for (q = 0; q < npix; ++q) {
                orc_pixel o;
                const double bg[3] = {0.0, 0.0, 0.0};
                blend_pixel(P, &V, bg, px[q], py[q], list, ORC_LIST_CAP, &o);
                depth_out[q] = o.depth;
                if (flags_out) flags_out[q] = o.borderline;
            }
        }
        free(list);
    }
    view_free(&V);
    return rc;
}

/* ----------------------------------------------------------- keys / sorting
 * Sec. 3.2 "Global Sorting and Tiling" with the 3DGS key: each visible
 * primitive emits one entry per tile of its rectangle (tiles in row-major
 * order, primitives in record order view * n + i); key = (global tile << 32)
 * | depth bits, value = record index; entries are stably sorted by key. */
typedef struct { uint64_t key; uint32_t val; long long seq; } orc_entry;

static int cmp_entry(const void* a, const void* b) {
    const orc_entry *x = (const orc_entry*)a, *y = (const orc_entry*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->seq > y->seq) - (x->seq < y->seq);
}

int orc_keys(const orc_prims* P, const orc_camera* cams, int ncams, int tile, uint64_t* keys,
             uint32_t* vals, long long cap, long long* n_out, uint32_t* counts) {
    long long n = 0, tile_base = 0, q;
    orc_entry* E = NULL;
    int pass, c, i;
    for (pass = 0; pass < 2; ++pass) {
        n = 0;
        tile_base = 0;
        for (c = 0; c < ncams; ++c) {
            int tiles_x = (cams[c].width + tile - 1) / tile;
            int tiles_y = (cams[c].height + tile - 1) / tile;
            for (i = 0; i < P->n; ++i) {
                orc_keyfields kf;
                int tx, ty, cnt = 0;
                keyfields_f32(P, &cams[c], i, &kf);
                if (kf.visible && kf.px0 <= kf.px1 && kf.py0 <= kf.py1) {
                    for (ty = kf.py0 / tile; ty <= kf.py1 / tile; ++ty)
                        for (tx = kf.px0 / tile; tx <= kf.px1 / tile; ++tx) {
                            if (pass == 1) {
                                uint64_t gt = (uint64_t)(tile_base + (long long)ty * tiles_x + tx);
                                E[n].key = (gt << 32) | kf.zbits;
                                E[n].val = (uint32_t)((long long)c * P->n + i);
                                E[n].seq = n;
                            }
                            ++n;
                            ++cnt;
                        }
                }
                if (pass == 0 && counts) counts[(size_t)c * P->n + i] = (uint32_t)cnt;
            }
            tile_base += (long long)tiles_x * tiles_y;
        }
        if (pass == 0) {
            E = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)(n > 0 ? n : 1));
            if (!E) return -1;
        }
    }
    qsort(E, (size_t)n, sizeof(orc_entry), cmp_entry);
    *n_out = n;
    for (q = 0; q < n && q < cap; ++q) { keys[q] = E[q].key; vals[q] = E[q].val; }
    free(E);
    return n > cap ? -2 : 0;
}

/* ---------------------------------------------------------- test accessors */

/* Per-primitive preprocess for one camera.  out [n][16]:
 * {visible, zbits, px0, px1, py0, py1, pc.x, pc.y, pc.z, sigma, dmin,
 *  rgb.r, rgb.g, rgb.b, dist, 0}; pverts [n][nv][3] ray-space vertices. */
int orc_preprocess(const orc_prims* P, const orc_camera* cam, double* out, double* pverts) {
    int i, k, m;
    for (i = 0; i < P->n; ++i) {
        orc_pp pp;
        double* o = out + 16 * (size_t)i;
        preprocess(P, cam, i, &pp);
        o[0] = pp.kf.visible; o[1] = (double)pp.kf.zbits;
        o[2] = pp.kf.px0; o[3] = pp.kf.px1; o[4] = pp.kf.py0; o[5] = pp.kf.py1;
        o[6] = pp.pc[0]; o[7] = pp.pc[1]; o[8] = pp.pc[2];
        o[9] = pp.sigma; o[10] = pp.dmin;
        o[11] = pp.rgb[0]; o[12] = pp.rgb[1]; o[13] = pp.rgb[2]; o[14] = pp.dist; o[15] = 0.0;
        if (pverts)
            for (k = 0; k < P->nv; ++k)
                for (m = 0; m < 3; ++m) pverts[((size_t)i * P->nv + k) * 3 + m] = pp.p[k][m];
    }
    return 0;
}

/* Span of the pixel ray (rx, ry) through primitive i under both formulations.
 * out = {hit_mtia, i1, i2, hit_clip, c1, c2}. */
int orc_span(const orc_prims* P, const orc_camera* cam, int i, double rx, double ry, double* out) {
    orc_pp pp;
    double i1 = 0, i2 = 0, c1 = 0, c2 = 0;
    int f1 = -1, f2 = -1;
    preprocess(P, cam, i, &pp);
    out[0] = span_mtia(&pp, P->nv, rx, ry, &i1, &i2, &f1, &f2);
    out[1] = i1; out[2] = i2;
    out[3] = span_clip(&pp, P->nv, rx, ry, &c1, &c2);
    out[4] = c1; out[5] = c2;
    return 0;
}

/* ------------------------------------------------------ parameter layer
 * Sec. 3.1: a primitive is its centre c, a rotation quaternion q = (w, x, y,
 * z) (normalised), per-corner distances and an opacity logit; vertices are
 *   octahedron  v_{2i} = c + d_i R e_i,  v_{2i+1} = c - d_i R e_i  (i = 0..2)
 *   tetrahedron v_k   = c + d_k R b_k   (b_k: the four regular directions)
 * and alpha = sigmoid(logit).  Reading: distances are linear (the paper
 * scales their learning rate by the scene extent, App. "Experimental
 * Setting"), so they are used as given. */
static void quat_to_R(const double q_in[4], double R[3][3], double* norm) {
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
    *norm = n;
}

static void tetra_dir(int k, double b[3]) {
    static const double s[4][3] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
    double r = 1.0 / sqrt(3.0);
    b[0] = s[k][0] * r; b[1] = s[k][1] * r; b[2] = s[k][2] * r;
}

/* Local direction of vertex k (before scaling by its distance) and the
 * distance index it uses. */
static void vertex_dir(int nv, int k, double e[3], int* di, double* sign) {
    if (nv == 6) {
        e[0] = e[1] = e[2] = 0.0;
        e[k / 2] = 1.0;
        *di = k / 2;
        *sign = (k % 2) ? -1.0 : 1.0;
    } else {
        tetra_dir(k, e);
        *di = k;
        *sign = 1.0;
    }
}

int orc_params_forward(int nv, int n, const double* centre, const double* quat, const double* dist,
                       const double* logit, double* verts, double* opacity) {
    int i, k, a, nd = nv == 6 ? 3 : 4;
    for (i = 0; i < n; ++i) {
        double R[3][3], qn;
        quat_to_R(quat + 4 * (size_t)i, R, &qn);
        for (k = 0; k < nv; ++k) {
            double e[3], s;
            int di;
            vertex_dir(nv, k, e, &di, &s);
            for (a = 0; a < 3; ++a) {
                double r = R[a][0] * e[0] + R[a][1] * e[1] + R[a][2] * e[2];
                verts[((size_t)i * nv + k) * 3 + a] = centre[3 * i + a] + s * dist[(size_t)i * nd + di] * r;
            }
        }
        opacity[i] = 1.0 / (1.0 + exp(-logit[i]));
    }
    return 0;
}

/* Adjoint of orc_params_forward.  dcentre is ADDED to (it may already hold
 * the renderer's direct centre gradient); dquat, ddist, dlogit are written. */
int orc_params_backward(int nv, int n, const double* quat, const double* dist, const double* logit,
                        const double* dverts, const double* dopacity, double* dcentre, double* dquat,
                        double* ddist, double* dlogit) {
    int i, k, a, b, nd = nv == 6 ? 3 : 4;
    for (i = 0; i < n; ++i) {
        const double* q = quat + 4 * (size_t)i;
        double R[3][3], dR[3][3] = {{0}}, qn, w, x, y, z, g[4], dot;
        quat_to_R(q, R, &qn);
        for (k = 0; k < nd; ++k) ddist[(size_t)i * nd + k] = 0.0;
        for (k = 0; k < nv; ++k) {
            double e[3], s, r[3];
            int di;
            const double* gv = dverts + ((size_t)i * nv + k) * 3;
            vertex_dir(nv, k, e, &di, &s);
            for (a = 0; a < 3; ++a) r[a] = R[a][0] * e[0] + R[a][1] * e[1] + R[a][2] * e[2];
            for (a = 0; a < 3; ++a) dcentre[3 * i + a] += gv[a];
            ddist[(size_t)i * nd + di] += s * (r[0] * gv[0] + r[1] * gv[1] + r[2] * gv[2]);
            for (a = 0; a < 3; ++a)
                for (b = 0; b < 3; ++b) dR[a][b] += s * dist[(size_t)i * nd + di] * gv[a] * e[b];
        }
        /* R(q_hat) with q_hat = q / |q| */
        w = q[0] / qn; x = q[1] / qn; y = q[2] / qn; z = q[3] / qn;
        g[0] = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        g[1] = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2] +
                    z * dR[2][0] + w * dR[2][1] - 2 * x * dR[2][2]);
        g[2] = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                    w * dR[2][0] + z * dR[2][1] - 2 * y * dR[2][2]);
        g[3] = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1] +
                    y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        dot = g[0] * w + g[1] * x + g[2] * y + g[3] * z;
        dquat[4 * (size_t)i + 0] = (g[0] - dot * w) / qn;
        dquat[4 * (size_t)i + 1] = (g[1] - dot * x) / qn;
        dquat[4 * (size_t)i + 2] = (g[2] - dot * y) / qn;
        dquat[4 * (size_t)i + 3] = (g[3] - dot * z) / qn;
        {
            double al = 1.0 / (1.0 + exp(-logit[i]));
            dlogit[i] = dopacity[i] * al * (1.0 - al);
        }
    }
    return 0;
}
