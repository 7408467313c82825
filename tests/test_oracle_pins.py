"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these retypes the oracle's own formula: each compares it with a
closed form, a library routine (scipy's spherical harmonics, numpy's linear
solver), an invariant, or central finite differences of its own forward.
"""
import json
import math
import os

import numpy as np
import pytest

import scenes

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
ALPHA_SCALE = GOLD["density_alpha_scale"]["value"]
STOP_T = 1.0 - GOLD["stop_cumulative_opacity"]["value"]


def one_scene(kind, centre, verts, opacity, rgb=(0.3, 0.6, 0.9), sh=None, degree=0):
    centre = np.atleast_2d(np.asarray(centre, np.float64))
    verts = np.asarray(verts, np.float64).reshape(centre.shape[0], kind, 3)
    n = centre.shape[0]
    if sh is None:
        sh = np.zeros((n, 1, 3))
        sh[:, 0, :] = scenes.sh_from_rgb(np.broadcast_to(np.asarray(rgb, np.float64), (n, 3)))
    return scenes.Scene(kind, centre, verts, np.broadcast_to(np.asarray(opacity, np.float64), (n,)).copy(),
                        np.asarray(sh, np.float64), degree)


def axis_octa(centre, a, b, c, R=None):
    R = np.eye(3) if R is None else R
    return scenes.octahedra_from_axes(np.atleast_2d(centre), R[None], np.array([[a, b, c]]))[0]


def cam_on_axis(D=4.0, W=33, H=33, fov=40.0):
    return scenes.make_camera((0.0, 0.0, D), W, H, fov)


# ----------------------------------------------------------------- SH basis

def test_sh_basis_matches_scipy(orc):
    """3DGS real-SH basis = sqrt(2) Re/Im of scipy's complex Y_l^m (with the
    Condon-Shortley phase); Sec. 3.1 colours follow 3DGS."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(5)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        th, ph = math.acos(d[2]), math.atan2(d[1], d[0])
        ref = []
        for l in range(4):
            for m in range(-l, l + 1):
                Y = sph_harm_y(l, abs(m), th, ph)
                ref.append(math.sqrt(2) * Y.real if m > 0 else
                           math.sqrt(2) * Y.imag if m < 0 else Y.real)
        Y, _ = orc.sh_basis(3, d)
        np.testing.assert_allclose(Y, ref, atol=1e-13)
        for deg in range(3):
            Yd, _ = orc.sh_basis(deg, d)
            k = (deg + 1) ** 2
            np.testing.assert_allclose(Yd[:k], ref[:k], atol=1e-13)
            assert np.all(Yd[k:] == 0)


def test_sh_basis_derivative_fd(orc):
    rng = np.random.default_rng(6)
    for _ in range(10):
        d = rng.normal(size=3)
        _, dY = orc.sh_basis(3, d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3); e[a] = h
            fd = (orc.sh_basis(3, d + e)[0] - orc.sh_basis(3, d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, a], fd, atol=1e-8)


# ---------------------------------------------------------------------- MTIA

def test_mtia_matches_linear_solve(orc):
    """Ray (rx, ry, 0) + t (0,0,1) against p0 + u e1 + v e2, solved by numpy."""
    rng = np.random.default_rng(7)
    hits = 0
    for _ in range(300):
        p = rng.normal(size=(3, 3)) * [5, 5, 1] + [10, 20, 4]
        rx, ry = 10 + rng.normal() * 4, 20 + rng.normal() * 4
        A = np.stack([p[1] - p[0], p[2] - p[0], -np.array([0, 0, 1.0])], axis=1)
        u, v, t = np.linalg.solve(A, np.array([rx, ry, 0.0]) - p[0])
        out, _ = orc.mtia(p[0], p[1], p[2], rx, ry)
        inside = u >= 0 and v >= 0 and u + v <= 1
        assert bool(out[0]) == inside
        np.testing.assert_allclose(out[1:3], [u, v], rtol=1e-9, atol=1e-11)
        np.testing.assert_allclose(out[4], t, rtol=1e-10, atol=1e-10)
        hits += inside
    assert hits > 30


def test_mtia_gradient_fd(orc):
    """App. 'Gradient Computation' derivatives of the hit depth w.r.t. the
    three corners, against central differences of the forward."""
    rng = np.random.default_rng(8)
    for _ in range(50):
        p = rng.normal(size=(3, 3)) * [5, 5, 1] + [0, 0, 4]
        rx, ry = rng.normal(size=2) * 2
        _, g = orc.mtia(p[0], p[1], p[2], rx, ry)
        h = 1e-6
        for k in range(3):
            for a in range(3):
                q1, q2 = p.copy(), p.copy()
                q1[k, a] += h
                q2[k, a] -= h
                fd = (orc.mtia(*q1, rx, ry)[0][4] - orc.mtia(*q2, rx, ry)[0][4]) / (2 * h)
                assert abs(g[k, a] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, a, g[k, a], fd)


# ------------------------------------------------------------ span closed forms

@pytest.mark.parametrize("D", [4.0, 30.0])
def test_span_axis_aligned_octahedron(orc, D):
    """On the optical axis the ray-space map is exactly a scaled orthographic
    projection, so the span through |x|/a + |y|/b + |z|/c <= 1 is
    2c (1 - |X|/a - |Y|/b) at world offset (X, Y)."""
    a, b, c = 0.3, 0.2, 0.1
    cam = cam_on_axis(D, 65, 65, 20.0)
    sc = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], a, b, c), 0.5)
    rng = np.random.default_rng(9)
    n_in = 0
    for _ in range(200):
        X, Y = rng.uniform(-a, a), rng.uniform(-b, b)
        rx = cam.cx + cam.fx * X / D           # camera x = world x
        ry = cam.cy + cam.fy * (-Y) / D        # camera y = -world y
        (hit, i1, i2), _ = orc.span(sc, cam, 0, rx, ry)
        expect = 2 * c * (1 - abs(X) / a - abs(Y) / b)
        if expect > 1e-9:
            assert hit
            assert abs((i2 - i1) - expect) < 1e-12 * D + 1e-12
            n_in += 1
        elif expect < -1e-9:
            assert not hit
    assert n_in > 50


def _chord_octa(R, d, w):
    return 2.0 / sum(abs(R[:, i] @ w) / d[i] for i in range(3))


def _chord_tetra(R, s, w):
    dirs = np.einsum("ij,kj->ki", R, scenes._TETRA_DIRS)
    n = -dirs                                # outward normal of the face opposite vertex k
    dots = n @ w
    fwd = min(s / (3 * x) for x in dots if x > 0)
    bwd = min(s / (3 * -x) for x in dots if x < 0)
    return fwd + bwd


@pytest.mark.parametrize("kind", [6, 4])
def test_span_centre_pixel_equals_world_chord(orc, kind):
    """The ray through the projected centre is exact under the ray-space
    approximation (J maps the viewing direction to +z at unit speed), so the
    span equals the world-space chord of the primitive along that ray."""
    rng = np.random.default_rng(10 + kind)
    cam = scenes.make_camera((0.5, -0.3, 5.0), 640, 480, 60.0)
    cam.viewmat = scenes.look_at((0.5, -0.3, 5.0))        # exactly orthonormal (binary64)
    Rw = cam.viewmat[:3, :3].astype(np.float64)
    eye = -Rw.T @ cam.viewmat[:3, 3].astype(np.float64)
    for _ in range(30):
        c = rng.uniform(-1.5, 1.5, 3)
        R = scenes.random_rotations(rng, 1)[0]
        if kind == 6:
            d = rng.uniform(0.05, 0.3, 3)
            verts = scenes.octahedra_from_axes(c[None], R[None], d[None])[0]
        else:
            s = rng.uniform(0.05, 0.3)
            verts = scenes.tetrahedra_from_scale(c[None], R[None], np.array([s]))[0]
        sc = one_scene(kind, c, verts, 0.5)
        pp = orc.preprocess(sc, cam)
        (hit, i1, i2), (hitc, c1, c2) = orc.span(sc, cam, 0, pp["pc"][0, 0], pp["pc"][0, 1])
        w = (c - eye) / np.linalg.norm(c - eye)
        expect = _chord_octa(R, d, w) if kind == 6 else _chord_tetra(R, s, w)
        assert hit and hitc
        assert abs((i2 - i1) - expect) < 1e-10
        assert abs((c2 - c1) - expect) < 1e-10


@pytest.mark.parametrize("kind", [6, 4])
def test_mtia_span_equals_halfspace_span(orc, kind):
    """Two formulations of the ray/convex-polyhedron span agree (the paper's
    MTIA and the half-space clipping the rasterizer uses)."""
    w = scenes.workload(0 if kind == 4 else 1, scale=0.01 if kind == 6 else 1.0)
    sc, cam = w.scene, w.cameras[0]
    pp = orc.preprocess(sc, cam)
    rng = np.random.default_rng(11)
    agree = hits = 0
    for i in np.nonzero(pp["visible"])[0][:40]:
        pv = pp["pverts"][i]
        lo, hi = pv[:, :2].min(0), pv[:, :2].max(0)
        for _ in range(25):
            rx, ry = rng.uniform(lo, hi)
            (h1, a1, b1), (h2, a2, b2) = orc.span(sc, cam, int(i), rx, ry)
            assert h1 == h2
            if h1:
                hits += 1
                scale = abs(b1) + abs(a1)
                assert abs(a1 - a2) <= 1e-12 * scale and abs(b1 - b2) <= 1e-12 * scale
            agree += 1
    assert hits > 100


# -------------------------------------------------------- density and blending

def centred_octa_scene(depth_offsets, extents, alphas, rgbs):
    cs, vs = [], []
    for z, (a, b, c) in zip(depth_offsets, extents):
        cen = np.array([0.0, 0.0, z])
        cs.append(cen)
        vs.append(axis_octa(cen, a, b, c))
    n = len(cs)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = scenes.sh_from_rgb(np.asarray(rgbs, np.float64))
    return scenes.Scene(6, np.array(cs), np.array(vs), np.asarray(alphas, np.float64), sh, 0)


@pytest.mark.parametrize("alpha", [0.05, 0.5, 0.9, 0.999])
def test_thin_axis_opacity_is_099_alpha(orc, alpha):
    """Eq. 1 with o = 1 - exp(-sigma (i2 - i1)): through the thinnest diameter
    (span 2 d_min) the opacity is exactly 0.99 alpha; one primitive on black
    gives C = o * rgb at the centre pixel."""
    rgb = np.array([0.2, 0.5, 0.8])
    sc = centred_octa_scene([0.0], [(0.3, 0.25, 0.1)], [alpha], [rgb])
    cam = cam_on_axis(4.0, 33, 33, 30.0)       # pixel 16's centre is the axis
    img = orc.render(sc, [cam]).reshape(3, 33, 33)
    np.testing.assert_allclose(img[:, 16, 16], ALPHA_SCALE * alpha * rgb, rtol=1e-12, atol=1e-15)


def test_general_axis_opacity(orc):
    """Along an axis of length 2 d_k: o = 1 - (1 - 0.99 alpha)^(d_k / d_min)."""
    alpha = 0.7
    rgb = np.array([1.0, 1.0, 1.0])
    d = (0.1, 0.15, 0.25)                      # viewed along z: d_k = 0.25, d_min = 0.1
    sc = centred_octa_scene([0.0], [d], [alpha], [rgb])
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    img = orc.render(sc, [cam]).reshape(3, 33, 33)
    expect = 1 - (1 - ALPHA_SCALE * alpha) ** (d[2] / d[0])
    np.testing.assert_allclose(img[:, 16, 16], expect, rtol=1e-12)


def test_two_layer_compositing_and_background(orc):
    """Front-to-back: C = o1 c1 + (1-o1) o2 c2 + (1-o1)(1-o2) bg, with the
    nearer primitive first whatever the input order."""
    a1, a2 = 0.6, 0.8
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.1, 0.3, 0.9])
    bg = np.array([0.25, 0.5, 0.75])
    # the second entry is nearer the camera (camera at z = +4)
    sc = centred_octa_scene([-1.0, 1.0], [(0.3, 0.3, 0.1), (0.3, 0.3, 0.1)], [a2, a1], [c2, c1])
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    img = orc.render(sc, [cam], bg=bg).reshape(3, 33, 33)
    o1, o2 = ALPHA_SCALE * a1, ALPHA_SCALE * a2
    expect = o1 * c1 + (1 - o1) * o2 * c2 + (1 - o1) * (1 - o2) * bg
    np.testing.assert_allclose(img[:, 16, 16], expect, rtol=1e-12)
    # a pixel that misses both primitives shows the background exactly
    np.testing.assert_array_equal(img[:, 0, 0], bg)


@pytest.mark.parametrize("alpha", [0.5, 0.8])
def test_early_stop_at_cumulative_opacity_0999(orc, alpha):
    """Sec. 3.2 'Compositing': with K equal layers of opacity o the pixel
    blends the first n layers, n the least with (1-o)^n < 1e-3, and stops."""
    K = 30
    o = ALPHA_SCALE * alpha
    n = next(j for j in range(1, K + 1) if (1 - o) ** j < STOP_T)
    assert abs((1 - o) ** n / STOP_T - 1) > 1e-3      # not a borderline case
    sc = centred_octa_scene(np.linspace(1.0, -1.0, K), [(0.3, 0.3, 0.02)] * K, [alpha] * K,
                            [[1.0, 1.0, 1.0]] * K)
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    bg = (0.5, 0.5, 0.5)
    img, info = orc.render(sc, [cam], bg=bg, info=True)
    img = img.reshape(3, 33, 33)
    info = info.reshape(33, 33, 4)
    assert info[16, 16, 0] == n
    T = (1 - o) ** n
    assert abs(info[16, 16, 1] - T) < 1e-14
    np.testing.assert_allclose(img[:, 16, 16], (1 - T) * 1.0 + T * 0.5, rtol=1e-12)


@pytest.mark.parametrize("rel, flagged", [(2e-4, True), (-2e-4, True), (5e-3, False), (-5e-3, False)])
def test_borderline_stop_flag(orc, rel, flagged):
    """Two layers through their thin axes (opacity exactly 0.99 alpha each)
    take T to (1 + rel) 1e-3.  Within 1e-3 (relative) of the stop threshold
    the pixel is flagged (info bit 0): binary32 may stop one primitive
    earlier or later there.  Farther from it, it is not."""
    o1 = 0.96
    t_end = STOP_T * (1 + rel)
    o2 = 1 - t_end / (1 - o1)
    sc = centred_octa_scene([1.0, -1.0], [(0.3, 0.3, 0.1)] * 2, [o1 / ALPHA_SCALE, o2 / ALPHA_SCALE],
                            [[1.0, 1.0, 1.0]] * 2)
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    _, info = orc.render(sc, [cam], info=True)
    info = info.reshape(33, 33, 4)
    assert info[16, 16, 0] == 2
    assert abs(info[16, 16, 1] - t_end) < 1e-14
    assert bool(int(info[16, 16, 2]) & 1) == flagged


@pytest.mark.parametrize("o, flagged", [(0.5 + 2e-5, True), (0.5 - 2e-5, True), (0.5 + 1e-3, False),
                                        (0.5 - 1e-3, False)])
def test_borderline_depth_flag(orc, o, flagged):
    """The depth map reads the first primitive that takes the cumulative
    opacity above 0.5.  When the transmittance after a primitive lands within
    1e-4 (relative) of 0.5, binary32 may choose the next primitive or none,
    so the pixel is flagged (info bit 2); farther from it, it is not."""
    sc = centred_octa_scene([0.0], [(0.3, 0.3, 0.1)], [o / ALPHA_SCALE], [[1.0, 1.0, 1.0]])
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    _, info = orc.render(sc, [cam], info=True)
    info = info.reshape(33, 33, 4)
    assert abs(info[16, 16, 1] - (1 - o)) < 1e-14
    assert bool(int(info[16, 16, 2]) & 4) == flagged


def test_transmittance_bounds_and_empty_pixels(orc):
    w = scenes.workload(0)
    img, info = orc.render(w.scene, w.cameras, info=True)
    T = info[:, 1]
    assert np.all(T >= 0) and np.all(T <= 1)
    empty = info[:, 0] == 0
    assert np.all(T[empty] == 1.0)
    assert np.all(img.reshape(3, -1)[:, empty] == 0.0)    # black background
    assert empty.sum() > 0 and (~empty).sum() > 0


def test_permutation_invariance(orc):
    w = scenes.workload(0)
    img = orc.render(w.scene, w.cameras)
    perm = np.random.default_rng(12).permutation(w.scene.n)
    img_p = orc.render(w.scene.subset(perm), w.cameras)
    np.testing.assert_array_equal(img, img_p)


# ------------------------------------------------------------- keys and tiles

def _frustum_scene(pos, dist=0.05):
    c = np.array([pos], np.float64)
    v = scenes.octahedra_from_axes(c, np.eye(3)[None], np.array([[dist, dist, dist]]))
    return scenes.Scene(6, c.astype(np.float32), v.astype(np.float32), np.array([0.8], np.float32),
                        np.full((1, 1, 3), 0.5, np.float32), 0)


def test_view_frustum_cull(orc):
    """A primitive is drawn only if its projected centre lies within 1.3
    times the image (normalised device coordinates in [-1.3, 1.3]): centres at
    x_ndc = 1.25 are kept, at 1.35 culled (both axes, both sides).  A primitive
    beside the camera, just in front of the near plane, would otherwise get a
    linearised box covering the whole image."""
    cam = scenes.make_camera((0.0, 0.0, 0.0), 160, 100, 60.0, target=(0.0, 0.0, 1.0))
    M = cam.viewmat.astype(np.float64)
    z = 3.0
    for axis, size, f_, c_ in ((0, cam.width, cam.fx, cam.cx), (1, cam.height, cam.fy, cam.cy)):
        for ndc, keep in ((1.25, True), (1.35, False), (-1.25, True), (-1.35, False)):
            pix = (ndc + 1.0) * size / 2.0                # pixel coordinate of that NDC
            t = np.zeros(3)
            t[axis] = (pix - float(c_)) * z / float(f_)   # camera-space offset
            t[2] = z
            world = M[:3, :3].T @ (t - M[:3, 3])
            pp = orc.preprocess(_frustum_scene(world), cam)
            assert bool(pp["visible"][0]) == keep, (axis, ndc)
    # beside the camera, 0.21 in front of it and 5 to the side: its ray-space
    # box (x_c +- |J02| d, J02 = -f_x x / z^2) would span the whole image, yet
    # it is culled; the same primitive straight ahead is drawn
    z, side, d = 0.21, 5.0, 0.3
    xc = float(cam.fx) * side / z + float(cam.cx)
    half = float(cam.fx) * side / z ** 2 * d
    assert xc - half < 0 and xc + half > cam.width
    for side_, keep in ((side, False), (0.0, True)):
        t = np.array([side_, 0.0, z])
        world = M[:3, :3].T @ (t - M[:3, 3])
        sc = _frustum_scene(world, dist=d)
        pp = orc.preprocess(sc, cam)
        assert bool(pp["visible"][0]) == keep
        img = orc.render(sc, [cam]).reshape(3, -1)
        assert (np.abs(img).max() > 0) == keep


def test_near_plane_cull(orc):
    """A primitive whose centre lies at camera depth 0.2 or less (the near
    plane), or behind the camera, is not drawn: a small primitive straight
    ahead at depth 0.19 is dropped, at 0.21 drawn, and 1.0 behind the camera
    dropped."""
    cam = scenes.make_camera((0.0, 0.0, 0.0), 160, 100, 60.0, target=(0.0, 0.0, 1.0))
    M = cam.viewmat.astype(np.float64)
    for z, keep in ((0.19, False), (0.21, True), (-1.0, False)):
        world = M[:3, :3].T @ (np.array([0.0, 0.0, z]) - M[:3, 3])
        sc = _frustum_scene(world, dist=0.01)
        assert bool(orc.preprocess(sc, cam)["visible"][0]) == keep, z
        img = orc.render(sc, [cam]).reshape(3, -1)
        assert (np.abs(img).max() > 0) == keep, z


def test_colour_direction_is_from_the_camera(orc):
    """Sec. 3.1 (view-dependent colour as in 3DGS): the SH are evaluated at
    the unit direction from the camera's position to the primitive's centre.
    The camera position here is the eye the camera was built from (the
    oracle recovers it from the view matrix), the basis is the one pinned to
    scipy above, and the colour is max(0, SH + 0.5)."""
    rng = np.random.default_rng(17)
    eye = np.array([1.5, -0.7, 4.0])
    cam = scenes.make_camera(tuple(eye), 64, 48, 50.0, target=(0.1, 0.2, -0.3))
    for _ in range(10):
        c = rng.uniform(-0.6, 0.6, 3)
        sh = rng.normal(0.0, 0.4, (1, 16, 3))
        sc = one_scene(6, c, axis_octa(c, 0.1, 0.08, 0.06), 0.6, sh=sh, degree=3)
        pp = orc.preprocess(sc, cam)
        assert pp["visible"][0]
        d = c - eye
        np.testing.assert_allclose(pp["dist"][0], np.linalg.norm(d), rtol=1e-6)
        Y, _ = orc.sh_basis(3, d / np.linalg.norm(d))
        want = np.maximum(Y @ sh[0] + 0.5, 0.0)
        np.testing.assert_allclose(pp["rgb"][0], want, atol=1e-5)


def test_keyfields_are_binary32_replay(orc):
    """The culling / depth key / pixel rectangle come from binary32 with one
    rounding per operation (the centre transformed to the camera frame, each
    vertex's offset from the centre rotated into it and mapped by the ray-space
    Jacobian); numpy float32 scalars reproduce them exactly, and the rectangle
    brackets the binary64 footprint to within one pixel."""
    w = scenes.workload(1, scale=0.05)
    sc, cam = w.scene, w.cameras[0]
    pp = orc.preprocess(sc, cam)
    f = np.float32
    M = cam.viewmat.astype(np.float32)
    def tr(x):
        return [f(f(f(M[i, 0] * f(x[0])) + f(M[i, 1] * f(x[1]))) + f(M[i, 2] * f(x[2]))) + M[i, 3]
                for i in range(3)]
    checked = 0
    for i in range(sc.n):
        tc = tr(sc.centre[i])
        assert np.array([tc[2]], np.float32).view(np.uint32)[0] == pp["zbits"][i]
        vis = bool(tc[2] > f(0.2))
        if vis:
            u, w_ = f(tc[0] / tc[2]), f(tc[1] / tc[2])
            xc, yc = f(f(f(cam.fx) * u) + f(cam.cx)), f(f(f(cam.fy) * w_) + f(cam.cy))
            W, H = f(cam.width), f(cam.height)
            vis = bool(f(f(-0.15) * W) <= xc <= f(f(1.15) * W) and f(f(-0.15) * H) <= yc <= f(f(1.15) * H))
        assert vis == pp["visible"][i]
        if not vis:
            continue
        j00, j11 = f(f(cam.fx) / tc[2]), f(f(cam.fy) / tc[2])
        j02, j12 = -f(j00 * u), -f(j11 * w_)
        qx, qy = [], []
        c32 = sc.centre[i].astype(np.float32)
        for v in sc.verts[i]:
            wv = [f(f(v[k]) - c32[k]) for k in range(3)]
            d = [f(f(f(M[k, 0] * wv[0]) + f(M[k, 1] * wv[1])) + f(M[k, 2] * wv[2])) for k in range(3)]
            qx.append(f(f(j00 * d[0]) + f(j02 * d[2])))
            qy.append(f(f(j11 * d[1]) + f(j12 * d[2])))
        x0 = max(np.ceil(f(f(xc + min(qx)) - f(0.5))), f(0))
        x1 = min(np.floor(f(f(xc + max(qx)) - f(0.5))), f(cam.width - 1))
        y0 = max(np.ceil(f(f(yc + min(qy)) - f(0.5))), f(0))
        y1 = min(np.floor(f(f(yc + max(qy)) - f(0.5))), f(cam.height - 1))
        r = pp["rect"][i]
        if x0 <= x1 and y0 <= y1:
            assert list(r) == [int(x0), int(x1), int(y0), int(y1)], i
            pv = pp["pverts"][i]
            assert abs(np.ceil(pv[:, 0].min() - 0.5) - max(x0, 0)) <= 1 or x0 == 0
            checked += 1
        else:
            assert r[0] > r[1] or r[2] > r[3]
    assert checked > 50


def test_keys_structure(orc):
    """Keys ascend; every record emits exactly its rectangle's tiles; equal
    keys keep emission (record-index) order; values are record indices."""
    w = scenes.workload(1, scale=0.2)
    sc, cam = w.scene, w.cameras[0]
    k, v, counts = orc.keys(sc, [cam], tile=16)
    assert np.all(np.diff(k.astype(np.uint64)) >= 0)
    pp = orc.preprocess(sc, cam)
    tiles_x = (cam.width + 15) // 16
    for i in range(sc.n):
        r = pp["rect"][i]
        if pp["visible"][i] and r[0] <= r[1] and r[2] <= r[3]:
            n_exp = (r[1] // 16 - r[0] // 16 + 1) * (r[3] // 16 - r[2] // 16 + 1)
        else:
            n_exp = 0
        assert counts[i] == n_exp
    assert len(k) == counts.sum()
    tile = (k >> np.uint64(32)).astype(np.int64)
    depth = (k & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    assert np.all(depth == pp["zbits"][v])
    for q in np.random.default_rng(13).choice(len(k), 200, replace=False):
        r = pp["rect"][v[q]]
        ty, tx = divmod(int(tile[q]), tiles_x)
        assert r[0] // 16 <= tx <= r[1] // 16 and r[2] // 16 <= ty <= r[3] // 16
    same = (k[1:] == k[:-1])
    assert np.all(v[1:][same] > v[:-1][same])


def test_keys_multiview_tile_bases(orc):
    w = scenes.workload(3, scale=0.0005)
    cams = w.cameras[::5]
    k, v, counts = orc.keys(w.scene, cams, tile=16)
    n = w.scene.n
    base = 0
    tile = (k >> np.uint64(32)).astype(np.int64)
    for c, cam in enumerate(cams):
        nt = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
        sel = (v // n) == c
        assert sel.sum() == counts[c * n:(c + 1) * n].sum()
        assert np.all((tile[sel] >= base) & (tile[sel] < base + nt))
        base += nt


# ----------------------------------------------------------------- gradients

def _fd_check(orc, sc, cam, bg, gimg, params, px=None, py=None, h_geo=1e-6, h_app=1e-5, aa=0.0):
    """Central FD of L = <g, image> against the oracle adjoint, d_min frozen."""
    dmin = orc.preprocess(sc, cam, aa=aa)["dmin"]
    if px is None:
        _, grads = orc.render(sc, [cam], bg=bg, dL_dimage=gimg, dmin=dmin, aa=aa)
        loss = lambda s: float(np.dot(orc.render(s, [cam], bg=bg, dmin=dmin, aa=aa), gimg))
    else:
        _, _, grads = orc.render_pixels(sc, cam, px, py, bg=bg, dL_dC=gimg, dmin=dmin, aa=aa)
        loss = lambda s: float(np.sum(orc.render_pixels(s, cam, px, py, bg=bg, dmin=dmin, aa=aa)[0] * gimg))
    base = dict(centre=sc.centre.astype(np.float64), verts=sc.verts.astype(np.float64),
                opacity=sc.opacity.astype(np.float64), sh=sc.sh.astype(np.float64))
    ok = 0
    for name, idx in params:
        h = h_app if name in ("opacity", "sh") else h_geo
        def L(delta):
            arrs = {k: v.copy() for k, v in base.items()}
            arrs[name].reshape(-1)[idx] += delta
            s = scenes.Scene(sc.kind, arrs["centre"], arrs["verts"], arrs["opacity"], arrs["sh"],
                             sc.sh_degree)
            return L_(s)
        L_ = loss
        fd1 = (L(h) - L(-h)) / (2 * h)
        fd2 = (L(h / 2) - L(-h / 2)) / h
        if abs(fd1 - fd2) > 1e-4 * max(abs(fd1), 1e-3):
            continue                               # a kink (face switch, order swap, stop)
        g = grads[name].reshape(-1)[idx]
        assert abs(g - fd1) <= 2e-4 * max(abs(fd1), 1e-2), (name, idx, g, fd1)
        ok += 1
    return ok


def test_adjoint_fd_tetrahedra(orc):
    w = scenes.workload(0)
    sc, cam = w.scene, w.cameras[0]
    rng = np.random.default_rng(14)
    gimg = rng.normal(size=3 * cam.pixels)
    pp = orc.preprocess(sc, cam)
    vis = np.nonzero(pp["visible"])[0]
    params = []
    for i in rng.choice(vis, 6, replace=False):
        params += [("centre", 3 * i + a) for a in range(3)]
        params += [("verts", 12 * i + a) for a in rng.choice(12, 5, replace=False)]
        params += [("opacity", i), ("sh", 3 * i + int(rng.integers(3)))]
    ok = _fd_check(orc, sc, cam, (0.1, 0.2, 0.3), gimg, params)
    assert ok >= 0.8 * len(params)


def test_adjoint_fd_octahedra_sh3(orc):
    """SH degree 3 octahedra, on a crop around sampled primitives."""
    w = scenes.workload(1, scale=0.1)
    sc, cam = w.scene, w.cameras[0]
    pp = orc.preprocess(sc, cam)
    rng = np.random.default_rng(15)
    area = (pp["rect"][:, 1] - pp["rect"][:, 0]) * (pp["rect"][:, 3] - pp["rect"][:, 2])
    cand = np.nonzero(pp["visible"] & (area > 60))[0]
    params = []
    mask = np.zeros((cam.height, cam.width), bool)
    for i in rng.choice(cand, 4, replace=False):
        params += [("centre", 3 * i + a) for a in range(3)]
        params += [("verts", 18 * i + a) for a in rng.choice(18, 4, replace=False)]
        params += [("opacity", i)] + [("sh", 48 * i + int(k)) for k in rng.choice(48, 3, replace=False)]
        r = pp["rect"][i]
        mask[max(r[2] - 2, 0):r[3] + 3, max(r[0] - 2, 0):r[1] + 3] = True
    py, px = [a.astype(np.int32) for a in np.nonzero(mask)]
    gpx = rng.normal(size=(px.shape[0], 3))
    ok = _fd_check(orc, sc, cam, (0.0, 0.0, 0.0), gpx, params, px, py)
    assert ok >= 0.8 * len(params)


def test_clamped_colour_channel_has_no_gradient(orc):
    """Sec. 3.1 (colour as in 3DGS): rgb = max(0, SH + 0.5).  A channel whose
    SH value sits well below -0.5 is clamped to 0 on a whole neighbourhood of
    the parameters, so the loss does not depend on that channel's SH
    coefficients there, nor on the view direction through them: central
    differences give zero, and the adjoint must too, for the SH coefficients
    and for the centre (degree 1, so the direction term is live)."""
    R = scenes.random_rotations(np.random.default_rng(3), 1)[0]
    sh = np.zeros((1, 4, 3))
    sh[0, 0, :] = scenes.sh_from_rgb(np.array([-0.4, 0.5, 0.7]))
    sh[0, 1:, :] = [[0.06, -0.04, 0.05], [-0.05, 0.07, 0.03], [0.04, 0.05, -0.06]]
    sc = one_scene(6, (0.05, -0.03, 0.0), axis_octa((0.05, -0.03, 0.0), 0.5, 0.4, 0.3, R), 0.8, sh=sh, degree=1)
    cam = cam_on_axis(D=3.0, W=41, H=41)
    img = orc.render(sc, [cam], bg=(0.1, 0.2, 0.3)).reshape(3, cam.height, cam.width)
    assert np.count_nonzero(img[1] != 0.2) > 60           # the primitive covers pixels
    gimg = np.random.default_rng(16).normal(size=3 * cam.pixels)
    dmin = orc.preprocess(sc, cam)["dmin"]
    _, grads = orc.render(sc, [cam], bg=(0.1, 0.2, 0.3), dL_dimage=gimg, dmin=dmin)
    assert np.all(grads["sh"].reshape(4, 3)[:, 0] == 0.0)  # the clamped channel
    assert np.all(np.abs(grads["sh"].reshape(4, 3)[:, 1:]) > 0.0)
    params = [("sh", 3 * k + ch) for k in range(4) for ch in range(3)] + [("centre", a) for a in range(3)]
    ok = _fd_check(orc, sc, cam, (0.1, 0.2, 0.3), gimg, params)
    assert ok >= 0.8 * len(params)


def test_ray_space_map_is_first_order_perspective(orc):
    """App. 'Ray Space Approximation': each ray-space vertex is the local affine
    (first-order) approximation of (fx x/z + cx, fy y/z + cy, |t|) around the
    centre, so for a primitive of size eps it matches the exact pinhole
    projection and camera distance of the vertex up to O(eps^2)."""
    rng = np.random.default_rng(16)
    cam = scenes.make_camera((0.7, 0.4, 4.5), 800, 600, 60.0)
    cam.viewmat = scenes.look_at((0.7, 0.4, 4.5))
    M = cam.viewmat.astype(np.float64)
    for _ in range(10):
        c = rng.uniform(-1.5, 1.5, 3)
        R = scenes.random_rotations(rng, 1)[0]
        errs = []
        for eps in (1e-2, 5e-3):
            verts = scenes.octahedra_from_axes(c[None], R[None], np.array([[eps, 0.7 * eps, 1.3 * eps]]))[0]
            sc = one_scene(6, c, verts, 0.5)
            pv = orc.preprocess(sc, cam)["pverts"][0]
            e = 0.0
            for k in range(6):
                t = M[:3, :3] @ verts[k] + M[:3, 3]
                exact = np.array([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy,
                                  np.linalg.norm(t)])
                e = max(e, np.max(np.abs(pv[k] - exact) / [cam.fx, cam.fy, 1.0]))
            errs.append(e)
        # second order: halving eps divides the error by ~4
        assert errs[0] < 2e-4 and 3.0 < errs[0] / errs[1] < 5.0, errs


def test_depth_ties_keep_index_order(orc):
    """Reading for equal depth keys: ascending primitive index (stable order).
    Two primitives with the same centre blend lower index first, and equal
    keys in the sorted tile list keep ascending record order."""
    c1, c2 = np.array([1.0, 0.1, 0.1]), np.array([0.1, 0.2, 1.0])
    sc = centred_octa_scene([0.0, 0.0], [(0.3, 0.3, 0.1), (0.25, 0.35, 0.1)], [0.6, 0.7], [c1, c2])
    cam = cam_on_axis(4.0, 33, 33, 30.0)
    img = orc.render(sc, [cam]).reshape(3, 33, 33)
    o1, o2 = ALPHA_SCALE * 0.6, ALPHA_SCALE * 0.7
    np.testing.assert_allclose(img[:, 16, 16], o1 * c1 + (1 - o1) * o2 * c2, rtol=1e-12)
    w = scenes.workload(1, scale=0.05)
    dup = w.scene.subset(np.repeat(np.arange(w.scene.n), 2))
    k, v, _ = orc.keys(dup, w.cameras, tile=16)
    same = k[1:] == k[:-1]
    assert same.sum() > 100
    assert np.all(v[1:][same] > v[:-1][same])


def test_degenerate_primitive_is_invisible(orc):
    """Eq. 1 divides by the smallest centre-vertex distance: a primitive with a
    vertex on its centre (a flat octahedron, d_z = 0) has no density and is
    not visible -- no tile entries, no colour, zero and finite gradients."""
    good = axis_octa((0.0, 0.0, 0.0), 0.6, 0.5, 0.4)
    flat = axis_octa((0.1, 0.0, 0.2), 0.7, 0.6, 0.0)
    both = one_scene(6, [[0.0, 0.0, 0.0], [0.1, 0.0, 0.2]], np.stack([good, flat]), 0.8,
                     rgb=[[0.9, 0.2, 0.1], [0.1, 0.9, 0.2]])
    alone = both.subset(np.array([0]))
    cam = cam_on_axis(W=40, H=36)
    dL = np.random.default_rng(4).normal(size=3 * 40 * 36)
    img, g = orc.render(both, [cam], dL_dimage=dL)
    img1, g1 = orc.render(alone, [cam], dL_dimage=dL)
    np.testing.assert_array_equal(img, img1)
    for k in g:
        assert np.all(np.isfinite(g[k]))
        assert np.all(g[k][1] == 0.0), k
        np.testing.assert_allclose(g[k][0], g1[k][0], rtol=1e-12, atol=1e-13)   # summation order only
    _, _, counts = orc.keys(both, [cam])
    assert counts[1] == 0 and counts[0] > 0


# ------------------------------------------------------------ 2D filter (Sec. 3.3)
AA = 0.1   # the paper's 2D filter size in pixels (App. "Experimental Setting")


@pytest.mark.parametrize("D", [4.0, 30.0])
def test_aa_filter_octahedron_span_closed_form(orc, D):
    """On the optical axis an axis-aligned octahedron's ray-space image is the
    octahedron with half-axes (fx a / D, fy b / D, c).  The 2D filter moves the
    four vertices on the projected box outward by half the filter size each,
    so the span becomes 2c (1 - |x|/(fx a/D + s) - |y|/(fy b/D + s)) with
    s = 0.05 px, (x, y) the pixel offset from the projected centre."""
    a, b, c = 0.3, 0.2, 0.1
    cam = cam_on_axis(D, 65, 65, 20.0)
    sc = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], a, b, c), 0.5)
    Xr, Yr, s = cam.fx * a / D, cam.fy * b / D, float(np.float32(AA / 2))   # the move is binary32
    rng = np.random.default_rng(19)
    n_in = n_grown = 0
    pts = [(rng.uniform(-Xr - s, Xr + s), rng.uniform(-Yr - s, Yr + s)) for _ in range(300)]
    # points just inside the filtered footprint's boundary, hence outside the
    # unfiltered one (the band is s / max(Xr, Yr) ~ 1e-3 wide in relative terms)
    for t in np.linspace(0.0, 1.0, 11):
        for sx, sy in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
            pts.append((sx * t * (Xr + s) * (1 - 1e-4), sy * (1 - t) * (Yr + s) * (1 - 1e-4)))
    for x, y in pts:
        (hit, i1, i2), (hit2, j1, j2) = orc.span(sc, cam, 0, cam.cx + x, cam.cy + y, aa=AA)
        expect = 2 * c * (1 - abs(x) / (Xr + s) - abs(y) / (Yr + s))
        if expect > 1e-9:
            assert hit and hit2
            assert abs((i2 - i1) - expect) < 1e-12 * D + 1e-12
            n_in += 1
            n_grown += abs(x) / Xr + abs(y) / Yr > 1      # outside the unfiltered primitive
        elif expect < -1e-9:
            assert not hit
    assert n_in > 100 and n_grown > 0


def test_aa_filter_moves_box_vertices(orc):
    """Only the vertices on the projected bounding box move, outward and
    parallel to the screen: by half the filter for an octahedron (its
    opposite vertices mirror the move), by the whole filter for a
    tetrahedron."""
    rng = np.random.default_rng(23)
    w0 = scenes.workload(0)
    cam = w0.cameras[0]
    for sc, step in ((scenes.workload(1, scale=0.01).scene, float(np.float32(AA / 2))),
                     (w0.scene, float(np.float32(AA)))):
        p0 = orc.preprocess(sc, cam)["pverts"]
        p1 = orc.preprocess(sc, cam, aa=AA)
        vis = p1["visible"]
        d = p1["pverts"] - p0
        assert np.all(d[..., 2] == 0)
        for i in np.nonzero(vis)[0][:200]:
            for ax in (0, 1):
                q = p0[i, :, ax]
                want = np.where(q == q.max(), step, np.where(q == q.min(), -step, 0.0))
                np.testing.assert_allclose(d[i, :, ax], want, atol=1e-12)
        assert rng is not None


def test_aa_filter_widens_the_pixel_rectangle(orc):
    """The tile rectangle is taken over the moved vertices: a box whose right
    edge sits 0.03 px short of a pixel centre gains that column."""
    a, c = 0.3, 0.1
    D = 4.0
    cam = cam_on_axis(D, 65, 65, 20.0)
    Xr = cam.fx * a / D
    # shift the primitive so that its right edge is 0.03 px left of pixel 40's centre
    cx_target = 40.5 - 0.03 - Xr
    X0 = (cx_target - cam.cx) * D / cam.fx
    sc = one_scene(6, [X0, 0, 0], axis_octa([X0, 0, 0], a, 0.2, c), 0.5)
    r0 = orc.preprocess(sc, cam)["rect"][0]
    r1 = orc.preprocess(sc, cam, aa=AA)["rect"][0]
    assert r0[1] == 39 and r1[1] == 40
    # and a box whose left edge sits 0.03 px right of pixel 10's centre
    X1 = (10.5 + 0.03 + Xr - cam.cx) * D / cam.fx
    sc1 = one_scene(6, [X1, 0, 0], axis_octa([X1, 0, 0], a, 0.2, c), 0.5)
    assert orc.preprocess(sc1, cam)["rect"][0][0] == 11
    assert orc.preprocess(sc1, cam, aa=AA)["rect"][0][0] == 10
    k0, _, n0 = orc.keys(sc, [cam])
    k1, _, n1 = orc.keys(sc, [cam], aa=AA)
    assert n1[0] >= n0[0]


def test_aa_filter_adjoint_fd(orc):
    """The move is piecewise constant in the geometry, so the adjoint with the
    filter on still matches central finite differences."""
    w = scenes.workload(0)
    sc, cam = w.scene, w.cameras[0]
    rng = np.random.default_rng(29)
    gimg = rng.normal(size=3 * cam.pixels)
    pp = orc.preprocess(sc, cam, aa=AA)
    vis = np.nonzero(pp["visible"])[0]
    params = []
    for i in rng.choice(vis, 6, replace=False):
        params += [("centre", 3 * i + a) for a in range(3)]
        params += [("verts", 12 * i + a) for a in rng.choice(12, 5, replace=False)]
        params += [("opacity", i)]
    ok = _fd_check(orc, sc, cam, (0.1, 0.2, 0.3), gimg, params, aa=AA)
    assert ok >= 0.8 * len(params)


def test_silhouette_grazing_pixels_are_flagged(orc):
    """A ray through a silhouette vertex has a zero span: the oracle flags it
    (bit 1 of the borderline word), and rays well inside, off the faces'
    edges, are not flagged."""
    D, a = 4.0, 0.3
    cam = cam_on_axis(D, 65, 65, 20.0)
    # the +x vertex projects onto the centre of pixel (40, 32)
    X = (40.5 - cam.cx) * D / cam.fx
    sc = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], X, 0.2, 0.1), 0.5)
    px = np.array([40, 38, 36], np.int32)
    py = np.array([32, 30, 29], np.int32)
    _, info = orc.render_pixels(sc, cam, px, py)
    flags = info[:, 2].astype(int)
    assert flags[0] & 2 and not flags[1] & 2 and not flags[2] & 2


def test_interior_edge_pixels_are_flagged(orc):
    """An axis-aligned octahedron on the optical axis: its front faces meet
    (and its back faces meet) along the image axes through the centre, where
    the span is continuous but its derivative switches between faces.  Rays
    through those edges are flagged (bit 1), a ray between them is not."""
    D = 4.0
    cam = cam_on_axis(D, 65, 65, 20.0)      # pixel 32 is centred on each axis
    sc = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], 0.17, 0.2, 0.1), 0.5)
    px = np.array([32, 36, 32, 36], np.int32)
    py = np.array([29, 32, 32, 29], np.int32)
    _, info = orc.render_pixels(sc, cam, px, py)
    flags = info[:, 2].astype(int)
    assert info[:, 0].min() == 1                       # each ray crosses the primitive
    assert flags[0] & 2 and flags[1] & 2 and flags[2] & 2 and not flags[3] & 2


# --------------------------------------------------- depth (App. "Depth and Surface Reconstruction")
def test_depth_front_surface_closed_form(orc):
    """An opaque-enough axis-aligned octahedron on the optical axis: the depth
    of pixel offset (x, y) is where the ray enters its front surface,
    D - c (1 - |x|/X - |y|/Y) with (X, Y) its projected half-axes; pixels whose
    span is too short to reach opacity 0.5 get no depth (0)."""
    D, a, b, c = 4.0, 0.3, 0.2, 0.1
    cam = cam_on_axis(D, 65, 65, 20.0)
    sc = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], a, b, c), 0.95)
    X, Y = cam.fx * a / D, cam.fy * b / D
    yy, xx = np.mgrid[0:65, 0:65]
    px, py = xx.reshape(-1).astype(np.int32), yy.reshape(-1).astype(np.int32)
    d, f = orc.depth_pixels(sc, cam, px, py)
    x = px + 0.5 - cam.cx
    y = py + 0.5 - cam.cy
    u = 1 - np.abs(x) / X - np.abs(y) / Y
    pp = orc.preprocess(sc, cam)
    sigma = pp["sigma"][0]
    reach = 1 - np.exp(-sigma * 2 * c * np.clip(u, 0, None)) > 0.5     # opacity of the full span
    ok = (f == 0)
    np.testing.assert_allclose(d[reach & ok], (D - c * u)[reach & ok], atol=1e-12)
    assert np.all(d[~reach & ok] == 0)
    assert reach.sum() > 100 and (~reach & (u > 0)).sum() > 10


def test_depth_two_layers(orc):
    """A front layer of opacity 0.3 leaves the depth to the layer behind it;
    one of opacity 0.7 takes it; the background never does."""
    cam = cam_on_axis(4.0, 33, 33, 40.0)
    front = axis_octa([0, 0, 1.0], 1.0, 1.0, 0.05)
    back = axis_octa([0, 0, -1.0], 1.0, 1.0, 0.05)
    for a_front, want in ((0.30, 5.0 - 0.05), (0.70, 3.0 - 0.05)):
        sc = one_scene(6, [[0, 0, 1.0], [0, 0, -1.0]], np.stack([front, back]), [a_front, 0.9])
        sig = orc.preprocess(sc, cam)["sigma"]
        # through the centres each layer's span is its full thickness 2c: opacity 0.99 alpha
        assert abs((1 - np.exp(-sig[0] * 0.1)) - 0.99 * a_front) < 1e-12
        d, f = orc.depth_pixels(sc, cam, np.array([16], np.int32), np.array([16], np.int32))
        # the axis ray meets both layers at their vertices, where faces meet
        # (bit 1); the 0.5 crossing itself is not borderline (bit 2)
        assert not f[0] & 4 and abs(d[0] - want) < 1e-12, (a_front, d[0])
    empty = one_scene(6, [0, 0, 0], axis_octa([0, 0, 0], 0.1, 0.1, 0.1), 0.9)
    d, _ = orc.depth_pixels(empty, cam, np.array([0], np.int32), np.array([0], np.int32))
    assert d[0] == 0.0


# ------------------------------------------- exact mode (App. "Ray Space Approximation")
def _hull_chord(verts_world, cam_pos, w):
    """Length of the ray cam_pos + l w (l > 0) inside the convex hull of the
    vertices, from scipy's hull facets (independent of the face topology)."""
    from scipy.spatial import ConvexHull
    h = ConvexHull(verts_world)
    lo, hi = 0.0, np.inf
    for eq in h.equations:                    # n . x + off <= 0 inside
        n, off = eq[:3], eq[3]
        den = n @ w
        num = -(off + n @ cam_pos)
        if abs(den) < 1e-15:
            if num < 0:
                return 0.0
            continue
        t = num / den
        if den > 0:
            hi = min(hi, t)
        else:
            lo = max(lo, t)
    return max(hi - lo, 0.0) * np.linalg.norm(w)


@pytest.mark.parametrize("kind", [6, 4])
def test_exact_span_is_the_world_chord(orc, kind):
    """Without the ray-space approximation the span of any pixel is the
    length of that pixel's perspective ray inside the primitive."""
    rng = np.random.default_rng(31 + kind)
    cam = scenes.make_camera((0.4, -0.3, 3.0), 96, 80, 50.0)
    cam.viewmat = scenes.look_at((0.4, -0.3, 3.0))        # exactly orthonormal (binary64)
    M = np.asarray(cam.viewmat, np.float64).reshape(4, 4)
    Rm, Tv = M[:3, :3], M[:3, 3]
    cam_pos = -Rm.T @ Tv
    R = scenes.random_rotations(rng, 1)
    c = np.array([[0.1, 0.05, -0.2]])
    if kind == 6:
        v = scenes.octahedra_from_axes(c, R, np.array([[0.5, 0.35, 0.25]]))[0]
    else:
        v = scenes.tetrahedra_from_scale(c, R, np.array([0.6]))[0]
    sc = one_scene(kind, c[0], v, 0.5)
    rect = orc.preprocess(sc, cam, exact=True)["rect"][0]
    n_hit = 0
    for _ in range(400):
        x, y = rng.uniform(rect[0] - 3, rect[1] + 4), rng.uniform(rect[2] - 3, rect[3] + 4)
        d_cam = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
        w = Rm.T @ d_cam
        want = _hull_chord(v, cam_pos, w)
        (hit, i1, i2), (hit2, j1, j2) = orc.span(sc, cam, 0, x, y, exact=True)
        if want > 1e-9:
            assert hit and hit2
            assert abs((i2 - i1) - want) < 1e-10
            assert abs((j2 - j1) - want) < 1e-10
            n_hit += 1
        elif want == 0.0:
            assert not hit
    assert n_hit > 50
    # every pixel whose centre ray meets the primitive lies in the tile rectangle
    for py in range(cam.height):
        for px in range(cam.width):
            (hit, _, _), _ = orc.span(sc, cam, 0, px + 0.5, py + 0.5, exact=True)
            if hit:
                assert rect[0] <= px <= rect[1] and rect[2] <= py <= rect[3]


def test_exact_culls_primitives_reaching_the_near_plane(orc):
    """Reading: in exact mode the perspective box needs every vertex in front,
    so a primitive with a vertex at depth <= 0.2 is not visible."""
    cam = cam_on_axis(4.0, 33, 33, 40.0)
    near = one_scene(6, [0, 0, 3.5], axis_octa([0, 0, 3.5], 0.2, 0.2, 0.35), 0.5)   # front vertex at depth 0.15
    far = one_scene(6, [0, 0, 3.5], axis_octa([0, 0, 3.5], 0.2, 0.2, 0.25), 0.5)    # front vertex at depth 0.25
    assert not orc.preprocess(near, cam, exact=True)["visible"][0]
    assert orc.preprocess(near, cam)["visible"][0]                # the ray-space mode keeps it
    assert orc.preprocess(far, cam, exact=True)["visible"][0]


@pytest.mark.parametrize("kind", [6, 4])
def test_exact_adjoint_fd(orc, kind):
    if kind == 4:
        w = scenes.workload(0)
    else:
        w = scenes.workload(1, scale=0.02)
    sc, cam = w.scene, w.cameras[0]
    rng = np.random.default_rng(37 + kind)
    pp = orc.preprocess(sc, cam, exact=True)
    area = (pp["rect"][:, 1] - pp["rect"][:, 0]) * (pp["rect"][:, 3] - pp["rect"][:, 2])
    cand = np.nonzero(pp["visible"] & (area > 30))[0]
    params = []
    mask = np.zeros((cam.height, cam.width), bool)
    for i in rng.choice(cand, min(4, cand.size), replace=False):
        params += [("centre", 3 * i + a) for a in range(3)]
        params += [("verts", 3 * kind * i + a) for a in rng.choice(3 * kind, 6, replace=False)]
        params += [("opacity", i)]
        r = pp["rect"][i]
        mask[max(r[2] - 2, 0):r[3] + 3, max(r[0] - 2, 0):r[1] + 3] = True
    py, px = [a.astype(np.int32) for a in np.nonzero(mask)]
    gpx = rng.normal(size=(px.shape[0], 3))
    ok = _fd_check_exact(orc, sc, cam, gpx, params, px, py)
    assert ok >= 0.8 * len(params)


def _fd_check_exact(orc, sc, cam, gimg, params, px, py, h=1e-6):
    dmin = orc.preprocess(sc, cam, exact=True)["dmin"]
    _, _, grads = orc.render_pixels(sc, cam, px, py, dL_dC=gimg, dmin=dmin, exact=True)
    base = dict(centre=sc.centre.astype(np.float64), verts=sc.verts.astype(np.float64),
                opacity=sc.opacity.astype(np.float64), sh=sc.sh.astype(np.float64))
    ok = 0
    for name, idx in params:
        hh = 1e-5 if name == "opacity" else h
        def L(delta):
            arrs = {k: v.copy() for k, v in base.items()}
            arrs[name].reshape(-1)[idx] += delta
            s2 = scenes.Scene(sc.kind, arrs["centre"], arrs["verts"], arrs["opacity"], arrs["sh"], sc.sh_degree)
            return float(np.sum(orc.render_pixels(s2, cam, px, py, dmin=dmin, exact=True)[0] * gimg))
        fd1 = (L(hh) - L(-hh)) / (2 * hh)
        fd2 = (L(hh / 2) - L(-hh / 2)) / hh
        if abs(fd1 - fd2) > 1e-4 * max(abs(fd1), 1e-3):
            continue
        g = grads[name].reshape(-1)[idx]
        assert abs(g - fd1) <= 2e-4 * max(abs(fd1), 1e-2), (name, idx, g, fd1)
        ok += 1
    return ok

