"""Pins of the population-control oracle (Sec. 3.4 "Adaptive Population
Control", App. "Experimental Setting") against geometry, closed forms, brute
force and finite differences of the oracle's forward render."""
import math

import numpy as np
import pytest

import scenes
from oracle import population as pop

f32 = np.float32


@pytest.fixture(scope="module")
def orc():
    import oracle
    return oracle


def _params(kind, n, rng, deg=0):
    D = 3 if kind == 6 else 4
    return dict(centre=rng.normal(size=(n, 3)), quat=scenes.random_quaternions(rng, n),
                dist=rng.uniform(0.05, 0.3, size=(n, D)), logit=rng.normal(size=n),
                sh=rng.normal(size=(n, (deg + 1) ** 2, 3)))


# ------------------------------------------------------------ size

@pytest.mark.parametrize("kind", [6, 4])
def test_size_matches_the_vertex_geometry(orc, kind):
    """Octahedron: the longest axis (vertex to opposite vertex); tetrahedron:
    sqrt(2) times the distance to the furthest corner, both measured on the
    vertices of the parameter layer."""
    rng = np.random.default_rng(1)
    p = _params(kind, 40, rng)
    p["dist"][::3] *= -1.0            # distances enter by magnitude
    v, _ = orc.params_forward(kind, p["centre"], p["quat"], p["dist"], p["logit"])
    for i in range(40):
        if kind == 6:
            ref = max(np.linalg.norm(v[i, 2 * a] - v[i, 2 * a + 1]) for a in range(3))
        else:
            ref = math.sqrt(2.0) * max(np.linalg.norm(v[i, k] - p["centre"][i]) for k in range(4))
        assert abs(float(pop.size32(kind, p["dist"][i])) - ref) <= 2e-6 * ref


# ------------------------------------------------------------ decision

def _one(kind, dist, logit, gsum=0.0, gcnt=1, px=0, extent=10.0):
    return int(pop.decide(kind, np.array([dist], f32), np.array([logit], f32), np.array([gsum], f32),
                          np.array([gcnt], np.uint32), np.array([px], np.uint32), extent)[0])


def test_decide_opacity_threshold():
    p = float(f32(0.025))
    thr = math.log(p / (1.0 - p))
    below = float(np.nextafter(f32(thr), f32(-10)))
    assert 1.0 / (1.0 + math.exp(-below)) < 0.025
    assert _one(6, [0.1] * 3, below) == pop.PRUNE
    assert _one(6, [0.1] * 3, float(f32(thr))) == pop.KEEP
    assert _one(6, [0.1] * 3, 0.0) == pop.KEEP


@pytest.mark.parametrize("kind", [6, 4])
def test_decide_world_size_threshold(kind):
    """Removed above 40% of the scene extent (strictly), by Sec. 3.4's size."""
    ext = 10.0
    big = f32(f32(0.4) * f32(ext))
    k = 2.0 if kind == 6 else math.sqrt(2.0)
    D = 3 if kind == 6 else 4
    # the largest distance whose size is exactly the bound (if representable)
    d = f32(big / f32(k))
    while pop.size32(kind, [d] * D) > big:
        d = np.nextafter(d, f32(0))
    while pop.size32(kind, [np.nextafter(d, f32(np.inf))] * D) <= big:
        d = np.nextafter(d, f32(np.inf))
    assert _one(kind, [float(d)] + [0.01] * (D - 1), 0.0, extent=ext) == pop.KEEP
    assert _one(kind, [float(np.nextafter(d, f32(np.inf)))] + [0.01] * (D - 1), 0.0, extent=ext) == pop.PRUNE
    assert _one(kind, [-float(np.nextafter(d, f32(np.inf)))] + [0.01] * (D - 1), 0.0, extent=ext) == pop.PRUNE


def test_decide_screen_size_threshold():
    assert _one(6, [0.1] * 3, 0.0, px=20) == pop.KEEP
    assert _one(6, [0.1] * 3, 0.0, px=21) == pop.PRUNE


@pytest.mark.parametrize("kind", [6, 4])
def test_decide_clone_bound(kind):
    """Cloned strictly below 1% of the scene extent: a size exactly on the
    bound is split."""
    ext = 7.0
    small = f32(f32(0.01) * f32(ext))
    D = 3 if kind == 6 else 4
    d = f32(small / f32(2.0 if kind == 6 else math.sqrt(2.0)))
    while pop.size32(kind, [d] * D) > small:
        d = np.nextafter(d, f32(0))
    while pop.size32(kind, [np.nextafter(d, f32(np.inf))] * D) <= small:
        d = np.nextafter(d, f32(np.inf))
    below = np.nextafter(d, f32(0))
    while pop.size32(kind, [below] * D) >= small:     # sqrt(2) d: neighbours can round alike
        below = np.nextafter(below, f32(0))
    assert _one(kind, [float(below)] * D, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.CLONE
    if pop.size32(kind, [d] * D) == small:
        assert _one(kind, [float(d)] * D, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.SPLIT
    assert _one(kind, [float(np.nextafter(d, f32(np.inf)))] * D, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.SPLIT


@pytest.mark.parametrize("cnt", [1, 2, 4])
def test_decide_gradient_bound(cnt):
    """Densified only strictly above the threshold: a mean exactly on it is kept."""
    thr = f32(1.5e-4)
    on = f32(thr * f32(cnt))                  # exact: cnt is a power of two
    assert _one(6, [0.01] * 3, 0.0, gsum=float(on), gcnt=cnt) == pop.KEEP
    up = np.nextafter(on, f32(1))
    assert _one(6, [0.01] * 3, 0.0, gsum=float(up), gcnt=cnt) == pop.CLONE


def test_decide_densification():
    ext = 10.0
    # mean gradient strictly above 1.5e-4 over the visible views
    assert _one(6, [0.01] * 3, 0.0, gsum=3 * 1.5e-4, gcnt=3) == pop.KEEP      # equal: not above
    assert _one(6, [0.01] * 3, 0.0, gsum=3 * 1.6e-4, gcnt=3) == pop.CLONE
    assert _one(6, [0.01] * 3, 0.0, gsum=1.6e-4, gcnt=0) == pop.KEEP          # never visible
    # clone strictly below 1% of the extent (size 2 d for an octahedron)
    assert _one(6, [0.0499] * 3, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.CLONE
    assert _one(6, [0.05] * 3, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.SPLIT
    assert _one(4, [0.0707] * 4, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.CLONE
    assert _one(4, [0.0708] * 4, 0.0, gsum=1.0, gcnt=1, extent=ext) == pop.SPLIT
    # pruning has priority over densification
    assert _one(6, [0.01] * 3, -5.0, gsum=1.0, gcnt=1) == pop.PRUNE
    assert _one(6, [0.01] * 3, 0.0, gsum=1.0, gcnt=1, px=25) == pop.PRUNE


def test_destinations_brute_force():
    rng = np.random.default_rng(3)
    act = rng.integers(0, 4, size=1000)
    dest, total = pop.destinations(act)
    run = 0
    for i, a in enumerate(act):
        assert dest[i] == run
        run += [0, 1, 2, 2][a]
    assert total == run


# ------------------------------------------------------------ application

@pytest.mark.parametrize("kind", [6, 4])
def test_apply_order_copies_and_states(kind):
    rng = np.random.default_rng(5)
    n = 50
    p = _params(kind, n, rng, deg=1)
    states = [{k: rng.normal(size=np.shape(v)) for k, v in p.items()} for _ in range(2)]
    act = rng.integers(0, 4, size=n)
    normals = rng.normal(size=(n, 2, 3))
    q, qs = pop.apply(kind, p, states, act, normals)
    dest, total = pop.destinations(act)
    assert q["centre"].shape[0] == total
    for i in range(n):
        o = dest[i]
        if act[i] in (pop.KEEP, pop.CLONE):
            for k in p:
                assert np.array_equal(q[k][o], p[k][i])
                for s, st in zip(qs, states):
                    assert np.array_equal(s[k][o], st[k][i])
        if act[i] == pop.CLONE:
            for k in p:
                assert np.array_equal(q[k][o + 1], p[k][i])
                for s in qs:
                    assert not np.any(s[k][o + 1])
        if act[i] == pop.SPLIT:
            for j in range(2):
                np.testing.assert_allclose(q["dist"][o + j], p["dist"][i] / 1.2, rtol=1e-15)
                for k in ("quat", "logit", "sh"):
                    assert np.array_equal(q[k][o + j], p[k][i])
                for s in qs:
                    for k in p:
                        assert not np.any(s[k][o + j])


def test_split_octahedron_child_on_a_vertex(orc):
    """With the draw z = +-e_a the child lands on the origin's vertex along
    rotated axis a (standard deviation = that distance, along that axis)."""
    rng = np.random.default_rng(7)
    p = _params(6, 8, rng)
    p["dist"][1] *= -1.0
    v, _ = orc.params_forward(6, p["centre"], p["quat"], p["dist"], p["logit"])
    for a in range(3):
        normals = np.zeros((8, 2, 3))
        normals[:, 0, a] = 1.0
        normals[:, 1, a] = -1.0
        q, _ = pop.apply(6, p, [], np.full(8, pop.SPLIT), normals)
        for i in range(8):
            ends = sorted([v[i, 2 * a], v[i, 2 * a + 1]], key=lambda x: tuple(x))
            got = sorted([q["centre"][2 * i], q["centre"][2 * i + 1]], key=lambda x: tuple(x))
            np.testing.assert_allclose(got, ends, atol=1e-12)


def test_split_octahedron_std_is_the_distance_magnitude(orc):
    """A standard deviation is non-negative: with the draw z = +e_a the child
    is offset by |d_a| along the rotated axis R e_a, which the parameter layer
    gives as (v_2a - c) / d_a, whatever the sign of d_a."""
    rng = np.random.default_rng(17)
    p = _params(6, 8, rng)
    p["dist"][::2] *= -1.0
    v, _ = orc.params_forward(6, p["centre"], p["quat"], p["dist"], p["logit"])
    for a in range(3):
        normals = np.zeros((8, 2, 3))
        normals[:, 0, a] = 1.0
        q, _ = pop.apply(6, p, [], np.full(8, pop.SPLIT), normals)
        axis = (v[:, 2 * a] - p["centre"]) / p["dist"][:, a:a + 1]
        np.testing.assert_allclose(q["centre"][0::2], p["centre"] + np.abs(p["dist"][:, a:a + 1]) * axis,
                                   atol=1e-12)


def test_split_tetrahedron_child_halfway_to_corner(orc):
    """Isotropic standard deviation of half the largest distance: with equal
    distances and z the unit direction to a corner, the child lies halfway
    between the centre and that corner."""
    rng = np.random.default_rng(8)
    p = _params(4, 8, rng)
    p["dist"][:] = rng.uniform(0.1, 0.3, size=(8, 1))
    v, _ = orc.params_forward(4, p["centre"], p["quat"], p["dist"], p["logit"])
    for k in range(4):
        u = v[:, k] - p["centre"]
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        normals = np.stack([u, u], axis=1)
        q, _ = pop.apply(4, p, [], np.full(8, pop.SPLIT), normals)
        np.testing.assert_allclose(q["centre"][0::2], 0.5 * (p["centre"] + v[:, k]), atol=1e-12)


@pytest.mark.parametrize("kind", [6, 4])
def test_split_offset_covariance(kind):
    """Over many draws the child offsets have covariance R diag(d^2) R^T
    (octahedron) or (max|d| / 2)^2 I (tetrahedron)."""
    rng = np.random.default_rng(9)
    p = _params(kind, 1, rng)
    m = 40_000
    rep = {k: np.repeat(v, m, axis=0) for k, v in p.items()}
    normals = rng.normal(size=(m, 2, 3))
    q, _ = pop.apply(kind, rep, [], np.full(m, pop.SPLIT), normals)
    off = q["centre"] - p["centre"][0]
    cov = off.T @ off / off.shape[0]
    d = np.abs(p["dist"][0])
    if kind == 6:
        R = pop.quat_rotation(p["quat"][0])
        ref = R @ np.diag(d ** 2) @ R.T
    else:
        ref = (d.max() / 2) ** 2 * np.eye(3)
    assert np.max(np.abs(cov - ref)) < 0.03 * np.max(np.abs(ref))


# ------------------------------------------------------------ statistics

@pytest.mark.parametrize("dists", [(0.31, 0.07, 0.05), (0.06, 0.27, 0.05)])
def test_screen_pixels_of_a_facing_octahedron(orc, dists):
    """An axis-aligned octahedron straight ahead of the camera projects its x
    (y) vertices to x_c +- f_x d_x / z (y_c +- f_y d_y / z): the covered
    columns (rows) are the pixel centres in that interval; the size is the
    larger count."""
    cam = scenes.make_camera((0.0, 0.0, 0.0), 96, 64, 60.0, target=(0.0, 0.0, 1.0))
    M = cam.viewmat.astype(np.float64)
    z = 3.0
    c = np.array([[0.0, 0.0, z]])
    R = M[:3, :3].T                          # camera axes in world coordinates
    verts = scenes.octahedra_from_axes(c, R[None], np.array([dists]))
    sc = scenes.Scene(6, c.astype(f32), verts.astype(f32), np.array([0.5], f32),
                      np.zeros((1, 1, 3), f32), 0)
    ext = pop.screen_pixels(orc, sc, [cam])
    tc = M[:3, :3] @ c[0] + M[:3, 3]
    xc = float(cam.fx) * tc[0] / tc[2] + float(cam.cx)
    yc = float(cam.fy) * tc[1] / tc[2] + float(cam.cy)
    wx = float(cam.fx) * dists[0] / tc[2]
    wy = float(cam.fy) * dists[1] / tc[2]
    cols = [x for x in range(cam.width) if xc - wx <= x + 0.5 <= xc + wx]
    rows = [y for y in range(cam.height) if yc - wy <= y + 0.5 <= yc + wy]
    assert ext[0] == max(len(cols), len(rows)) and abs(len(cols) - len(rows)) > 5


def test_view_gradient_matches_finite_differences(orc):
    """The NDC view-space position gradient against central differences of
    <g, image> under a translation of one primitive parallel to the image
    plane (centre and vertices moved together)."""
    w = scenes.workload(0)
    sc = w.scene
    # an oblique, non-square view (a generic rotation; W != H) with
    # non-square pixels (f_y != f_x), so that each axis's scale is its own
    cam = scenes.make_camera((2.6, -1.3, 2.9), 112, 72, 55.0)
    cam.fy = float(np.float32(1.25 * cam.fx))
    rng = np.random.default_rng(11)
    gimg = rng.normal(size=3 * cam.pixels)
    dmin = orc.preprocess(sc, cam)["dmin"]
    _, g = orc.render(sc, [cam], dL_dimage=gimg, dmin=dmin)
    vg = pop.view_gradient(cam, sc.centre, g["centre"], g["verts"])
    M = cam.viewmat.astype(np.float64)
    pp = orc.preprocess(sc, cam)
    z = sc.centre.astype(np.float64) @ M[2, :3] + M[2, 3]
    checked = 0
    for i in rng.permutation(np.nonzero(pp["visible"])[0])[:12]:
        for ax in range(2):
            scale = (cam.width if ax == 0 else cam.height) * z[i] / (2.0 * float(cam.fx if ax == 0 else cam.fy))
            t = M[ax, :3] * scale                 # world direction of a unit NDC shift

            def L(h):
                c = sc.centre.astype(np.float64).copy()
                v = sc.verts.astype(np.float64).copy()
                c[i] += h * t
                v[i] += h * t
                s2 = scenes.Scene(sc.kind, c, v, sc.opacity.astype(np.float64), sc.sh.astype(np.float64),
                                  sc.sh_degree)
                return float(np.dot(orc.render(s2, [cam], dmin=dmin), gimg))

            h = 1e-6
            fd1 = (L(h) - L(-h)) / (2 * h)
            fd2 = (L(h / 2) - L(-h / 2)) / h
            if abs(fd1 - fd2) > 1e-4 * max(abs(fd1), 1e-3):
                continue                          # a kink
            assert abs(vg[i, ax] - fd1) <= 2e-4 * max(abs(fd1), 1e-2), (i, ax, vg[i, ax], fd1)
            checked += 1
    assert checked >= 10


def test_gradient_stats_sum_over_views(orc):
    """Per-view norms add up; the count is the number of views with a
    non-empty pixel rectangle."""
    w = scenes.workload(0)
    rng = np.random.default_rng(12)
    cams = scenes.sphere_cameras(rng, [(48, 40), (40, 32)], 4.0, 60.0)
    sc = w.scene
    dL = [rng.normal(size=3 * c.pixels) for c in cams]
    acc, cnt = pop.gradient_stats(orc, sc, cams, np.concatenate(dL))
    ref_acc = np.zeros(sc.n)
    ref_cnt = np.zeros(sc.n, np.int64)
    for c, d in zip(cams, dL):
        a1, c1 = pop.gradient_stats(orc, sc, [c], d)
        ref_acc += a1
        ref_cnt += c1
        r = orc.preprocess(sc, c)["rect"]
        vis = orc.preprocess(sc, c)["visible"] & (r[:, 0] <= r[:, 1]) & (r[:, 2] <= r[:, 3])
        assert np.array_equal(c1, vis.astype(np.int64))
        assert np.all(a1[~vis] == 0.0)
    np.testing.assert_allclose(acc, ref_acc, rtol=1e-12)
    assert np.array_equal(cnt, ref_cnt) and cnt.max() == 2
