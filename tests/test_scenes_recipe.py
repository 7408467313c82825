"""The seeded input generators against the input recipe they implement
(sizes, camera rigs, value ranges and the primitives' geometry), on the CPU.
The generators hold none of the renderer's arithmetic; these checks keep the
benchmark's stand-in workloads what the documentation says they are."""
import math

import numpy as np
import pytest

import scenes


def _eyes(cams):
    out = []
    for c in cams:
        M = np.asarray(c.viewmat, np.float64)
        out.append(-M[:3, :3].T @ M[:3, 3])
    return np.array(out)


def test_workloads_are_deterministic():
    for i in (0, 1, 2, 3, 4):
        a, b = scenes.workload(i, scale=0.01), scenes.workload(i, scale=0.01)
        for k in ("centre", "verts", "opacity", "sh"):
            assert np.array_equal(getattr(a.scene, k), getattr(b.scene, k)), (i, k)
        assert all(np.array_equal(x.viewmat, y.viewmat) for x, y in zip(a.cameras, b.cameras))
    g1 = scenes.image_gradient(scenes.workload(0), seed=3)
    assert np.array_equal(g1, scenes.image_gradient(scenes.workload(0), seed=3))
    assert g1.dtype == np.float32 and g1.shape == (3 * 128 * 128,)


@pytest.mark.parametrize("index, kind, n, views, degree", [
    (0, scenes.TETRAHEDRON, 64, [(128, 128)], 0),
    (1, scenes.OCTAHEDRON, 10_000, [(512, 512)], 3),
    (2, scenes.OCTAHEDRON, 500_000, [(1264, 832)] * 8, 3),
    (3, scenes.TETRAHEDRON, 1_000_000, [(1920, 1080)] * 6 + [(1280, 720)] * 6 + [(640, 480)] * 4, 3),
    (4, scenes.OCTAHEDRON, 2_000_000, [(1600, 1064)] * 4, 3),
])
def test_workload_sizes(index, kind, n, views, degree):
    scale = 1.0 if n <= 500_000 else 0.05
    w = scenes.workload(index, scale=scale)
    m = int(round(n * scale))
    assert w.scene.kind == kind and w.scene.sh_degree == degree
    assert w.scene.centre.shape == (m, 3) and w.scene.verts.shape == (m, kind, 3)
    assert w.scene.opacity.shape == (m,) and w.scene.sh.shape == (m, (degree + 1) ** 2, 3)
    assert [(c.width, c.height) for c in w.cameras] == views
    for arr in (w.scene.centre, w.scene.verts, w.scene.opacity, w.scene.sh):
        assert arr.dtype == np.float32 and arr.flags.c_contiguous


def test_camera_rigs():
    # workload 2: a radius-4 ring around the origin, +-15 deg of jitter, 50 deg vertical FOV
    w = scenes.workload(2, scale=0.001)
    eyes = _eyes(w.cameras)
    assert np.allclose(np.linalg.norm(eyes, axis=1), 4.0, rtol=1e-5)
    assert np.all(np.abs(np.degrees(np.arcsin(eyes[:, 1] / 4.0))) <= 15.0 + 1e-3)
    az = np.degrees(np.arctan2(eyes[:, 0], eyes[:, 2])) % 360.0
    nominal = np.arange(8) * 45.0
    assert np.all(np.abs((az - nominal + 180.0) % 360.0 - 180.0) <= 15.0 + 1e-3)
    for c in w.cameras:
        assert c.fy == pytest.approx(416.0 / math.tan(math.radians(25.0)), rel=1e-6)
        assert (c.fx, c.cx, c.cy) == (c.fy, 632.0, 416.0)
        # the optical axis (third row of the rotation) points at the origin
        M = np.asarray(c.viewmat, np.float64)
        eye = -M[:3, :3].T @ M[:3, 3]
        assert np.allclose(M[2, :3], -eye / np.linalg.norm(eye), atol=1e-6)
        assert np.allclose(M[:3, :3] @ M[:3, :3].T, np.eye(3), atol=1e-6)
    # workload 3: 16 cameras on a radius-6 sphere, 60 deg; workload 1: radius 3, 50 deg
    w3 = scenes.workload(3, scale=0.0001)
    assert np.allclose(np.linalg.norm(_eyes(w3.cameras), axis=1), 6.0, rtol=1e-5)
    assert w3.cameras[0].fy == pytest.approx(540.0 / math.tan(math.radians(30.0)), rel=1e-6)
    w1 = scenes.workload(1, scale=0.01)
    assert np.linalg.norm(_eyes(w1.cameras)[0]) == pytest.approx(3.0, rel=1e-5)


def _octa_axes(sc):
    c = sc.centre.astype(np.float64)
    v = sc.verts.astype(np.float64)
    half = (v[:, 0::2] - v[:, 1::2]) / 2.0                 # the three half-axes
    mid = (v[:, 0::2] + v[:, 1::2]) / 2.0
    return c, half, mid


def test_capture_like_octahedra():
    w = scenes.workload(2, scale=0.05)                      # 25k primitives, same distributions
    c, half, mid = _octa_axes(w.scene)
    assert np.allclose(mid, c[:, None, :], atol=1e-5)       # vertices symmetric about the centre
    d = np.linalg.norm(half, axis=2)
    u = half / d[:, :, None]
    gram = np.einsum("nia,nja->nij", u, u)
    assert np.allclose(gram, np.eye(3), atol=1e-4)           # orthogonal axes (a rotation)
    n = c.shape[0]
    n_core = int(round(0.7 * n))
    core, shell = slice(0, n_core), slice(n_core, n)
    assert d[core].min() >= 0.01 * (1 - 1e-4) and d[core].max() <= 0.08 * (1 + 1e-4)
    assert d[shell].min() >= 0.1 * (1 - 1e-4) and d[shell].max() <= 0.5 * (1 + 1e-4)
    r = np.linalg.norm(c[shell], axis=1)
    assert r.min() >= 8.0 * (1 - 1e-6) and r.max() <= 20.0 * (1 + 1e-6)
    # core centres N(0, I)
    assert np.abs(c[core].mean(0)).max() < 0.05 and np.allclose(c[core].std(0), 1.0, atol=0.05)
    # log-uniform extents: log d uniform, so its mean is the midpoint
    assert np.log(d[core]).mean() == pytest.approx(0.5 * (math.log(0.01) + math.log(0.08)), abs=0.02)
    # opacity sigmoid(N(0, 1.5)): logit mean 0, std 1.5
    o = w.scene.opacity.astype(np.float64)
    logit = np.log(o / (1 - o))
    assert abs(logit.mean()) < 0.05 and logit.std() == pytest.approx(1.5, rel=0.03)
    # SH: DC coefficient U[0, 1], higher bands N(0, 0.05)
    sh = w.scene.sh.astype(np.float64)
    assert sh[:, 0].min() >= 0.0 and sh[:, 0].max() <= 1.0 and sh[:, 0].mean() == pytest.approx(0.5, abs=0.01)
    assert sh[:, 1:].std() == pytest.approx(0.05, rel=0.02) and abs(sh[:, 1:].mean()) < 1e-3


def test_tetrahedra_are_regular_and_colours_reproduce_the_draw():
    w = scenes.workload(3, scale=0.02)                      # 20k tetrahedra in [-3, 3]^3
    c = w.scene.centre.astype(np.float64)
    v = w.scene.verts.astype(np.float64)
    assert np.abs(c).max() <= 3.0
    # circumradius, equal for the 4 vertices up to the binary32 rounding of
    # coordinates of magnitude <= 3 (half an ulp there is 1.2e-7)
    s = np.linalg.norm(v - c[:, None, :], axis=2)
    assert np.allclose(s, s[:, :1], rtol=0.0, atol=1e-6)
    assert s.min() >= 0.005 * (1 - 1e-4) and s.max() <= 0.05 * (1 + 1e-4)
    edges = np.linalg.norm(v[:, [0, 0, 0, 1, 1, 2]] - v[:, [1, 2, 3, 2, 3, 3]], axis=2)
    assert np.allclose(edges, s[:, :1] * math.sqrt(8.0 / 3.0), rtol=0.0, atol=2e-6)   # regular
    # workload 0: degree-0 colours drawn in [0, 1]^3 are what Y00 * sh0 + 0.5 gives back
    w0 = scenes.workload(0)
    rgb = 0.5 / math.sqrt(math.pi) * w0.scene.sh[:, 0].astype(np.float64) + 0.5
    assert rgb.min() >= -1e-6 and rgb.max() <= 1 + 1e-6


def test_uniform_rotations():
    R = scenes.random_rotations(np.random.default_rng(5), 200_000)
    assert np.allclose(np.einsum("nij,nkj->nik", R, R), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)
    # Haar measure on SO(3): every entry has mean 0 and variance 1/3
    assert np.abs(R.mean(0)).max() < 0.005
    assert np.allclose((R ** 2).mean(0), 1.0 / 3.0, atol=0.005)


def test_optimisation_workload_recipe():
    w = scenes.optimisation_workload(scale=0.005)             # 10k primitives, 4 x 1600x1064
    assert [(c.width, c.height) for c in w.cameras] == [(1600, 1064)] * 4
    t, p = w.truth, w.init
    n = t.centre.shape[0]
    assert n == 10_000 and p.centre.shape == (n, 3)
    q = np.asarray(t.quat, np.float64)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-6)
    # the start perturbs centres and distances by N(0, 0.01) and SH by N(0, 0.1);
    # rotations and opacities are unchanged
    dc = np.asarray(p.centre, np.float64) - np.asarray(t.centre, np.float64)
    assert dc.std() == pytest.approx(0.01, rel=0.05)
    dsh = np.asarray(p.sh, np.float64) - np.asarray(t.sh, np.float64)
    assert dsh.std() == pytest.approx(0.1, rel=0.05)
    assert np.array_equal(np.asarray(p.quat), np.asarray(t.quat))
    assert np.array_equal(np.asarray(p.logit), np.asarray(t.logit))
    assert np.asarray(p.dist).min() >= 1e-3
