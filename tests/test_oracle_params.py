"""Pins of the oracle's parameter layer (Sec. 3.1): (centre, quaternion,
distances, opacity logit) -> (vertices, opacity), and its adjoint."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle


def random_params(kind, n, seed):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(n, 3))
    q = rng.normal(size=(n, 4)) * rng.uniform(0.5, 2.0, (n, 1))     # unnormalised on purpose
    d = rng.uniform(0.05, 0.3, (n, 3 if kind == 6 else 4))
    l = rng.normal(size=n)
    return c, q, d, l


@pytest.mark.parametrize("kind", [6, 4])
def test_vertices_match_scipy_rotation(kind):
    """R(q) from scipy (scalar-last quaternion): octahedron vertices at
    c +- d_i R e_i, tetrahedron vertices at c + d_k R b_k."""
    c, q, d, l = random_params(kind, 50, 1)
    v, o = oracle.params_forward(kind, c, q, d, l)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    if kind == 6:
        for i in range(3):
            np.testing.assert_allclose(v[:, 2 * i], c + d[:, i:i + 1] * R[:, :, i], atol=1e-12)
            np.testing.assert_allclose(v[:, 2 * i + 1], c - d[:, i:i + 1] * R[:, :, i], atol=1e-12)
    else:
        b = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]]) / math.sqrt(3)
        for k in range(4):
            np.testing.assert_allclose(v[:, k], c + d[:, k:k + 1] * (R @ b[k]), atol=1e-12)
    np.testing.assert_allclose(o, 1 / (1 + np.exp(-l)), rtol=1e-14)


def test_octahedron_geometry_closed_forms():
    """Sec. 3.1: opposite vertices share a distance, the centre is the true
    geometric centre and the three axes are orthogonal."""
    c, q, d, l = random_params(6, 40, 2)
    v, _ = oracle.params_forward(6, c, q, d, l)
    for i in range(3):
        np.testing.assert_allclose(np.linalg.norm(v[:, 2 * i] - c, axis=1), d[:, i], rtol=1e-12)
        np.testing.assert_allclose(0.5 * (v[:, 2 * i] + v[:, 2 * i + 1]), c, atol=1e-12)
    a = [v[:, 2 * i] - c for i in range(3)]
    for i in range(3):
        for j in range(i + 1, 3):
            assert np.abs(np.sum(a[i] * a[j], axis=1)).max() < 1e-12


def test_regular_tetrahedron_and_identity_rotation():
    """Equal corner distances give a regular tetrahedron (edge d sqrt(8/3));
    the identity quaternion keeps octahedron axes on the coordinate axes."""
    c, q, _, l = random_params(4, 20, 3)
    d = np.full((20, 4), 0.2)
    v, _ = oracle.params_forward(4, c, q, d, l)
    for a in range(4):
        for b in range(a + 1, 4):
            np.testing.assert_allclose(np.linalg.norm(v[:, a] - v[:, b], axis=1), 0.2 * math.sqrt(8 / 3),
                                       rtol=1e-12)
    qi = np.tile([1.0, 0, 0, 0], (20, 1))
    v6, _ = oracle.params_forward(6, c, qi, np.full((20, 3), 0.1), l)
    np.testing.assert_allclose(v6[:, 0], c + [0.1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(v6[:, 5], c - [0, 0, 0.1], atol=1e-15)
    # a quaternion and any positive multiple give the same vertices
    v2, _ = oracle.params_forward(4, c, 3.7 * q, d, l)
    np.testing.assert_allclose(v2, v, atol=1e-13)


@pytest.mark.parametrize("kind", [6, 4])
def test_params_adjoint_fd(kind):
    c, q, d, l = random_params(kind, 6, 4)
    rng = np.random.default_rng(5)
    gv = rng.normal(size=(6, kind, 3))
    go = rng.normal(size=6)
    gc = rng.normal(size=(6, 3))
    out = oracle.params_backward(kind, q, d, l, gv, go, gc)

    def L(c_, q_, d_, l_):
        v, o = oracle.params_forward(kind, c_, q_, d_, l_)
        return float(np.sum(v * gv) + np.sum(o * go) + np.sum(c_ * gc))
    h = 1e-6
    for name, arr in (("centre", c), ("quat", q), ("dist", d), ("logit", l)):
        flat = arr.reshape(-1)
        for idx in range(flat.size):
            args = {"centre": c, "quat": q, "dist": d, "logit": l}
            p1 = {k: v.copy() for k, v in args.items()}
            p2 = {k: v.copy() for k, v in args.items()}
            p1[name].reshape(-1)[idx] += h
            p2[name].reshape(-1)[idx] -= h
            fd = (L(p1["centre"], p1["quat"], p1["dist"], p1["logit"]) -
                  L(p2["centre"], p2["quat"], p2["dist"], p2["logit"])) / (2 * h)
            g = out[name].reshape(-1)[idx]
            assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (name, idx, g, fd)
