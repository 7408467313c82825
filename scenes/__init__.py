"""Seeded synthetic scenes and pinhole cameras for the LinPrim rasterizer.

This module only *draws inputs*: primitive centres, world-space vertices,
opacities, spherical-harmonic (SH) coefficients and cameras, from numpy's
PCG64 generator with a fixed draw order.  It contains none of the rendering
arithmetic (no projection, intersection, density, blending or gradients), so
both the FP64 oracle and the CUDA path can take their inputs from here without
sharing any of the method.

Primitive geometry follows the paper's parameterisation (Sec. 3.1):

* octahedron: six vertices on the rotated coordinate axes around the centre,
  opposite vertices at the same distance; vertex order is
  (+a0, -a0, +a1, -a1, +a2, -a2) where a_i = R . (d_i e_i);
* tetrahedron: four vertices along the equally spaced directions of a regular
  tetrahedron (circumradius 1 before scaling), rotated by R.

Rotations are uniform random quaternions (Shoemake's subgroup algorithm).
Cameras are world->camera 4x4 matrices in OpenCV axes (x right, y down,
z forward) with square pixels and the principal point at the image centre.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

OCTAHEDRON = 6
TETRAHEDRON = 4

# Unit directions of a regular tetrahedron (circumradius 1): the (+-1, +-1, +-1)
# corners of a cube with an even number of minus signs, normalised.
_TETRA_DIRS = np.array(
    [[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]]
) / math.sqrt(3.0)

# Zeroth-order real SH normalisation 1/(2 sqrt(pi)); used only to turn a drawn
# RGB colour into the DC coefficient that reproduces it.
_SH_Y00 = 0.5 / math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    """A population of primitives in the boundary's structure-of-arrays form."""

    kind: int                 # OCTAHEDRON (6 vertices) or TETRAHEDRON (4)
    centre: np.ndarray        # f32 [N, 3]
    verts: np.ndarray         # f32 [N, V, 3]
    opacity: np.ndarray       # f32 [N], in (0, 1)
    sh: np.ndarray            # f32 [N, K, 3], K = (sh_degree + 1)^2
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.centre.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.kind, self.centre[idx].copy(), self.verts[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.sh_degree)


@dataclasses.dataclass
class Camera:
    viewmat: np.ndarray       # f32 [4, 4], world -> camera, row-major
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def pixels(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cameras: List[Camera]
    bg: tuple = (0.0, 0.0, 0.0)

    @property
    def pixels(self) -> int:
        return sum(c.pixels for c in self.cameras)


# ---------------------------------------------------------------- draw helpers

def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices [n, 3, 3] via Shoemake's quaternions."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qx = a * np.sin(2 * np.pi * u2)
    qy = a * np.cos(2 * np.pi * u2)
    qz = b * np.sin(2 * np.pi * u3)
    qw = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def octahedra_from_axes(centre, R, dists) -> np.ndarray:
    """Vertices [n, 6, 3]: centre +- R[:, :, i] * d_i for i = 0, 1, 2."""
    n = centre.shape[0]
    v = np.empty((n, 6, 3))
    for i in range(3):
        axis = R[:, :, i] * dists[:, i:i + 1]
        v[:, 2 * i] = centre + axis
        v[:, 2 * i + 1] = centre - axis
    return v


def tetrahedra_from_scale(centre, R, s) -> np.ndarray:
    """Vertices [n, 4, 3]: centre + s * R . dir_k for the four tetrahedron directions."""
    d = np.einsum("nij,kj->nki", R, _TETRA_DIRS)
    return centre[:, None, :] + s[:, None, None] * d


def sh_from_rgb(rgb: np.ndarray) -> np.ndarray:
    """DC coefficient whose degree-0 colour (Y00 * sh0 + 0.5) equals rgb."""
    return (rgb - 0.5) / _SH_Y00


def draw_sh(rng, n, degree, dc, rest_std=0.05) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = dc
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def _finish(kind, centre, verts, opacity, sh, degree) -> Scene:
    return Scene(kind, np.ascontiguousarray(centre, np.float32),
                 np.ascontiguousarray(verts, np.float32),
                 np.ascontiguousarray(opacity, np.float32),
                 np.ascontiguousarray(sh, np.float32), degree)


# --------------------------------------------------------------------- cameras

def intrinsics(width: int, height: int, fov_y_deg: float):
    fy = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return fy, fy, width / 2.0, height / 2.0


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera matrix, OpenCV axes (x right, y down, z toward the target).

    If the viewing direction is within 1e-3 of the up vector, +z is used as up.
    """
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(abs(np.dot(fwd, up / np.linalg.norm(up))) - 1.0) < 1e-3:
        up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)           # camera +x
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)         # camera +y
    Rw = np.stack([right, down, fwd])   # rows: camera axes in world coords
    M = np.eye(4)
    M[:3, :3] = Rw
    M[:3, 3] = -Rw @ eye
    return M


def make_camera(eye, width, height, fov_y_deg, target=(0.0, 0.0, 0.0)) -> Camera:
    """Camera whose matrix and intrinsics are exactly representable in binary32,
    so both the binary32 renderer and a binary64 reference see the same values."""
    f32 = lambda x: float(np.float32(x))
    fx, fy, cx, cy = intrinsics(width, height, fov_y_deg)
    return Camera(look_at(eye, target).astype(np.float32), f32(fx), f32(fy),
                  f32(cx), f32(cy), int(width), int(height))


def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ------------------------------------------------------------------- workloads

def tetra_scene(seed=0, n=64, box=1.0, s_range=(0.05, 0.2), sh_degree=0,
                rest_std=0.05, rng=None) -> Scene:
    """Random tetrahedra: centres uniform in [-box, box]^3, log-uniform scale,
    opacity sigmoid(N(0,1)), DC colour uniform in [0,1]^3."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    centre = rng.uniform(-box, box, (n, 3))
    s = log_uniform(rng, s_range[0], s_range[1], n)
    R = random_rotations(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.0, n))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = draw_sh(rng, n, sh_degree, sh_from_rgb(rgb), rest_std)
    return _finish(TETRAHEDRON, centre, tetrahedra_from_scale(centre, R, s),
                   opacity, sh, sh_degree)


def octa_scene(seed=1, n=10_000, centre_std=0.5, ext_range=(0.01, 0.08),
               opacity_std=1.5, sh_degree=3, rest_std=0.05, rng=None) -> Scene:
    """Random octahedra: centres N(0, centre_std^2 I), per-axis log-uniform
    extents, opacity sigmoid(N(0, opacity_std^2)), DC coefficient U[0,1]."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    centre = rng.normal(0.0, centre_std, (n, 3))
    d = log_uniform(rng, ext_range[0], ext_range[1], (n, 3))
    R = random_rotations(rng, n)
    opacity = _sigmoid(rng.normal(0.0, opacity_std, n))
    sh = draw_sh(rng, n, sh_degree, rng.uniform(0.0, 1.0, (n, 3)), rest_std)
    return _finish(OCTAHEDRON, centre, octahedra_from_axes(centre, R, d),
                   opacity, sh, sh_degree)


def capture_like_octa_scene(seed=2, n=500_000, core_frac=0.7, sh_degree=3,
                            rng=None) -> Scene:
    """Unbounded-capture stand-in: an object core (centres N(0, I), extents
    log-U[0.01, 0.08]) plus a background shell (uniform directions at radius
    U[8, 20], extents log-U[0.1, 0.5])."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    n_core = int(round(core_frac * n))
    n_shell = n - n_core
    centre = np.concatenate([
        rng.normal(0.0, 1.0, (n_core, 3)),
        _unit_vectors(rng, n_shell) * rng.uniform(8.0, 20.0, (n_shell, 1)),
    ])
    d = np.concatenate([
        log_uniform(rng, 0.01, 0.08, (n_core, 3)),
        log_uniform(rng, 0.1, 0.5, (n_shell, 3)),
    ])
    R = random_rotations(rng, n)
    opacity = _sigmoid(rng.normal(0.0, 1.5, n))
    sh = draw_sh(rng, n, sh_degree, rng.uniform(0.0, 1.0, (n, 3)))
    return _finish(OCTAHEDRON, centre, octahedra_from_axes(centre, R, d),
                   opacity, sh, sh_degree)


@dataclasses.dataclass
class ParamScene:
    """Primitives in the optimised parameter form: centre [n,3], quaternion
    (w, x, y, z) [n,4], distances [n,3] (octahedron) or [n,4] (tetrahedron),
    opacity logit [n], SH [n,K,3]; all float32."""
    kind: int
    centre: np.ndarray
    quat: np.ndarray
    dist: np.ndarray
    logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.centre.shape[0])


def random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z) [n, 4] (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    return np.stack([b * np.cos(2 * np.pi * u3), a * np.sin(2 * np.pi * u2),
                     a * np.cos(2 * np.pi * u2), b * np.sin(2 * np.pi * u3)], axis=1)


def capture_like_octa_params(n=2_000_000, core_frac=0.7, sh_degree=3, rng=None, seed=4) -> ParamScene:
    """The capture-like octahedron distribution (object core plus background
    shell, as capture_like_octa_scene) drawn directly in parameter form."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    n_core = int(round(core_frac * n))
    n_shell = n - n_core
    centre = np.concatenate([
        rng.normal(0.0, 1.0, (n_core, 3)),
        _unit_vectors(rng, n_shell) * rng.uniform(8.0, 20.0, (n_shell, 1)),
    ])
    dist = np.concatenate([
        log_uniform(rng, 0.01, 0.08, (n_core, 3)),
        log_uniform(rng, 0.1, 0.5, (n_shell, 3)),
    ])
    quat = random_quaternions(rng, n)
    logit = rng.normal(0.0, 1.5, n)
    sh = draw_sh(rng, n, sh_degree, rng.uniform(0.0, 1.0, (n, 3)))
    f = lambda a: np.ascontiguousarray(a, np.float32)
    return ParamScene(OCTAHEDRON, f(centre), f(quat), f(dist), f(logit), f(sh), sh_degree)


def perturb_params(p: ParamScene, rng, pos_std=0.01, sh_std=0.1, dist_floor=1e-3) -> ParamScene:
    """Starting point of an optimisation towards p: centres and distances
    moved by N(0, pos_std) (distances kept >= dist_floor), SH by N(0, sh_std);
    rotations and opacities unchanged."""
    f = lambda a: np.ascontiguousarray(a, np.float32)
    centre = p.centre + rng.normal(0.0, pos_std, p.centre.shape)
    dist = np.maximum(np.abs(p.dist + rng.normal(0.0, pos_std, p.dist.shape)), dist_floor)
    sh = p.sh + rng.normal(0.0, sh_std, p.sh.shape)
    return ParamScene(p.kind, f(centre), p.quat.copy(), f(dist), p.logit.copy(), f(sh), p.sh_degree)


@dataclasses.dataclass
class ParamWorkload:
    name: str
    truth: ParamScene
    init: ParamScene
    cameras: List[Camera]

    @property
    def pixels(self) -> int:
        return sum(c.pixels for c in self.cameras)


def optimisation_workload(scale: float = 1.0) -> ParamWorkload:
    """The optimisation-step workload: 2M capture-like octahedra in parameter
    form (ground truth), its perturbation (the starting point) and 4 views
    1600x1064 (50 deg) on a radius-4 ring; `scale` scales the primitive count."""
    rng = np.random.default_rng(4)
    n = max(1, int(round(2_000_000 * scale)))
    truth = capture_like_octa_params(n=n, rng=rng)
    cams = ring_cameras(rng, 4, 4.0, 1600, 1064, 50.0)
    init = perturb_params(truth, rng)
    return ParamWorkload("octa2M_4x1600x1064_train" if n == 2_000_000 else f"octa{n}_4x1600x1064_train",
                         truth, init, cams)


def ring_cameras(rng, n_views, radius, width, height, fov_y_deg, jitter_deg=15.0):
    cams = []
    for i in range(n_views):
        az = 2 * math.pi * i / n_views + math.radians(rng.uniform(-jitter_deg, jitter_deg))
        el = math.radians(rng.uniform(-jitter_deg, jitter_deg))
        eye = radius * np.array([math.cos(el) * math.sin(az), math.sin(el),
                                 math.cos(el) * math.cos(az)])
        cams.append(make_camera(eye, width, height, fov_y_deg))
    return cams


def sphere_cameras(rng, sizes: Sequence[tuple], radius, fov_y_deg):
    cams = []
    dirs = _unit_vectors(rng, len(sizes))
    for (w, h), d in zip(sizes, dirs):
        cams.append(make_camera(radius * d, w, h, fov_y_deg))
    return cams


def workload(index: int, scale: float = 1.0) -> Workload:
    """The five evaluation workloads (index 0..4), optionally with the primitive
    count scaled by `scale` (same distributions, fewer primitives).

    0: 64 tetrahedra, one 128x128 view (60 deg), SH degree 0.
    1: 10k octahedra, one 512x512 view on a radius-3 sphere (50 deg), SH 3.
    2: 500k capture-like octahedra, 8 views 1264x832 on a radius-4 ring.
    3: 1M tetrahedra in [-3,3]^3, 16 mixed-resolution views (60 deg), SH 3.
    4: 2M capture-like octahedra, 4 views 1600x1064 (50 deg), SH 3.
    """
    rng = np.random.default_rng(index)
    sn = lambda n: max(1, int(round(n * scale)))
    if index == 0:
        sc = tetra_scene(n=sn(64), rng=rng)
        cams = [make_camera((0.0, 0.0, 4.0), 128, 128, 60.0)]
        return Workload("tetra64_128x128", sc, cams)
    if index == 1:
        sc = octa_scene(n=sn(10_000), rng=rng)
        eye = 3.0 * _unit_vectors(rng, 1)[0]
        return Workload("octa10k_512x512", sc, [make_camera(eye, 512, 512, 50.0)])
    if index == 2:
        sc = capture_like_octa_scene(n=sn(500_000), rng=rng)
        cams = ring_cameras(rng, 8, 4.0, 1264, 832, 50.0)
        return Workload("octa500k_8x1264x832", sc, cams)
    if index == 3:
        sc = tetra_scene(n=sn(1_000_000), box=3.0, s_range=(0.005, 0.05),
                         sh_degree=3, rng=rng)
        sizes = [(1920, 1080)] * 6 + [(1280, 720)] * 6 + [(640, 480)] * 4
        cams = sphere_cameras(rng, sizes, 6.0, 60.0)
        return Workload("tetra1M_16mixed", sc, cams)
    if index == 4:
        sc = capture_like_octa_scene(n=sn(2_000_000), rng=rng)
        cams = ring_cameras(rng, 4, 4.0, 1600, 1064, 50.0)
        return Workload("octa2M_4x1600x1064", sc, cams)
    raise ValueError(f"no workload {index}")


def image_gradient(workload: Workload, seed: int = 0) -> np.ndarray:
    """dL/dimage ~ N(0,1), packed [cam][3][H][W] in camera order, float32."""
    rng = np.random.default_rng(1000 + seed)
    return rng.normal(0.0, 1.0, 3 * workload.pixels).astype(np.float32)
