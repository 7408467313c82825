"""Adaptive population control (Sec. 3.4 "Adaptive Population Control",
App. "Experimental Setting") -- TEST INFRASTRUCTURE ONLY: imported by the
tests, the smoke check and the benchmark's CPU baseline, never by the product.

Plain numpy, one primitive at a time.  Integer outcomes (the action of each
primitive, the output order, the new count) are decided in binary32 with the
same operands and operations as the GPU kernels, so they compare exactly;
everything else is binary64.

Readings of the paper (each also listed with the design notes):
  * size: an octahedron's longest axis, twice its largest distance; a
    tetrahedron's sqrt(2) times the distance to its furthest corner (Sec. 3.4).
    Distances enter by magnitude.
  * prune (App.): opacity sigmoid(logit) below 0.025 -- decided as logit below
    the binary32 rounding of log(p / (1 - p)), p the binary32 0.025 evaluated
    in binary64; size above 40% of the scene
    extent; or more than 20 pixels of a known view -- the largest side, in
    pixels, of the primitive's pixel rectangle (clipped to the image) over the
    views rendered since the last adjustment.
  * densify (App.): primitives whose mean view-space position gradient is
    above 1.5e-4.  The view-space position gradient of one view is the
    gradient of the loss w.r.t. a translation of the whole primitive parallel
    to that view's image plane, in NDC units (x_ndc = 2 px / W - 1); its norm
    is summed over the views in which the primitive was visible (non-empty
    pixel rectangle) and divided by their number.
  * pruning has priority: a pruned primitive is not densified.  The rest are
    cloned when smaller than 1% of the scene extent, else split.
  * clone (Sec. 3.4): a copy with the same features and zero optimiser state
    placed right after its origin, which keeps its state.
  * split (App.): the origin is replaced by two children, in its place, with
    distances divided by 1.2 and zero optimiser state; child j's centre is the
    origin's plus, for an octahedron, R(q) (|d| * z_j) (standard deviations
    equal to the distances along the rotated axes), for a tetrahedron,
    (max |d| / 2) z_j, with z_j a standard-normal draw passed in.
  * the scene extent is the caller's (the optimiser uses the largest distance
    between a camera and the mean camera position, the scale the paper gives
    the distance learning rate).
"""
from __future__ import annotations

import math

import numpy as np

PRUNE_OPACITY = 0.025
PRUNE_SCENE_FRAC = 0.4
PRUNE_PIXELS = 20
DENSIFY_GRAD = 1.5e-4
CLONE_SCENE_FRAC = 0.01
SPLIT_SHRINK = 1.2

PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3

f32 = np.float32


def quat_rotation(q):
    """Rotation matrix of the quaternion (w, x, y, z), normalised first."""
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def size32(kind, d):
    """Sec. 3.4's size of one primitive, in binary32."""
    m = f32(np.max(np.abs(np.asarray(d, f32))))
    return f32(f32(2.0) * m) if kind == 6 else f32(f32(math.sqrt(2.0)) * m)


# ------------------------------------------------------------ statistics

def screen_pixels(orc, scene, cameras, aa=0.0, exact=False):
    """Per primitive, the largest side of its pixel rectangle over the views
    (0 where never visible); the rectangle is the oracle's binary32 one."""
    ext = np.zeros(scene.n, np.int64)
    for cam in cameras:
        pp = orc.preprocess(scene, cam, aa=aa, exact=exact)
        r = pp["rect"]                    # inclusive px0, px1, py0, py1
        ok = pp["visible"] & (r[:, 0] <= r[:, 1]) & (r[:, 2] <= r[:, 3])
        side = np.maximum(r[:, 1] - r[:, 0] + 1, r[:, 3] - r[:, 2] + 1)
        ext = np.maximum(ext, np.where(ok, side, 0))
    return ext


def view_gradient(camera, centre, g_centre, g_verts):
    """NDC view-space position gradient of each primitive for one view, from
    that view's world-space gradients of the renderer's inputs.  A translation
    by t moves the centre and every vertex by t, so its gradient is
    g_centre + sum_k g_verts[k]; a shift of the NDC x coordinate by delta at
    fixed depth z is a camera-space shift of delta W z / (2 f_x)."""
    M = np.asarray(camera.viewmat, np.float64).reshape(4, 4)
    g = np.asarray(g_centre, np.float64) + np.asarray(g_verts, np.float64).sum(axis=1)
    gc = g @ M[:3, :3].T                                  # camera frame
    z = np.asarray(centre, np.float64) @ M[2, :3] + M[2, 3]
    gx = gc[:, 0] * camera.width * z / (2.0 * float(camera.fx))
    gy = gc[:, 1] * camera.height * z / (2.0 * float(camera.fy))
    return np.stack([gx, gy], axis=1)


def gradient_stats(orc, scene, cameras, dL_dimage, bg=(0.0, 0.0, 0.0), aa=0.0, exact=False):
    """(sum of view-space gradient norms, number of visible views) per
    primitive for one backward over `cameras` with image gradient dL_dimage
    (the cameras' images concatenated, 3 H W floats each)."""
    dL = np.asarray(dL_dimage, np.float64).reshape(-1)
    acc = np.zeros(scene.n)
    cnt = np.zeros(scene.n, np.int64)
    off = 0
    for cam in cameras:
        m = 3 * cam.width * cam.height
        _, g = orc.render(scene, [cam], bg=bg, dL_dimage=dL[off:off + m], aa=aa, exact=exact)
        off += m
        pp = orc.preprocess(scene, cam, aa=aa, exact=exact)
        r = pp["rect"]
        vis = pp["visible"] & (r[:, 0] <= r[:, 1]) & (r[:, 2] <= r[:, 3])
        vg = view_gradient(cam, scene.centre, g["centre"], g["verts"])
        acc += np.where(vis, np.linalg.norm(vg, axis=1), 0.0)
        cnt += vis
    return acc, cnt


# ------------------------------------------------------------ decision

def decide(kind, dist, logit, grad_sum, grad_count, max_pixels, scene_extent, grad_threshold=DENSIFY_GRAD):
    """Per primitive: PRUNE, KEEP, CLONE or SPLIT (binary32 decisions).  The
    thresholds are the paper's; the gradient one may be overridden."""
    n = len(logit)
    act = np.zeros(n, np.int64)
    p = float(f32(PRUNE_OPACITY))          # the threshold is a binary32 operand
    logit_min = f32(math.log(p / (1.0 - p)))
    big = f32(f32(PRUNE_SCENE_FRAC) * f32(scene_extent))
    small = f32(f32(CLONE_SCENE_FRAC) * f32(scene_extent))
    thr = f32(grad_threshold)
    for i in range(n):
        s = size32(kind, dist[i])
        if f32(logit[i]) < logit_min or s > big or int(max_pixels[i]) > PRUNE_PIXELS:
            act[i] = PRUNE
            continue
        c = int(grad_count[i])
        g = f32(f32(grad_sum[i]) / f32(c)) if c > 0 else f32(0.0)
        if g > thr:
            act[i] = CLONE if s < small else SPLIT
        else:
            act[i] = KEEP
    return act


def destinations(act):
    """Exclusive prefix sum of the output counts (0, 1, 2, 2) and the total."""
    per = np.array([0, 1, 2, 2], np.int64)[np.asarray(act, np.int64)]
    dest = np.concatenate([[0], np.cumsum(per)])
    return dest[:-1], int(dest[-1])


# ------------------------------------------------------------ application

def apply(kind, params, states, act, normals):
    """New population.  params: dict centre [n,3], quat [n,4], dist [n,D],
    logit [n], sh [n,K,3]; states: list of dicts of the same shapes (the
    optimiser's moments); normals: [n, 2, 3] standard-normal draws for the
    split children.  Returns (params, states) in binary64."""
    keys = list(params)
    out = {k: [] for k in keys}
    sout = [{k: [] for k in keys} for _ in states]
    for i in range(len(act)):
        a = int(act[i])
        if a == PRUNE:
            continue
        if a == KEEP:
            rows = [(None, False)]
        elif a == CLONE:
            rows = [(None, False), (None, True)]
        else:
            rows = [(0, True), (1, True)]
        for child, fresh in rows:
            row = {k: np.array(params[k][i], np.float64) for k in keys}
            if child is not None:
                d = row["dist"]
                if kind == 6:
                    off = quat_rotation(row["quat"]) @ (np.abs(d) * normals[i, child])
                else:
                    off = (np.max(np.abs(d)) / 2.0) * np.asarray(normals[i, child], np.float64)
                row["centre"] = row["centre"] + off
                row["dist"] = d / SPLIT_SHRINK
            for k in keys:
                out[k].append(row[k])
            for s, st in zip(sout, states):
                for k in keys:
                    s[k].append(np.zeros(np.shape(params[k][i])) if fresh else np.array(st[k][i], np.float64))

    def stack(lst, k):
        return np.array(lst) if lst else np.zeros((0,) + np.shape(params[k])[1:])

    return ({k: stack(out[k], k) for k in keys},
            [{k: stack(s[k], k) for k in keys} for s in sout])
