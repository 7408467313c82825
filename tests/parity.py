"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the FP64 oracle on the same seeded inputs.

Tolerances (from the rasterizer's specification):
  * tile lists, keys, values and per-record tile counts: bit-exact;
  * images: |gpu - oracle| <= 1e-4 per channel, except pixels the oracle
    flags as borderline (the transmittance at some step is within 1e-3
    relative of the 1e-3 stop threshold, so binary32 and binary64 may stop at
    different primitives); those may number at most max(2, 1e-4 * pixels);
  * gradients: per array, ||g - g*|| / ||g*|| <= 1e-3, and per element
    |g - g*| <= 1e-3 max(|g*|, 1e-2 rms(g*)), for a dL/dimage that is zero at
    the borderline pixels (both sides get the same dL).  As borderline pixels
    may differ in number at most max(2, 1e-4 P), primitives may have an
    element over the per-element bound in number at most max(8, 1e-3 n) per
    array, each within 5e-2: binary32 resolves some rays only to about 1e-3
    -- a ray that grazes a primitive, crosses a face seen nearly edge-on, or
    passes within rounding of an edge between two faces -- and a primitive
    whose gradient comes from few pixels inherits that error from one of
    them (each such element traces back to one pixel; see the design notes).
    The count and the worst element are reported.  The
    oracle also flags pixels whose ray passes within rounding of some
    primitive's silhouette: the colour is continuous there but its
    derivative with respect to the vertices jumps, so binary32 and binary64
    may take different sides.
"""
import numpy as np

IMG_TOL = 1e-4
GRAD_REL_L2 = 1e-3


def gpu_forward_backward(rast, scene, cameras, bg, dL=None, device="cuda:0"):
    import torch
    from paper_2501_16312_gb300 import Primitives
    prims = Primitives.from_scene(scene, device)
    img = rast.forward(prims, cameras, bg)
    grads = None
    if dL is not None:
        g = rast.backward(torch.as_tensor(dL, dtype=torch.float32, device=device))
        grads = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    torch.cuda.synchronize()
    rast.sync_status()
    return img.cpu().numpy().astype(np.float64), grads


def compare_images(gpu, ref, info, cameras):
    """Returns (max error over non-borderline pixels, #borderline violations)."""
    P = sum(c.width * c.height for c in cameras)
    err = np.zeros(P)
    off = 0
    for c in cameras:
        n = c.width * c.height
        e = np.abs(gpu[3 * off:3 * (off + n)] - ref[3 * off:3 * (off + n)]).reshape(3, n).max(0)
        err[off:off + n] = e
        off += n
    border = info[:, 2] > 0
    bad = err > IMG_TOL
    return float(err[~border].max(initial=0.0)), int((bad & border).sum()), int(bad.sum())


def assert_images_match(gpu, ref, info, cameras):
    P = sum(c.width * c.height for c in cameras)
    max_clean, n_border_bad, n_bad = compare_images(gpu, ref, info, cameras)
    assert max_clean <= IMG_TOL, f"max image error {max_clean:.3e} on non-borderline pixels"
    assert n_border_bad <= max(2, 1e-4 * P), f"{n_border_bad} borderline pixels differ"
    return max_clean


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64).reshape(-1), np.asarray(b, np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


GRAD_ELEM = 1e-3
GRAD_ELEM_FLOOR = 1e-2
GRAD_ELEM_OUTLIER_FRAC = 1e-3
GRAD_ELEM_OUTLIER_MIN = 8
GRAD_ELEM_OUTLIER_MAX = 5e-2


def outlier_allowance(n):
    """Primitives that may exceed the per-element bound, of n."""
    return max(GRAD_ELEM_OUTLIER_MIN, int(GRAD_ELEM_OUTLIER_FRAC * n))


def elem_ratios(a, b):
    """|a - b| / max(|b|, 1e-2 rms(b)) per element of one array (the
    per-element gradient bound is ratio <= 1e-3).  An all-zero reference
    admits only exact zeros."""
    a = np.asarray(a, np.float64).reshape(-1)
    b = np.asarray(b, np.float64).reshape(-1)
    if a.size == 0:
        return np.zeros(0)
    rms = float(np.sqrt(np.mean(b * b)))
    scale = np.maximum(np.abs(b), GRAD_ELEM_FLOOR * rms)
    d = np.abs(a - b)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d > 0, np.inf, 0.0))


def elem_stats(a, b, tol=GRAD_ELEM):
    """(worst ratio, its index, primitives with an element over tol, primitives
    allowed over tol); the arrays' first axis is the primitive."""
    r = elem_ratios(a, b)
    if r.size == 0:
        return 0.0, -1, 0, 0
    n = max(1, np.asarray(b).shape[0])
    i = int(np.argmax(r))
    over = int((r.reshape(n, -1) > tol).any(1).sum())
    return float(r[i]), i, over, outlier_allowance(n)


def assert_grads_match(gpu, ref, tol=GRAD_REL_L2, elem_tol=GRAD_ELEM):
    """Relative L2 per array and the per-element bound (with its counted
    allowance); returns the relative L2 errors."""
    out, stats = {}, {}
    for k in ("centre", "verts", "opacity", "sh"):
        out[k] = rel_l2(gpu[k], ref[k])
        stats[k] = elem_stats(gpu[k], ref[k], elem_tol)
    bad = {k: v for k, v in out.items() if not v <= tol}
    assert not bad, f"gradient relative L2 errors {out}"
    bad_e = {k: v for k, v in stats.items() if not (v[2] <= v[3] and v[0] <= GRAD_ELEM_OUTLIER_MAX)}
    assert not bad_e, ("per-element gradient bound: (worst ratio, index, primitives over 1e-3, allowed) "
                       f"{bad_e}; all arrays {stats}")
    print(f"per-element gradient check (worst ratio, index, primitives over 1e-3, allowed): {stats}")
    return out


def mask_borderline(dL, info, cameras):
    """dL (packed [cam][3][H][W]) with every channel zeroed at the pixels the
    oracle flags as borderline (info[:, 2] != 0, pixels in camera order)."""
    out = np.array(dL, np.float64, copy=True).reshape(-1)
    off = 0
    for c in cameras:
        n = c.width * c.height
        b = info[off:off + n, 2] > 0
        seg = out[3 * off:3 * (off + n)].reshape(3, n)
        seg[:, b] = 0.0
        off += n
    return out



def trimmed_rel_l2(a, b):
    """Relative L2 error of one array without the outlier_allowance(n)
    primitives (first axis) whose errors are largest, for checks on few
    primitives, where one sensitive primitive can dominate the norm."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = max(1, b.shape[0])
    d = ((a - b).reshape(n, -1) ** 2).sum(1)
    keep = np.argsort(d)[:max(0, n - outlier_allowance(n))]
    nb = np.sqrt((b.reshape(n, -1)[keep] ** 2).sum())
    return float(np.sqrt(d[keep].sum()) / nb) if nb > 0 else float(np.sqrt(d[keep].sum()))
