"""FP64 CPU oracle for the LinPrim rasterizer -- TEST INFRASTRUCTURE ONLY.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The product path never does, and the
oracle never imports the product package: the two share nothing but the
seeded input generators in `scenes`.

The arithmetic lives in `linprim_oracle.c` (plain C, binary64); this module
only marshals numpy arrays through ctypes.  Every stage cites the paper
section it restates; see that file's header.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class _Prims(C.Structure):
    _fields_ = [("nv", C.c_int), ("n", C.c_int), ("sh_degree", C.c_int),
                ("centre", C.c_void_p), ("verts", C.c_void_p), ("opacity", C.c_void_p),
                ("sh", C.c_void_p), ("dmin", C.c_void_p), ("aa_kernel", C.c_double), ("exact", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("viewmat", C.c_double * 16), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int),
                ("height", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


class use_library:
    """Temporarily route every call through another build of the oracle
    (used by the mutation tests, which compile deliberately broken copies)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.prev = _lib
        _lib = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.prev
        return False


def _load(path):
    L = C.CDLL(path)
    dp = C.c_void_p
    L.orc_render.argtypes = [dp, dp, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_render_pixels.argtypes = [dp, dp, dp, C.c_longlong, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    L.orc_keys.argtypes = [dp, dp, C.c_int, C.c_int, dp, dp, C.c_longlong, dp, dp]
    L.orc_depth_pixels.argtypes = [dp, dp, C.c_longlong, dp, dp, dp, dp]
    L.orc_preprocess.argtypes = [dp, dp, dp, dp]
    L.orc_span.argtypes = [dp, dp, C.c_int, C.c_double, C.c_double, dp]
    L.orc_mtia.argtypes = [dp, dp, dp, C.c_double, C.c_double, dp, dp]
    L.orc_sh_basis.argtypes = [C.c_int, dp, dp, dp]
    L.orc_params_forward.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
    L.orc_params_backward.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp, dp]
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Bound:
    """Keeps the float64 copies alive while the C call runs."""

    def __init__(self, scene, dmin=None, aa=0.0, exact=False):
        self.centre = np.ascontiguousarray(scene.centre, np.float64)
        self.verts = np.ascontiguousarray(scene.verts, np.float64)
        self.opacity = np.ascontiguousarray(scene.opacity, np.float64)
        self.sh = np.ascontiguousarray(scene.sh, np.float64)
        self.dmin = None if dmin is None else np.ascontiguousarray(dmin, np.float64)
        self.s = _Prims(int(scene.kind), int(scene.centre.shape[0]), int(scene.sh_degree),
                        _ptr(self.centre), _ptr(self.verts), _ptr(self.opacity),
                        _ptr(self.sh), _ptr(self.dmin), float(aa), int(bool(exact)))


def _cams(cameras):
    arr = (_Camera * max(1, len(cameras)))()
    for i, c in enumerate(cameras):
        vm = np.asarray(c.viewmat, np.float64).reshape(16)
        arr[i].viewmat[:] = [float(x) for x in vm]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


def set_threads(n: int) -> int:
    """Threads of the oracle's loops over pixels (n <= 0: all); returns the
    count in effect.  For timing the oracle on one core or all cores."""
    L = lib()
    L.orc_set_threads.restype = C.c_int
    return int(L.orc_set_threads(int(n)))


def render(scene, cameras, bg=(0.0, 0.0, 0.0), dL_dimage=None, dmin=None, info=False, aa=0.0, exact=False):
    """Images packed [cam][3][H][W] (float64).  With dL_dimage, also returns
    the gradients of L = <dL_dimage, image> w.r.t. centre, verts, opacity, sh.
    aa: size in pixels of the 2D anti-aliasing filter (Sec. 3.3), 0 = off.
    exact: spans along the true perspective ray instead of the ray-space
    approximation (App. "Ray Space Approximation"; the filter is then off)."""
    b = _Bound(scene, dmin, aa, exact)
    cams = _cams(cameras)
    P = sum(c.width * c.height for c in cameras)
    img = np.zeros(3 * P, np.float64)
    inf = np.zeros(4 * P, np.float64) if info else None
    bgv = np.asarray(bg, np.float64)
    g = None if dL_dimage is None else np.ascontiguousarray(dL_dimage, np.float64).reshape(-1)
    grads = None
    if g is not None:
        grads = dict(centre=np.zeros_like(b.centre), verts=np.zeros_like(b.verts),
                     opacity=np.zeros_like(b.opacity), sh=np.zeros_like(b.sh))
    rc = lib().orc_render(C.byref(b.s), cams, len(cameras), _ptr(bgv), _ptr(img), _ptr(inf),
                          _ptr(g), *(None if grads is None else _ptr(grads[k])
                                     for k in ("centre", "verts", "opacity", "sh")))
    if rc:
        raise RuntimeError(f"oracle render failed ({rc})")
    out = [img]
    if info:
        out.append(inf.reshape(P, 4))
    if grads is not None:
        out.append(grads)
    return out[0] if len(out) == 1 else tuple(out)


def render_pixels(scene, camera, px, py, bg=(0.0, 0.0, 0.0), dL_dC=None, dmin=None, aa=0.0, exact=False):
    """Colours [npix][3] and info [npix][4] = (n_contrib, T_final, borderline,
    min_span) of the listed pixels; with dL_dC [npix][3] also the gradients."""
    b = _Bound(scene, dmin, aa, exact)
    cams = _cams([camera])
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = px.shape[0]
    rgb = np.zeros((n, 3))
    inf = np.zeros((n, 4))
    bgv = np.asarray(bg, np.float64)
    g = None if dL_dC is None else np.ascontiguousarray(dL_dC, np.float64).reshape(n, 3)
    grads = None
    if g is not None:
        grads = dict(centre=np.zeros_like(b.centre), verts=np.zeros_like(b.verts),
                     opacity=np.zeros_like(b.opacity), sh=np.zeros_like(b.sh))
    rc = lib().orc_render_pixels(C.byref(b.s), cams, _ptr(bgv), n, _ptr(px), _ptr(py),
                                 _ptr(rgb), _ptr(inf), _ptr(g),
                                 *(None if grads is None else _ptr(grads[k])
                                   for k in ("centre", "verts", "opacity", "sh")))
    if rc:
        raise RuntimeError(f"oracle render_pixels failed ({rc})")
    return (rgb, inf) if grads is None else (rgb, inf, grads)


def depth_pixels(scene, camera, px, py, aa=0.0, exact=False):
    """Depth (App. "Depth and Surface Reconstruction") of the listed pixels:
    the ray entry depth of the first primitive after which the cumulative
    opacity exceeds 0.5, 0 where it never does; and each pixel's borderline
    word (bit 2: the 0.5 crossing is within 1e-4 of 0.5)."""
    b = _Bound(scene, None, aa, exact)
    cams = _cams([camera])
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    d = np.zeros(px.shape[0])
    f = np.zeros(px.shape[0], np.int32)
    rc = lib().orc_depth_pixels(C.byref(b.s), cams, px.shape[0], _ptr(px), _ptr(py), _ptr(d), _ptr(f))
    if rc:
        raise RuntimeError(f"oracle depth_pixels failed ({rc})")
    return d, f


def depth(scene, cameras, aa=0.0, exact=False):
    """Depth maps packed [cam][H][W] and the borderline words, all pixels."""
    ds, fs = [], []
    for c in cameras:
        yy, xx = np.mgrid[0:c.height, 0:c.width]
        d, f = depth_pixels(scene, c, xx.reshape(-1), yy.reshape(-1), aa=aa, exact=exact)
        ds.append(d)
        fs.append(f)
    return np.concatenate(ds), np.concatenate(fs)


def keys(scene, cameras, tile=16, aa=0.0, exact=False):
    """Sorted (keys u64, values u32) and per-record tile counts u32 [cam*n]."""
    b = _Bound(scene, None, aa, exact)
    cams = _cams(cameras)
    n_out = C.c_longlong(0)
    counts = np.zeros(len(cameras) * scene.n, np.uint32)
    L = lib()
    rc = L.orc_keys(C.byref(b.s), cams, len(cameras), tile, None, None, 0, C.byref(n_out),
                    _ptr(counts))
    n = n_out.value
    k = np.zeros(max(n, 1), np.uint64)
    v = np.zeros(max(n, 1), np.uint32)
    rc = L.orc_keys(C.byref(b.s), cams, len(cameras), tile, _ptr(k), _ptr(v), n,
                    C.byref(n_out), None)
    if rc:
        raise RuntimeError(f"oracle keys failed ({rc})")
    return k[:n], v[:n], counts


def preprocess(scene, camera, dmin=None, aa=0.0, exact=False):
    b = _Bound(scene, dmin, aa, exact)
    cams = _cams([camera])
    out = np.zeros((scene.n, 16))
    pv = np.zeros((scene.n, scene.kind, 3))
    lib().orc_preprocess(C.byref(b.s), cams, _ptr(out), _ptr(pv))
    return dict(visible=out[:, 0].astype(bool), zbits=out[:, 1].astype(np.uint32),
                rect=out[:, 2:6].astype(np.int64), pc=out[:, 6:9], sigma=out[:, 9],
                dmin=out[:, 10], rgb=out[:, 11:14], dist=out[:, 14], pverts=pv)


def span(scene, camera, i, rx, ry, aa=0.0, exact=False):
    """(hit, i1, i2) by MTIA and (hit, i1, i2) by half-space clipping."""
    b = _Bound(scene, None, aa, exact)
    cams = _cams([camera])
    out = np.zeros(6)
    lib().orc_span(C.byref(b.s), cams, int(i), float(rx), float(ry), _ptr(out))
    return (bool(out[0]), out[1], out[2]), (bool(out[3]), out[4], out[5])


def mtia(p0, p1, p2, rx, ry):
    """(hit, u, v, det, depth), d depth / d (p0, p1, p2) as [3][3]."""
    a = [np.ascontiguousarray(p, np.float64) for p in (p0, p1, p2)]
    out = np.zeros(5)
    grad = np.zeros(9)
    lib().orc_mtia(_ptr(a[0]), _ptr(a[1]), _ptr(a[2]), float(rx), float(ry), _ptr(out), _ptr(grad))
    return out, grad.reshape(3, 3)


def sh_basis(degree, direction):
    d = np.ascontiguousarray(direction, np.float64)
    Y = np.zeros(16)
    dY = np.zeros(48)
    lib().orc_sh_basis(int(degree), _ptr(d), _ptr(Y), _ptr(dY))
    return Y, dY.reshape(16, 3)


# ------------------------------------------------------------ parameter layer
def params_forward(kind, centre, quat, dist, logit):
    """Sec. 3.1 parameterisation: (centre, quaternion (w,x,y,z), distances,
    opacity logit) -> (verts [n][kind][3], opacity [n]), binary64."""
    c, q, d, l = (np.ascontiguousarray(a, np.float64) for a in (centre, quat, dist, logit))
    n = c.shape[0]
    v = np.zeros((n, kind, 3))
    o = np.zeros(n)
    lib().orc_params_forward(int(kind), n, _ptr(c), _ptr(q), _ptr(d), _ptr(l), _ptr(v), _ptr(o))
    return v, o


def params_backward(kind, quat, dist, logit, dverts, dopacity, dcentre_render=None):
    """Adjoint of params_forward; dcentre includes the renderer's direct term."""
    q, d, l = (np.ascontiguousarray(a, np.float64) for a in (quat, dist, logit))
    gv = np.ascontiguousarray(dverts, np.float64)
    go = np.ascontiguousarray(dopacity, np.float64)
    n = q.shape[0]
    dc = np.zeros((n, 3)) if dcentre_render is None else np.array(dcentre_render, np.float64)
    dq, dd, dl = np.zeros_like(q), np.zeros_like(d), np.zeros_like(l)
    lib().orc_params_backward(int(kind), n, _ptr(q), _ptr(d), _ptr(l), _ptr(gv), _ptr(go), _ptr(dc),
                              _ptr(dq), _ptr(dd), _ptr(dl))
    return dict(centre=dc, quat=dq, dist=dd, logit=dl)
