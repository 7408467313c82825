"""GB300-native LinPrim rasterizer (arXiv 2501.16312).

Differentiable tile rasterization of transparent octahedra and tetrahedra on
one sm_103a GPU.  The work happens in the CUDA library behind
include/linprim.h; this package marshals torch tensors to it (device memory
and streams come from PyTorch) and wraps it in a torch.autograd.Function.

    rast = Rasterizer(device=0)
    img = render(centre, verts, opacity, sh, cameras, kind=OCTAHEDRON,
                 rasterizer=rast)            # packed [cam][3][H][W], flat
    img.backward(grad)                       # grads on the four leaves
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

from . import _native
from ._native import LP_OCTAHEDRON as OCTAHEDRON, LP_TETRAHEDRON as TETRAHEDRON, LinPrimError

__all__ = ["OCTAHEDRON", "TETRAHEDRON", "Primitives", "Rasterizer", "render", "split_images",
           "LinPrimError"]


def _torch():
    import torch
    return torch


def _fptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


class Primitives:
    """Device-resident primitive arrays in the boundary's layout."""

    def __init__(self, kind: int, centre, verts, opacity, sh, sh_degree: Optional[int] = None):
        torch = _torch()
        if kind not in (OCTAHEDRON, TETRAHEDRON):
            raise ValueError(f"kind must be OCTAHEDRON (6) or TETRAHEDRON (4), got {kind}")
        n = centre.shape[0]
        K = sh.shape[1] if sh.dim() == 3 else sh.numel() // max(1, 3 * n)
        if sh_degree is None:
            sh_degree = {1: 0, 4: 1, 9: 2, 16: 3}[K]
        arrays = (("centre", centre, (n, 3)), ("verts", verts, (n, kind, 3)),
                  ("opacity", opacity, (n,)), ("sh", sh, (n, (sh_degree + 1) ** 2, 3)))
        for name, t, shape in arrays:
            if tuple(t.shape) != shape:
                raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
        for name, t, _ in arrays:
            if t.dtype != torch.float32 or not t.is_cuda:
                raise ValueError(f"{name} must be a float32 CUDA tensor")
        self.kind, self.n, self.sh_degree = kind, n, sh_degree
        self.centre, self.verts = centre.contiguous(), verts.contiguous()
        self.opacity, self.sh = opacity.contiguous(), sh.contiguous()

    @classmethod
    def from_scene(cls, scene, device="cuda"):
        torch = _torch()
        t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
        return cls(int(scene.kind), t(scene.centre), t(scene.verts), t(scene.opacity), t(scene.sh),
                   int(scene.sh_degree))

    def struct(self):
        return _native.lp_prims(self.kind, self.n, self.sh_degree, _fptr(self.centre).value,
                                _fptr(self.verts).value, _fptr(self.opacity).value,
                                _fptr(self.sh).value)


def split_images(flat, cameras):
    """Views [3, H, W] of a packed image buffer, one per camera."""
    out, off = [], 0
    for c in cameras:
        n = 3 * c.width * c.height
        out.append(flat[off:off + n].view(3, c.height, c.width))
        off += n
    return out


class Rasterizer:
    """One C-ABI context: workspace, tuning and the state of the last forward."""

    def __init__(self, device: int = 0, tuning: Optional[dict] = None):
        self.lib = _native.load()
        torch = _torch()
        self.device = torch.device("cuda", device)
        h = C.c_void_p()
        _native.check(None, self.lib.lp_create(C.byref(h), device), "lp_create")
        self.ctx = h
        self.generation = 0
        self._fwd = None
        self._timing = False
        if tuning:
            self.set_tuning(**tuning)

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.lp_destroy(self.ctx)
            self.ctx = None

    def _stream(self):
        return C.c_void_p(_torch().cuda.current_stream(self.device).cuda_stream)

    def set_tuning(self, tile=None, batch=None, blocks_per_sm=None, sort_mode=None,
                   pixels_per_thread=None, chain_split=None, radix_bits=None,
                   tile_order=None, onesweep=None):
        t = _native.lp_tuning()
        _native.check(self.ctx, self.lib.lp_get_tuning(self.ctx, C.byref(t)), "lp_get_tuning")
        for k, v in (("tile", tile), ("batch", batch), ("blocks_per_sm", blocks_per_sm),
                     ("sort_mode", sort_mode), ("pixels_per_thread", pixels_per_thread),
                     ("chain_split", chain_split), ("radix_bits", radix_bits),
                     ("tile_order", tile_order), ("onesweep", onesweep)):
            if v is not None:
                setattr(t, k, int(v))
        _native.check(self.ctx, self.lib.lp_set_tuning(self.ctx, C.byref(t)), "lp_set_tuning")

    def set_filter_2d(self, kernel_px: float):
        """Sec. 3.3 2D anti-aliasing filter size in pixels (0 = off; the paper
        uses 0.1).  Applies to later forward calls."""
        _native.check(self.ctx, self.lib.lp_set_filter_2d(self.ctx, float(kernel_px)), "lp_set_filter_2d")

    def set_exact(self, exact: bool):
        """Spans along the true perspective ray instead of the ray-space
        approximation (App. "Ray Space Approximation"); applies to later
        forward calls."""
        _native.check(self.ctx, self.lib.lp_set_exact(self.ctx, int(bool(exact))), "lp_set_exact")

    def set_densify_stats(self, grad_sum=None, grad_count=None, px_max=None):
        """Gather densification statistics (Sec. 3.4 "Adaptive Population
        Control") into device tensors of one entry per primitive: float32
        grad_sum and int32 grad_count (view-space position-gradient norms and
        visible views, added by each backward) and int32 px_max (largest
        pixel-rectangle side, raised by each forward).  No arguments: stop."""
        ts = (grad_sum, grad_count, px_max)
        if all(t is None for t in ts):
            st = self.lib.lp_set_densify_stats(self.ctx, None, None, None, 0)
        else:
            n = min(int(t.numel()) for t in ts)
            st = self.lib.lp_set_densify_stats(self.ctx, _fptr(grad_sum), _fptr(grad_count), _fptr(px_max), n)
        _native.check(self.ctx, st, "lp_set_densify_stats")
        self._densify_stats = ts

    def exact(self) -> bool:
        v = C.c_int()
        _native.check(self.ctx, self.lib.lp_get_exact(self.ctx, C.byref(v)), "lp_get_exact")
        return bool(v.value)

    def filter_2d(self) -> float:
        v = C.c_float()
        _native.check(self.ctx, self.lib.lp_get_filter_2d(self.ctx, C.byref(v)), "lp_get_filter_2d")
        return v.value

    def tuning(self) -> dict:
        t = _native.lp_tuning()
        _native.check(self.ctx, self.lib.lp_get_tuning(self.ctx, C.byref(t)), "lp_get_tuning")
        return {k: getattr(t, k) for k, _ in t._fields_}

    def reserve(self, records, entries, pixels, tiles):
        _native.check(self.ctx, self.lib.lp_reserve(self.ctx, int(records), int(entries),
                                                    int(pixels), int(tiles)), "lp_reserve")

    def forward(self, prims: Primitives, cameras: Sequence, bg=(0.0, 0.0, 0.0), images=None):
        torch = _torch()
        P = sum(c.width * c.height for c in cameras)
        if images is None:
            images = torch.empty(3 * P, dtype=torch.float32, device=self.device)
        cams = _native.camera_struct(cameras)
        bgv = (C.c_float * 3)(*[float(x) for x in bg])
        ps = prims.struct()
        st = self.lib.lp_render_forward(self.ctx, C.byref(ps), cams, len(cameras), bgv,
                                        _fptr(images), self._stream())
        _native.check(self.ctx, st, "lp_render_forward")
        self.generation += 1
        self._fwd = (prims, list(cameras), tuple(bg))
        return images

    def backward(self, dL_dimages, grads=None, accumulate=False):
        torch = _torch()
        if self._fwd is None:
            raise LinPrimError(_native.LP_ERR_STATE, "backward without forward")
        prims = self._fwd[0]
        if grads is None:
            grads = dict(centre=torch.empty_like(prims.centre), verts=torch.empty_like(prims.verts),
                         opacity=torch.empty_like(prims.opacity), sh=torch.empty_like(prims.sh))
        g = dL_dimages.contiguous()
        st = self.lib.lp_render_backward(self.ctx, _fptr(g), _fptr(grads["centre"]),
                                         _fptr(grads["verts"]), _fptr(grads["opacity"]),
                                         _fptr(grads["sh"]), int(bool(accumulate)), self._stream())
        _native.check(self.ctx, st, "lp_render_backward")
        return grads

    def depth(self, out=None):
        """Depth map of the last forward (App. "Depth and Surface
        Reconstruction"): per pixel, packed [cam][H][W], the distance at which
        the ray enters the first primitive taking the cumulative opacity above
        0.5; 0 where none does."""
        torch = _torch()
        if self._fwd is None:
            raise LinPrimError(_native.LP_ERR_STATE, "depth without forward")
        P = sum(c.width * c.height for c in self._fwd[1])
        if out is None:
            out = torch.empty(P, dtype=torch.float32, device=self.device)
        _native.check(self.ctx, self.lib.lp_render_depth(self.ctx, _fptr(out), self._stream()), "lp_render_depth")
        return out

    def sync_status(self):
        _native.check(self.ctx, self.lib.lp_sync_status(self.ctx, self._stream()), "lp_sync_status")

    def stats(self) -> dict:
        s = _native.lp_stats()
        _native.check(self.ctx, self.lib.lp_get_stats(self.ctx, C.byref(s)), "lp_get_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def debug_keys(self):
        import numpy as np
        n = C.c_longlong(0)
        _native.check(self.ctx, self.lib.lp_debug_keys(self.ctx, None, None, 0, C.byref(n)),
                      "lp_debug_keys")
        k = np.zeros(max(1, n.value), np.uint64)
        v = np.zeros(max(1, n.value), np.uint32)
        _native.check(self.ctx, self.lib.lp_debug_keys(self.ctx, k.ctypes.data, v.ctypes.data,
                                                       n.value, C.byref(n)), "lp_debug_keys")
        return k[:n.value], v[:n.value]

    def debug_counts(self):
        import numpy as np
        m = self.stats()["records"]
        out = np.zeros(max(1, m), np.uint32)
        _native.check(self.ctx, self.lib.lp_debug_counts(self.ctx, out.ctypes.data, m),
                      "lp_debug_counts")
        return out[:m]

    def pixel_state(self):
        import numpy as np
        m = self.stats()["pixels"]
        last = np.zeros(max(1, m), np.uint32)
        tl = np.zeros(max(1, m), np.float32)
        _native.check(self.ctx, self.lib.lp_debug_pixel_state(self.ctx, last.ctypes.data,
                                                              tl.ctypes.data, m),
                      "lp_debug_pixel_state")
        return last[:m], tl[:m]

    def debug_scan(self, counts):
        """The forward's tile-count scan on a uint32 numpy array: (exclusive
        offsets as uint32, total).  Raises LinPrimError (LP_ERR_CAPACITY)
        when the total reaches 2^32 - 1."""
        import numpy as np
        import torch
        c = np.ascontiguousarray(counts, dtype=np.uint32)
        d_in = torch.from_numpy(c.view(np.int32).copy()).to(self.device)
        d_out = torch.empty_like(d_in)
        total = C.c_uint(0)
        _native.check(self.ctx, self.lib.lp_debug_scan(self.ctx, d_in.data_ptr(), c.size, d_out.data_ptr(),
                                                       C.byref(total), self._stream()), "lp_debug_scan")
        return d_out.cpu().numpy().view(np.uint32), total.value

    def set_debug_guard(self, enabled=True):
        """Canary zones after every workspace buffer allocated from now on
        (a debugging aid; see check_guards)."""
        _native.check(self.ctx, self.lib.lp_set_debug_guard(self.ctx, int(bool(enabled))), "lp_set_debug_guard")

    def check_guards(self) -> dict:
        """Synchronise and read every canary zone back: the number of guarded
        buffers and of zone bytes that changed (0 unless a kernel wrote past
        a buffer's capacity), with the first damaged buffer's name."""
        checked, damaged = C.c_longlong(0), C.c_longlong(0)
        _native.check(self.ctx, self.lib.lp_check_guards(self.ctx, C.byref(checked), C.byref(damaged)),
                      "lp_check_guards")
        return {"checked": checked.value, "damaged": damaged.value,
                "first": self.lib.lp_last_error(self.ctx).decode() if damaged.value else ""}

    def set_timing(self, enabled=True):
        _native.check(self.ctx, self.lib.lp_set_timing(self.ctx, int(bool(enabled))), "lp_set_timing")
        self._timing = bool(enabled)

    def timing(self) -> bool:
        """Whether per-stage CUDA events are recorded (`set_timing`)."""
        return self._timing

    def stage_times(self) -> dict:
        ms = (C.c_float * len(_native.STAGES))()
        _native.check(self.ctx, self.lib.lp_stage_times(self.ctx, ms), "lp_stage_times")
        return dict(zip(_native.STAGES, [float(x) for x in ms]))

    def count_pairs(self) -> dict:
        """(pixel, primitive) pair counts of the last forward: iterated,
        evaluated (face planes evaluated), intersected, and evaluated up to
        each pixel's last contributor (the backward's work)."""
        out = (C.c_longlong * 4)()
        _native.check(self.ctx, self.lib.lp_count_pairs(self.ctx, out), "lp_count_pairs")
        return dict(iterated=out[0], evaluated=out[1], intersected=out[2], iterated_to_last=out[3])


def _make_fn():
    torch = _torch()

    class RenderFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, centre, verts, opacity, sh, rast, kind, sh_degree, cameras, bg):
            prims = Primitives(kind, centre.detach(), verts.detach(), opacity.detach(),
                               sh.detach(), sh_degree)
            img = rast.forward(prims, cameras, bg)
            ctx.rast, ctx.gen, ctx.prims, ctx.cameras, ctx.bg = rast, rast.generation, prims, cameras, bg
            return img

        @staticmethod
        def backward(ctx, gimg):
            rast = ctx.rast
            if rast.generation != ctx.gen:
                # another forward ran on this context since: rebuild its state
                rast.forward(ctx.prims, ctx.cameras, ctx.bg)
                ctx.gen = rast.generation
            g = rast.backward(gimg.contiguous())
            return g["centre"], g["verts"], g["opacity"], g["sh"], None, None, None, None, None

    return RenderFn


_fn_cache = {}


def render(centre, verts, opacity, sh, cameras, kind=OCTAHEDRON, sh_degree=None,
           bg=(0.0, 0.0, 0.0), rasterizer: Optional[Rasterizer] = None):
    """Differentiable render of all `cameras` in one batched launch sequence.
    Returns the packed images (flat float32, [cam][3][H][W])."""
    if "fn" not in _fn_cache:
        _fn_cache["fn"] = _make_fn()
    rast = rasterizer if rasterizer is not None else _default_rasterizer(centre.device)
    if sh_degree is None:
        sh_degree = {1: 0, 4: 1, 9: 2, 16: 3}[sh.shape[1]]
    return _fn_cache["fn"].apply(centre, verts, opacity, sh, rast, kind, sh_degree, list(cameras),
                                 tuple(bg))


_default = {}


def _default_rasterizer(device):
    idx = device.index if device.index is not None else _torch().cuda.current_device()
    if idx not in _default:
        _default[idx] = Rasterizer(idx)
    return _default[idx]
