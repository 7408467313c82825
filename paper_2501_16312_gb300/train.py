"""The optimisation step of LinPrim primitives, on device-resident parameters.

    parameter layer (Sec. 3.1) -> batched render of the training views ->
    L1 image-loss gradient -> render backward -> parameter-layer backward ->
    fused Adam (Sec. 3.4)

Every stage is a kernel of the C-ABI library.  Two front ends:

* `params_layer` / `render` are torch.autograd.Functions, so a user can write
  an ordinary PyTorch loop (any loss, any optimiser) around them;
* `Trainer` runs the fixed step above on one flat parameter array (group
  blocks [centre n*3 | quaternion n*4 | distances n*D | opacity logit n |
  SH n*K*3], gradients and both Adam moments in the same layout), can capture
  it into one CUDA graph and replays it.

Learning rates are the paper's (App. "Experimental Setting", Table 16):
colour (SH DC) 2.5e-3, higher SH bands 1.25e-4, opacity 2.5e-2, rotation
1e-3, distance 1e-4 / 2.6 times the scene extent; position as in 3DGS,
1.6e-4 decaying log-linearly to 1.6e-6 over 30k steps, times the extent.
The extent is the largest distance between a camera and the mean camera
position.  Adam uses beta = (0.9, 0.999), eps = 1e-15 (3DGS's optimiser,
which the paper keeps).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _native
from . import OCTAHEDRON, TETRAHEDRON, Primitives, Rasterizer


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else C.c_void_p(0)


def _stream(device):
    return C.c_void_p(_torch().cuda.current_stream(device).cuda_stream)


def _check(st, what):
    _native.check(None, st, what)


def _ndist(kind: int) -> int:
    return 3 if kind == OCTAHEDRON else 4


def camera_extent(cameras) -> float:
    """Largest distance between a camera centre and the mean camera centre."""
    pos = []
    for c in cameras:
        M = np.asarray(c.viewmat, np.float64).reshape(4, 4)
        pos.append(-M[:3, :3].T @ M[:3, 3])
    pos = np.array(pos)
    return float(np.max(np.linalg.norm(pos - pos.mean(0), axis=1))) if len(pos) > 1 else 1.0


# ---------------------------------------------------------------- functional

def params_forward(kind, centre, quat, dist, logit, verts=None, opacity=None):
    """Vertices [n, kind, 3] and opacities [n] of the parameter form (Sec. 3.1)."""
    torch = _torch()
    n = centre.shape[0]
    verts = torch.empty(n, kind, 3, device=centre.device) if verts is None else verts
    opacity = torch.empty(n, device=centre.device) if opacity is None else opacity
    L = _native.load()
    _check(L.lp_params_forward(int(kind), n, _ptr(centre), _ptr(quat), _ptr(dist), _ptr(logit), _ptr(verts),
                               _ptr(opacity), _stream(centre.device)), "lp_params_forward")
    return verts, opacity


def params_backward(kind, quat, dist, logit, dverts, dopacity, dcentre):
    """Adjoint of params_forward.  dcentre is added to (it holds the
    renderer's direct centre gradient on entry); returns (dquat, ddist, dlogit)."""
    torch = _torch()
    n = quat.shape[0]
    dquat, ddist, dlogit = torch.empty_like(quat), torch.empty_like(dist), torch.empty_like(logit)
    L = _native.load()
    _check(L.lp_params_backward(int(kind), n, _ptr(quat), _ptr(dist), _ptr(logit), _ptr(dverts),
                                _ptr(dopacity), _ptr(dcentre), _ptr(dquat), _ptr(ddist), _ptr(dlogit),
                                _stream(quat.device)), "lp_params_backward")
    return dquat, ddist, dlogit


def l1_loss_grad(image, target, grad=None, loss=None):
    """mean |image - target| (added into the float64 `loss`) and its gradient."""
    torch = _torch()
    grad = torch.empty_like(image) if grad is None else grad
    if loss is None:
        loss = torch.zeros(1, dtype=torch.float64, device=image.device)
    L = _native.load()
    _check(L.lp_l1_loss_grad(_ptr(image), _ptr(target), image.numel(), _ptr(grad), _ptr(loss),
                             _stream(image.device)), "lp_l1_loss_grad")
    return loss, grad


def adam_group(offset, count, lr, lr_final=0.0, decay_steps=0, period=0, head=0, lr_tail=0.0):
    return _native.lp_adam_group(int(offset), int(count), float(lr), float(lr_final), int(decay_steps),
                                 int(period), int(head), float(lr_tail))


def adam_step(params, grads, m, v, groups, step, beta1=0.9, beta2=0.999, eps=1e-15):
    """One fused Adam update of the flat `params` over `groups`
    (lp_adam_group list); `step` is a device int32 tensor of completed steps."""
    arr = (_native.lp_adam_group * len(groups))(*groups)
    L = _native.load()
    _check(L.lp_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), arr, len(groups), float(beta1),
                          float(beta2), float(eps), _ptr(step), _stream(params.device)), "lp_adam_step")


def population_rules(extent: float, min_opacity=0.025, max_scene_frac=0.4, max_pixels=20,
                     grad_threshold=1.5e-4, clone_scene_frac=0.01):
    """App. "Experimental Setting"'s population thresholds (the defaults)."""
    return _native.lp_population_rules(float(extent), float(min_opacity), float(max_scene_frac), int(max_pixels),
                                       float(grad_threshold), float(clone_scene_frac))


def population_decide(kind, dist, logit, grad_sum, grad_count, px_max, rules):
    """Per-primitive action (uint8: 0 prune, 1 keep, 2 clone, 3 split), the
    destination row of each primitive (int32) and the new count (int32 [1]),
    all on the device."""
    torch = _torch()
    dev = logit.device
    n = int(logit.shape[0])
    L = _native.load()
    action = torch.empty(n, dtype=torch.uint8, device=dev)
    dest = torch.empty(n, dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    scratch = torch.empty(max(1, int(L.lp_population_scratch(n))), dtype=torch.int32, device=dev)
    _check(L.lp_population_decide(int(kind), n, _ptr(dist), _ptr(logit), _ptr(grad_sum), _ptr(grad_count),
                                  _ptr(px_max), C.byref(rules), _ptr(action), _ptr(dest), _ptr(n_out),
                                  _ptr(scratch), _stream(dev)), "lp_population_decide")
    return action, dest, n_out


_FIELDS = ("centre", "quat", "dist", "logit", "sh")


def _arrays(d):
    return _native.lp_param_arrays(*(C.c_void_p(d[k].data_ptr()) for k in _FIELDS))


def population_apply(kind, action, dest, normals, sets, n_out: int, out_sets=None):
    """Compact every set (dicts of the parameter-layer arrays; set 0 the
    parameters, the rest optimiser state) into n_out rows.  normals: device
    float32 [n, 2, 3] standard-normal draws for split children."""
    torch = _torch()
    if out_sets is None:
        out_sets = [{k: torch.empty((n_out,) + tuple(s[k].shape[1:]), dtype=torch.float32, device=s[k].device)
                     for k in _FIELDS} for s in sets]
    n = int(action.shape[0])
    K = int(sets[0]["sh"].shape[1])
    src = (_native.lp_param_arrays * len(sets))(*(_arrays(s) for s in sets))
    dst = (_native.lp_param_arrays * len(sets))(*(_arrays(s) for s in out_sets))
    L = _native.load()
    _check(L.lp_population_apply(int(kind), K, n, _ptr(action), _ptr(dest), _ptr(normals), src, dst, len(sets),
                                 _stream(action.device)), "lp_population_apply")
    return out_sets


def _make_params_fn():
    torch = _torch()

    class _Params(torch.autograd.Function):
        @staticmethod
        def forward(ctx, centre, quat, dist, logit, kind):
            c, q, d, l = (t.detach().contiguous() for t in (centre, quat, dist, logit))
            verts, opacity = params_forward(kind, c, q, d, l)
            ctx.kind = kind
            ctx.save_for_backward(q, d, l)
            return verts, opacity

        @staticmethod
        def backward(ctx, gverts, gopacity):
            q, d, l = ctx.saved_tensors
            n = q.shape[0]
            gv = torch.zeros(n, ctx.kind, 3, device=q.device) if gverts is None else gverts.contiguous()
            go = torch.zeros(n, device=q.device) if gopacity is None else gopacity.contiguous()
            dc = torch.zeros(n, 3, device=q.device)
            dq, dd, dl = params_backward(ctx.kind, q, d, l, gv, go, dc)
            return dc, dq, dd, dl, None

    return _Params


_PARAMS_FN = None


def params_layer(kind: int, centre, quat, dist, logit):
    """Differentiable parameter layer: (verts, opacity) from (centre, quaternion
    (w, x, y, z), distances, opacity logit).  The vertices also depend on the
    centre directly; pass the same centre tensor to `render` so that autograd
    adds the renderer's own centre gradient."""
    global _PARAMS_FN
    if _PARAMS_FN is None:
        _PARAMS_FN = _make_params_fn()
    return _PARAMS_FN.apply(centre, quat, dist, logit, int(kind))


def paper_learning_rates(extent: float) -> dict:
    return dict(centre=1.6e-4 * extent, centre_final=1.6e-6 * extent, centre_decay_steps=30_000,
                quat=1e-3, dist=1e-4 / 2.6 * extent, logit=2.5e-2, sh_dc=2.5e-3, sh_rest=1.25e-4)


# ---------------------------------------------------------------- fused step

class Trainer:
    """Fixed L1 + Adam optimisation step over all `cameras` per step."""

    GROUPS = ("centre", "quat", "dist", "logit", "sh")

    def __init__(self, kind: int, centre, quat, dist, logit, sh, cameras: Sequence, targets,
                 bg=(0.0, 0.0, 0.0), rasterizer: Optional[Rasterizer] = None, lrs: Optional[dict] = None,
                 extent: Optional[float] = None, device: int = 0):
        torch = _torch()
        if kind not in (OCTAHEDRON, TETRAHEDRON):
            raise ValueError(f"kind must be OCTAHEDRON (6) or TETRAHEDRON (4), got {kind}")
        self.lib = _native.load()
        self.kind = kind
        self.cameras = list(cameras)
        self.bg = tuple(float(x) for x in bg)
        self.rast = rasterizer if rasterizer is not None else Rasterizer(device)
        dev = self.rast.device
        self.D, self.K = _ndist(kind), int(sh.shape[1])
        self._layout(int(np.asarray(centre.shape)[0]))
        for k, src in zip(self.GROUPS, (centre, quat, dist, logit, sh)):
            self.p[k].copy_(torch.as_tensor(src, dtype=torch.float32).reshape(self.p[k].shape))
        self.pixels = sum(c.width * c.height for c in self.cameras)
        self.targets = torch.as_tensor(targets, dtype=torch.float32).reshape(3 * self.pixels).to(dev)
        self.images = torch.empty(3 * self.pixels, device=dev)
        self.dimages = torch.empty_like(self.images)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.step_count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.extent = camera_extent(self.cameras) if extent is None else float(extent)
        lr = paper_learning_rates(self.extent)
        if lrs:
            lr.update(lrs)
        self.lr = lr
        self._cams = _native.camera_struct(self.cameras)
        self._bgv = (C.c_float * 3)(*self.bg)
        self.stats = None
        self._bind()

    def _layout(self, n: int):
        """Flat parameter, gradient and moment arrays for n primitives (the
        parameters uninitialised, the rest zero) and the per-primitive buffers."""
        torch = _torch()
        dev = self.rast.device
        D, K = self.D, self.K
        self.n = n
        self.shapes = dict(centre=(n, 3), quat=(n, 4), dist=(n, D), logit=(n,), sh=(n, K, 3))
        self.sizes = {k: int(np.prod(s)) for k, s in self.shapes.items()}
        self.offsets, off = {}, 0
        for k in self.GROUPS:
            self.offsets[k] = off
            off += self.sizes[k]
        self.total = off
        self.P = torch.empty(off, device=dev)
        self.G = torch.zeros(off, device=dev)
        self.m = torch.zeros(off, device=dev)
        self.v = torch.zeros(off, device=dev)
        self.p, self.g = self._views(self.P), self._views(self.G)
        self.verts = torch.empty(n, self.kind, 3, device=dev)
        self.opacity = torch.empty(n, device=dev)
        self.dverts = torch.empty_like(self.verts)
        self.dopacity = torch.empty_like(self.opacity)

    def _views(self, buf):
        return {k: buf[self.offsets[k]:self.offsets[k] + self.sizes[k]].view(*self.shapes[k]) for k in self.GROUPS}

    def _bind(self):
        """Adam groups and the boundary structs of the current arrays."""
        lr, o, sz = self.lr, self.offsets, self.sizes
        self.groups = [
            adam_group(o["centre"], sz["centre"], lr["centre"], lr["centre_final"], lr["centre_decay_steps"]),
            adam_group(o["quat"], sz["quat"], lr["quat"]),
            adam_group(o["dist"], sz["dist"], lr["dist"]),
            adam_group(o["logit"], sz["logit"], lr["logit"]),
            adam_group(o["sh"], sz["sh"], lr["sh_dc"], period=3 * self.K, head=3, lr_tail=lr["sh_rest"]),
        ]
        self._groups_arr = (_native.lp_adam_group * len(self.groups))(*self.groups)
        self.prims = Primitives(self.kind, self.p["centre"], self.verts, self.opacity, self.p["sh"])
        self._ps = self.prims.struct()
        self.graph = None

    # ------------------------------------------------ population control
    def enable_densify_stats(self):
        """Gather the densification statistics from the next step on (zeroed
        here).  A captured graph is dropped: capture again afterwards."""
        torch = _torch()
        dev = self.rast.device
        self.stats = dict(grad_sum=torch.zeros(self.n, device=dev),
                          grad_count=torch.zeros(self.n, dtype=torch.int32, device=dev),
                          px_max=torch.zeros(self.n, dtype=torch.int32, device=dev))
        self.rast.set_densify_stats(self.stats["grad_sum"], self.stats["grad_count"], self.stats["px_max"])
        self.graph = None

    def densify(self, rules=None, normals=None, generator=None) -> dict:
        """Adjust the population once (Sec. 3.4 "Adaptive Population
        Control"; the paper does so every 250 steps): prune, clone and split
        by the gathered statistics, compact parameters and Adam moments into
        new arrays, zero the gradients and the statistics.  normals: optional
        device float32 [n, 2, 3] draws for split children (else drawn with
        `generator`).  Synchronises once to read the new count; drops a
        captured graph.  Returns the per-action counts."""
        torch = _torch()
        if self.stats is None:
            raise RuntimeError("enable_densify_stats() before densify()")
        dev = self.rast.device
        rules = population_rules(self.extent) if rules is None else rules
        st = self.stats
        action, dest, n_out = population_decide(self.kind, self.p["dist"], self.p["logit"], st["grad_sum"],
                                                st["grad_count"], st["px_max"], rules)
        if normals is None:
            normals = torch.randn(self.n, 2, 3, device=dev, generator=generator)
        n_new = int(n_out.item())
        counts = torch.bincount(action.long(), minlength=4).tolist()
        old = [self.p, self._views(self.m), self._views(self.v)]
        keep = (self.P, self.m, self.v, action, dest, normals)   # alive until the copies ran
        self._layout(n_new)
        population_apply(self.kind, action, dest, normals, old, n_new,
                         out_sets=[self.p, self._views(self.m), self._views(self.v)])
        self._bind()
        self.enable_densify_stats()
        torch.cuda.current_stream(dev).synchronize()
        del keep
        return dict(pruned=counts[0], kept=counts[1], cloned=counts[2], split=counts[3], n=n_new)

    def step(self):
        """Enqueue one optimisation step on the current stream; the loss of
        the step lands in self.loss (float64, device)."""
        L, s = self.lib, _stream(self.rast.device)
        n, kind, p, g = self.n, self.kind, self.p, self.g
        _check(L.lp_params_forward(kind, n, _ptr(p["centre"]), _ptr(p["quat"]), _ptr(p["dist"]),
                                   _ptr(p["logit"]), _ptr(self.verts), _ptr(self.opacity), s),
               "lp_params_forward")
        _native.check(self.rast.ctx, L.lp_render_forward(self.rast.ctx, C.byref(self._ps), self._cams,
                                                         len(self.cameras), self._bgv, _ptr(self.images), s),
                      "lp_render_forward")
        self.rast._fwd = (self.prims, self.cameras, self.bg)
        self.loss.zero_()
        _check(L.lp_l1_loss_grad(_ptr(self.images), _ptr(self.targets), 3 * self.pixels, _ptr(self.dimages),
                                 _ptr(self.loss), s), "lp_l1_loss_grad")
        _native.check(self.rast.ctx, L.lp_render_backward(self.rast.ctx, _ptr(self.dimages), _ptr(g["centre"]),
                                                          _ptr(self.dverts), _ptr(self.dopacity), _ptr(g["sh"]),
                                                          0, s), "lp_render_backward")
        _check(L.lp_params_backward(kind, n, _ptr(p["quat"]), _ptr(p["dist"]), _ptr(p["logit"]),
                                    _ptr(self.dverts), _ptr(self.dopacity), _ptr(g["centre"]), _ptr(g["quat"]),
                                    _ptr(g["dist"]), _ptr(g["logit"]), s), "lp_params_backward")
        _check(L.lp_adam_step(_ptr(self.P), _ptr(self.G), _ptr(self.m), _ptr(self.v), self._groups_arr,
                              len(self.groups), 0.9, 0.999, 1e-15, _ptr(self.step_count), s), "lp_adam_step")

    def capture(self, entry_margin: float = 1.5):
        """Size the workspace with one eager step, reserve it with a margin for
        growth of the tile list, then capture one step into a CUDA graph.  The
        two steps run here are real steps (the parameters move)."""
        torch = _torch()
        dev = self.rast.device
        self.step()
        torch.cuda.synchronize(dev)
        self.rast.sync_status()
        st = self.rast.stats()
        self.rast.reserve(st["records"], int(st["entries"] * entry_margin) + 4096, st["pixels"], st["tiles"])
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self.step()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self, n: int = 1, losses=None):
        """Replay the captured step n times; with `losses` (a float64 device
        tensor of length >= n) also record each step's loss."""
        for i in range(n):
            self.graph.replay()
            if losses is not None:
                losses[i:i + 1].copy_(self.loss)

    def steps_done(self) -> int:
        return int(self.step_count.item())

    def loss_value(self) -> float:
        return float(self.loss.item())

    def params_numpy(self) -> dict:
        return {k: v.detach().cpu().numpy() for k, v in self.p.items()}
