"""Forward + backward steps streamed from and to pinned host memory.

A caller whose primitives and image gradients live on the host (a data
loader, another process, a CPU-side optimiser) pays for two host<->device
transfers per step.  `HostPipeline` hides them behind the GPU work of the
neighbouring steps: step i's inputs are copied in while step i-1 computes,
its images are copied out while its own backward runs, and its gradients
while step i+1 runs.  Two device buffer sets alternate between steps; the
forward and backward of each set are captured as CUDA graphs (one per set
and pass), so no call reads a size back to the host.

Every step still moves all of its inputs in and all of its outputs out; the
rendering runs in the library's kernels exactly as `Rasterizer.forward` /
`Rasterizer.backward` do.  PyTorch supplies the streams, events and memory.

Usage::

    pipe = HostPipeline(rast, kind, n, sh_degree, cameras, bg)
    for step in range(k):
        pipe.submit(host_inputs, host_outputs)   # pinned tensors, see submit()
    pipe.synchronize()
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

from . import Primitives, Rasterizer

INPUTS = ("centre", "verts", "opacity", "sh", "dL")
GRADS = ("centre", "verts", "opacity", "sh")


def _torch():
    import torch
    return torch


class HostPipeline:
    """Streams forward + backward steps of one scene layout (primitive kind,
    count and SH degree, and one camera set) between pinned host tensors and
    the GPU.  The first `submit` sizes the workspace with one plain step on its
    inputs and reserves `entry_margin` times the tile-list length it needed;
    a later step whose tile list outgrows that raises from `synchronize`."""

    def __init__(self, rast: Rasterizer, kind: int, n: int, sh_degree: int, cameras: Sequence,
                 bg=(0.0, 0.0, 0.0), entry_margin: float = 1.25):
        torch = _torch()
        self.rast, self.kind, self.n, self.sh_degree = rast, int(kind), int(n), int(sh_degree)
        self.cameras, self.bg = list(cameras), tuple(float(x) for x in bg)
        self.entry_margin = float(entry_margin)
        dev = rast.device
        K = (self.sh_degree + 1) ** 2
        self.pixels = sum(c.width * c.height for c in self.cameras)
        shapes = dict(centre=(n, 3), verts=(n, kind, 3), opacity=(n,), sh=(n, K, 3), dL=(3 * self.pixels,))
        self.shapes = shapes
        self.sets = []
        for _ in range(2):
            inp = {k: torch.zeros(s, device=dev) for k, s in shapes.items()}
            out = dict(images=torch.zeros(3 * self.pixels, device=dev),
                       **{k: torch.zeros(shapes[k], device=dev) for k in GRADS})
            prims = Primitives(self.kind, inp["centre"], inp["verts"], inp["opacity"], inp["sh"], self.sh_degree)
            self.sets.append(dict(inp=inp, out=out, prims=prims))
        self.s_comp = torch.cuda.Stream(dev)
        self.s_in = torch.cuda.Stream(dev)
        self.s_out = torch.cuda.Stream(dev)
        ev = lambda: [torch.cuda.Event() for _ in range(2)]
        self.ev_prims_in, self.ev_dl_in, self.ev_fwd, self.ev_done, self.ev_out = ev(), ev(), ev(), ev(), ev()
        self.graphs = None
        self.steps = 0

    # ------------------------------------------------------------ capture
    def _run(self, b):
        s = self.sets[b]
        self.rast.forward(s["prims"], self.cameras, self.bg, images=s["out"]["images"])

    def _run_bwd(self, b):
        s = self.sets[b]
        grads = {k: s["out"][k] for k in GRADS}
        self.rast.backward(s["inp"]["dL"], grads=grads)

    def _prepare(self, host_in: Dict):
        """Size the workspace on the first inputs, then capture the forward and
        backward of both buffer sets (each set's backward right after its
        forward, since a backward reads the state its forward left)."""
        torch = _torch()
        dev = self.rast.device
        for s in self.sets:
            for k in INPUTS:
                s["inp"][k].copy_(host_in[k])
        torch.cuda.synchronize(dev)
        self._run(0)
        self._run_bwd(0)
        torch.cuda.synchronize(dev)
        self.rast.sync_status()
        st = self.rast.stats()
        self.rast.reserve(st["records"], int(st["entries"] * self.entry_margin) + 4096, st["pixels"], st["tiles"])
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):       # warm the reserved workspace outside capture
            self._run(0)
            self._run_bwd(0)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        graphs = []
        for b in range(2):
            gf, gb = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
            with torch.cuda.graph(gf):
                self._run(b)
            with torch.cuda.graph(gb):
                self._run_bwd(b)
            graphs.append((gf, gb))
        torch.cuda.synchronize(dev)
        self.graphs = graphs

    # ------------------------------------------------------------ steps
    def submit(self, host_in: Dict, host_out: Dict):
        """Enqueue one step.  host_in: pinned float32 tensors centre [n,3],
        verts [n,kind,3], opacity [n], sh [n,K,3] and dL [3 P] (the image
        gradient, cameras' [3][H][W] planes back to back); host_out: pinned
        tensors images [3 P] and the gradients centre, verts, opacity, sh.
        Returns without waiting; the host tensors must stay untouched until
        `synchronize` (or `step_done`) says the step has finished."""
        torch = _torch()
        if self.graphs is None:
            self._prepare(host_in)
        b = self.steps % 2
        s = self.sets[b]
        # inputs of set b: after step i-2's compute is done with them
        self.s_in.wait_event(self.ev_done[b])
        with torch.cuda.stream(self.s_in):
            for k in ("centre", "verts", "opacity", "sh"):
                s["inp"][k].copy_(host_in[k], non_blocking=True)
            self.ev_prims_in[b].record(self.s_in)
            s["inp"]["dL"].copy_(host_in["dL"], non_blocking=True)
            self.ev_dl_in[b].record(self.s_in)
        # compute: after the inputs landed and step i-2's outputs were copied out
        self.s_comp.wait_event(self.ev_prims_in[b])
        self.s_comp.wait_event(self.ev_out[b])
        gf, gb = self.graphs[b]
        with torch.cuda.stream(self.s_comp):
            gf.replay()
            self.ev_fwd[b].record(self.s_comp)
            self.s_comp.wait_event(self.ev_dl_in[b])
            gb.replay()
            self.ev_done[b].record(self.s_comp)
        # outputs: images once the forward is done, gradients after the backward
        self.s_out.wait_event(self.ev_fwd[b])
        with torch.cuda.stream(self.s_out):
            host_out["images"].copy_(s["out"]["images"], non_blocking=True)
            self.s_out.wait_event(self.ev_done[b])
            for k in GRADS:
                host_out[k].copy_(s["out"][k], non_blocking=True)
            self.ev_out[b].record(self.s_out)
        self.steps += 1

    def synchronize(self):
        """Wait for every submitted step; raises if a step's tile list
        overflowed the reserved workspace."""
        for s in (self.s_in, self.s_comp, self.s_out):
            s.synchronize()
        self.rast.sync_status()

    def bytes_per_step(self):
        """(host->device, device->host) bytes moved per step."""
        h2d = sum(4 * _numel(self.shapes[k]) for k in INPUTS)
        d2h = 4 * 3 * self.pixels + sum(4 * _numel(self.shapes[k]) for k in GRADS)
        return h2d, d2h


def _numel(shape):
    n = 1
    for x in shape:
        n *= int(x)
    return n
