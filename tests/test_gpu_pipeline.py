"""HostPipeline: forward + backward steps streamed between pinned host
memory and the GPU, overlapped across steps, against direct calls of the
same rasterizer on device tensors."""
import numpy as np
import pytest

import scenes
from tests.parity import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _workload():
    w = scenes.workload(3, scale=0.004)
    rng = np.random.default_rng(3)
    cams = scenes.sphere_cameras(rng, [(200, 120), (97, 61), (64, 48)], 6.0, 60.0)
    return scenes.Workload("tetra4k_3mixed", w.scene, cams)


def test_pipeline_matches_direct_calls(torch):
    from paper_2501_16312_gb300 import Primitives, Rasterizer
    from paper_2501_16312_gb300.pipeline import HostPipeline
    w = _workload()
    sc, bg = w.scene, (0.1, 0.2, 0.3)
    P = sum(c.width * c.height for c in w.cameras)
    steps = 5
    rng = np.random.default_rng(1)
    # per step: slightly moved primitives and its own image gradient
    ins, outs = [], []
    for s in range(steps):
        d = {"centre": sc.centre + 0.002 * s, "verts": sc.verts + 0.002 * s, "opacity": sc.opacity,
             "sh": sc.sh, "dL": rng.normal(size=3 * P)}
        ins.append({k: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float32).pin_memory()
                    for k, v in d.items()})
        outs.append({"images": torch.empty(3 * P, pin_memory=True),
                     **{k: torch.empty(ins[-1][k].shape, pin_memory=True)
                        for k in ("centre", "verts", "opacity", "sh")}})
    pipe = HostPipeline(Rasterizer(0), sc.kind, sc.n, sc.sh_degree, w.cameras, bg)
    for s in range(steps):
        pipe.submit(ins[s], outs[s])
    pipe.synchronize()
    h2d, d2h = pipe.bytes_per_step()
    assert h2d == sum(4 * ins[0][k].numel() for k in ins[0])
    assert d2h == 4 * 3 * P + sum(4 * ins[0][k].numel() for k in ("centre", "verts", "opacity", "sh"))

    rast = Rasterizer(0)
    for s in range(steps):
        dev = {k: v.to("cuda:0") for k, v in ins[s].items()}
        prims = Primitives(sc.kind, dev["centre"], dev["verts"], dev["opacity"], dev["sh"], sc.sh_degree)
        img = rast.forward(prims, w.cameras, bg).clone()
        g = rast.backward(dev["dL"])
        torch.cuda.synchronize()
        assert torch.equal(outs[s]["images"], img.cpu()), s
        for k in g:
            assert rel_l2(outs[s][k].numpy(), g[k].cpu().numpy()) <= 1e-5, (s, k)   # atomics order
