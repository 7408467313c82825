"""lp_render_forward_noalloc: the allocation-free single-camera forward for
callers that cannot call cudaMalloc (graph capture, pooled or budgeted device
memory, hosts that forbid allocation after start-up).

Its image must match lp_render_forward's within the image tolerance the
parity tests use (1e-4 per channel; the two run the same kernels, so they
agree bit for bit), on two calls in a row -- the second call reuses the shared
scratch array and must not see the first call's leftovers.  This file is
collected last so that, if it fails, a run stopped at the first failure has
already run everything else."""
import ctypes as C

import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4


def _noalloc(lib, prims, cam, bg, image, stream):
    from paper_2501_16312_gb300 import _native
    ps = prims.struct()
    cs = _native.camera_struct([cam])
    bgv = (C.c_float * 3)(*bg)
    return lib.lp_render_forward_noalloc(C.byref(ps), cs, bgv, C.c_void_p(image.data_ptr()), stream)


def test_noalloc_matches_forward_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import Primitives, Rasterizer, _native
    lib = _native.load()
    rast = Rasterizer(0)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(scenes.workload(1, scale=0.5), (0.1, 0.2, 0.3)),   # 5k octahedra, 512x512
             (scenes.workload(0), (0.0, 0.0, 0.0))]             # 64 tetrahedra, 128x128
    for w, bg in cases:
        cam = w.cameras[0]
        prims = Primitives.from_scene(w.scene, "cuda:0")
        ref = rast.forward(prims, [cam], bg).clone()
        for _ in range(2):
            img = torch.full((3 * cam.width * cam.height,), -1.0, device="cuda:0")
            st = _noalloc(lib, prims, cam, bg, img, stream)
            assert st == _native.LP_OK, lib.lp_status_string(st)
            torch.cuda.synchronize()
            err = (img - ref).abs().max().item()
            assert err <= IMG_TOL, err


def test_noalloc_rejects_oversized_inputs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import Primitives, _native
    lib = _native.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    w = scenes.workload(0)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    big = scenes.make_camera((0, 0, 4), 1024, 1024, 60)        # more than 512 * 512 pixels
    img = torch.empty(3 * 1024 * 1024, device="cuda:0")
    assert _noalloc(lib, prims, big, (0, 0, 0), img, stream) == _native.LP_ERR_CAPACITY
    many = scenes.workload(1, scale=2.0).scene                 # 20k > 16384 primitives
    pm = Primitives.from_scene(many, "cuda:0")
    cam = scenes.make_camera((0, 0, 4), 64, 64, 60)
    img2 = torch.empty(3 * 64 * 64, device="cuda:0")
    assert _noalloc(lib, pm, cam, (0, 0, 0), img2, stream) == _native.LP_ERR_CAPACITY
