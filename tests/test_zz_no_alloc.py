"""lp_render_forward_noalloc: the allocation-free single-camera forward for
callers that cannot call cudaMalloc (pooled or budgeted device memory, hosts
that forbid allocation after start-up).

Its image must match lp_render_forward's within the image tolerance the
parity tests use (1e-4 per channel; the two run the same kernels, so they
agree bit for bit), on two calls in a row -- the second call reuses the shared
scratch array and must not see the first call's leftovers -- and the FP64
oracle's within the same tolerance.  This file is collected last so that, if
it fails, a run stopped at the first failure has already run everything
else."""
import ctypes as C

import numpy as np
import pytest

import oracle
import scenes
from tests.parity import assert_images_match

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
        orc, info = oracle.render(w.scene, [cam], bg=bg, info=True)
        for _ in range(2):
            img = torch.full((3 * cam.width * cam.height,), -1.0, device="cuda:0")
            st = _noalloc(lib, prims, cam, bg, img, stream)
            assert st == _native.LP_OK, lib.lp_status_string(st)
            torch.cuda.synchronize()
            err = (img - ref).abs().max().item()
            assert err <= IMG_TOL, err
            assert_images_match(img.cpu().numpy().astype(np.float64), orc, info, [cam])


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


def test_noalloc_rejects_a_tile_list_over_capacity():
    """300 primitives that each cover the whole 512x512 image make a tile
    list of 300 x 1024 entries, past the 262144 the scratch array holds: the
    call returns LP_ERR_CAPACITY after the key scan and leaves the image
    untouched; a call within the limits then renders normally."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import Primitives, Rasterizer, _native
    lib = _native.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 300
    rng = np.random.default_rng(3)
    c = np.zeros((n, 3))
    c[:, 2] = np.linspace(1.0, 2.0, n)
    v = scenes.octahedra_from_axes(c, np.repeat(np.eye(3)[None], n, 0), np.tile([[4.0, 4.0, 0.01]], (n, 1)))
    sh = scenes.sh_from_rgb(rng.uniform(0, 1, (n, 3)))[:, None, :]
    big = scenes.Scene(6, c.astype(np.float32), v.astype(np.float32), np.full(n, 0.05, np.float32),
                       sh.astype(np.float32), 0)
    cam = scenes.make_camera((0, 0, 4), 512, 512, 60)
    prims = Primitives.from_scene(big, "cuda:0")
    img = torch.full((3 * 512 * 512,), -1.0, device="cuda:0")
    assert _noalloc(lib, prims, cam, (0, 0, 0), img, stream) == _native.LP_ERR_CAPACITY
    torch.cuda.synchronize()
    assert torch.all(img == -1.0)
    # the same primitives fewer times fit: 200 x 1024 entries
    few = big.subset(np.arange(200))
    pf = Primitives.from_scene(few, "cuda:0")
    assert _noalloc(lib, pf, cam, (0, 0, 0), img, stream) == _native.LP_OK
    torch.cuda.synchronize()
    ref = Rasterizer(0).forward(pf, [cam], (0, 0, 0))
    assert torch.equal(img, ref)
