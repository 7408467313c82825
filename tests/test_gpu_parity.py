"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Sizes are chosen so the oracle finishes in seconds while spanning many tiles
with ragged edges; the full-size workload is checked on sampled pixels."""
import numpy as np
import pytest

import oracle
import scenes
from tests.parity import (assert_grads_match, assert_images_match, gpu_forward_backward,
                          mask_borderline, rel_l2)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rast():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import Rasterizer
    return Rasterizer(0)


def multiview_small():
    """Mixed-resolution cameras (ragged tile edges) on a scaled-down version of
    the 1M-tetrahedron box workload."""
    w = scenes.workload(3, scale=0.004)
    rng = np.random.default_rng(3)
    sizes = [(200, 120), (97, 61), (64, 48)]
    cams = scenes.sphere_cameras(rng, sizes, 6.0, 60.0)
    return scenes.Workload("tetra4k_3mixed", w.scene, cams)


CASES = {
    "cfg0_tetra64": lambda: scenes.workload(0),
    "cfg1_octa10k": lambda: scenes.workload(1),
    "multiview_tetra": multiview_small,
}


@pytest.mark.parametrize("onesweep", [0, 1])
@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("sort_mode", [0, 1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_tile_lists_bit_exact(rast, case, sort_mode, tile, onesweep):
    """Sec. 3.2 "Global Sorting and Tiling" at every tile edge the tuner
    may pick and in every sort form: counts, keys and values equal the
    oracle's bit for bit."""
    w = CASES[case]()
    base = rast.tuning()
    rast.set_tuning(sort_mode=sort_mode, tile=tile, pixels_per_thread=2, onesweep=onesweep)
    try:
        gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0))
    finally:
        rast.set_tuning(**base)
    k, v = rast.debug_keys()
    ko, vo, co = oracle.keys(w.scene, w.cameras, tile=tile)
    np.testing.assert_array_equal(rast.debug_counts(), co)
    assert k.shape == ko.shape
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)


def _crowded_tiles():
    """9,000 large tetrahedra filling a 96x64 view: tiles list up to about
    6,700 entries, so that the per-tile sort takes all three of its forms."""
    scene = scenes.tetra_scene(seed=11, n=9000, box=0.6, s_range=(0.4, 0.9))
    return scene, [scenes.make_camera((0.0, 0.0, 3.0), 96, 64, 60.0)]


@pytest.mark.parametrize("sort_mode", [1, 2])
@pytest.mark.parametrize("tile", [8, 16])
def test_tile_lists_bit_exact_long_runs(rast, sort_mode, tile):
    """Tile lists far longer than a warp's run in the per-tile sort (512
    entries), which sort mode 2 sorts with a block per run in shared memory
    up to 2,048 entries and through global scratch beyond:
    keys and values bit-exact, images within the bar."""
    scene, cams = _crowded_tiles()
    base = rast.tuning()
    rast.set_tuning(sort_mode=sort_mode, tile=tile, pixels_per_thread=2)
    try:
        img, _ = gpu_forward_backward(rast, scene, cams, (0.1, 0.1, 0.1))
        k, v = rast.debug_keys()
    finally:
        rast.set_tuning(**base)
    ko, vo, _ = oracle.keys(scene, cams, tile=tile)
    runs = np.unique(ko >> np.uint64(32), return_counts=True)[1]   # entries per tile
    assert runs.max() > 2048 and runs.min() <= 512, (runs.min(), runs.max())
    assert ((runs > 512) & (runs <= 2048)).any(), runs
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)
    ref, info = oracle.render(scene, cams, bg=(0.1, 0.1, 0.1), info=True)
    assert_images_match(img, ref, info, cams)


@pytest.mark.parametrize("onesweep", [0, 1])
@pytest.mark.parametrize("radix_bits", [4, 6, 11])
@pytest.mark.parametrize("tile", [8, 16])
@pytest.mark.parametrize("sort_mode", [0, 1, 2])
def test_tile_lists_bit_exact_every_digit_width(rast, sort_mode, tile, radix_bits, onesweep):
    """The radix sort at each widest digit the tuner may pick: a sort of k key
    bits takes ceil(k / radix_bits) passes of evenly spread digits, so these
    cases run digits of 4, 5, 6, 10 and 11 bits (10k octahedra at 512x512:
    tile ids of 10 or 12 bits, 32-bit depths, 42- or 44-bit combined keys;
    the full-size 8x8 cases add 7, 8 and 9).  Keys and values equal the
    oracle's bit for bit."""
    w = CASES["cfg1_octa10k"]()
    base = rast.tuning()
    rast.set_tuning(sort_mode=sort_mode, tile=tile, pixels_per_thread=2, radix_bits=radix_bits,
                    onesweep=onesweep)
    try:
        gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0))
    finally:
        rast.set_tuning(**base)
    k, v = rast.debug_keys()
    ko, vo, _ = oracle.keys(w.scene, w.cameras, tile=tile)
    assert k.shape == ko.shape
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)


@pytest.mark.parametrize("case", sorted(CASES))
def test_forward_backward_parity(rast, case):
    w = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    ref, info = oracle.render(w.scene, w.cameras, bg=bg, info=True)
    dL = mask_borderline(scenes.image_gradient(w, seed=1), info, w.cameras)
    img, grads = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
    _, ref_g = oracle.render(w.scene, w.cameras, bg=bg, dL_dimage=dL)
    err = assert_images_match(img, ref, info, w.cameras)
    rel = assert_grads_match(grads, ref_g)
    print(f"{case}: max image err {err:.2e}, grad rel L2 {rel}")


AA = float(np.float32(0.1))   # the paper's 2D filter size; both sides get the same binary32 value


@pytest.mark.parametrize("sort_mode", [0, 1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_filter_2d_parity(rast, case, sort_mode):
    """Sec. 3.3 2D filter on: tile lists bit-exact, images and gradients
    within the parity bars, and the filter visibly changes the image."""
    w = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    ref, info = oracle.render(w.scene, w.cameras, bg=bg, info=True, aa=AA)
    dL = mask_borderline(scenes.image_gradient(w, seed=2), info, w.cameras)
    rast.set_tuning(sort_mode=sort_mode)
    rast.set_filter_2d(AA)
    try:
        assert rast.filter_2d() == AA
        img, grads = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
        k, v = rast.debug_keys()
    finally:
        rast.set_filter_2d(0.0)
        rast.set_tuning(sort_mode=0)
    ko, vo, _ = oracle.keys(w.scene, w.cameras, tile=16, aa=AA)
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)
    _, ref_g = oracle.render(w.scene, w.cameras, bg=bg, dL_dimage=dL, aa=AA)
    err = assert_images_match(img, ref, info, w.cameras)
    rel = assert_grads_match(grads, ref_g)
    img0, _ = gpu_forward_backward(rast, w.scene, w.cameras, bg)
    assert np.abs(img - img0).max() > 1e-3
    print(f"{case}: 2D filter on, max image err {err:.2e}, grad rel L2 {rel}")


def test_filter_2d_rejects_bad_sizes(rast):
    from paper_2501_16312_gb300 import LinPrimError
    for bad in (-0.1, 17.0, float("nan")):
        with pytest.raises(LinPrimError):
            rast.set_filter_2d(bad)
    assert rast.filter_2d() == 0.0


def _depth_match(d, do, flags, tol=2e-5):
    ok = flags == 0
    assert np.array_equal(d[ok] == 0, do[ok] == 0), "pixels with / without depth differ"
    np.testing.assert_allclose(d[ok], do[ok], rtol=tol, atol=tol)
    return int(ok.sum()), int((do[ok] > 0).sum())


@pytest.mark.parametrize("case", sorted(CASES))
def test_depth_parity(rast, case):
    """App. "Depth and Surface Reconstruction": depth of the first primitive
    taking the cumulative opacity above 0.5, against the oracle on every
    pixel that is not borderline."""
    w = CASES[case]()
    dL = scenes.image_gradient(w, seed=3)
    _, g_ref = gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0), dL)
    d = rast.depth().cpu().numpy().astype(np.float64)
    # the depth pass leaves the forward state alone: a backward now is unchanged
    import torch
    g2 = rast.backward(torch.as_tensor(dL, device="cuda:0"))
    for k in g_ref:
        assert rel_l2(g2[k].cpu().numpy(), g_ref[k]) <= 1e-5, k   # float atomics reorder
    do, flags = oracle.depth(w.scene, w.cameras)
    n_ok, n_valid = _depth_match(d, do, flags)
    assert n_valid > 0
    print(f"{case}: depth on {n_ok} pixels ({n_valid} with a depth)")


@pytest.mark.parametrize("case", sorted(CASES))
def test_exact_mode_parity(rast, case):
    """App. "Ray Space Approximation", the variant without it: tile lists
    bit-exact, images, gradients and depth against the oracle's exact mode."""
    w = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    ref, info = oracle.render(w.scene, w.cameras, bg=bg, info=True, exact=True)
    dL = mask_borderline(scenes.image_gradient(w, seed=4), info, w.cameras)
    rast.set_exact(True)
    try:
        assert rast.exact()
        img, grads = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
        k, v = rast.debug_keys()
        depth = rast.depth().cpu().numpy().astype(np.float64)
    finally:
        rast.set_exact(False)
    ko, vo, _ = oracle.keys(w.scene, w.cameras, tile=16, exact=True)
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)
    _, ref_g = oracle.render(w.scene, w.cameras, bg=bg, dL_dimage=dL, exact=True)
    err = assert_images_match(img, ref, info, w.cameras)
    rel = assert_grads_match(grads, ref_g)
    do, flags = oracle.depth(w.scene, w.cameras, exact=True)
    _depth_match(depth, do, flags)
    img_rs, _ = gpu_forward_backward(rast, w.scene, w.cameras, bg)
    print(f"{case}: exact mode, max image err {err:.2e}, grad rel L2 {rel}, "
          f"max difference to the ray-space image {np.abs(img - img_rs).max():.2e}")


def test_exact_mode_edge_cases(rast):
    """Near cull (a vertex at depth <= 0.2), the 2D filter switched off, and a
    primitive covering the whole image."""
    bg = (0.25, 0.5, 0.75)
    cam = scenes.make_camera((0, 0, 4), 48, 40, 60)
    near = scenes.Scene(6, np.array([[0, 0, 3.5]], np.float32),
                        scenes.octahedra_from_axes(np.array([[0, 0, 3.5]]), np.eye(3)[None],
                                                   np.array([[0.2, 0.2, 0.35]])).astype(np.float32),
                        np.array([0.8], np.float32), np.zeros((1, 1, 3), np.float32), 0)
    big = scenes.Scene(6, np.array([[0, 0, 2.0]], np.float32),
                       scenes.octahedra_from_axes(np.array([[0, 0, 2.0]]), np.eye(3)[None],
                                                  np.array([[3.0, 2.5, 0.5]])).astype(np.float32),
                       np.array([0.7], np.float32), np.full((1, 1, 3), 0.4, np.float32), 0)
    rast.set_exact(True)
    rast.set_filter_2d(0.1)
    try:
        img_near, _ = gpu_forward_backward(rast, near, [cam], bg)
        img_big, g_big = gpu_forward_backward(rast, big, [cam], bg,
                                              np.ones(3 * cam.pixels, np.float32))
    finally:
        rast.set_exact(False)
        rast.set_filter_2d(0.0)
    np.testing.assert_array_equal(img_near.reshape(3, -1), np.repeat(np.array(bg)[:, None], cam.pixels, 1).astype(np.float32))
    ref, info, ref_g = oracle.render(big, [cam], bg=bg, dL_dimage=np.ones(3 * cam.pixels), info=True, exact=True)
    assert_images_match(img_big, ref, info, [cam])
    assert_grads_match(g_big, ref_g)


def test_full_size_workload(rast):
    """The 500k-octahedron, 8 x 1264x832 workload in the launch configuration
    the benchmark times: every pixel of camera 0 and sampled pixels of camera 5
    against the oracle."""
    w = scenes.workload(2)
    img, _ = gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0))
    depth = rast.depth().cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(7)
    off = 0
    for ci, cam in enumerate(w.cameras):
        n = cam.width * cam.height
        if ci in (0, 5):
            q = np.arange(n) if ci == 0 else rng.choice(n, 4000, replace=False)
            px, py = (q % cam.width).astype(np.int32), (q // cam.width).astype(np.int32)
            ref, info = oracle.render_pixels(w.scene, cam, px, py)
            got = img[3 * off:3 * (off + n)].reshape(3, n)[:, q].T
            err = np.abs(got - ref).max(1)
            clean = info[:, 2] == 0
            assert err[clean].max() <= 1e-4, err[clean].max()
            assert (err[~clean] > 1e-4).sum() <= max(2, 1e-4 * len(q))
            s = q[:4000] if ci == 0 else q
            do, flags = oracle.depth_pixels(w.scene, cam, (s % cam.width).astype(np.int32),
                                            (s // cam.width).astype(np.int32))
            _depth_match(depth[off:off + n][s], do, flags)
        off += n


def test_full_size_sampled_gradient(rast):
    """Gradients at full size (500k octahedra, all 8 cameras in one batched
    forward + backward, the benchmark's schedule) for a loss on 4096 random
    pixels of camera 0, against the oracle's adjoint of the same pixels."""
    w = scenes.workload(2)
    cam = w.cameras[0]
    q = np.random.default_rng(9).choice(cam.width * cam.height, 4096, replace=False)
    px, py = (q % cam.width).astype(np.int32), (q // cam.width).astype(np.int32)
    _, info = oracle.render_pixels(w.scene, cam, px, py)
    dLc = np.random.default_rng(8).normal(size=(px.size, 3))
    dLc[info[:, 2] > 0] = 0.0                      # borderline pixels (stop or graze)
    dL = np.zeros(3 * sum(c.width * c.height for c in w.cameras))
    n0 = cam.width * cam.height
    for ch in range(3):
        dL[ch * n0 + py * cam.width + px] = dLc[:, ch]
    base = rast.tuning()
    try:
        rast.set_tuning(sort_mode=1, batch=32, pixels_per_thread=4, chain_split=0)
        _, g = gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0), dL)
    finally:
        rast.set_tuning(**base)
    _, _, ref = oracle.render_pixels(w.scene, cam, px, py, dL_dC=dLc)
    rel = assert_grads_match(g, ref)
    touched = int((np.abs(ref["opacity"]) > 0).sum())
    print(f"full-size sampled gradient: {touched} primitives touched, relative L2 {rel}")
    assert touched > 1000


def test_permutation_invariance(rast):
    w = scenes.workload(1, scale=0.3)
    img, _ = gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0))
    perm = np.random.default_rng(4).permutation(w.scene.n)
    img_p, _ = gpu_forward_backward(rast, w.scene.subset(perm), w.cameras, (0, 0, 0))
    np.testing.assert_array_equal(img, img_p)


def test_batched_equals_per_view(rast):
    w = multiview_small()
    img, _ = gpu_forward_backward(rast, w.scene, w.cameras, (0.2, 0.2, 0.2))
    parts = [gpu_forward_backward(rast, w.scene, [c], (0.2, 0.2, 0.2))[0] for c in w.cameras]
    np.testing.assert_array_equal(img, np.concatenate(parts))


def test_per_view_accumulated_gradients_equal_batched(rast):
    import torch
    from paper_2501_16312_gb300 import Primitives
    w = multiview_small()
    dL = scenes.image_gradient(w, seed=2)
    _, gb = gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0), dL)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    acc = None
    off = 0
    for c in w.cameras:
        n = 3 * c.width * c.height
        rast.forward(prims, [c])
        g = torch.as_tensor(dL[off:off + n], device="cuda:0")
        acc = rast.backward(g, grads=acc, accumulate=acc is not None)
        off += n
    for k in gb:
        assert rel_l2(acc[k].cpu().numpy(), gb[k]) <= 1e-5, k


@pytest.mark.parametrize("kind", ["empty", "culled", "ragged", "huge", "one_pixel", "degenerate"])
def test_edge_cases(rast, kind):
    bg = (0.25, 0.5, 0.75)
    if kind == "empty":
        sc = scenes.workload(0).scene.subset(np.arange(0))
        cams = [scenes.make_camera((0, 0, 4), 40, 24, 60)]
    elif kind == "culled":
        sc = scenes.workload(0).scene
        cams = [scenes.make_camera((0, 0, 4), 48, 32, 60, target=(0, 0, 8))]   # looks away
    elif kind == "ragged":
        sc = scenes.workload(0).scene
        cams = [scenes.make_camera((0.3, 0.2, 3.5), 37, 23, 60)]
    elif kind == "huge":
        # one primitive around the camera's view axis covering the whole image
        c = np.array([[0.0, 0.0, 2.5]])
        R = np.eye(3)[None]
        v = scenes.octahedra_from_axes(c, R, np.array([[3.0, 2.0, 0.5]]))
        sh = scenes.sh_from_rgb(np.array([[0.9, 0.1, 0.4]]))[:, None, :]
        sc = scenes.Scene(6, c.astype(np.float32), v.astype(np.float32),
                          np.array([0.7], np.float32), sh.astype(np.float32), 0)
        cams = [scenes.make_camera((0, 0, 4), 160, 96, 60)]
    elif kind == "degenerate":
        # every fourth primitive has a vertex on its centre: no density, not visible
        sc = scenes.workload(0).scene.subset(np.arange(64))
        sc.verts[::4, 1] = sc.centre[::4]
        cams = [scenes.make_camera((0.3, 0.2, 3.5), 70, 50, 60)]
    else:
        sc = scenes.workload(0).scene
        cams = [scenes.make_camera((0, 0, 4), 1, 1, 60)]
    P = sum(c.width * c.height for c in cams)
    ref, info = oracle.render(sc, cams, bg=bg, info=True)
    dL = mask_borderline(np.random.default_rng(0).normal(size=3 * P), info, cams)
    img, grads = gpu_forward_backward(rast, sc, cams, bg, dL)
    _, ref_g = oracle.render(sc, cams, bg=bg, dL_dimage=dL)
    assert_images_match(img, ref, info, cams)
    if kind in ("empty", "culled"):
        np.testing.assert_array_equal(img.reshape(3, -1), np.repeat(np.array(bg)[:, None], P, 1).astype(np.float32))
        for k in grads:
            assert np.all(grads[k] == 0)
    else:
        assert_grads_match(grads, ref_g)
    if kind == "degenerate":
        k, v = rast.debug_keys()
        ko, vo, co = oracle.keys(sc, cams, tile=16)
        np.testing.assert_array_equal(k, ko)
        np.testing.assert_array_equal(v, vo)
        assert np.all(co[::4] == 0)
        for name in grads:
            assert np.all(np.isfinite(grads[name]))
            assert np.all(grads[name][::4] == 0), name


def test_autograd_function(rast):
    import torch
    from paper_2501_16312_gb300 import render
    w = scenes.workload(0)
    t = lambda a: torch.tensor(a, device="cuda:0", requires_grad=True)
    leaves = [t(w.scene.centre), t(w.scene.verts), t(w.scene.opacity), t(w.scene.sh)]
    img = render(*leaves, w.cameras, kind=w.scene.kind, rasterizer=rast)
    g = torch.as_tensor(scenes.image_gradient(w), device="cuda:0")
    (img * g).sum().backward()
    _, ref_g = oracle.render(w.scene, w.cameras, dL_dimage=g.cpu().numpy().astype(np.float64))
    for leaf, k in zip(leaves, ("centre", "verts", "opacity", "sh")):
        assert rel_l2(leaf.grad.cpu().numpy(), ref_g[k]) <= 1e-3, k


def test_cuda_graph_capture_replays(rast):
    import torch
    from paper_2501_16312_gb300 import Primitives, Rasterizer
    w = multiview_small()
    r2 = Rasterizer(0)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    P = w.pixels
    img0 = r2.forward(prims, w.cameras, (0, 0, 0)).clone()
    g = torch.as_tensor(scenes.image_gradient(w), device="cuda:0")
    gr0 = {k: v.clone() for k, v in r2.backward(g).items()}
    st = r2.stats()
    r2.reserve(st["records"], 2 * st["entries"] + 1024, P, st["tiles"])
    img = torch.empty(3 * P, device="cuda:0")
    grads = {k: torch.empty_like(v) for k, v in gr0.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        r2.forward(prims, w.cameras, (0, 0, 0), images=img)     # warm-up outside capture
        r2.backward(g, grads=grads)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        r2.forward(prims, w.cameras, (0, 0, 0), images=img)
        r2.backward(g, grads=grads)
    img.zero_()
    for k in grads:
        grads[k].zero_()
    graph.replay()
    torch.cuda.synchronize()
    r2.sync_status()
    assert torch.equal(img, img0)
    for k in grads:
        assert rel_l2(grads[k].cpu().numpy(), gr0[k].cpu().numpy()) <= 1e-5


def test_every_tuning_renders_identical_images(rast):
    """Tile edge, tile order, sort mode, radix width, pixels per thread,
    batch, grid size and chain form change the schedule, never the
    arithmetic of a pixel: images are bitwise identical and
    gradients agree to float rounding (atomics and the chain form reorder the
    sums)."""
    import itertools
    w = multiview_small()
    dL = scenes.image_gradient(w, seed=3)
    base = rast.tuning()
    tile_pix = [(8, 1), (8, 2), (16, 1), (16, 2), (16, 4), (32, 2), (32, 4)]
    try:
        rast.set_tuning(tile=16, pixels_per_thread=4)
        img16, g16 = gpu_forward_backward(rast, w.scene, w.cameras, (0.1, 0.1, 0.1), dL)
        for (tile, pix), sm, rb, batch, bps, cs, to, ow in itertools.product(
                tile_pix, [0, 1], [4, 11, 8], [32, 128], [0, 1], [0, 1], [0, 1], [0, 1]):
            if (rb != 8 or to or ow) and (batch, bps, cs) != (32, 0, 0):
                continue    # the digit width, sort form and tile order touch one stage each
            rast.set_tuning(tile=tile, sort_mode=sm, radix_bits=rb, pixels_per_thread=pix, batch=batch,
                            blocks_per_sm=bps, chain_split=cs, tile_order=to, onesweep=ow)
            img, g = gpu_forward_backward(rast, w.scene, w.cameras, (0.1, 0.1, 0.1), dL)
            np.testing.assert_array_equal(img, img16)
            for k in g:
                assert rel_l2(g[k], g16[k]) <= 1e-5, (tile, sm, rb, pix, batch, bps, cs, to, ow, k)
    finally:
        rast.set_tuning(**base)


def test_tuning_rejects_unbuilt_schedules(rast):
    from paper_2501_16312_gb300 import LinPrimError
    base = rast.tuning()
    for bad in (dict(tile=12), dict(tile=8, pixels_per_thread=4), dict(tile=32, pixels_per_thread=1)):
        with pytest.raises(LinPrimError):
            rast.set_tuning(**dict(base, **bad))
    assert rast.tuning() == base


@pytest.mark.parametrize("tile", [8, 32])
@pytest.mark.parametrize("case", sorted(CASES))
def test_tile_sizes_vs_oracle(rast, case, tile):
    """Images and gradients at the other tile edges against the oracle (the
    tile changes only which tile lists a pixel walks, never its order)."""
    w = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    ref, info = oracle.render(w.scene, w.cameras, bg=bg, info=True)
    dL = mask_borderline(scenes.image_gradient(w, seed=1), info, w.cameras)
    base = rast.tuning()
    try:
        rast.set_tuning(tile=tile, pixels_per_thread=2)
        img, grads = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
    finally:
        rast.set_tuning(**base)
    _, ref_g = oracle.render(w.scene, w.cameras, bg=bg, dL_dimage=dL)
    assert_images_match(img, ref, info, w.cameras)
    assert_grads_match(grads, ref_g)


@pytest.mark.parametrize("case", sorted(CASES))
def test_chain_split_vs_oracle(rast, case):
    """The two-pass backward chain (geometry, then colour) against the oracle's
    adjoint, and against the one-pass chain: the same terms in another order."""
    w = CASES[case]()
    bg = (0.1, 0.2, 0.3)
    _, info = oracle.render(w.scene, w.cameras, bg=bg, info=True)
    dL = mask_borderline(scenes.image_gradient(w, seed=6), info, w.cameras)
    base = rast.tuning()
    try:
        rast.set_tuning(chain_split=1)
        _, g1 = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
        rast.set_tuning(chain_split=0)
        _, g0 = gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
    finally:
        rast.set_tuning(**base)
    _, ref_g = oracle.render(w.scene, w.cameras, bg=bg, dL_dimage=dL)
    assert_grads_match(g1, ref_g)
    for k in g1:   # float atomics order the per-record sums differently run to run
        assert rel_l2(g1[k], g0[k]) <= 1e-5, k


def test_unaligned_sh_array(rast):
    """SH coefficients at an address that is not 16-byte aligned (a view into
    a larger array): the one-pass chain, which re-reads SH rows per camera,
    falls back to 4-byte loads; images equal those of an aligned copy and
    gradients agree to the run-to-run rounding of float atomics."""
    import torch
    from paper_2501_16312_gb300 import Primitives
    w = scenes.workload(1)       # SH degree 3: 48-float rows
    dL = torch.as_tensor(scenes.image_gradient(w, seed=7), dtype=torch.float32, device="cuda:0")
    base_p = Primitives.from_scene(w.scene, "cuda:0")
    buf = torch.zeros(base_p.sh.numel() + 1, device="cuda:0")
    buf[1:].copy_(base_p.sh.reshape(-1))
    sh_off = buf[1:].view_as(base_p.sh)
    assert sh_off.data_ptr() % 16 == 4
    odd = Primitives(base_p.kind, base_p.centre, base_p.verts, base_p.opacity, sh_off)
    saved = rast.tuning()
    try:
        rast.set_tuning(chain_split=0)
        outs = []
        for prims in (base_p, odd):
            img = rast.forward(prims, w.cameras).clone()
            g = {k: v.clone() for k, v in rast.backward(dL).items()}
            torch.cuda.synchronize()
            outs.append((img, g))
    finally:
        rast.set_tuning(**saved)
    assert torch.equal(outs[0][0], outs[1][0])
    for k in outs[0][1]:
        assert rel_l2(outs[1][1][k].cpu().numpy(), outs[0][1][k].cpu().numpy()) <= 1e-5, k   # atomics order


def test_pair_counters_match_oracle_contributors(rast):
    """The intersected-pair counter equals the oracle's number of blended
    (pixel, primitive) pairs up to binary32 ties at silhouettes; the counters
    are ordered iterated >= evaluated >= intersected and iterated >=
    iterated-to-last >= intersected, and iterated-to-last sums the pixels'
    last-contributor list positions."""
    w = scenes.workload(1)
    gpu_forward_backward(rast, w.scene, w.cameras, (0, 0, 0))
    c = rast.count_pairs()
    _, info = oracle.render(w.scene, w.cameras, info=True)
    n_contrib = int(info[:, 0].sum())
    assert abs(c["intersected"] - n_contrib) <= 1e-4 * n_contrib + 2, (c, n_contrib)
    assert c["iterated"] >= c["evaluated"] >= c["intersected"] >= 0
    assert c["iterated"] >= c["iterated_to_last"] >= c["intersected"]
    last, _ = rast.pixel_state()
    assert c["iterated_to_last"] == int(last.astype(np.int64).sum())
    assert c["evaluated"] >= c["intersected"] > 0
