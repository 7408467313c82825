"""Capacity overflow inside a captured CUDA graph.

A captured forward cannot read the tile-list length back, so it sorts up to
the capacity reserved with lp_reserve and latches LP_ERR_CAPACITY on the
device when the list is longer; lp_sync_status returns it.  The kernels must
write nothing past any buffer's capacity meanwhile: every workspace buffer
here carries a canary zone (lp_set_debug_guard) that is read back.  After
the workspace is regrown and the graph re-captured, the replay must equal
the plain call."""
import numpy as np
import pytest

import scenes
from tests.parity import rel_l2

pytestmark = pytest.mark.gpu


def _capture(rast, prims, cams, bg, img, dL, grads):
    import torch
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rast.forward(prims, cams, bg, images=img)
            rast.backward(dL, grads=grads)
    torch.cuda.current_stream().wait_stream(s)
    return g


@pytest.mark.parametrize("sort_mode", [0, 1, 2])
def test_capacity_latch_in_captured_graph(sort_mode):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import LinPrimError, Primitives, Rasterizer, _native
    w = scenes.workload(1, scale=0.5)            # 5k octahedra, 512x512
    bg = (0.25, 0.5, 0.75)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    dL = torch.as_tensor(scenes.image_gradient(w, seed=5), device="cuda:0")
    P = w.pixels

    ref = Rasterizer(0)
    ref.set_tuning(sort_mode=sort_mode)
    img_ref = ref.forward(prims, w.cameras, bg).clone()
    g_ref = {k: v.clone() for k, v in ref.backward(dL).items()}
    torch.cuda.synchronize()
    st = ref.stats()
    E = st["entries"]
    assert E > 1000

    rast = Rasterizer(0)
    rast.set_debug_guard(True)
    rast.set_tuning(sort_mode=sort_mode)
    rast.reserve(st["records"], E // 2, P, st["tiles"])
    img = torch.full((3 * P,), -1.0, device="cuda:0")
    grads = {k: torch.full_like(v, 7.0) for k, v in g_ref.items()}
    graph = _capture(rast, prims, w.cameras, bg, img, dL, grads)
    graph.replay()
    torch.cuda.synchronize()
    with pytest.raises(LinPrimError) as e:
        rast.sync_status()
    assert e.value.status == _native.LP_ERR_CAPACITY
    guards = rast.check_guards()
    assert guards["checked"] >= 10 and guards["damaged"] == 0, guards
    # an overflowed list yields no tile ranges: every pixel is background
    # and every gradient zero -- nothing stale, nothing past capacity
    expect = torch.tensor(bg, device="cuda:0").repeat_interleave(P)
    assert torch.equal(img, expect)
    for k in grads:
        assert torch.count_nonzero(grads[k]).item() == 0, k
    # the latch was cleared by the read
    rast.sync_status()

    # regrow, re-capture: the replay equals the plain call
    del graph
    rast.reserve(st["records"], E + 1024, P, st["tiles"])
    graph = _capture(rast, prims, w.cameras, bg, img, dL, grads)
    img.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    rast.sync_status()
    assert torch.equal(img, img_ref)
    for k in grads:
        assert rel_l2(grads[k].cpu().numpy(), g_ref[k].cpu().numpy()) <= 1e-5, k
    guards = rast.check_guards()
    assert guards["damaged"] == 0, guards


def test_guard_zones_are_checked():
    """The canary check itself: a fresh guarded context reports its buffers
    intact after a plain forward + backward, and a context without guards
    reports none checked."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import Primitives, Rasterizer
    w = scenes.workload(0)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    plain = Rasterizer(0)
    plain.forward(prims, w.cameras)
    assert plain.check_guards() == {"checked": 0, "damaged": 0, "first": ""}
    r = Rasterizer(0)
    r.set_debug_guard(True)
    r.forward(prims, w.cameras)
    r.backward(torch.ones(3 * w.pixels, device="cuda:0"))
    g = r.check_guards()
    assert g["checked"] >= 10 and g["damaged"] == 0, g


@pytest.mark.parametrize("sort_mode", [0, 1, 2])
def test_sort_wait_times_out_and_recovers(sort_mode):
    """The onesweep sort's look-back waits are bounded: when one block of the first
    pass never publishes its counts (a test hook), the blocks after it give
    up after about a second, latch LP_ERR_TIMEOUT and write nothing past any
    buffer; with the hook off, the next call renders correctly again."""
    import time
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import LinPrimError, Primitives, Rasterizer, _native
    w = scenes.workload(1, scale=0.5)            # 5k octahedra, 512x512: tens of sort blocks
    prims = Primitives.from_scene(w.scene, "cuda:0")
    ref = Rasterizer(0)
    ref.set_tuning(sort_mode=sort_mode)
    img_ref = ref.forward(prims, w.cameras).clone()
    torch.cuda.synchronize()
    assert ref.stats()["entries"] > 3 * 4096

    rast = Rasterizer(0)
    rast.set_debug_guard(True)
    rast.set_tuning(sort_mode=sort_mode, onesweep=1)
    rast.forward(prims, w.cameras)               # sizes the workspace (with guard zones)
    torch.cuda.synchronize()
    _native.check(rast.ctx, rast.lib.lp_debug_sort_stall(rast.ctx, 1), "lp_debug_sort_stall")
    t0 = time.time()
    rast.forward(prims, w.cameras)
    with pytest.raises(LinPrimError) as e:
        rast.sync_status()
    assert e.value.status == _native.LP_ERR_TIMEOUT
    assert time.time() - t0 < 30
    g = rast.check_guards()
    assert g["checked"] > 0 and g["damaged"] == 0, g
    _native.check(rast.ctx, rast.lib.lp_debug_sort_stall(rast.ctx, -1), "lp_debug_sort_stall")
    img = rast.forward(prims, w.cameras)
    rast.sync_status()
    assert torch.equal(img, img_ref)


def test_scan_total_is_64_bit():
    """The tile-count scan (Sec. 3.2: a record's entries start at the
    exclusive prefix sum of the tile counts) keeps its total in 64 bits: a sum
    below 2^32 - 1 comes back exact with exact 32-bit offsets; a sum that
    reaches 2^32 - 1 -- within one block of 4096 counts, or only across
    blocks -- raises LP_ERR_CAPACITY instead of wrapping, and leaves no status
    latched for the next forward."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16312_gb300 import LinPrimError, Primitives, Rasterizer, _native
    r = Rasterizer(0)
    rng = np.random.default_rng(21)

    def exact(c):
        off, tot = r.debug_scan(c)
        ex = np.concatenate([[0], np.cumsum(c.astype(np.uint64))[:-1]]) if c.size else np.zeros(0, np.uint64)
        np.testing.assert_array_equal(off, ex.astype(np.uint32))
        assert tot == int(c.astype(np.uint64).sum()), (tot, int(c.astype(np.uint64).sum()))

    exact(np.zeros(0, np.uint32))
    exact(rng.integers(0, 5000, 10007).astype(np.uint32))            # several blocks, ragged tail
    exact(np.array([0xFFFFFFFE], np.uint32))                          # largest representable list
    exact(np.full(3, (0xFFFFFFFE) // 3, np.uint32))
    overflowing = [
        np.array([0xFFFFFFFF], np.uint32),                            # exactly the sentinel
        np.full(4, 1 << 30, np.uint32),                               # 2^32 in four counts
        np.full(4096, 1 << 20, np.uint32),                            # one block's total is 2^32
        np.concatenate([np.full(4096, 1 << 19, np.uint32),           # each block 2^31, together 2^32
                        np.full(4096, 1 << 19, np.uint32)]),
        np.full(40000, 1 << 28, np.uint32),                           # far past 32 bits
    ]
    for c in overflowing:
        with pytest.raises(LinPrimError) as e:
            r.debug_scan(c)
        assert e.value.status == _native.LP_ERR_CAPACITY
    r.sync_status()                                                   # nothing left latched
    w = scenes.workload(0)
    prims = Primitives.from_scene(w.scene, "cuda:0")
    img = r.forward(prims, w.cameras).clone()
    r.sync_status()
    ref = Rasterizer(0)
    assert torch.equal(img, ref.forward(prims, w.cameras))
