"""Population control on the GPU (Sec. 3.4 "Adaptive Population Control",
App. "Experimental Setting") against the oracle: the densification
statistics gathered by the forward and backward kernels, the decision and
destination scan (bit-exact), the compaction of parameters and Adam moments,
and the optimiser's densify call end to end."""
import ctypes as C

import numpy as np
import pytest

import oracle
import scenes
from oracle import population as pop
from tests.parity import gpu_forward_backward, mask_borderline, rel_l2

pytestmark = pytest.mark.gpu

AA = float(np.float32(0.1))


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def multiview_small():
    w = scenes.workload(3, scale=0.004)
    rng = np.random.default_rng(3)
    cams = scenes.sphere_cameras(rng, [(200, 120), (97, 61), (64, 48)], 6.0, 60.0)
    return scenes.Workload("tetra4k_3mixed", w.scene, cams)


CASES = {
    "cfg0_tetra64": lambda: scenes.workload(0),
    "cfg1_octa10k": lambda: scenes.workload(1),
    "multiview_tetra": multiview_small,
}
MODES = {"ray": dict(), "filter": dict(aa=AA), "exact": dict(exact=True)}


def _stats_gpu(torch, w, dL, mode, bg):
    from paper_2501_16312_gb300 import Rasterizer
    rast = Rasterizer(0)
    if mode.get("aa"):
        rast.set_filter_2d(mode["aa"])
    if mode.get("exact"):
        rast.set_exact(True)
    n = w.scene.n
    gs = torch.zeros(n, device="cuda:0")
    gc = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    px = torch.zeros(n, dtype=torch.int32, device="cuda:0")
    rast.set_densify_stats(gs, gc, px)
    gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)
    # a second forward alone raises px_max to the same values; a backward adds
    gpu_forward_backward(rast, w.scene, w.cameras, bg, None)
    rast.set_densify_stats()
    gpu_forward_backward(rast, w.scene, w.cameras, bg, dL)   # not gathered
    torch.cuda.synchronize()
    return gs.cpu().numpy().astype(np.float64), gc.cpu().numpy(), px.cpu().numpy()


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("case", sorted(CASES))
def test_densify_stats_vs_oracle(torch, case, mode):
    w = CASES[case]()
    kw = MODES[mode]
    bg = (0.1, 0.2, 0.3)
    _, info = oracle.render(w.scene, w.cameras, bg=bg, info=True, **kw)
    dL = mask_borderline(scenes.image_gradient(w, seed=5), info, w.cameras)
    gs, gc, px = _stats_gpu(torch, w, dL, kw, bg)
    ref_px = pop.screen_pixels(oracle, w.scene, w.cameras, **kw)
    ref_gs, ref_gc = pop.gradient_stats(oracle, w.scene, w.cameras, dL, bg=bg, **kw)
    np.testing.assert_array_equal(px, ref_px)
    np.testing.assert_array_equal(gc, ref_gc)
    assert ref_gs.max() > 0 and gc.max() >= 1
    assert rel_l2(gs, ref_gs) <= 1e-3, rel_l2(gs, ref_gs)
    np.testing.assert_allclose(gs, ref_gs, rtol=2e-3, atol=1e-3 * ref_gs.max())


def test_densify_stats_argument_errors(torch):
    from paper_2501_16312_gb300 import Primitives, Rasterizer, _native
    rast = Rasterizer(0)
    L = _native.load()
    x = torch.zeros(4, device="cuda:0")
    p = C.c_void_p(x.data_ptr())
    assert L.lp_set_densify_stats(rast.ctx, p, None, p, 4) == _native.LP_ERR_INVALID
    assert L.lp_set_densify_stats(rast.ctx, p, p, p, -1) == _native.LP_ERR_INVALID
    assert L.lp_set_densify_stats(rast.ctx, None, None, None, 0) == _native.LP_OK
    # statistics smaller than the population: the forward refuses
    w = scenes.workload(0)
    assert L.lp_set_densify_stats(rast.ctx, p, p, p, 4) == _native.LP_OK
    with pytest.raises(_native.LinPrimError):
        rast.forward(Primitives.from_scene(w.scene, "cuda:0"), w.cameras)
    rast.set_densify_stats()


# ------------------------------------------------------------ decide + scan

def _random_decide_inputs(kind, n, seed, extent=5.0):
    rng = np.random.default_rng(seed)
    D = 3 if kind == 6 else 4
    f = np.float32
    scale = np.exp(rng.uniform(np.log(0.002), np.log(1.2), (n, 1)))      # sizes on both sides of both bounds
    dist = (scale * rng.uniform(0.5, 1.0, (n, D)) * rng.choice([-1, 1], (n, D))).astype(f)
    logit = rng.normal(0.0, 2.0, n).astype(f)
    cnt = rng.integers(0, 6, n).astype(np.uint32)
    gsum = (rng.uniform(0, 3e-4, n) * cnt).astype(f)
    px = rng.integers(0, 30, n).astype(np.uint32)
    # values on the thresholds
    k = n // 10
    p = float(f(0.025))
    logit[:k] = f(np.log(p / (1 - p)))
    gsum[k:2 * k] = (f(1.5e-4) * cnt[k:2 * k].astype(f)).astype(f)
    dist[2 * k:3 * k] = f(f(0.4) * f(extent)) / (f(2.0) if kind == 6 else f(np.sqrt(2.0)))
    dist[3 * k:4 * k] = f(f(0.01) * f(extent)) / (f(2.0) if kind == 6 else f(np.sqrt(2.0)))
    px[4 * k:5 * k] = 20
    return dist, logit, gsum, cnt, px


@pytest.mark.parametrize("n", [0, 1, 4095, 4096, 13_001])
@pytest.mark.parametrize("kind", [6, 4])
def test_decide_and_destinations_bit_exact(torch, kind, n):
    from paper_2501_16312_gb300 import train
    extent = 5.0
    dist, logit, gsum, cnt, px = _random_decide_inputs(kind, n, 31 + n + kind, extent)
    t = lambda a, dt=torch.float32: torch.as_tensor(a, dtype=dt, device="cuda:0")
    action, dest, n_out = train.population_decide(
        kind, t(dist), t(logit), t(gsum), t(cnt.astype(np.int32), torch.int32), t(px.astype(np.int32), torch.int32),
        train.population_rules(extent))
    torch.cuda.synchronize()
    ref = pop.decide(kind, dist, logit, gsum, cnt, px, extent)
    ref_dest, ref_total = pop.destinations(ref)
    np.testing.assert_array_equal(action.cpu().numpy(), ref)
    np.testing.assert_array_equal(dest.cpu().numpy(), ref_dest)
    assert int(n_out.item()) == ref_total
    if n >= 4096:
        assert len(set(ref.tolist())) == 4          # every action occurs


# ------------------------------------------------------------ apply

def _random_population(kind, n, K, seed):
    rng = np.random.default_rng(seed)
    D = 3 if kind == 6 else 4
    f = np.float32
    params = dict(centre=rng.normal(size=(n, 3)).astype(f), quat=rng.normal(size=(n, 4)).astype(f),
                  dist=(rng.uniform(0.01, 0.3, (n, D)) * rng.choice([-1, 1], (n, D))).astype(f),
                  logit=rng.normal(size=n).astype(f), sh=rng.normal(size=(n, K, 3)).astype(f))
    states = [{k: rng.normal(size=v.shape).astype(f) for k, v in params.items()} for _ in range(2)]
    return params, states


@pytest.mark.parametrize("n,K", [(1, 1), (5003, 16), (20_000, 4)])
@pytest.mark.parametrize("kind", [6, 4])
def test_apply_vs_oracle(torch, kind, n, K):
    from paper_2501_16312_gb300 import train
    params, states = _random_population(kind, n, K, 41 + n)
    rng = np.random.default_rng(n)
    act = rng.integers(0, 4, n)
    normals = rng.normal(size=(n, 2, 3)).astype(np.float32)
    dest, total = pop.destinations(act)
    t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")
    sets = [{k: t(v) for k, v in s.items()} for s in [params] + states]
    out = train.population_apply(kind, t(act, torch.uint8), t(dest, torch.int32), t(normals), sets, total)
    torch.cuda.synchronize()
    ref_p, ref_s = pop.apply(kind, params, states, act, normals.astype(np.float64))
    split_rows = np.zeros(total, bool)
    for i in np.nonzero(act == pop.SPLIT)[0]:
        split_rows[dest[i]:dest[i] + 2] = True
    for k in params:
        got = out[0][k].cpu().numpy()
        if k == "centre":
            np.testing.assert_array_equal(got[~split_rows], ref_p[k][~split_rows])
            np.testing.assert_allclose(got[split_rows], ref_p[k][split_rows], atol=2e-6, rtol=0)
        elif k == "dist":
            np.testing.assert_array_equal(got[~split_rows], ref_p[k][~split_rows])
            np.testing.assert_allclose(got[split_rows], ref_p[k][split_rows], rtol=3e-7, atol=0)
        else:
            np.testing.assert_array_equal(got, ref_p[k])
        for s_gpu, s_ref in zip(out[1:], ref_s):
            np.testing.assert_array_equal(s_gpu[k].cpu().numpy(), s_ref[k])


# ------------------------------------------------------------ optimiser

@pytest.mark.parametrize("kind", [6, 4])
def test_trainer_densify_end_to_end(torch, kind):
    """A few optimisation steps with the statistics on, then one densify with
    fixed draws: the new parameters and moments equal the oracle's decision
    and compaction of the arrays read back before the call; the step after
    it runs and the statistics restart."""
    from paper_2501_16312_gb300 import train
    rng = np.random.default_rng(50 + kind)
    n = 3000
    D = 3 if kind == 6 else 4
    centre = rng.normal(0, 0.6, (n, 3))
    quat = scenes.random_quaternions(rng, n)
    dist = rng.uniform(0.01, 0.15, (n, D))
    logit = rng.normal(-1.0, 2.0, n)
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = rng.normal(0, 1, (n, 3))
    cams = scenes.sphere_cameras(rng, [(96, 64), (80, 80)], 4.0, 60.0)
    targets = rng.uniform(0, 1, 3 * sum(c.width * c.height for c in cams))
    tr = train.Trainer(kind, centre, quat, dist, logit, sh, cams, targets)
    tr.enable_densify_stats()
    for _ in range(3):
        tr.step()
    torch.cuda.synchronize()
    before = {k: v.cpu().numpy() for k, v in tr.p.items()}
    mom = [{k: v.cpu().numpy() for k, v in tr._views(b).items()} for b in (tr.m, tr.v)]
    st = {k: v.cpu().numpy() for k, v in tr.stats.items()}
    normals = torch.randn(n, 2, 3, device="cuda:0", generator=torch.Generator("cuda").manual_seed(3))
    counts = tr.densify(normals=normals, rules=train.population_rules(tr.extent, grad_threshold=2e-5))
    ref_act = pop.decide(kind, before["dist"], before["logit"], st["grad_sum"], st["grad_count"].astype(np.uint32),
                         st["px_max"].astype(np.uint32), tr.extent, grad_threshold=2e-5)
    dest, total = pop.destinations(ref_act)
    assert counts["n"] == total == tr.n
    assert [counts[k] for k in ("pruned", "kept", "cloned", "split")] == [int((ref_act == a).sum()) for a in range(4)]
    assert counts["cloned"] + counts["split"] > 0 and counts["pruned"] > 0
    ref_p, ref_s = pop.apply(kind, before, mom, ref_act, normals.cpu().numpy().astype(np.float64))
    for k in before:
        np.testing.assert_allclose(tr.p[k].cpu().numpy(), ref_p[k], atol=2e-6, rtol=3e-7, err_msg=k)
        for b, s in zip((tr.m, tr.v), ref_s):
            np.testing.assert_array_equal(tr._views(b)[k].cpu().numpy(), s[k])
    assert not tr.G.any().item()
    tr.step()
    torch.cuda.synchronize()
    assert int(tr.stats["grad_count"].max().item()) >= 1
    assert np.isfinite(tr.loss_value())

