"""Host logic of the autotuner, on the CPU: the coordinate search picks each
group's fastest candidate at the earlier groups' choices, and `tune` caches,
reuses and restores state.  A fake rasterizer stands in for the GPU: its stage
times are a known function of the knobs."""
import json
import types

import pytest

from paper_2501_16312_gb300 import autotune

BASE = dict(tile=16, batch=64, blocks_per_sm=0, sort_mode=0, pixels_per_thread=4, chain_split=0,
            radix_bits=8, tile_order=0, onesweep=0)


def stage_model(k):
    """Stage times (ms) with a unique best setting per group; the blend and
    chain times depend on earlier groups' knobs too, so the order matters.
    The sort group is best at (1, 11); the blend group at tile 16, 4 pixels,
    batch 64 -- though 8x8 tiles would make a faster blend, their longer tile
    lists cost more in the sort stages, which the tile group is judged on."""
    sort = (0.5 if k["sort_mode"] == 1 else 0.9) * {4: 1.3, 6: 1.1, 8: 1.0, 11: 0.9}[k["radix_bits"]]
    sort *= {8: 3.0, 16: 1.0, 32: 0.6}[k["tile"]]
    fwd = {(2, 32): 1.9, (2, 64): 1.7, (4, 32): 1.6, (4, 64): 1.4, (1, 32): 2.0, (1, 64): 1.8,
           (1, 128): 1.85, (2, 128): 1.75, (4, 128): 1.5}[
        (k["pixels_per_thread"], k["batch"])]
    fwd *= {8: 0.9, 16: 1.0, 32: 1.3}[k["tile"]]
    bwd = 3.0 + (0.3 if k["pixels_per_thread"] == 2 else 0.0)
    if k["sort_mode"] == 1:
        fwd += 0.05                      # a slower blend must not change the sort choice
    chain = 0.5 if k["chain_split"] == 1 else 0.6
    return {"preprocess": 0.3, "scan_emit": sort * 0.6, "sort": sort * 0.35, "ranges": sort * 0.05,
            "blend_fwd": fwd, "blend_bwd": bwd, "chain": chain}


class FakeRast:
    def __init__(self):
        import torch
        self.device = torch.device("cpu")
        self.knobs = dict(BASE)
        self.timing_calls = []
        self._timing = False
        self.measured = 0

    def tuning(self):
        return dict(self.knobs)

    def set_tuning(self, **kw):
        assert set(kw) <= set(BASE), kw
        self.knobs.update(kw)

    def timing(self):
        return self._timing

    def set_timing(self, enabled=True):
        self.timing_calls.append(bool(enabled))
        self._timing = bool(enabled)

    def forward(self, prims, cameras, bg, images=None):
        assert self._timing
        return images

    def backward(self, dL, grads=None):
        return grads

    def stage_times(self):
        self.measured += 1
        return stage_model(self.knobs)


def test_search_picks_each_groups_best_in_order():
    knobs = dict(BASE)
    applied = []

    def apply(setting):
        applied.append(dict(setting))
        knobs.update(setting)

    entry = autotune.search(apply, lambda: stage_model(knobs), BASE)
    want = dict(BASE, sort_mode=1, radix_bits=11, tile=16, pixels_per_thread=4, batch=64, blocks_per_sm=0,
                chain_split=1)
    assert entry["tuning"] == want
    assert knobs == want                                # the winners are left applied
    assert len(entry["trials"]) == 24 + 18 + 24 + 2 + 2
    # the sort group is judged on its own stages only, at both visits
    assert entry["best_ms"]["sort_mode+radix_bits+onesweep"] == pytest.approx(0.45)
    assert entry["best_ms"]["sort_mode+radix_bits+onesweep (again)"] == pytest.approx(0.45)
    # the tile group on the sort and blend stages together
    assert entry["best_ms"]["tile+pixels_per_thread+batch+blocks_per_sm"] == pytest.approx(0.45 + 1.45 + 3.0)
    # each trial of a later group ran at the earlier groups' winners
    for t in entry["trials"]:
        if "chain_split" in t:
            assert t["blend_fwd"] == pytest.approx(1.45)
        if t.get("tile") == 16:                            # timed at sort mode 1, 11-bit digits
            assert t["scan_emit"] == pytest.approx(0.45 * 0.6)


def test_sort_knobs_are_settled_again_at_the_chosen_tile():
    """The best digit width depends on the key width, and so on the tile
    edge: here 8-bit digits are best at 16x16 tiles and 11-bit digits at 8x8.
    8x8 tiles win the tile group even with 8-bit digits, and the second visit
    of the sort group then moves to 11 bits."""
    knobs = dict(BASE)

    def model(k):
        t = stage_model(k)
        sort = {16: {4: 1.3, 6: 1.1, 8: 1.0, 11: 1.2}, 8: {4: 1.6, 6: 1.25, 8: 1.25, 11: 1.0},
                32: {4: 2.0, 6: 2.0, 8: 2.0, 11: 2.0}}[k["tile"]][k["radix_bits"]]
        t.update(scan_emit=sort * 0.6, sort=sort * 0.35, ranges=sort * 0.05)
        t["blend_fwd"] = 1.0 if k["tile"] == 8 else 1.5
        return t

    entry = autotune.search(knobs.update, lambda: model(knobs), BASE)
    assert entry["tuning"]["tile"] == 8
    assert entry["tuning"]["radix_bits"] == 11
    first = [t for t in entry["trials"][:16] if t["radix_bits"] == 8 and t["sort_mode"] == 0]
    assert first and all(t["sort"] == pytest.approx(0.35) for t in first)   # timed at 16x16


def test_search_ties_keep_the_first_candidate():
    knobs = dict(BASE)
    flat = {"preprocess": 0.0, "scan_emit": 1.0, "sort": 1.0, "ranges": 1.0, "blend_fwd": 1.0,
            "blend_bwd": 1.0, "chain": 1.0}
    entry = autotune.search(knobs.update, lambda: flat, BASE)
    assert entry["tuning"] == dict(BASE, sort_mode=0, radix_bits=4, tile=8, pixels_per_thread=1, batch=32,
                                   chain_split=0)


def test_cache_key_buckets():
    cam = types.SimpleNamespace(width=1264, height=832)
    k1 = autotune.cache_key("G", 6, 500000, [cam] * 8)
    k2 = autotune.cache_key("G", 6, 520000, [cam] * 8)        # same power-of-two bucket
    k3 = autotune.cache_key("G", 6, 2000000, [cam] * 8)
    k4 = autotune.cache_key("G", 4, 500000, [cam] * 8)
    assert k1 == k2 and k1 != k3 and k1 != k4
    assert autotune.cache_key("G", 6, 500000, [cam] * 7) != k1


def _fake_workload(torch):
    n, K = 10, 16
    prims = types.SimpleNamespace(kind=6, n=n, centre=torch.zeros(n, 3), verts=torch.zeros(n, 6, 3),
                                  opacity=torch.zeros(n), sh=torch.zeros(n, K, 3))
    cams = [types.SimpleNamespace(width=8, height=4), types.SimpleNamespace(width=6, height=2)]
    return prims, cams


@pytest.fixture
def fake_cuda(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    return torch


def test_tune_caches_reuses_and_restores_timing(fake_cuda, tmp_path):
    torch = fake_cuda
    prims, cams = _fake_workload(torch)
    cache = str(tmp_path / "sub" / "tuning.json")
    rast = FakeRast()
    entry = autotune.tune(rast, prims, cams, reps=2, cache=cache)
    want = dict(BASE, sort_mode=1, radix_bits=11, pixels_per_thread=4, batch=64, chain_split=1)
    assert entry["tuning"] == want and rast.knobs == want
    assert rast.measured == 70 * 3                       # 70 trials x (warm-up + 2 timed)
    assert rast.timing_calls == [True, False]            # timing restored to off
    stored = json.load(open(cache))
    key = autotune.cache_key("FakeGPU", 6, 10, cams)
    assert stored[key]["tuning"] == want

    # a fresh context takes the cached choice without timing anything
    rast2 = FakeRast()
    entry2 = autotune.tune(rast2, prims, cams, reps=2, cache=cache)
    assert entry2["tuning"] == want and rast2.knobs == want and rast2.measured == 0
    # force re-times; timing that was on stays on
    rast3 = FakeRast()
    rast3.set_timing(True)
    autotune.tune(rast3, prims, cams, reps=1, cache=cache, force=True)
    assert rast3.measured == 70 * 2 and rast3.timing() is True
    # other workloads share the file
    autotune.tune(FakeRast(), prims, cams[:1], reps=1, cache=cache)
    assert len(json.load(open(cache))) == 2


def test_tune_retimes_a_cached_entry_with_other_knobs(fake_cuda, tmp_path):
    """An entry written by a build with another set of knobs is not applied:
    the search runs again and replaces it."""
    torch = fake_cuda
    prims, cams = _fake_workload(torch)
    cache = tmp_path / "tuning.json"
    key = autotune.cache_key("FakeGPU", 6, 10, cams)
    stale = dict(BASE, sparse_lanes=8)
    cache.write_text(json.dumps({key: {"tuning": stale, "best_ms": {}, "trials": []}}))
    assert autotune.load_cache(str(cache), key)["tuning"] == stale
    assert autotune.load_cache(str(cache), key, knobs=BASE) is None
    rast = FakeRast()
    entry = autotune.tune(rast, prims, cams, reps=1, cache=str(cache))
    assert rast.measured == 70 * 2 and set(entry["tuning"]) == set(BASE)   # warm-up + 1 timed
    assert json.load(open(cache))[key]["tuning"] == entry["tuning"]


def test_tune_tolerates_a_corrupt_cache(fake_cuda, tmp_path):
    torch = fake_cuda
    prims, cams = _fake_workload(torch)
    cache = tmp_path / "tuning.json"
    cache.write_text("{not json")
    entry = autotune.tune(FakeRast(), prims, cams, reps=1, cache=str(cache))
    assert entry["tuning"]["sort_mode"] == 1
    assert autotune.load_cache(str(cache), autotune.cache_key("FakeGPU", 6, 10, cams))["tuning"] == entry["tuning"]
    # no cache at all: nothing written, nothing read
    assert autotune.load_cache(None, "k") is None
    autotune.store_cache(None, "k", {"tuning": {}})
