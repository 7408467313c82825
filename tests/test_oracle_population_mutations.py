"""Each plausible mistake planted in a copy of the population-control oracle
must make at least one of its pins fail (the pins are not tautologies)."""
import os
import types

import pytest

import tests.test_oracle_population as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "population.py")

MUTANTS = {
    # Sec. 3.4's size: octahedron longest axis is twice the distance
    "octa_size_not_doubled": ("f32(f32(2.0) * m) if kind == 6", "f32(m) if kind == 6"),
    # tetrahedron size factor sqrt(2)
    "tetra_size_factor": ("f32(f32(math.sqrt(2.0)) * m)", "f32(f32(math.sqrt(3.0)) * m)"),
    # distances by magnitude
    "size_signed": ("np.max(np.abs(np.asarray(d, f32)))", "np.max(np.asarray(d, f32))"),
    # view gradient: the vertices move with the centre
    "no_vertex_term": ("+ np.asarray(g_verts, np.float64).sum(axis=1)", ""),
    # camera rotation applied transposed
    "rotation_transposed": ("gc = g @ M[:3, :3].T", "gc = g @ M[:3, :3]"),
    # NDC scale uses W for x and H for y
    "width_height_swapped": ("gc[:, 0] * camera.width", "gc[:, 0] * camera.height"),
    # gradient counted in every view, visible or not
    "count_invisible": ("cnt += vis", "cnt += 1"),
    # screen size: the larger of the two sides
    "screen_width_only": ("side = np.maximum(r[:, 1] - r[:, 0] + 1, r[:, 3] - r[:, 2] + 1)",
                          "side = r[:, 1] - r[:, 0] + 1"),
    # thresholds are strict
    "prune_size_inclusive": ("s > big", "s >= big"),
    "densify_inclusive": ("if g > thr:", "if g >= thr:"),
    "clone_inclusive": ("CLONE if s < small", "CLONE if s <= small"),
    "pixels_inclusive": ("int(max_pixels[i]) > PRUNE_PIXELS", "int(max_pixels[i]) >= PRUNE_PIXELS"),
    # pruning has priority
    "densify_before_prune": ("        if f32(logit[i]) < logit_min or s > big or int(max_pixels[i]) > PRUNE_PIXELS:\n"
                             "            act[i] = PRUNE\n            continue\n",
                             "        if f32(logit[i]) < logit_min and s > big and int(max_pixels[i]) > PRUNE_PIXELS:\n"
                             "            act[i] = PRUNE\n            continue\n"),
    # clone and split swapped
    "clone_split_swapped": ("CLONE if s < small else SPLIT", "SPLIT if s < small else CLONE"),
    # a clone keeps the optimiser state
    "clone_keeps_state": ("rows = [(None, False), (None, True)]", "rows = [(None, False), (None, False)]"),
    # split: standard deviations = |d|, unrotated, halved for tetrahedra, children shrink
    "split_unrotated": ("off = quat_rotation(row[\"quat\"]) @ (np.abs(d) * normals[i, child])",
                        "off = np.abs(d) * normals[i, child]"),
    "split_signed_std": ("(np.abs(d) * normals[i, child])", "(d * normals[i, child])"),
    "tetra_std_not_halved": ("(np.max(np.abs(d)) / 2.0)", "np.max(np.abs(d))"),
    "split_no_shrink": ("row[\"dist\"] = d / SPLIT_SHRINK", "row[\"dist\"] = d"),
    "prefix_inclusive": ("return dest[:-1], int(dest[-1])", "return dest[1:], int(dest[-1])"),
    "dest_split_one_row": ("per = np.array([0, 1, 2, 2], np.int64)", "per = np.array([0, 1, 2, 1], np.int64)"),
    # view gradient: NDC scale grows with depth, uses the axis's own focal
    # length, and the depth is the camera-space z row
    "ndc_scale_no_depth": ("gx = gc[:, 0] * camera.width * z / (2.0 * float(camera.fx))",
                           "gx = gc[:, 0] * camera.width / (2.0 * float(camera.fx))"),
    "ndc_y_uses_fx": ("gy = gc[:, 1] * camera.height * z / (2.0 * float(camera.fy))",
                      "gy = gc[:, 1] * camera.height * z / (2.0 * float(camera.fx))"),
    "depth_from_x_row": ("z = np.asarray(centre, np.float64) @ M[2, :3] + M[2, 3]",
                         "z = np.asarray(centre, np.float64) @ M[0, :3] + M[0, 3]"),
    # the densification statistic is a mean over visible views
    "grad_sum_not_mean": ("g = f32(f32(grad_sum[i]) / f32(c)) if c > 0 else f32(0.0)", "g = f32(grad_sum[i])"),
    # the opacity threshold is compared as a logit
    "opacity_threshold_not_logit": ("logit_min = f32(math.log(p / (1.0 - p)))", "logit_min = f32(p)"),
    # split children start with fresh optimiser state and their own draws
    "split_keeps_state": ("rows = [(0, True), (1, True)]", "rows = [(0, False), (1, False)]"),
    "split_children_share_draw": ("off = quat_rotation(row[\"quat\"]) @ (np.abs(d) * normals[i, child])",
                                  "off = quat_rotation(row[\"quat\"]) @ (np.abs(d) * normals[i, 0])"),
}


def _mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("population_mutant")
    exec(compile(src.replace(old, new), SRC + " (mutant)", "exec"), mod.__dict__)
    return mod


def _run_pins(mod, stop_at_first=True):
    import oracle
    failed = []
    saved = pins.pop
    pins.pop = mod
    try:
        for name in dir(pins):
            if not name.startswith("test_"):
                continue
            fn = getattr(pins, name)
            marks = getattr(fn, "pytestmark", [])
            params = [m for m in marks if m.name == "parametrize"]
            calls = [{}]
            for m in params:
                calls = [dict(c, **{m.args[0]: v}) for c in calls for v in m.args[1]]
            for kw in calls:
                if "orc" in fn.__code__.co_varnames[:fn.__code__.co_argcount]:
                    kw = dict(kw, orc=oracle)
                try:
                    fn(**kw)
                except AssertionError:
                    failed.append(name)
                    if stop_at_first:
                        return failed
    finally:
        pins.pop = saved
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    failed = _run_pins(_mutant(*MUTANTS[name]))
    assert failed, f"mutant {name} passed every pin"


def test_unmutated_passes():
    mod = _mutant("PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3", "PRUNE, KEEP, CLONE, SPLIT = 0, 1, 2, 3")
    assert _run_pins(mod, stop_at_first=False) == []
