#!/usr/bin/env python3
"""Benchmark of the GB300 LinPrim rasterizer: forward + backward Mpixel/s.

One step = the whole hot path over one batch: preprocess, key emission, radix
sort, tile ranges, front-to-back blend, back-to-front blend backward and the
chain to world-space gradients, for every camera of the workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 2|3]
  python bench.py --config 4 ...            (the graph-captured optimisation step)
  python bench.py --impl reference ...      (the FP64 CPU oracle arm)

Default workload: 500,000 capture-like octahedra, SH degree 3, eight
1264x832 cameras (8.4 Mpixel per step), rendered as one batched launch
sequence captured in a CUDA graph.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 1080p-class (batched vs per-view, same GB300, ≤1e-4 img err)"
UNIT = "Mpixel/s"


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=2, choices=[0, 1, 2, 3, 4],
                   help="0-3: render fwd+bwd workloads; 4: the optimisation step "
                        "(parameter layer, render, L1, backward, Adam) on 2M octahedra")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-per-view", action="store_true")
    p.add_argument("--no-other-configs", action="store_true",
                   help="skip the second 1080p-class workload (1M tetrahedra, 16 mixed cameras)")
    p.add_argument("--tuning", default="",
                   help="fixed schedule instead of autotuning, e.g. sort_mode=1,pixels_per_thread=4,batch=32")
    p.add_argument("--scale", type=float, default=1.0,
                   help="primitive-count scale of the workload (profiling runs only)")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--exact", action="store_true",
                   help="spans along the true perspective ray (no ray-space approximation)")
    p.add_argument("--filter-2d", type=float, default=0.0,
                   help="2D anti-aliasing filter size in pixels (the paper uses 0.1)")
    return p.parse_args()


# ------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in self.rows:
            for name, val in zip(self.NAMES, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


# ------------------------------------------------------------------- helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic FP32 work of the blend kernels, in flops (an FMA counts 2), on
# the pair counts of the paper's algorithm (every tile-list entry a pixel
# walks; the kernels skip the ones they prove uncovered, so this is the work
# the method asks for, not the work a schedule happens to do):
#   per iterated (pixel, primitive) pair: F planes x 2 FMA + F min/max +
#   span subtraction + span test                 = 5F + 2
#   forward, per intersected pair: sigma*s, exp, 1 - tau, T*(1-tau),
#   3 colour FMA, T*tau, stop test               = 12
#   backward, per pair iterated up to the pixel's last contributor: 5F + 2;
#   per contributor: tau, T division, 3 colour grads, dL/do (3 FMA), suffix
#   colour (3 FMA + 3 mul), span/sigma grads, (x, y, 1) weights of two faces ~ 40
def blend_flops(F, pairs):
    fwd = (5 * F + 2) * pairs["iterated"] + 12 * pairs["intersected"]
    bwd = (5 * F + 2) * pairs["iterated_to_last"] + 40 * pairs["intersected"]
    return fwd, bwd


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture (-k that kernel, -c 1) of a workload
# at one blend schedule, with the sha1 of the kernel's sources: a figure is
# reported only for the same workload (primitives, cameras) and schedule, and
# is ignored once the sources change (profiles/dram_traffic_blend_bwd_*.md).
MEASURED_TRAFFIC = {
    "blend_bwd": [
        {"primitives": 500000, "cameras": 8, "schedule": {"tile": 16, "pixels_per_thread": 2, "batch": 128},
         "bytes": 520.0e6 + 122.2e6, "sources_sha1": "842f1cd18749163eb0709eafe0deb4847a51d9ba",
         "capture": "ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:^k_blend_bwd$ -s 2 -c 1"},
    ],
    "blend_fwd": [
        {"primitives": 500000, "cameras": 8, "schedule": {"tile": 16, "pixels_per_thread": 2, "batch": 128},
         "bytes": 245.9e6 + 128.8e6, "sources_sha1": "13240ec9bb4abeaf414ff91478da354e58002f15",
         "capture": "ncu --set full -k regex:^k_blend_fwd$ -s 2 -c 1 (dram__bytes_read.sum, dram__bytes_write.sum)"},
    ],
}
KERNEL_SOURCES = {
    "blend_fwd": ("lp_blend_fwd.cuh", "lp_blend.cuh", "lp_device.cuh"),
    "blend_bwd": ("lp_blend_bwd.cuh", "lp_blend.cuh", "lp_device.cuh"),
}


def sources_sha1(kernel):
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2501_16312_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, n=None, n_cams=None, tuning=None):
    """The captured DRAM bytes of one launch of kernel on this workload and
    schedule, or None."""
    if kernel not in KERNEL_SOURCES:
        return None
    sha = sources_sha1(kernel)
    for t in MEASURED_TRAFFIC.get(kernel, ()):
        if t["sources_sha1"] != sha or (n, n_cams) != (t["primitives"], t["cameras"]):
            continue
        if tuning is not None and any(tuning.get(k) != v for k, v in t["schedule"].items()):
            continue
        return t["bytes"]
    return None


def hbm_bytes(kind_v, K, n, n_cams, E, passes, tiles, sort_mode=0, key_bits=0, radix_bits=8):
    """Algorithmic bytes per launch of the HBM-bound stages: each radix pass
    reads and writes every key and value once (histogram reads excluded).
    Sort mode 0 emits 64-bit (tile, depth) keys and sorts them; mode 1 sorts
    the records by depth inside the scan/emit stage, emits 32-bit tile keys in
    that order and sorts those."""
    F = 8 if kind_v == 6 else 4
    R = n_cams * n
    rec = (8 + 3 * F) * 4
    prim_in = (3 + 3 * kind_v + 1 + 3 * K) * 4
    out = {
        "preprocess": n * prim_in + R * (rec + 4 + 16 + 4),
        "ranges": E * 4 * (2 if sort_mode == 0 else 1) + tiles * 8,
        "chain": n * prim_in + R * (F * 3 + 4 + 1) * 4 + n * prim_in,
    }
    if sort_mode == 0:
        out["scan_emit"] = R * (4 + 4 + 4 + 16 + 4) + E * 12
        out["sort"] = passes * E * 24
    else:
        p2 = (key_bits + radix_bits - 1) // radix_bits
        p1 = max(passes - p2, 0)
        out["scan_emit"] = (R * (4 + 4 + 8)            # depth keys
                            + p1 * R * 16             # record sort by depth
                            + R * (4 + 4 + 4)         # gather counts
                            + R * 8                   # scan
                            + R * (4 + 4 + 4 + 16) + E * 8)   # emission
        out["sort"] = p2 * E * 16
    return out


def roofline(rast, stages, kind, sh_degree, n, n_cams, clk, dev):
    """Roofline entry of the dominant render stage, per-stage rates, the
    device pair counters and the context stats of the last forward."""
    import torch
    pairs = rast.count_pairs()
    st = rast.stats()
    F = 8 if kind == 6 else 4
    fl_fwd, fl_bwd = blend_flops(F, pairs)
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = peaks.get("sm_max_mhz") or clk.get("sm_max_mhz") or 2070.0
    alu_peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12   # TFLOP/s
    tun = rast.tuning()
    hb = hbm_bytes(kind, (sh_degree + 1) ** 2, n, n_cams, st["entries"], st["sort_passes"], st["tiles"],
                   tun["sort_mode"], st["key_bits"], tun.get("radix_bits", 8))
    render_stages = {k: v for k, v in stages.items() if k in hb or k in ("blend_fwd", "blend_bwd")}
    dom = max(render_stages, key=render_stages.get)
    if dom in ("blend_fwd", "blend_bwd"):
        work = fl_fwd if dom == "blend_fwd" else fl_bwd
        achieved = work / (stages[dom] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": alu_peak,
                "unit": "TFLOP/s", "frac": achieved / alu_peak,
                # the captured traffic is the ray-space kernel's; the exact mode runs other kernels
                "traffic": None if rast.exact() else measured_traffic(dom, n, n_cams, tun),
                "peak_source": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x "
                               f"{sm_max:.0f} MHz ({peak_src} max clock)"}
    else:
        achieved = hb[dom] / (stages[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": measured_traffic(dom, n, n_cams, tun),
                "peak_source": f"{peak_src} copy bandwidth"}
    stage_report = {}
    for k, ms in stages.items():
        if k in hb:
            stage_report[k] = {"ms": ms, "GB/s": hb[k] / (ms * 1e-3) / 1e9 if ms > 0 else None}
        elif k == "blend_fwd":
            stage_report[k] = {"ms": ms, "TFLOP/s": fl_fwd / (ms * 1e-3) / 1e12 if ms > 0 else None}
        elif k == "blend_bwd":
            stage_report[k] = {"ms": ms, "TFLOP/s": fl_bwd / (ms * 1e-3) / 1e12 if ms > 0 else None}
        else:
            stage_report[k] = {"ms": ms}
    return roof, stage_report, pairs, st


# ---------------------------------------------------------------- CPU oracle
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(workload, target_s, gpu_image=None, seed=11):
    """Time the FP64 oracle (forward + adjoint) on a bounded sample of pixels:
    random pixels of camera 0 (a sample grown until one run takes a third of
    the budget, or all of the camera), then whole further cameras while the
    budget lasts; returns the rate in Mpixel/s."""
    import numpy as np
    import oracle
    rng = np.random.default_rng(seed)

    def run(ci, q):
        cam = workload.cameras[ci]
        px, py = (q % cam.width).astype(np.int32), (q // cam.width).astype(np.int32)
        g = rng.normal(size=(q.shape[0], 3))
        t0 = time.perf_counter()
        rgb, info, _ = oracle.render_pixels(workload.scene, cam, px, py, bg=workload.bg, dL_dC=g)
        return time.perf_counter() - t0, rgb, info

    cam0 = workload.cameras[0]
    n0 = cam0.width * cam0.height
    # random pixels of camera 0, the sample growing 4x while a run stays under
    # a third of the budget (the cost per pixel varies too much between scenes
    # to extrapolate from one small run); the last run is the sample, between
    # a third of the budget and four thirds of it
    npix0 = min(n0, 1024)
    while True:
        q0 = rng.choice(n0, npix0, replace=False)
        dt, rgb, info = run(0, q0)
        if npix0 >= n0 or dt >= target_s / 3:
            break
        npix0 = min(n0, npix0 * 4)
    total_px, total_t, cams_used = npix0, dt, 1
    for ci in range(1, len(workload.cameras)):
        c = workload.cameras[ci]
        # a whole further camera only if, at the rate just measured, it fits
        # in what is left of the budget
        if total_t + dt / npix0 * c.width * c.height > target_s:
            break
        dtc, _, _ = run(ci, np.arange(c.width * c.height))
        total_px += c.width * c.height
        total_t += dtc
        cams_used += 1
    threads = oracle.set_threads(0)
    out = {"value": total_px / total_t / 1e6, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{total_px} pixels: {npix0} random pixels of camera 0 ({cam0.width}x{cam0.height})"
                     + (f" and all pixels of cameras 1..{cams_used - 1}" if cams_used > 1 else "")
                     + ", forward + adjoint, binary64, OpenMP over pixels", "seconds": round(total_t, 2),
           "cpu_model": cpu_model()}
    # one core, on a slice of the sample sized for a quarter of the budget
    oracle.set_threads(1)
    try:
        n1 = max(64, min(npix0, int(npix0 * (target_s / 4) / max(dt * threads, 1e-9))))
        dt1, _, _ = run(0, q0[:n1])
        out["single_core"] = {"value": n1 / dt1 / 1e6, "unit": UNIT, "pixels": n1, "seconds": round(dt1, 2)}
    finally:
        oracle.set_threads(0)
    if gpu_image is not None:
        got = gpu_image[:3 * n0].reshape(3, n0)[:, q0].T
        clean = info[:, 2] == 0
        err = np.abs(got - rgb).max(1)
        out["max_img_err_vs_gpu"] = float(err[clean].max()) if clean.any() else None
        # pixels the oracle flags (a stop within rounding of the threshold, or
        # a ray grazing a silhouette): how many of them differ by more than
        # 1e-4, against the cap the parity tests allow
        out["borderline_pixels"] = int((~clean).sum())
        out["borderline_differ"] = int((err[~clean] > 1e-4).sum())
        out["borderline_differ_cap"] = max(2, int(1e-4 * npix0))
        out["max_img_err_vs_gpu_all"] = float(err.max())
    return out


def reference_arm(args, workload, metric=METRIC):
    """--impl reference: the FP64 oracle on the host cores, each step a
    bounded sample of the workload's pixels (forward + adjoint)."""
    import numpy as np
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cam = workload.cameras[0]
    n_all = cam.width * cam.height
    rng = np.random.default_rng(5)
    per_step_s = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))

    def step(npix):
        q = rng.choice(n_all, npix, replace=False)
        px, py = (q % cam.width).astype(np.int32), (q // cam.width).astype(np.int32)
        g = rng.normal(size=(npix, 3))
        t0 = time.perf_counter()
        oracle.render_pixels(workload.scene, cam, px, py, bg=workload.bg, dL_dC=g)
        return time.perf_counter() - t0

    # grow the per-step sample 4x while one step stays under a quarter of its
    # time (extrapolating from a small run misjudges scenes whose per-pixel
    # cost varies)
    npix = min(n_all, 1024)
    while npix < n_all and step(npix) < per_step_s / 4:
        npix = min(n_all, npix * 4)
    for _ in range(args.warmup):
        step(npix)
    times = [step(npix) for _ in range(args.steps)]
    total = sum(times)
    value = npix * args.steps / total / 1e6
    sample = (f"{npix} random pixels of camera 0 ({cam.width}x{cam.height}) per step, "
              "forward + adjoint, binary64, OpenMP over pixels")
    line = {"impl": "reference", "metric": metric, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(config_dict(args, workload),
                           form="the FP64 oracle on the host cores, a sample of camera 0's pixels per step"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.set_threads(0), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(args, w):
    s = w.scene
    return {"workload": w.name + f" (workload {args.config})",
            "primitives": s.n, "kind": "octahedron" if s.kind == 6 else "tetrahedron",
            "sh_degree": s.sh_degree, "cameras": len(w.cameras),
            "resolutions": sorted({f"{c.width}x{c.height}" for c in w.cameras}),
            "pixels_per_step": w.pixels, "tile": 16,
            "form": "batched: all cameras in one launch sequence, fwd+bwd captured in one CUDA graph",
            "l2": "inputs larger than L2 (primitives, records, tile lists and images > 129 MB)",
            "parallelism": f"replicas x{args.gpus}",
            "spans": "exact perspective ray" if getattr(args, "exact", False) else "ray-space approximation",
            "filter_2d_px": getattr(args, "filter_2d", 0.0)}


# ------------------------------------------------------------------- our arm
def measure_render(args, w, local, dev, world, barrier, max_over_ranks, tuning_arg="", per_view_on=True):
    """Tune, capture and time the batched fwd+bwd of workload w (and its
    per-view form); returns the figures and the objects the end-to-end and
    CPU legs reuse."""
    import numpy as np
    import torch
    import scenes
    from paper_2501_16312_gb300 import Primitives, Rasterizer, autotune

    P = w.pixels
    rast = Rasterizer(local)
    rast.set_exact(args.exact)
    rast.set_filter_2d(args.filter_2d)
    prims = Primitives.from_scene(w.scene, dev)
    dL = torch.as_tensor(scenes.image_gradient(w), device=dev)
    img = torch.empty(3 * P, device=dev)
    grads = dict(centre=torch.empty_like(prims.centre), verts=torch.empty_like(prims.verts),
                 opacity=torch.empty_like(prims.opacity), sh=torch.empty_like(prims.sh))

    # tune the schedule on this workload (untimed), size the workspace with one
    # plain call, then capture fwd+bwd in a graph
    tuned_pv = None
    if tuning_arg:
        fixed = dict(rast.tuning(), **{k: int(v) for k, v in
                                       (kv.split("=") for kv in tuning_arg.split(","))})
        tuned = tuned_pv = fixed
        rast.set_tuning(**fixed)
    else:
        if per_view_on:
            tuned_pv = autotune.tune(rast, prims, w.cameras[:1], w.bg, cache=None)["tuning"]
        tuned = autotune.tune(rast, prims, w.cameras, w.bg, dL, cache=None)["tuning"]
    rast.forward(prims, w.cameras, w.bg, images=img)
    rast.backward(dL, grads=grads)
    torch.cuda.synchronize()
    st = rast.stats()
    E = st["entries"]
    rast.reserve(st["records"], int(E * 1.1) + 4096, P, st["tiles"])
    rast.set_timing(True)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        rast.forward(prims, w.cameras, w.bg, images=img)
        rast.backward(dL, grads=grads)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rast.forward(prims, w.cameras, w.bg, images=img)
        rast.backward(dL, grads=grads)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    rast.sync_status()

    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    stage_sum = {}
    step_ms = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        ev0.record(stream)
        graph.replay()
        ev1.record(stream)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k, v in rast.stage_times().items():
            stage_sum[k] = stage_sum.get(k, 0.0) + v
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    rast.sync_status()
    t_step = max_over_ranks(sum(step_ms) / len(step_ms))
    stages = {k: v / args.steps for k, v in stage_sum.items()}
    value = world * P / (t_step * 1e-3) / 1e6

    # ---- per-view form: one camera per launch sequence, plain (not captured)
    per_view = None
    if per_view_on:
        rast.set_timing(False)
        rast.set_tuning(**tuned_pv)
        pv_img = torch.empty(3 * P, device=dev)
        offs = np.cumsum([0] + [3 * c.width * c.height for c in w.cameras])

        def per_view_step():
            for ci, cam in enumerate(w.cameras):
                rast.forward(prims, [cam], w.bg, images=pv_img[offs[ci]:offs[ci + 1]])
                rast.backward(dL[offs[ci]:offs[ci + 1]], grads=grads, accumulate=ci > 0)

        for _ in range(max(2, args.warmup // 2)):
            per_view_step()
        torch.cuda.synchronize()
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            per_view_step()
        ev1.record(stream)
        ev1.synchronize()
        t_pv = max_over_ranks(ev0.elapsed_time(ev1) / args.steps)
        # per camera: a separate pass with events around each camera's
        # forward + backward (kept out of the aggregate timing above)
        cam_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in w.cameras]
        cam_ms = [0.0] * len(w.cameras)
        reps = max(2, args.steps // 4)
        for _ in range(reps):
            for ci, cam in enumerate(w.cameras):
                cam_ev[ci][0].record(stream)
                rast.forward(prims, [cam], w.bg, images=pv_img[offs[ci]:offs[ci + 1]])
                rast.backward(dL[offs[ci]:offs[ci + 1]], grads=grads, accumulate=ci > 0)
                cam_ev[ci][1].record(stream)
            torch.cuda.synchronize()
            for ci in range(len(w.cameras)):
                cam_ms[ci] += cam_ev[ci][0].elapsed_time(cam_ev[ci][1]) / reps
        per_camera = [{"camera": ci, "resolution": f"{c.width}x{c.height}", "ms": cam_ms[ci],
                       "Mpixel/s": c.width * c.height / (cam_ms[ci] * 1e-3) / 1e6}
                      for ci, c in enumerate(w.cameras)]
        per_view = {"value": world * P / (t_pv * 1e-3) / 1e6, "ms_per_step": t_pv,
                    "form": "one camera per launch sequence, not captured, same kernels",
                    "batched_over_per_view": t_pv / t_step, "tuning": tuned_pv,
                    "per_camera": per_camera,
                    "per_camera_note": "forward + backward of each camera alone (events around its calls); "
                                       "the batched form renders all cameras in one launch sequence, so only "
                                       "its aggregate exists"}
        rast.set_tuning(**tuned)

    # ---- roofline of the dominant kernel: one eager batched step first, so
    # that the context's host-side state (the last forward's sizes, which the
    # pair counter uses) is the batched workload's again after the per-view
    # runs, then the captured step
    rast.forward(prims, w.cameras, w.bg, images=img)
    rast.backward(dL, grads=grads)
    graph.replay()
    torch.cuda.synchronize()
    roof, stage_report, pairs, st = roofline(rast, stages, w.scene.kind, w.scene.sh_degree, w.scene.n,
                                             len(w.cameras), clk, dev)
    return {"value": value, "ms_per_step": t_step, "per_view": per_view, "tuning": tuned, "clocks": clk,
            "roofline": roof, "stages": stage_report, "pairs": pairs, "stats": st,
            "rast": rast, "prims": prims, "dL": dL, "img": img, "grads": grads, "graph": graph}


def ours(args, workload):
    import numpy as np
    import torch
    import torch.distributed as dist
    import scenes
    from paper_2501_16312_gb300 import Rasterizer

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2501_16312_gb300 import dist as pdist
    barrier = pdist.barrier

    def max_over_ranks(x):
        return pdist.max_over_ranks(x, dev)

    w = workload
    P = w.pixels
    m = measure_render(args, w, local, dev, world, barrier, max_over_ranks, args.tuning,
                       per_view_on=not args.no_per_view)
    rast, prims, dL, img, grads = m["rast"], m["prims"], m["dL"], m["img"], m["grads"]
    st = m["stats"]

    # ---- end to end through the public API with host buffers: every step
    # copies the primitives and dL/dimage in from pinned host memory and the
    # images and all gradients out, overlapped with the neighbouring steps'
    # GPU work by HostPipeline (its own context, so that its workspace
    # reservation leaves the graph timed above untouched)
    from paper_2501_16312_gb300.pipeline import HostPipeline
    host_in = {k: getattr(prims, k).cpu().pin_memory() for k in ("centre", "verts", "opacity", "sh")}
    host_in["dL"] = dL.cpu().pin_memory()
    host_out = {"images": torch.empty(3 * P, pin_memory=True),
                **{k: torch.empty(v.shape, pin_memory=True) for k, v in grads.items()}}
    pipe_rast = Rasterizer(local, tuning=rast.tuning())   # same span mode, filter and schedule
    pipe_rast.set_exact(rast.exact())
    pipe_rast.set_filter_2d(rast.filter_2d())
    pipe = HostPipeline(pipe_rast, prims.kind, prims.n, prims.sh_degree, w.cameras, w.bg)
    for _ in range(2):
        pipe.submit(host_in, host_out)
    pipe.synchronize()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pipe.submit(host_in, host_out)
    pipe.synchronize()
    t_e2e = max_over_ranks(1000 * (time.perf_counter() - t0) / args.steps)
    h2d, d2h = pipe.bytes_per_step()
    e2e_err = float(np.abs(host_out["images"].numpy() - img.cpu().numpy()).max())
    e2e = {"value": world * P / (t_e2e * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e,
           "path": "HostPipeline: pinned host -> device (primitives, dL/dimage), forward + backward "
                   "(CUDA graphs of lp_render_forward / lp_render_backward), device -> host (images, "
                   "gradients); copies overlap the neighbouring steps' kernels; host wall clock over all steps",
           "max_abs_diff_vs_device_images": e2e_err}
    del pipe, pipe_rast, host_in, host_out

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, args.cpu_seconds, gpu_image=img.cpu().numpy().astype(np.float64))

    # ---- the other 1080p-class workload (1M tetrahedra, 16 cameras of mixed
    # size) measured the same way, batched and per view, beside the headline
    others = {}
    if args.config == 2 and not args.no_other_configs and args.scale == 1.0:
        for k in ("rast", "prims", "dL", "img", "grads", "graph"):
            m.pop(k)
        del rast, prims, dL, img, grads
        torch.cuda.empty_cache()
        w3 = scenes.workload(3)
        m3 = measure_render(args, w3, local, dev, world, barrier, max_over_ranks, "",
                            per_view_on=not args.no_per_view)
        others["3"] = {"workload": w3.name + " (workload 3)", "value": m3["value"], "unit": UNIT,
                       "ms_per_step": m3["ms_per_step"], "steps": args.steps, "warmup": args.warmup,
                       "pixels_per_step": w3.pixels, "per_view": m3["per_view"], "tuning": m3["tuning"],
                       "clocks": m3["clocks"], "roofline": m3["roofline"], "stages": m3["stages"],
                       "workload_counts": {"records": m3["stats"]["records"],
                                           "tile_list_entries": m3["stats"]["entries"],
                                           "pairs": m3["pairs"], "sort_passes": m3["stats"]["sort_passes"]},
                       "gpu_launches": (m3["stats"]["launches_fwd"] + m3["stats"]["launches_bwd"]) * args.steps}
        del m3

    if rank == 0:
        cfg = config_dict(args, w)
        cfg["tuning"] = m["tuning"]
        cfg["tile"] = m["tuning"]["tile"]
        line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "per_view": m["per_view"], "e2e": e2e,
                "gpu_launches": (st["launches_fwd"] + st["launches_bwd"]) * args.steps,
                "roofline": m["roofline"], "stages": m["stages"], "clocks": m["clocks"],
                "workload_counts": {"records": st["records"], "tile_list_entries": st["entries"],
                                    "pairs": m["pairs"],
                                    "sort_passes": st["sort_passes"]},
                "cpu_baseline": cpu}
        if others:
            line["other_configs"] = others
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- optimisation step
TRAIN_METRIC = ("optimisation-step Mpixel/s (parameter layer, batched render fwd+bwd, L1, "
                "parameter adjoint, fused Adam; graph-captured)")


def hbm_train_bytes(n, D, K, pixels):
    """Algorithmic bytes per launch of the optimisation-step kernels."""
    V = 6 if D == 3 else 4
    n_par = 3 + 4 + D + 1 + 3 * K
    return {
        "params_fwd": n * (3 + 4 + D + 1) * 4 + n * (3 * V + 1) * 4,
        "l1": 3 * pixels * 12,
        "params_bwd": n * (4 + D + 1 + 3 * V + 1 + 3) * 4 + n * (3 + 4 + D + 1) * 4,
        "adam": n * n_par * 28,
    }


def train_arm(args):
    import numpy as np
    import torch
    import scenes
    from paper_2501_16312_gb300 import Primitives, Rasterizer, autotune, train

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_2501_16312_gb300 import dist as pdist
    barrier = pdist.barrier

    def max_over_ranks(x):
        return pdist.max_over_ranks(x, dev)

    w = scenes.optimisation_workload(scale=args.scale)
    P = w.pixels
    rast = Rasterizer(local)
    # targets: the ground-truth parameters rendered by the same path (untimed)
    tp = w.truth
    c = torch.as_tensor(tp.centre, device=dev)
    v, o = train.params_forward(tp.kind, c, torch.as_tensor(tp.quat, device=dev),
                                torch.as_tensor(tp.dist, device=dev), torch.as_tensor(tp.logit, device=dev))
    target = rast.forward(Primitives(tp.kind, c, v, o, torch.as_tensor(tp.sh, device=dev)), w.cameras).clone()
    del c, v, o
    p = w.init
    tr = train.Trainer(p.kind, p.centre, p.quat, p.dist, p.logit, p.sh, w.cameras, target, rasterizer=rast)
    # schedule tuned on the starting point (untimed)
    if args.tuning:
        tuned = dict(rast.tuning(), **{k: int(x) for k, x in (kv.split("=") for kv in args.tuning.split(","))})
        rast.set_tuning(**tuned)
    else:
        tr.step()
        tune_entry = autotune.tune(rast, tr.prims, w.cameras, tr.bg, tr.dimages, cache=None)
        tuned = tune_entry["tuning"]
    rast.set_timing(True)
    tr.capture()
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        tr.graph.replay()
    torch.cuda.synchronize()
    rast.sync_status()

    losses = torch.zeros(args.steps, dtype=torch.float64, device=dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    step_ms, stage_sum = [], {}
    for i in range(args.steps):
        ev0.record(stream)
        tr.graph.replay()
        ev1.record(stream)
        losses[i:i + 1].copy_(tr.loss)
        ev1.synchronize()
        step_ms.append(ev0.elapsed_time(ev1))
        for k, x in rast.stage_times().items():
            stage_sum[k] = stage_sum.get(k, 0.0) + x
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    rast.sync_status()
    t_step = max_over_ranks(sum(step_ms) / len(step_ms))
    stages = {k: x / args.steps for k, x in stage_sum.items()}
    value = world * P / (t_step * 1e-3) / 1e6
    loss_curve = losses.cpu().numpy()

    # the optimisation-step kernels timed alone (eager, same stream, events)
    L = tr.lib
    sp = train._stream(dev)
    ptr = train._ptr
    n, kind = tr.n, tr.kind

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / reps

    scratch = {k: torch.empty_like(x) for k, x in tr.g.items()}
    dv_copy = tr.dverts.clone()
    extra = {
        "params_fwd": timed(lambda: L.lp_params_forward(kind, n, ptr(tr.p["centre"]), ptr(tr.p["quat"]),
                                                        ptr(tr.p["dist"]), ptr(tr.p["logit"]), ptr(tr.verts),
                                                        ptr(tr.opacity), sp)),
        "l1": timed(lambda: L.lp_l1_loss_grad(ptr(tr.images), ptr(tr.targets), 3 * P, ptr(tr.dimages),
                                              ptr(tr.loss), sp)),
        "params_bwd": timed(lambda: L.lp_params_backward(kind, n, ptr(tr.p["quat"]), ptr(tr.p["dist"]),
                                                         ptr(tr.p["logit"]), ptr(dv_copy), ptr(tr.dopacity),
                                                         ptr(scratch["centre"]), ptr(scratch["quat"]),
                                                         ptr(scratch["dist"]), ptr(scratch["logit"]), sp)),
    }
    m2, v2, P2 = torch.zeros_like(tr.m), torch.zeros_like(tr.v), tr.P.clone()
    step2 = torch.zeros(1, dtype=torch.int32, device=dev)
    extra["adam"] = timed(lambda: L.lp_adam_step(ptr(P2), ptr(tr.G), ptr(m2), ptr(v2), tr._groups_arr,
                                                 len(tr.groups), 0.9, 0.999, 1e-15, ptr(step2), sp))
    hb = hbm_train_bytes(n, tr.D, tr.K, P)
    for k, ms in extra.items():
        stages[k] = ms
    tr.graph.replay()
    torch.cuda.synchronize()
    roof, stage_report, pairs, st = roofline(rast, stages, kind, tr.prims.sh_degree, n, len(w.cameras), clk, dev)
    for k in extra:
        stage_report[k] = {"ms": extra[k], "GB/s": hb[k] / (extra[k] * 1e-3) / 1e9, "timed": "alone, eager"}

    # ---- end to end through the public API: each step streams its target
    # images in from pinned host memory and reads the loss back
    h_target = target.cpu().pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64, pin_memory=True)

    def e2e_step():
        tr.targets.copy_(h_target, non_blocking=True)
        tr.replay(1)                      # the captured step (Trainer's public replay)
        h_loss.copy_(tr.loss, non_blocking=True)

    rast.set_timing(False)
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    ev0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(max(ev0.elapsed_time(ev1), 1000 * (time.perf_counter() - t0)) / args.steps)
    e2e = {"value": world * P / (t_e2e * 1e-3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": h_target.numel() * 4,
           "d2h_bytes_per_step": 8, "ms_per_step": t_e2e,
           "path": "pinned host targets -> device, Trainer.replay (the captured step), loss -> host"}

    popm = population_measure(tr, dev, timed)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(param_workload_scene(w, tr.params_numpy()), args.cpu_seconds)
        cpu["sample"] += "; parameters at the end of the timed steps"

    if rank == 0:
        cfg = {"workload": w.name + " (workload 4, optimisation step)", "primitives": n, "kind": "octahedron",
               "sh_degree": tr.prims.sh_degree, "cameras": len(w.cameras),
               "resolutions": sorted({f"{c.width}x{c.height}" for c in w.cameras}), "pixels_per_step": P,
               "tile": tuned["tile"], "form": "params -> render -> L1 -> backward -> params adjoint -> Adam, one CUDA graph",
               "l2": "inputs larger than L2 (2M primitives x 59 parameters x 4 arrays, images > 129 MB)",
               "parallelism": f"replicas x{world}", "tuning": tuned, "learning_rates": tr.lr}
        line = {"metric": TRAIN_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg, "e2e": e2e,
                "gpu_launches": (st["launches_fwd"] + st["launches_bwd"] + 5) * args.steps,
                "roofline": roof, "stages": stage_report, "clocks": clk,
                "loss": {"first_timed": float(loss_curve[0]), "last_timed": float(loss_curve[-1]),
                         "steps_before_timing": args.warmup + 2},
                "workload_counts": {"records": st["records"], "tile_list_entries": st["entries"],
                                    "pairs": pairs, "sort_passes": st["sort_passes"]},
                "population": popm,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def hbm_population_bytes(n, n_pruned, n_new, n_split, D, K):
    """Algorithmic bytes of one population adjustment: decide (distances,
    logit, three statistics in; action and count out), the scan (counts read
    twice, destinations written) and the compaction of three array sets
    (parameters and both Adam moments): action and destination of every
    primitive, the rows of the surviving ones read, normals of the split
    ones, the new rows written."""
    n_par = 3 + 4 + D + 1 + 3 * K
    decide = n * (4 * D + 4 + 12 + 1 + 4) + n * 12
    apply = n * 5 + (n - n_pruned) * 3 * n_par * 4 + n_split * 24 + n_new * 3 * n_par * 4
    return decide, apply


def population_measure(tr, dev, timed):
    """Population control at the workload's size (App. "Experimental
    Setting": every 250 steps), each kernel timed alone with events (10
    repetitions on unchanged inputs).  Two states: the workload's own
    statistics, gathered over one optimisation step, and seeded synthetic
    statistics that send about 10% of the primitives to densification and
    5% to pruning (a mid-training mix that exercises every branch)."""
    import ctypes as C
    import torch
    from paper_2501_16312_gb300 import _native, train
    tr.enable_densify_stats()
    tr.step()
    torch.cuda.synchronize()
    L, sp, ptr = tr.lib, train._stream(dev), train._ptr
    n, kind = tr.n, tr.kind
    K = int(tr.p["sh"].shape[1])
    rules = train.population_rules(tr.extent)
    action = torch.empty(n, dtype=torch.uint8, device=dev)
    dest = torch.empty(n, dtype=torch.int32, device=dev)
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    scratch = torch.empty(int(L.lp_population_scratch(n)), dtype=torch.int32, device=dev)
    normals = torch.randn(n, 2, 3, device=dev, generator=torch.Generator(dev).manual_seed(0))
    sets = [tr.p, tr._views(tr.m), tr._views(tr.v)]
    src = (_native.lp_param_arrays * 3)(*(train._arrays(x) for x in sets))
    peak = measured_peaks()[0].get("hbm_gbs")

    def one(st):
        def decide():
            return L.lp_population_decide(kind, n, ptr(tr.p["dist"]), ptr(tr.p["logit"]), ptr(st["grad_sum"]),
                                          ptr(st["grad_count"]), ptr(st["px_max"]), C.byref(rules), ptr(action),
                                          ptr(dest), ptr(n_out), ptr(scratch), sp)
        t_decide = timed(decide)
        n_new = int(n_out.item())
        counts = torch.bincount(action.long(), minlength=4).tolist()
        outs = [{k: torch.empty((n_new,) + tuple(x.shape[1:]), device=dev) for k, x in s_.items()} for s_ in sets]
        dst = (_native.lp_param_arrays * 3)(*(train._arrays(x) for x in outs))
        t_apply = timed(lambda: L.lp_population_apply(kind, K, n, ptr(action), ptr(dest), ptr(normals), src, dst,
                                                      3, sp))
        b_dec, b_app = hbm_population_bytes(n, counts[0], n_new, counts[3], tr.D, K)
        del outs
        gbs = b_app / (t_apply * 1e-3) / 1e9
        return {"ms": t_decide + t_apply, "primitives_out": n_new,
                "actions": dict(zip(("pruned", "kept", "cloned", "split"), counts)),
                "decide_scan": {"ms": t_decide, "GB/s": b_dec / (t_decide * 1e-3) / 1e9},
                "apply": {"ms": t_apply, "GB/s": gbs, "frac_hbm": gbs / peak if peak else None, "bytes": b_app}}

    own = one(tr.stats)
    g = torch.Generator(dev).manual_seed(1)
    thr = float(rules.grad_threshold)
    cnt = torch.full((n,), 4, dtype=torch.int32, device=dev)
    # mean gradients uniform in [0.9, 1.01) x threshold: about 10% above it
    synth = {"grad_count": cnt,
             "grad_sum": 4 * thr * (0.9 + 0.11 * torch.rand(n, device=dev, generator=g)),
             "px_max": (torch.rand(n, device=dev, generator=g) < 0.05).to(torch.int32) * 21}
    mixed = one(synth)
    return {"primitives_in": n, "timed": "alone, eager, events, 10 repetitions",
            "amortised_ms_per_step": own["ms"] / 250.0,
            "workload_state": dict(own, statistics="one optimisation step (4 views) with gathering on"),
            "mixed_state": dict(mixed, statistics="seeded: about 10% above the gradient threshold, 5% over 20 px")}


def param_workload_scene(w, params):
    """The optimisation workload as a renderable scene for the oracle: the
    oracle's own parameter layer applied to the given parameters."""
    import numpy as np
    import oracle
    import scenes
    v, o = oracle.params_forward(w.init.kind, params["centre"], params["quat"], params["dist"], params["logit"])
    sc = scenes.Scene(w.init.kind, params["centre"].astype(np.float32), v.astype(np.float32),
                      o.astype(np.float32), params["sh"].astype(np.float32), w.init.sh_degree)
    return scenes.Workload(w.name, sc, w.cameras)


def main():
    args = parse_args()
    import scenes
    if args.config == 4:
        if args.impl == "reference":
            w = scenes.optimisation_workload(scale=args.scale)
            reference_arm(args, param_workload_scene(w, {k: getattr(w.init, k) for k in
                                                         ("centre", "quat", "dist", "logit", "sh")}),
                          metric=TRAIN_METRIC)
        else:
            train_arm(args)
        return
    w = scenes.workload(args.config, scale=args.scale)
    if args.impl == "reference":
        reference_arm(args, w)
    else:
        ours(args, w)


if __name__ == "__main__":
    main()
