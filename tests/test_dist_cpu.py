"""The multi-process path on CPU: two gloo ranks.

A camera-sharded step (each rank renders its own cameras, then one sum
all-reduce of the per-primitive gradients) must give every rank the gradient
of all cameras; the replica timing aggregation must report the slowest rank's
time and the units of all ranks.  Per-rank rendering uses the FP64 oracle,
so this runs without a GPU."""
import os
import socket

import numpy as np
import pytest

import scenes


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(r, n, port, out_dir, task):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=r, world_size=n)
    try:
        from paper_2501_16312_gb300 import dist as pdist
        if task == "grad":
            import oracle
            w = _multiview()
            mine = pdist.balanced_shards(w.cameras, n)[r]
            dL = scenes.image_gradient(w).astype(np.float64)
            offs = np.cumsum([0] + [3 * c.width * c.height for c in w.cameras])
            cams = [w.cameras[i] for i in mine]
            g_local = np.concatenate([dL[offs[i]:offs[i + 1]] for i in mine]) if mine else np.zeros(0)
            if cams:
                _, g = oracle.render(w.scene, cams, dL_dimage=g_local)
            else:
                g = {k: np.zeros_like(getattr(w.scene, k), np.float64) for k in ("centre", "verts", "opacity", "sh")}
            gt = {k: torch.as_tensor(np.asarray(v, np.float64)) for k, v in g.items()}
            pdist.allreduce_gradients(gt)
            np.savez(os.path.join(out_dir, f"grad{r}.npz"), **{k: v.numpy() for k, v in gt.items()})
        else:
            t = [3.0, 5.0][r]
            units = [100.0, 300.0][r]
            mx = pdist.max_over_ranks(t)
            tot = pdist.sum_over_ranks(units)
            pdist.barrier()
            np.save(os.path.join(out_dir, f"agg{r}.npy"), np.array([mx, tot]))
    finally:
        dist.destroy_process_group()


def _multiview():
    w = scenes.workload(0)
    rng = np.random.default_rng(21)
    cams = scenes.sphere_cameras(rng, [(48, 40), (64, 32), (40, 40)], 4.0, 60.0)
    return scenes.Workload("tetra64_3views", w.scene, cams)


def _spawn(task, tmp_path, n=2):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(n, _free_port(), str(tmp_path), task), nprocs=n, start_method="spawn",
                       join=True)


def test_balanced_shards_cover_every_camera_once():
    from paper_2501_16312_gb300.dist import balanced_shards
    rng = np.random.default_rng(3)
    sizes = [(1920, 1080)] * 6 + [(1280, 720)] * 6 + [(640, 480)] * 4
    cams = scenes.sphere_cameras(rng, sizes, 6.0, 60.0)
    for n in (1, 2, 3, 4, 8, 20):
        sh = balanced_shards(cams, n)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(len(cams)))
        px = [sum(cams[i].width * cams[i].height for i in s) for s in sh]
        if n <= len(cams):
            assert max(px) - min(px) <= 1920 * 1080      # greedy: within one largest camera


def test_camera_sharded_gradients_sum_to_the_full_gradient(tmp_path):
    import oracle
    _spawn("grad", tmp_path)
    w = _multiview()
    dL = scenes.image_gradient(w).astype(np.float64)
    _, full = oracle.render(w.scene, w.cameras, dL_dimage=dL)
    for r in range(2):
        got = np.load(tmp_path / f"grad{r}.npz")
        for k in full:
            np.testing.assert_allclose(got[k], full[k], rtol=1e-9, atol=1e-12, err_msg=k)


def test_replica_timing_aggregation(tmp_path):
    _spawn("agg", tmp_path)
    for r in range(2):
        mx, tot = np.load(tmp_path / f"agg{r}.npy")
        assert mx == 5.0 and tot == 400.0
