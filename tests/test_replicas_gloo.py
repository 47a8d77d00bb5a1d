"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2) run the
host logic the GPU ranks run -- rank / world from the torchrun environment,
one frame per replica, the barrier, the maximum of the per-rank timings and
the whole-job throughput.  The path shards by replica (every rank holds the
scene and renders its own frame), so no data-path collective is involved.
No GPU.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        dist.barrier()
        # per-rank step and forward times (ms): rank 1 is the slower one in
        # the first, rank 0 in the second
        ms = bench.max_over_ranks([2.0 + r, 1.5 - 0.25 * r], w, "cpu")
        frame = bench.replica_frame(r)
        value = bench.job_value(w, 1920 * 1280 / 1e6, ms[0])
        dist.barrier()
        out.put((r, w, local, ms, frame, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    # every rank sees the slowest rank's times
    for r in res:
        assert r[3] == [3.0, 1.5]
    # distinct frames, whole-job throughput = 2 x one frame per slowest step
    assert res[0][4] != res[1][4]
    assert res[0][5] == pytest.approx(2 * 1920 * 1280 / 1e6 / 3e-3)
    assert res[0][5] == res[1][5]


def test_single_process_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 1, 0)
    assert bench.max_over_ranks([1.25, 2.5], 1, "cpu") == [1.25, 2.5]
    assert bench.job_value(1, 2.4576, 2.0) == pytest.approx(1228.8)


def _dp_rank_main(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2311_18561_gb300 import render as R
    from paper_2311_18561_gb300 import synth

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        scene = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in synth.make_fd_scene(seed=0, n=7).items()}
        flat, grads = R.flat_gradients(scene)
        for j, k in enumerate(R.PARAM_NAMES):  # a rank's gradients: (rank + 1) (j + 1) everywhere
            assert grads[k].shape == scene[k].shape and grads[k].data_ptr() >= flat.data_ptr()
            grads[k].fill_((rank + 1) * (j + 1))
        R.allreduce_gradients(flat)
        out.put((rank, {k: grads[k].clone().numpy() for k in R.PARAM_NAMES}))
    finally:
        dist.destroy_process_group()


def test_data_parallel_gradient_sum():
    """The exchange step of a data-parallel training step: each rank's
    per-Gaussian gradients (views of one flat buffer) are summed over the
    ranks by one all-reduce."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_dp_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2311_18561_gb300 import render as R

    total = sum(r + 1 for r in range(world))  # 1 + 2
    for _, g in res:
        for j, k in enumerate(R.PARAM_NAMES):
            assert (g[k] == total * (j + 1)).all(), k

