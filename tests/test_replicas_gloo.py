"""The multi-GPU path on the CPU: bench.py runs one replica per rank (independent
spectra, no data-path collective) and reduces only its timing: total work over
the slowest rank's time. Two gloo ranks stand in for two GPUs."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    red = bench.RankReduce(world, "cpu")
    work, secs = 10.0 * (rank + 1), 1.0 + rank        # rank 0: 10 units in 1 s, rank 1: 20 in 2 s
    red.barrier()
    out[rank] = (red.sum(work), red.max(secs), red.rate(work, secs))
    b = bench.replica_workload("single_hn_k50", rank)
    out[10 + rank] = (b.S, int(b.K.sum()), float(b.params[0, 0]))
    red.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_only():
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        tmp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        assert res[r] == (30.0, 2.0, 15.0)
    # every rank fits a batch of the same shape
    assert res[10][:2] == res[11][:2]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    red = bench.RankReduce(1)
    red.barrier()
    assert (red.sum(3.0), red.max(4.0), red.rate(8.0, 2.0)) == (3.0, 4.0, 4.0)
    b0, b1 = bench.replica_workload("mixed_1024", 0), bench.replica_workload("mixed_1024", 1)
    assert b0.S == b1.S and not np.array_equal(b0.K, b1.K)


def _split_rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.split_workload("mixed_1024", rank, world)
    w = float(np.sum(256 * b.K * (b.n_poles + 2.0) ** 2))
    red = bench.RankReduce(world, "cpu")
    out[rank] = (b.S, w, red.sum(w), red.sum(float(b.S)), float(b.omega[0]), int(b.K[0]))
    dist.destroy_process_group()


def test_weight_balanced_split_over_two_gloo_ranks():
    # the strong-scaling mode: one batch split by the work weight P K (N + 2)^2, contiguous,
    # every spectrum on exactly one rank, the ranks' weights within 1 % of each other
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    world, port = 2, _free_port()
    ctx = tmp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        tmp.start_processes(_split_rank_main, args=(world, port, out), nprocs=world, join=True,
                            start_method="spawn")
        res = dict(out)
    full = W.workload("mixed_1024")
    wtot = float(np.sum(256 * full.K * (full.n_poles + 2.0) ** 2))
    assert res[0][0] + res[1][0] == full.S
    assert abs(res[0][2] - wtot) <= 1e-9 * wtot and res[0][3] == full.S
    assert abs(res[0][1] - res[1][1]) <= 0.01 * wtot / 2
    bounds = bench.split_by_weight(full, 2, 256)
    assert res[1][4] == full.omega[full.offsets[bounds[1]]] and res[1][5] == full.K[bounds[1]]
    for world in (1, 3, 8):
        bd = bench.split_by_weight(full, world, 256)
        assert bd[0] == 0 and bd[-1] == full.S and np.all(np.diff(bd) >= 0)
