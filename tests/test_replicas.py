"""Multi-process path of bench.py on CPU: world size 2 over gloo (no GPU).

Each rank solves its own replica; the job time is the slowest rank's, so the
reduction must return the maximum on every rank, and the oracle arm must run
on rank 0 only.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = bench.replica_rank_info()
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, w, r, lr, t))


def test_max_over_ranks_world_two_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    for rank, w, r, lr, t in res:
        assert (w, r, lr) == (2, rank, rank)
        assert t == 15.0  # the slower rank's time on both ranks


def test_single_process_reduction_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5


def test_oracle_arm_prints_on_rank_zero_only(capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload, steps, warmup, gpus = "poisson2d_q1_16", 1, 1, 2

    bench.run_reference(Args, rank=1)
    assert capsys.readouterr().out == ""
    bench.run_reference(Args, rank=0)
    line = capsys.readouterr().out.strip()
    assert '"impl": "reference"' in line and '"n_gpus": 2' in line
