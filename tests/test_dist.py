"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): replicas
with their own seeds and no data-path collective; the step time is the
maximum over ranks.  No GPU needed."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.5 + rank, dist)
        bench.barrier(dist)
        out.put((rank, t, bench.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_replica_seeds():
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
    assert [r[1] for r in res] == [2.5, 2.5]
    assert res[0][2] != res[1][2]


def test_reference_arm_runs_only_on_rank_zero(capsys):
    """Under torchrun the CPU reference arm works and prints on rank 0 only."""
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=3)
    assert bench.run_reference(args, 2, 1) == 0
    assert capsys.readouterr().out == ""
