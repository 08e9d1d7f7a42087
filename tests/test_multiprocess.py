"""The multi-GPU path of the benchmark is replicas (one independent design
sweep or request stream per rank, no data exchange): the only collective
step is the combination of per-rank figures — the slowest rank's time, the
sum of all ranks' work.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mx = bench._allreduce(dist, [1.0 + rank, 5.0 - rank], "max", "cpu")
    sm = bench._allreduce(dist, [10.0 * (rank + 1)], "sum", "cpu")
    out.put((rank, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_rank_figures_combine_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm in res:
        assert mx == [2.0, 5.0] and sm == [30.0]


def test_single_process_combination_is_identity():
    import bench

    assert bench._allreduce(None, [3, 4.5], "max", "cpu") == [3.0, 4.5]
