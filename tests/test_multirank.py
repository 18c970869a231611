"""The N > 1 benchmark path on CPU ranks (gloo, world size 2): every rank gets
its own batch of the same size, and the reported time is the slowest rank's."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    variants, inst = bench.batch_instances(12, small=True, rank=rank)
    cells = sum(variants[k].n_cell for k, _, _ in inst)
    slowest = bench.reduce_max(10.0 * (rank + 1), dist)
    taus = [round(t, 12) for _, t, _ in inst]
    out.put((rank, cells, slowest, taus))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_and_max_time():
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
    (r0, c0, m0, t0), (r1, c1, m1, t1) = res
    assert c0 == c1 > 0                 # same work per rank
    assert m0 == m1 == 20.0             # max over ranks
    assert t0 != t1                     # each rank its own instances
    assert bench_reduce_single() == 3.5


def bench_reduce_single():
    import bench
    return bench.reduce_max(3.5, None)
