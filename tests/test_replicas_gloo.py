"""The benchmark's multi-GPU path is replicas only (every GPU applies H to
its own copy of the orbitals; no data-path collective).  Its host logic,
the max-over-ranks time and the whole-job throughput, runs here as two
gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                     # the slower replica is rank 1
    m = bench.max_over_ranks(ms, torch.device("cpu"))
    v = bench.replica_throughput(world, 1e9, 4, m)
    out.put((rank, m, v))
    dist.destroy_process_group()


def test_replicas_max_over_ranks_two_gloo_ranks():
    import multiprocessing as mp
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
    for rank, m, v in res:
        assert m == 15.0                       # every rank sees the slowest time
        assert v == pytest.approx(2 * 1e9 * 4 / 15e-3 / 1e9)
