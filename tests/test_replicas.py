"""The N-replica bench path on CPU: two gloo ranks agree on the slowest
rank's time (max over ranks), which is what a replicated run reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = 10.0 + 7.5 * rank
    got = bench.max_over_ranks(mine, world, "cpu")
    single = bench.max_over_ranks(mine, 1, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, single))


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [17.5, 17.5]
    assert [o[2] for o in out] == [10.0, 17.5]
