"""The bench's multi-rank path on CPU ranks (gloo, world size 2): each rank
integrates its own problem (weak scaling, no collective on the data path);
only the timing is reduced, as the max over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank          # rank 1 is the slowest
    m = bench.max_over_ranks(ms, world)
    dist.barrier()
    q.put((rank, m, bench.whole_job_rate(5 * 20, m, world)))
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_gloo():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [150.0, 150.0]
    assert res[0][2] == pytest.approx(100 * 2 / 0.150)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10, 1000.0, 1) == pytest.approx(10.0)
