"""World-size-2 gloo checks (CPU) of the multi-replica helpers used by
bench.py: shards partition the right-hand sides, max/sum reductions."""
import os

import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2210_02698_gb300 import dist as hd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, e = hd.rhs_shard(13, rank, world)
    total = hd.sum_over_ranks(e - b)
    mx = hd.max_over_ranks(1.5 + rank)
    out.put((rank, b, e, total, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_rhs_shards_and_reductions_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, b0, e0, t0, m0), (r1, b1, e1, t1, m1) = res
    assert (b0, e0, b1, e1) == (0, 7, 7, 13)
    assert t0 == t1 == 13 and m0 == m1 == 2.5


@pytest.mark.parametrize("n,w", [(16, 1), (16, 4), (5, 8), (128, 3)])
def test_rhs_shard_partition(n, w):
    from paper_2210_02698_gb300 import dist as hd
    spans = [hd.rhs_shard(n, r, w) for r in range(w)]
    assert spans[0][0] == 0 and spans[-1][1] == n
    assert all(spans[i][1] == spans[i + 1][0] for i in range(w - 1))
    assert max(e - b for b, e in spans) - min(e - b for b, e in spans) <= 1
