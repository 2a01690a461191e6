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


def _shard_worker(rank, world, port, out, nx, ny, leaf):
    """One gloo rank of ShardedApply over a seeded dense stand-in operator
    (the collectives and the cell bookkeeping are under test; on a GPU the
    two callables are the library's hb_apply_shard / hb_apply_shard_adjoint,
    tested in tests/test_gpu_shards.py)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2210_02698_gb300 import binding
    from paper_2210_02698_gb300 import dist as hd
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nv = nx * ny
    perm, _ = binding.host_cluster_tree(nx, ny, leaf)
    bounds = [binding.host_shard_rows(nx, ny, leaf, world, r) for r in range(world)]
    cells = hd.shard_cells(torch.from_numpy(perm), bounds)
    rng = np.random.default_rng(5)
    A = torch.from_numpy(rng.standard_normal((nv, nv)) + 1j * rng.standard_normal((nv, nv)))
    mine = cells[rank]

    def fwd(s_full, u_full, n):           # this rank's rows of u = A s
        u_full[:, mine] = (s_full @ A.T)[:, mine]

    def adj(u_full, s_full, n):           # this rank's share of A^H u
        um = torch.zeros_like(u_full)
        um[:, mine] = u_full[:, mine]
        s_full[:] = um @ A.conj()

    sa = hd.ShardedApply(fwd, adj, cells, nv)
    S = torch.from_numpy(rng.standard_normal((3, nv)) + 1j * rng.standard_normal((3, nv)))
    U = torch.from_numpy(rng.standard_normal((3, nv)) + 1j * rng.standard_normal((3, nv)))
    u_loc = sa.forward(S[:, mine].contiguous())
    s_loc = sa.adjoint(U[:, mine].contiguous())
    e_f = float((u_loc - (S @ A.T)[:, mine]).abs().max())
    e_a = float((s_loc - (U @ A.conj())[:, mine]).abs().max())
    out.put((rank, bounds, e_f, e_a))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_row_shards_gloo(world):
    """Row shards of a 12 x 10 grid (leaf 8): the ranks' cells partition the
    grid into contiguous tree ranges, and the all-gather / all-reduce
    assembly gives every rank its cells of A s and A^H u."""
    import numpy as np
    from paper_2210_02698_gb300 import binding, build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + world + (os.getpid() % 500)
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q, 12, 10, 8)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    bounds = res[0][1]
    assert bounds[0][0] == 0 and bounds[-1][1] == 120
    assert all(bounds[i][1] == bounds[i + 1][0] and bounds[i][0] < bounds[i][1] for i in range(world - 1))
    perm, tb = binding.host_cluster_tree(12, 10, 8)
    k = int(np.log2(world))
    assert [tuple(b) for b in bounds] == [(int(tb[k][r]), int(tb[k][r + 1])) for r in range(world)]
    for _, _, ef, ea in res:
        assert ef < 1e-12 and ea < 1e-12
