"""Multi-process helpers: replicas of the apply, and the apply sharded by
rows of the operator.

Replicas: each rank applies the whole operator to its own batch of
right-hand sides (rhs_shard), with no exchange (weak scaling).

Row shards (Sec. 4.2: each off-diagonal butterfly K(o, s) of the HODBF
writes only the rows of o): rank r of P = 2^k owns node r of level k of the
cluster tree, i.e. its cells.  Forward: one all-gather of every rank's input
cells, then the library computes every task whose rows meet the rank's
(hb_apply_shard) and keeps its own cells.  Adjoint: each rank computes its
share of K^H u from its own cells (hb_apply_shard_adjoint), the shares are
summed across ranks and each rank keeps its cells.  Only the collectives and
the bookkeeping live here; every product runs in the library.
"""
import torch
import torch.distributed as dist


def rhs_shard(nrhs_total: int, rank: int, world: int):
    """Contiguous [begin, end) block of right-hand sides owned by ``rank``."""
    base, rem = divmod(nrhs_total, world)
    begin = rank * base + min(rank, rem)
    return begin, begin + base + (1 if rank < rem else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_cells(perm, bounds):
    """Natural indices of every rank's cells: perm[lo_r:hi_r] for the tree
    ranges [lo_r, hi_r) in ``bounds`` (one (lo, hi) per rank)."""
    return [perm[lo:hi] for lo, hi in bounds]


def _all_gather_rows(x, sizes, group=None):
    """All-gather (nrhs, n_r) complex128 blocks of different widths n_r:
    padded to the widest, gathered as real views, trimmed."""
    width = max(sizes)
    pad = torch.zeros((x.shape[0], width), dtype=x.dtype, device=x.device)
    pad[:, :x.shape[1]] = x
    parts = [torch.empty_like(pad) for _ in sizes]
    dist.all_gather([torch.view_as_real(p) for p in parts], torch.view_as_real(pad), group=group)
    return [p[:, :n] for p, n in zip(parts, sizes)]


class ShardedApply:
    """The apply and its adjoint with the rows of the operator split over the
    ranks of a process group.

    apply_shard(s_full, u_full, nrhs) and apply_shard_adjoint(u_full,
    s_full, nrhs) compute this rank's part (the library's hb_apply_shard /
    hb_apply_shard_adjoint for rank ``rank`` of ``world``; tests may pass
    other callables with the same contract).  ``cells[r]`` are the natural
    indices of rank r's cells (a LongTensor each), ``nv`` the number of
    cells.  Vectors are (nrhs, cells) complex128, one right-hand side per
    row, as the library's column-major N_v x nrhs buffers."""

    def __init__(self, apply_shard, apply_shard_adjoint, cells, nv, group=None):
        self.fwd, self.adj = apply_shard, apply_shard_adjoint
        self.cells = cells
        self.nv = nv
        self.group = group
        self.rank = dist.get_rank(group)
        self.sizes = [int(c.numel()) for c in cells]

    def forward(self, s_local):
        """u on this rank's cells from s on this rank's cells (one all-gather)."""
        nrhs = s_local.shape[0]
        parts = _all_gather_rows(s_local, self.sizes, self.group)
        s_full = torch.zeros((nrhs, self.nv), dtype=s_local.dtype, device=s_local.device)
        for c, p in zip(self.cells, parts):
            s_full[:, c.to(s_full.device)] = p
        u_full = torch.zeros_like(s_full)
        self.fwd(s_full, u_full, nrhs)
        return u_full[:, self.cells[self.rank].to(u_full.device)]

    def adjoint(self, u_local):
        """s = h^2 K^H u on this rank's cells from u on this rank's cells: the
        rank's share on every cell, summed over the ranks (all-reduce)."""
        nrhs = u_local.shape[0]
        mine = self.cells[self.rank].to(u_local.device)
        u_full = torch.zeros((nrhs, self.nv), dtype=u_local.dtype, device=u_local.device)
        u_full[:, mine] = u_local
        s_full = torch.zeros_like(u_full)
        self.adj(u_full, s_full, nrhs)
        dist.all_reduce(torch.view_as_real(s_full), op=dist.ReduceOp.SUM, group=self.group)
        return s_full[:, mine]


def library_sharded_apply(op, world, rank, group=None):
    """ShardedApply over a built binding.Operator: rank ``rank`` of
    ``world`` with the library's shard entry points and partition."""
    perm = torch.from_numpy(op.tree_perm())
    bounds = [op.shard_rows(world, r) for r in range(world)]
    cells = shard_cells(perm, bounds)
    return ShardedApply(lambda s, u, n: op.apply_shard(s, u, n, world, rank),
                        lambda u, s, n: op.apply_shard_adjoint(u, s, n, world, rank), cells, op.Nv, group)
