"""Row-sharded operator over torch.distributed, one process per GPU.

Each row of the stacked operator (Eq. 3) is the response of one (order,
pixel) to the whole source history (Sec. 3.1), so a contiguous block of rows
is an operator of its own.  Rank i of n builds block i of n of the
(order, pixel)-sorted rows (rtt_build_operator_shard; every rank passes the
whole ray table, so the whitening of Eq. 17-18 is the whole table's) and
holds the whole source x:

  * A x: each rank computes its own rows; no exchange.  The ranks' outputs,
    taken in rank order, are the rows of the whole operator in order.
  * A^T y: each rank applies the adjoint of its rows to its rows of y; the
    partial source vectors are summed over the ranks in rank order
    (`ordered_sum`), the one collective of the path.

The rank-order sum gathers every partial and adds them in the order
0, 1, ..., n-1 on every rank, so all ranks hold the same bits and repeated
runs agree; a library all-reduce chooses its own summation order.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def arm_row_range(total_rows_per_order, row_begin: int, row_end: int, arm_mask: int):
    """[start, end) of a row block's rows inside the whole operator's y of an
    arm.  The rows of the arm are the rows of its orders in (order, pixel)
    order, so the arm rows that fall in a contiguous block of the sorted rows
    are a contiguous range of the arm's y."""
    start = end = 0
    b = 0
    for n in range(3):
        c = int(total_rows_per_order[n])
        if arm_mask & (1 << n):
            lo, hi = max(b, row_begin), min(b + c, row_end)
            start += min(max(row_begin - b, 0), c)
            end += max(hi - lo, 0)
        b += c
    return start, start + end


def ordered_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of `t` over the ranks of `group`, added in rank order on every rank."""
    n = dist.get_world_size(group)
    t = t.contiguous()
    if n == 1:
        return t.clone()
    parts = [torch.empty_like(t) for _ in range(n)]
    dist.all_gather(parts, t, group=group)
    acc = parts[0].clone()
    for p in parts[1:]:
        acc += p
    return acc


def gather_rows(y_local: torch.Tensor, group=None) -> torch.Tensor:
    """The whole operator's y of an arm from every rank's rows (rank order)."""
    n = dist.get_world_size(group)
    if n == 1:
        return y_local.clone()
    rows = torch.tensor([y_local.shape[0]], dtype=torch.int64, device=y_local.device)
    counts = [torch.empty_like(rows) for _ in range(n)]
    dist.all_gather(counts, rows, group=group)
    counts = [int(c.item()) for c in counts]
    m = max(counts)
    pad = y_local.new_zeros((m,) + tuple(y_local.shape[1:]))
    pad[: y_local.shape[0]] = y_local
    parts = [torch.empty_like(pad) for _ in range(n)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


class ShardedOperator:
    """A and A^T of the whole operator from this rank's row block.

    `local` is the rank's row-block operator: an object with
    apply_A(x, arm_mask=...) / apply_AT(y, arm_mask=...) and the attributes
    shard_row_begin, total_rows_per_order and info.n_rows (rtt.Operator built
    with shard=(rank, world_size)).
    """

    def __init__(self, local, group=None):
        self.local = local
        self.group = group

    @classmethod
    def build(cls, workload, table, group=None, **kw):
        from . import rtt
        rank, n = dist.get_rank(group), dist.get_world_size(group)
        return cls(rtt.Operator(workload, table, shard=(rank, n), **kw), group)

    def rows(self, arm_mask: int = 7):
        """[start, end) of this rank's rows inside the whole y of the arm."""
        b = self.local.shard_row_begin
        return arm_row_range(self.local.total_rows_per_order, b, b + int(self.local.info.n_rows),
                             arm_mask)

    def local_rows(self, y: torch.Tensor, arm_mask: int = 7) -> torch.Tensor:
        """This rank's rows of a whole-operator y of the arm."""
        s, e = self.rows(arm_mask)
        return y[s:e]

    def apply_A(self, x: torch.Tensor, arm_mask: int = 7) -> torch.Tensor:
        """This rank's rows of A x (no exchange)."""
        return self.local.apply_A(x, arm_mask=arm_mask)

    def apply_AT(self, y_local: torch.Tensor, arm_mask: int = 7) -> torch.Tensor:
        """The whole A^T y from every rank's rows of y: one rank-order sum."""
        return ordered_sum(self.local.apply_AT(y_local, arm_mask=arm_mask), self.group)

    def normal(self, x: torch.Tensor, arm_mask: int = 7) -> torch.Tensor:
        """A^T A x of the whole operator."""
        return self.apply_AT(self.apply_A(x, arm_mask), arm_mask)
