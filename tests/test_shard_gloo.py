"""The row-sharded operator's host logic on CPU: the row partition, the arm
row ranges, and the collective steps of ShardedOperator (rows of A x from
every rank, one rank-order sum for A^T y) run by two spawned gloo ranks.

On CPU the per-rank operator is the oracle restricted to the rank's block of
rows (with the whole table's whitening scale); on a GPU it is the library's
rtt_build_operator_shard (tests/test_gpu_shard.py).  The whole operator's
A x must come out bit for bit (rows are independent, Sec. 3.1), and A^T y
within FP64 rounding of the whole oracle adjoint, with the same bits on both
ranks and on a second run.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _paths():
    for p in (ROOT, os.path.join(ROOT, "oracle")):
        if p not in sys.path:
            sys.path.insert(0, p)


_paths()
from paper_2609_05528_b300 import rtt  # noqa: E402
from paper_2609_05528_b300.shard import arm_row_range  # noqa: E402


def test_shard_rows_partition():
    for R in (1, 7, 1000, 36513):
        for n in (1, 2, 3, 8):
            if n > R:
                continue
            spans = [rtt.shard_rows(R, i, n) for i in range(n)]
            assert spans[0][0] == 0 and spans[-1][1] == R
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(rtt.RttError):
        rtt.shard_rows(10, 2, 2)
    with pytest.raises(rtt.RttError):
        rtt.shard_rows(10, 0, 0)


def test_arm_row_range_brute_force():
    rng = np.random.default_rng(3)
    for _ in range(300):
        counts = rng.integers(0, 9, size=3)
        R = int(counts.sum())
        order = np.repeat(np.arange(3), counts)
        lo = int(rng.integers(0, R + 1))
        hi = int(rng.integers(lo, R + 1))
        for mask in range(1, 8):
            arm = [g for g in range(R) if mask & (1 << order[g])]
            mine = [i for i, g in enumerate(arm) if lo <= g < hi]
            s, e = arm_row_range(counts, lo, hi, mask)
            assert list(range(s, e)) == mine, (counts, lo, hi, mask)


# --------------------------------------------------------------------------
# two gloo ranks

def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _OracleRows:
    """The oracle restricted to rows [begin, end) of a table, whitened with the
    whole table's scale: the CPU stand-in of a row-shard operator."""

    def __init__(self, O, w, tab, begin, end, scl):
        rows = np.arange(begin, end)
        idx = np.concatenate([np.arange(tab.row_ptr[i], tab.row_ptr[i + 1]) for i in rows])
        rp = np.zeros(rows.size + 1, np.int64)
        rp[1:] = np.cumsum(tab.row_ptr[rows + 1] - tab.row_ptr[rows])
        self.O, self.w, self.scl = O, w, scl
        self.tab = O.Table(tab.order[idx], tab.pixel[idx], tab.r[idx], tab.phi[idx],
                           tab.delay[idx], tab.weight[idx], tab.throughput[idx], rp,
                           tab.row_order[rows], tab.row_pixel[rows], tab.sample[idx])
        self.shard_row_begin = begin
        self.total_rows_per_order = [tab.rows_of_order(n) for n in range(3)]

        class _Info:
            n_rows = end - begin
        self.info = _Info()

    def _arm(self, mask):
        return self.tab.select(tuple(n for n in range(3) if mask & (1 << n)))

    def apply_A(self, x, arm_mask=7):
        return torch.from_numpy(self.O.apply_A(self.w, self._arm(arm_mask), x.numpy(), self.scl))

    def apply_AT(self, y, arm_mask=7):
        return torch.from_numpy(self.O.apply_AT(self.w, self._arm(arm_mask), y.numpy(), self.scl))


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    _paths()
    import torch.distributed as dist
    import oracle as O
    from paper_2609_05528_b300 import inputs as I
    from paper_2609_05528_b300 import rtt as R
    from paper_2609_05528_b300.shard import ShardedOperator, gather_rows
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = I.small_kerr(spin=0.5, incl_deg=50.0, nx=24, n_r=8, n_phi=12, n_frames=64,
                         n_hats=24, ss=1)
        tab = O.build_table(w, I.screen_samples(w))
        scl = O.scale(tab)
        lo, hi = R.shard_rows(tab.n_rows, rank, world)
        op = ShardedOperator(_OracleRows(O, w, tab, lo, hi, scl))
        out = {}
        x = torch.from_numpy(I.uniform_batch(w, range(3)))
        for mask in (7, 1, 6):
            sub = tab.select(tuple(n for n in range(3) if mask & (1 << n)))
            y_full = gather_rows(op.apply_A(x, mask))
            out[f"A{mask}"] = bool(np.array_equal(y_full.numpy(), O.apply_A(w, sub, x.numpy(), scl)))
            d = torch.from_numpy(I.noise((sub.n_rows, w.time.n_frames, 3), 40 + mask))
            g = op.apply_AT(op.local_rows(d, mask), mask)
            g2 = op.apply_AT(op.local_rows(d, mask), mask)
            ref = O.apply_AT(w, sub, d.numpy(), scl)
            out[f"AT{mask}"] = float(np.linalg.norm(g.numpy() - ref) / np.linalg.norm(ref))
            out[f"rep{mask}"] = bool(torch.equal(g, g2))
            both = [torch.empty_like(g) for _ in range(world)]
            dist.all_gather(both, g)
            out[f"same{mask}"] = bool(all(torch.equal(both[0], b) for b in both))
            out[f"rows{mask}"] = op.rows(mask)
            out[f"n{mask}"] = sub.n_rows
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_ranks_rows_and_rank_order_sum():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        assert p.exitcode == 0
    res = {}
    while not q.empty():
        rank, out = q.get()
        res[rank] = out
    assert sorted(res) == [0, 1]
    for mask in (7, 1, 6):
        # the ranks' row ranges tile the arm's rows
        (s0, e0), (s1, e1) = res[0][f"rows{mask}"], res[1][f"rows{mask}"]
        assert s0 == 0 and e0 == s1 and e1 == res[0][f"n{mask}"]
        for r in (0, 1):
            assert res[r][f"A{mask}"], (r, mask)
            assert res[r][f"AT{mask}"] <= 1e-13, (r, mask, res[r][f"AT{mask}"])
            assert res[r][f"rep{mask}"] and res[r][f"same{mask}"]
