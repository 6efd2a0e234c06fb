"""Sharding of one solve over k GPUs, one process per GPU: the partition, the one exchange
step of each iteration and the shapes of the collectives.

Host logic only: ownership, index sets, counts, and the data movement over
torch.distributed.  The arithmetic of an iteration stays in each rank's kernels.

Design: the one-exchange form of the transpose of Alg. 2 step 5 (Lemma 3.2).  The operand
is replicated instead of being split into the 1.5D blocks of Alg. 4.
- S (Cov), or X and Y^T (Obs), is replicated on every rank.  S is 17 GB at p = 65536,
  which fits a GB300's HBM many times over.
- The block pairs (I, J), I <= J, of the screening pass are split into k contiguous runs
  of near-equal work (a diagonal pair counts half).  A pair's two tiles W[I, J] and
  W[J, I] are formed on one rank, so the transpose never crosses ranks.
- Rows are owned in contiguous, tile-aligned blocks.  Every emitted candidate entry (i, j)
  is routed to owner(i): one all-to-all per iteration, the exchange step.
- The line search's FP64 partials are kept per block of rows (one row tile), for every
  tau of the window.  They are all-gathered and summed in block order on every rank, so
  the decision, and with it every iterate, is bitwise the same for any k.
- The rows of the accepted iterate are all-gathered into the replicated CSR.

No call here needs a GPU.  The functions take a torch.distributed process group (gloo or
NCCL); tests run them as gloo ranks on the CPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class ShardPlan:
    p: int
    k: int
    tile: int
    pairs: np.ndarray        # (npairs, 2) block pairs (I, J), I <= J, in the screening order
    pair_starts: np.ndarray  # (k + 1,) rank r forms pairs[pair_starts[r]:pair_starts[r + 1]]
    row_starts: np.ndarray   # (k + 1,) rank r owns rows row_starts[r] .. row_starts[r + 1] - 1

    @property
    def nblocks(self) -> int:
        return (self.p + self.tile - 1) // self.tile

    def my_pairs(self, rank: int) -> np.ndarray:
        return self.pairs[self.pair_starts[rank]:self.pair_starts[rank + 1]]

    def my_rows(self, rank: int) -> range:
        return range(int(self.row_starts[rank]), int(self.row_starts[rank + 1]))

    def my_blocks(self, rank: int) -> range:
        """Row blocks (tiles) of rank's rows: the units of its line-search partials."""
        return range(int(self.row_starts[rank]) // self.tile,
                     (int(self.row_starts[rank + 1]) + self.tile - 1) // self.tile)

    def owner(self, rows) -> np.ndarray:
        """Owning rank of each row."""
        return np.searchsorted(self.row_starts, np.asarray(rows), side="right") - 1


def block_pairs(p: int, tile: int) -> np.ndarray:
    """The block pairs (I, J), I <= J, row-major."""
    nb = (p + tile - 1) // tile
    I, J = np.triu_indices(nb)
    return np.stack([I, J], axis=1).astype(np.int64)


def make_plan(p: int, k: int, tile: int = 128) -> ShardPlan:
    """Split the block pairs into k runs of near-equal work and the rows into k
    tile-aligned ranges of near-equal length.  A diagonal pair is one tile, so it counts
    half of an off-diagonal pair (two tiles).  Every rank gets at least one row block
    when p allows it."""
    if p < 1 or k < 1 or tile < 1:
        raise ValueError("p, k and tile must be positive")
    pairs = block_pairs(p, tile)
    w = np.where(pairs[:, 0] == pairs[:, 1], 1.0, 2.0)
    cum = np.concatenate([[0.0], np.cumsum(w)])
    targets = cum[-1] * np.arange(k + 1) / k
    pair_starts = np.searchsorted(cum, targets, side="left").astype(np.int64)
    pair_starts[0], pair_starts[-1] = 0, len(pairs)
    pair_starts = np.maximum.accumulate(pair_starts)
    nb = (p + tile - 1) // tile
    bstarts = np.round(nb * np.arange(k + 1) / k).astype(np.int64)
    row_starts = np.minimum(bstarts * tile, p)
    return ShardPlan(p, k, tile, pairs, pair_starts, row_starts)


def route(plan: ShardPlan, rows) -> tuple[np.ndarray, np.ndarray]:
    """For a rank's emitted entries with these rows: a stable permutation that groups them
    by destination rank (owner of the row), and the number sent to each rank."""
    dest = plan.owner(rows)
    order = np.argsort(dest, kind="stable")
    counts = np.bincount(dest, minlength=plan.k).astype(np.int64)
    return order, counts


def exchange(arrays, send_counts, group=None):
    """The exchange step: an all-to-all of variable-size runs.  ``arrays`` are 1-D numpy
    arrays of equal length, already grouped by destination (route); ``send_counts[r]``
    entries go to rank r.  Returns the received arrays, grouped by source rank in rank
    order, and the counts received from each rank."""
    import torch
    import torch.distributed as dist

    k = dist.get_world_size(group)
    sc = torch.as_tensor(np.asarray(send_counts, dtype=np.int64))
    rc = torch.empty(k, dtype=torch.int64)
    dist.all_to_all_single(rc, sc, group=group)
    s_list, r_list = sc.tolist(), rc.tolist()
    out = []
    for a in arrays:
        a = np.ascontiguousarray(a)
        t_in = torch.from_numpy(a.view(np.int64) if a.dtype == np.float64 else a.astype(np.int64))
        t_out = torch.empty(sum(r_list), dtype=torch.int64)
        dist.all_to_all_single(t_out, t_in, r_list, s_list, group=group)
        v = t_out.numpy()
        out.append(v.view(np.float64) if a.dtype == np.float64 else v.astype(a.dtype))
    return out, np.asarray(r_list, dtype=np.int64)


def allgather_blocks(plan: ShardPlan, rank: int, local, group=None) -> np.ndarray:
    """All-gather per-row-block partials: ``local`` has one leading entry per block of
    plan.my_blocks(rank).  Returns the (nblocks, ...) array in block order, identical on
    every rank (its sums do not depend on k)."""
    import torch
    import torch.distributed as dist

    local = np.ascontiguousarray(local, dtype=np.float64)
    per = [len(plan.my_blocks(r)) for r in range(plan.k)]
    mx = max(per)
    pad = np.zeros((mx,) + local.shape[1:], dtype=np.float64)
    pad[:local.shape[0]] = local
    outs = [torch.empty(pad.shape, dtype=torch.float64) for _ in range(plan.k)]
    dist.all_gather(outs, torch.from_numpy(pad), group=group)
    parts = [o.numpy()[:per[r]] for r, o in enumerate(outs)]
    return np.concatenate(parts, axis=0)


def allgather_rows(plan: ShardPlan, rank: int, row_ptr, col, val, group=None):
    """All-gather the CSR rows each rank owns (row_ptr local to its row range) into the
    replicated CSR of all p rows.  Returns (row_ptr int64 (p+1,), col int64, val float64)."""
    import torch
    import torch.distributed as dist

    k = plan.k
    nnz = torch.tensor([len(col)], dtype=torch.int64)
    allnnz = [torch.empty(1, dtype=torch.int64) for _ in range(k)]
    dist.all_gather(allnnz, nnz, group=group)
    counts = [int(t.item()) for t in allnnz]
    mx = max(max(counts), 1)

    def gather(a, dtype):
        buf = np.zeros(mx, dtype=dtype)
        buf[:len(a)] = a
        t = torch.from_numpy(buf.view(np.int64) if dtype == np.float64 else buf.astype(np.int64))
        outs = [torch.empty(mx, dtype=torch.int64) for _ in range(k)]
        dist.all_gather(outs, t, group=group)
        res = []
        for r, o in enumerate(outs):
            v = o.numpy()[:counts[r]]
            res.append(v.view(np.float64) if dtype == np.float64 else v)
        return np.concatenate(res)

    cols = gather(np.asarray(col, dtype=np.int64), np.int64)
    vals = gather(np.asarray(val, dtype=np.float64), np.float64)
    lens = np.diff(np.asarray(row_ptr, dtype=np.int64))
    nrow = len(plan.my_rows(rank))
    lbuf = np.zeros(max(int(np.max(np.diff(plan.row_starts))), 1), dtype=np.int64)
    lbuf[:nrow] = lens
    outs = [torch.empty(len(lbuf), dtype=torch.int64) for _ in range(k)]
    dist.all_gather(outs, torch.from_numpy(lbuf), group=group)
    all_lens = np.concatenate([o.numpy()[:len(plan.my_rows(r))] for r, o in enumerate(outs)])
    rp = np.concatenate([[0], np.cumsum(all_lens)]).astype(np.int64)
    return rp, cols, vals
