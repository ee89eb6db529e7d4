"""Partition of a cell suspension over ranks (one process per GPU).

Cells do not interact inside the solver (Supplementary Sec. 2.1: each cell
is advanced from its own forces), and the paper distributes them evenly and
statically over the GPUs, independently of the fluid decomposition (Sec.
2.3).  Two partitions are provided:

* ``weak``  : every rank steps its own suspension of the full size (seeds
  offset by rank); per-GPU work is fixed as ranks are added.
* ``strong``: the cells of one suspension are split into contiguous,
  near-equal ranges per group; the union over ranks is the whole.

No collective is needed on the data path; ranks only meet for timing.
"""
from __future__ import annotations

from . import inputs as I


def cell_range(n: int, rank: int, world: int):
    """Contiguous near-equal split of n cells: [lo, hi) of ``rank``."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_groups(workload: str, rank: int, world: int, mode: str = "weak", scale: float = 1.0):
    """Materialised groups this rank steps."""
    groups = I.workload_groups(workload, scale)
    if mode == "weak":
        for g in groups:
            g.seed += 7919 * rank
            I.materialise(g)
        return groups
    if mode != "strong":
        raise ValueError(mode)
    out = []
    for g in groups:
        I.materialise(g)
        lo, hi = cell_range(g.n_cells, rank, world)
        out.append(I.subset(g, range(lo, hi)))
    return out
