"""Host-side partition of a mode-sorted COO stream across ranks.

The paper parallelises MTTKRP over nonzeros and resolves the race on output
rows with atomics or per-thread private outputs plus a global reduction
(Sec. 5.3).  Across GPUs the same two choices exist:

  * row-aligned ranges (`row_aligned_ranges`): cut the mode-n sorted stream
    into contiguous ranges of about equal entry counts, each cut moved forward
    to the start of an output row, so every rank owns a disjoint block of
    output rows and no reduction is needed (the rows are gathered if a
    consumer needs all of them);
  * arbitrary ranges (`even_ranges`, or `aligned_ranges` whose cuts are
    multiples of 4 entries, as the library's range calls
    pasta_mttkrp_range / pasta_cp_loss_fwd_bwd_range need) with a sum
    all-reduce of the partial outputs: the paper's privatization at GPU
    scale, and the form the loss gradient uses (data parallelism over
    entries).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def even_ranges(nnz: int, parts: int) -> list[tuple[int, int]]:
    """`parts` contiguous ranges covering [0, nnz) with sizes differing by at most one."""
    if parts < 1:
        raise ValueError("parts must be >= 1")
    bounds = [(nnz * p) // parts for p in range(parts + 1)]
    return [(bounds[p], bounds[p + 1]) for p in range(parts)]


def row_aligned_ranges(sorted_rows: Sequence[int] | np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Split a non-decreasing array of output-row indices into `parts`
    contiguous ranges of about nnz/parts entries, moving each cut forward to the
    first entry of the next row so that no row spans two ranges.  Ranges may be
    empty (e.g. when one row holds most entries)."""
    rows = np.asarray(sorted_rows)
    nnz = int(rows.shape[0])
    if parts < 1:
        raise ValueError("parts must be >= 1")
    if nnz and np.any(rows[1:] < rows[:-1]):
        raise ValueError("rows must be sorted (non-decreasing)")
    cuts = [0]
    for p in range(1, parts):
        c = max((nnz * p) // parts, cuts[-1])
        if 0 < c < nnz:
            # first index >= c whose row differs from the row just before c
            c = int(np.searchsorted(rows, rows[c - 1], side="right"))
        cuts.append(min(max(c, cuts[-1]), nnz))
    cuts.append(nnz)
    return [(cuts[p], cuts[p + 1]) for p in range(parts)]


def aligned_ranges(nnz: int, parts: int, align: int = 4) -> list[tuple[int, int]]:
    """`parts` contiguous ranges covering [0, nnz), every cut a multiple of
    `align` entries, sizes as equal as that allows (the last range takes the
    remainder; ranges may be empty when nnz < parts * align)."""
    if parts < 1 or align < 1:
        raise ValueError("parts and align must be >= 1")
    units = -(-nnz // align)
    cuts = [min(nnz, ((units * p) // parts) * align) for p in range(parts)] + [nnz]
    return [(cuts[p], cuts[p + 1]) for p in range(parts)]


def step_range(nnz: int, world: int, rank: int) -> tuple[int, int]:
    """The range of stored positions rank `rank` of `world` takes in every
    sorted copy for a sharded step (the cuts of `aligned_ranges`)."""
    return aligned_ranges(nnz, world)[rank]


def boundary_rows(first_row: int, last_row: int, device="cpu", group=None):
    """The output rows that ranges can share: the union over ranks of each
    range's first and last rows (first_row / last_row of this rank's range,
    -1 for an empty range), as an int64 tensor on `device`.  Only these rows
    can receive contributions from more than one rank.  Collective (one
    all-gather)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    ends = torch.tensor([first_row, last_row], dtype=torch.int64, device=device)
    if world == 1:
        rows = sorted({r for r in (first_row, last_row) if r >= 0})
    else:
        allends = [torch.empty_like(ends) for _ in range(world)]
        dist.all_gather(allends, ends, group=group)
        rows = sorted({int(r) for t in allends for r in t.tolist() if r >= 0})
    return torch.tensor(rows, dtype=torch.int64, device=device)


def sum_rows(M, rows, group=None) -> None:
    """Sum the rows `rows` of every rank's partial output M in place (one
    all-reduce of those rows only).  Collective."""
    import torch.distributed as dist
    if rows.numel() == 0 or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return
    sub = M.index_select(0, rows).contiguous()
    dist.all_reduce(sub, group=group)
    M.index_copy_(0, rows, sub)


def complete_boundary_rows(M, first_row: int, last_row: int, group=None) -> None:
    """Finish a range-split output in place: M is this rank's partial output
    (its range's contributions; rows it does not reach are 0) and
    first_row / last_row are the output rows of its range's first and last
    entries (-1 for an empty range).  Only rows at range ends can be shared
    by several ranks, so those rows' partials are summed across ranks
    (boundary_rows, then sum_rows).  Afterwards every rank holds the
    complete value of every row its range reaches; together the ranks hold
    the whole output.  Collective: every rank of `group` must call it."""
    sum_rows(M, boundary_rows(first_row, last_row, M.device, group), group)
