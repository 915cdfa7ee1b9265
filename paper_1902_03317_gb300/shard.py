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
