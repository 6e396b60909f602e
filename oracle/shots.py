"""Mask fracturing shot count, by exhaustive search (test infrastructure only).

Sec. II-C.3: a mask is fractured into rectangles that reproduce it exactly; the shot
count is the number of rectangles. Reading: the minimum number of non-overlapping
axis-aligned pixel rectangles whose union is the mask (a minimum rectangle
partition). The oracle finds it by search: the first pixel of the mask not yet
covered (row-major order) must be the top-left pixel of the rectangle that covers it
in any partition, so the search tries every rectangle of uncovered mask pixels with
that top-left corner and recurses on what is left (memoised on the uncovered set).
Exponential: tiny masks only.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


def min_partition(mask: np.ndarray) -> int:
    """Shot count of a small mask (Sec. II-C.3 reading): the fewest rectangles partitioning it, by memoised search."""
    M = (np.asarray(mask) != 0)
    H, W = M.shape
    full = 0
    for i in range(H):
        for j in range(W):
            if M[i, j]:
                full |= 1 << (i * W + j)

    @lru_cache(maxsize=None)
    def solve(rem: int) -> int:
        if rem == 0:
            return 0
        p = (rem & -rem).bit_length() - 1      # first uncovered pixel, row-major
        i0, j0 = divmod(p, W)
        best = None
        jmax = j0
        while jmax < W and rem >> (i0 * W + jmax) & 1:
            jmax += 1                           # columns j0 .. jmax-1 usable in row i0
        for j1 in range(j0 + 1, jmax + 1):      # rectangle columns [j0, j1)
            cells = 0
            for i1 in range(i0 + 1, H + 1):     # rows [i0, i1)
                row = 0
                ok = True
                for j in range(j0, j1):
                    b = 1 << ((i1 - 1) * W + j)
                    if not rem & b:
                        ok = False
                        break
                    row |= b
                if not ok:
                    break
                cells |= row
                r = 1 + solve(rem & ~cells)
                if best is None or r < best:
                    best = r
        return best

    return solve(full)
