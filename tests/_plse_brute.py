"""Independent brute-force helpers for pinning the oracle (test code only).

Nothing here shares code with the oracle: the evaluators count conflicts over
all cell pairs straight from the problem statement (Sec. 1 and Eq. 1-5), and the
exact PLSE solver is a depth-first search over fillings of the empty cells.
"""
from __future__ import annotations

import numpy as np


def fill_colouring(grid, cells, S):
    """Place colouring S (over reduced vertices ``cells``) into a copy of grid."""
    g = np.array(grid, dtype=np.int64, copy=True)
    n = g.shape[0]
    for v, cell in enumerate(cells):
        g[cell // n, cell % n] = S[v]
    return g


def count_f_c(grid, cells, S):
    """f = uncoloured vertices; c = same-row/column pairs of reduced vertices
    carrying the same nonzero colour (Eq. 1, 3, 4)."""
    n = grid.shape[0]
    f = int(np.sum(np.asarray(S) == 0))
    c = 0
    for a in range(len(cells)):
        ra, ca = divmod(int(cells[a]), n)
        for b in range(a + 1, len(cells)):
            rb, cb = divmod(int(cells[b]), n)
            if (ra == rb or ca == cb) and S[a] != 0 and S[a] == S[b]:
                c += 1
    return f, c


def is_partial_latin(g) -> bool:
    g = np.asarray(g)
    n = g.shape[0]
    for k in range(n):
        for line in (g[k, :], g[:, k]):
            vals = line[line != 0]
            if len(vals) != len(set(vals.tolist())):
                return False
    return bool(np.all((g >= 0) & (g <= n)))


def plse_optimum(grid) -> int:
    """Maximum number of filled cells of any extension of ``grid`` (exact DFS)."""
    g = np.asarray(grid, dtype=np.int64)
    n = g.shape[0]
    rowm = [0] * n
    colm = [0] * n
    for r in range(n):
        for c in range(n):
            k = int(g[r, c])
            if k:
                rowm[r] |= 1 << k
                colm[c] |= 1 << k
    empty = [(r, c) for r in range(n) for c in range(n) if g[r, c] == 0]
    prefilled = n * n - len(empty)
    best = [0]

    def dfs(idx, filled):
        if filled + (len(empty) - idx) <= best[0]:
            return
        if idx == len(empty):
            best[0] = filled
            return
        r, c = empty[idx]
        free = ~(rowm[r] | colm[c])
        for k in range(1, n + 1):
            if free >> k & 1:
                rowm[r] |= 1 << k
                colm[c] |= 1 << k
                dfs(idx + 1, filled + 1)
                rowm[r] &= ~(1 << k)
                colm[c] &= ~(1 << k)
        dfs(idx + 1, filled)

    dfs(0, 0)
    return prefilled + best[0]
