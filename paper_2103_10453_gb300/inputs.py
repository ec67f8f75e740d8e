"""Seeded synthetic PLSE instances (inputs only: no step of the method lives here).

Two generators follow the instance constructions the paper describes:

* ``random_insertion(n, r, seed)`` -- the construction of the PLSE benchmark of
  Sec. 4.1: starting from an empty n x n grid, a random empty cell receives a
  random symbol, kept only if the symbol is not yet in the cell's row or column,
  until round(r * n^2) cells are filled.  Such instances need not be completable.
  Reading: after 100 * n^2 consecutive rejections the construction restarts
  with seed + 1 (the paper does not say what happens on a stall).
* ``cyclic_delete(n, keep, seed)`` -- a completable (LSC-style) instance: the
  cyclic square L[i][j] = (i + j) mod n + 1 with random row, column and symbol
  permutations, each cell kept independently with probability ``keep``.  The
  permuted square is a hidden witness that the optimum is n^2.

The named workloads used by the tests and the benchmark are built here so that
the CUDA path and the oracle always receive byte-identical grids.  Random draws
use numpy's PCG64 ``default_rng`` and are independent of the method's Philox
streams.
"""
from __future__ import annotations

import numpy as np


def cyclic_delete(n: int, keep: float, seed: int):
    """Returns (grid int8 [n, n], witness int8 [n, n])."""
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    L = (i[:, None] + i[None, :]) % n + 1
    L = L[rng.permutation(n)][:, rng.permutation(n)]
    sym = np.concatenate([[0], rng.permutation(n) + 1])
    L = sym[L]
    mask = rng.random((n, n)) < keep
    grid = np.where(mask, L, 0).astype(np.int8)
    return grid, L.astype(np.int8)


def random_insertion(n: int, r: float, seed: int) -> np.ndarray:
    target = int(round(r * n * n))
    s = seed
    while True:
        rng = np.random.default_rng(s)
        grid = np.zeros((n, n), dtype=np.int8)
        row_has = np.zeros((n, n + 1), dtype=bool)
        col_has = np.zeros((n, n + 1), dtype=bool)
        empty = list(range(n * n))
        filled, fails = 0, 0
        while filled < target and fails < 100 * n * n:
            q = int(rng.integers(len(empty)))
            cell = empty[q]
            a, b = divmod(cell, n)
            k = int(rng.integers(1, n + 1))
            if row_has[a, k] or col_has[b, k]:
                fails += 1
                continue
            grid[a, b] = k
            row_has[a, k] = col_has[b, k] = True
            empty[q] = empty[-1]
            empty.pop()
            filled += 1
            fails = 0
        if filled == target:
            return grid
        s += 1


# --------------------------------------------------------------------------
# Named workloads (sizes of the paper's benchmark classes, Sec. 4.1-4.2).
# --------------------------------------------------------------------------
def tiny_n10() -> np.ndarray:
    """n = 10 cyclic square, permuted with seed 0, each cell kept with p = 0.4."""
    return cyclic_delete(10, 0.4, 0)[0]


def n50_r05() -> np.ndarray:
    """n = 50 random-insertion instance, 50% prefilled, seed 2000."""
    return random_insertion(50, 0.5, 2000)


N70_RATIOS = (0.3, 0.4, 0.5, 0.6, 0.7)


def n70(r: float) -> np.ndarray:
    """n = 70 instances: r in {0.3, 0.5, 0.7} by random insertion, r in {0.4, 0.6}
    by the cyclic construction (prefilled fraction r), seeds 3000 + k."""
    k = N70_RATIOS.index(r)
    if r in (0.4, 0.6):
        return cyclic_delete(70, r, 3000 + k)[0]
    return random_insertion(70, r, 3000 + k)


def batch_mix(count: int = 64, seed0: int = 4000):
    """Uneven instances for batching: n in {20..70 step 10}, r ~ U[0.3, 0.8],
    generator chosen by a coin; instance k uses seed seed0 + k."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        n = int(rng.choice([20, 30, 40, 50, 60, 70]))
        r = float(rng.uniform(0.3, 0.8))
        if rng.random() < 0.5:
            out.append(cyclic_delete(n, r, seed0 + k)[0])
        else:
            out.append(random_insertion(n, r, seed0 + k))
    return out


def serve_mix(count: int = 200, seed0: int = 5000):
    """Request mix of the serving workload: about a quarter LSC-style requests
    (cyclic-delete, n in [60, 100]), the rest random insertion with n uniform
    over {10..100}; r ~ U[0.3, 0.8]; request k uses seed seed0 + k."""
    out = []
    for k in range(count):
        rng = np.random.default_rng(seed0 + k)
        r = float(rng.uniform(0.3, 0.8))
        if rng.random() < 0.25:
            n = int(rng.integers(60, 101))
            out.append(cyclic_delete(n, r, seed0 + k)[0])
        else:
            n = int(rng.integers(10, 101))
            out.append(random_insertion(n, r, seed0 + k))
    return out


def poisson_arrivals(count: int, rate: float, seed: int = 5000):
    """Arrival times (seconds from 0) of a Poisson process with `rate` per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def serve_pop(grid) -> int:
    """Population of a serving request, fixed by its size alone (never by load):
    2^16 / (empty cells), rounded down to a power of two, within [32, 512]."""
    empty = max(int((np.asarray(grid) == 0).sum()), 1)
    p = 32
    while p * 2 <= 512 and p * 2 * empty <= (1 << 16):
        p *= 2
    return p
