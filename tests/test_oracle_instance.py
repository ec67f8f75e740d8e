"""Pins of the oracle's instance reduction (Sec. 2.1-2.2, Alg. 1)."""
import os

import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "n3_example.txt")


def read_golden():
    grid, facts = [], {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0].isdigit():
            grid.append([int(x) for x in parts])
        else:
            facts[parts[0]] = [int(x) for x in parts[1:]]
    return np.array(grid, dtype=np.int8), facts


def test_n3_worked_example(oracle_mod):
    grid, facts = read_golden()
    I = oracle_mod.Instance(grid)
    assert I.nv == facts["nv"][0]
    assert I.l == facts["l"][0]
    assert I.ub == facts["ub"][0]          # n^2 - 2 because l = 1 (Sec. 2.2)
    cells = I.vertices()
    # v7 (1-based, row-major) removed, prefilled cells are not vertices
    assert facts["removed_cell"][0] - 1 not in cells
    for c in facts["prefilled_cells"]:
        assert c - 1 not in cells
    dom = I.domains()
    v6 = list(cells).index(6 - 1)
    assert [k for k in range(4) if dom[v6, k]] == facts["v6_domain"]


def test_full_latin_square_graph_edge_count(oracle_mod):
    # Sec. 2.1: the Latin square graph of order n has n^2 vertices and n^2(n-1) edges
    for n in (1, 2, 3, 5, 8):
        I = oracle_mod.Instance(np.zeros((n, n), dtype=np.int8))
        assert I.nv == n * n and I.l == 0 and I.ub == n * n
        assert I.num_edges() == n * n * (n - 1)
        assert I.domains().sum() == n * n * (n + 1)


@pytest.mark.parametrize("seed", range(6))
def test_reduction_invariants(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 12))
    r = float(rng.uniform(0.2, 0.85))
    grid = inputs.random_insertion(n, r, seed)
    I = oracle_mod.Instance(grid)
    # every cell is prefilled, a reduced vertex, or counted in l
    assert I.nv + I.nfixed + I.l == n * n
    cells = I.vertices()
    assert np.all(np.diff(cells) > 0)                   # row-major order
    dom = I.domains()
    for v, cell in enumerate(cells):
        a, b = divmod(int(cell), n)
        used = set(grid[a, :].tolist()) | set(grid[:, b].tolist())
        expect = [1] + [0 if k in used else 1 for k in range(1, n + 1)]
        assert dom[v].tolist() == expect
        assert sum(expect) >= 2                        # D(v) != {0}
    # removed empty cells have every symbol blocked
    removed = [c for c in range(n * n) if grid.flat[c] == 0 and c not in set(cells.tolist())]
    assert len(removed) == I.l
    for cell in removed:
        a, b = divmod(cell, n)
        used = set(grid[a, :].tolist()) | set(grid[:, b].tolist())
        assert all(k in used for k in range(1, n + 1))
    # edges: pairs of reduced vertices sharing a row or a column
    rows = np.bincount(cells // n, minlength=n)
    cols = np.bincount(cells % n, minlength=n)
    assert I.num_edges() == int((rows * (rows - 1) // 2).sum() + (cols * (cols - 1) // 2).sum())
    assert I.ub == (n * n - 2 if I.l == 1 else n * n - I.l)


def test_invalid_grids_rejected(oracle_mod):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Instance(np.array([[1, 1], [0, 0]], dtype=np.int8))   # row repeat
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Instance(np.array([[2, 0], [2, 0]], dtype=np.int8))   # column repeat
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.Instance(np.array([[3, 0], [0, 0]], dtype=np.int8))   # symbol > n


def test_generators(oracle_mod):
    g, witness = inputs.cyclic_delete(9, 0.5, 3)
    assert np.all((g == 0) | (g == witness))
    for k in range(9):
        assert sorted(witness[k, :].tolist()) == list(range(1, 10))
        assert sorted(witness[:, k].tolist()) == list(range(1, 10))
    g2 = inputs.random_insertion(12, 0.6, 5)
    assert int((g2 != 0).sum()) == round(0.6 * 144)
    oracle_mod.Instance(g2)                                # a valid partial Latin square
    assert np.array_equal(inputs.random_insertion(12, 0.6, 5), g2)
