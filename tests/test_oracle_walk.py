"""Pins of the oracle's tabu walk (Alg. 3, Sec. 3.3), PartialCol (Sec. 3.7) and
the greedy repair (Sec. 3.7)."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _plse_brute import count_f_c

TABU = 2


def small_instances():
    return [inputs.cyclic_delete(6, 0.3, 1)[0], inputs.random_insertion(7, 0.5, 2),
            inputs.random_insertion(8, 0.7, 3), inputs.cyclic_delete(9, 0.5, 4)[0]]


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("phase", [1, 2])
def test_walk_self_checks_tiny(oracle_mod, k, phase):
    # debug=2: every scanned move's predicted 2dF equals the from-scratch change
    # of F2, and the incremental gamma equals a from-scratch gamma after each move
    I = oracle_mod.Instance(small_instances()[k])
    P = I.init_population(3, 11)
    for i in range(3):
        S, F2, st = I.tabu_walk(P[i], i, 0, phase, 300, 5, debug=2)
        f, c = count_f_c(I.grid, I.vertices(), S)
        phi2 = 1 if phase == 1 else 2 * I.nv
        assert F2 == 2 * f + phi2 * c
        f0, c0 = count_f_c(I.grid, I.vertices(), P[i])
        assert F2 <= 2 * f0 + phi2 * c0
        assert st["pairs"] > 0 and st["moves"] <= st["iterations"] <= 300


def test_walk_self_checks_n30(oracle_mod):
    I = oracle_mod.Instance(inputs.random_insertion(30, 0.6, 9))
    P = I.init_population(2, 3)
    S, F2, st = I.tabu_walk(P[0], 0, 4, 1, 3000, 8, debug=1)
    S2, F22, st2 = I.tabu_walk(S, 0, 4, 2, 2 * I.nv, 8, debug=1)
    f, c = count_f_c(I.grid, I.vertices(), S2)
    assert F22 == 2 * f + 2 * I.nv * c


def _first_move_by_brute_force(oracle_mod, I, S, ind, gen, phase, seed):
    """Best key (2dF, (v - r) mod |V|, j) over N0 u Nc at t = 1, with every F
    recomputed from scratch; r from the pinned Philox stream."""
    cells = I.vertices()
    dom = I.domains()
    phi2 = 1 if phase == 1 else 2 * I.nv
    f0, c0 = count_f_c(I.grid, cells, S)
    F0 = 2 * f0 + phi2 * c0
    u = oracle_mod.philox4x32_10([1, ind, (gen << 8) | (TABU << 4) | phase, 0],
                                 [seed & 0xFFFFFFFF, seed >> 32])
    r = (int(u[1]) * I.nv) >> 32
    n = I.n
    best = None
    for v in range(I.nv):
        i = int(S[v])
        a, b = divmod(int(cells[v]), n)
        conflicting = i != 0 and any(
            S[w] == i for w in range(I.nv) if w != v and
            (cells[w] // n == a or cells[w] % n == b))
        if i != 0 and not conflicting:
            continue
        for j in range(n + 1):
            if not dom[v, j] or j == i:
                continue
            T = S.copy()
            T[v] = j
            f1, c1 = count_f_c(I.grid, cells, T)
            key = ((2 * f1 + phi2 * c1) - F0, (v - r) % I.nv, j)
            if best is None or key < best[0]:
                best = (key, T)
    return F0, best


@pytest.mark.parametrize("k", range(4))
def test_first_move_is_brute_force_best(oracle_mod, k):
    I = oracle_mod.Instance(small_instances()[k])
    P = I.init_population(6, 21)
    checked = 0
    for i in range(6):
        for phase in (1, 2):
            F0, best = _first_move_by_brute_force(oracle_mod, I, P[i], i, 3, phase, 99)
            S1, F1, st = I.tabu_walk(P[i], i, 3, phase, 1, 99)
            assert F1 == min(F0, F0 + best[0][0])
            if best[0][0] < 0:                    # improving: S'* is the moved colouring
                assert np.array_equal(S1, best[1])
                checked += 1
    assert checked >= 6


def test_isolated_vertices_closed_form(oracle_mod):
    # one empty cell per row and column: the reduced graph has no edges, every
    # move colours one vertex (2dF = -2), and the walk stops after exactly |V|
    n = 9
    _, L = inputs.cyclic_delete(n, 1.0, 5)
    perm = np.random.default_rng(3).permutation(n)
    grid = L.copy()
    grid[np.arange(n), perm] = 0
    I = oracle_mod.Instance(grid)
    assert I.nv == n and I.num_edges() == 0
    S0 = np.zeros(n, dtype=np.uint8)
    for phase in (1, 2):
        S, F2, st = I.tabu_walk(S0, 0, 0, phase, 1000, 1)
        assert F2 == 0 and st["iterations"] == n and st["moves"] == n
        filled = grid.copy()
        filled[np.arange(n), perm] = S[np.argsort(I.vertices() // n)]
        assert np.array_equal(filled, L)


def test_zero_iterations_returns_start(oracle_mod):
    I = oracle_mod.Instance(small_instances()[2])
    P = I.init_population(1, 4)
    S, F2, st = I.tabu_walk(P[0], 0, 0, 1, 0, 4)
    assert np.array_equal(S, P[0]) and st["iterations"] == 0
    assert F2 == I.eval(P[0], 1)[0]


def test_repair_legalises_greedily(oracle_mod):
    I = oracle_mod.Instance(inputs.random_insertion(12, 0.3, 6))
    P = I.init_population(5, 2)
    cells = I.vertices()
    for i in range(5):
        S, steps = I.repair(P[i])
        f, c = count_f_c(I.grid, cells, S)
        assert c == 0
        changed = np.nonzero(S != P[i])[0]
        assert len(changed) == steps and np.all(S[changed] == 0)
        # each uncoloured vertex was coloured and conflicting in the input
        g0 = I.gamma(P[i])
        assert all(P[i][v] != 0 and g0[v, P[i][v]] > 0 for v in changed)
        # the first vertex removed is the most conflicting one, lowest index on ties
        conf = np.array([g0[v, P[i][v]] if P[i][v] else -1 for v in range(I.nv)])
        first = int(np.argmax(conf))
        if conf[first] > 0:
            assert S[first] == 0


def test_repair_tie_break_lowest_index(oracle_mod):
    # rows 0-1 empty, row 2 = [1, 2, 3]; S puts equal colours on v0/v1 (row 0)
    # and on v3/v5 (row 1): four vertices with gamma = 1 each
    grid = np.zeros((3, 3), dtype=np.int8)
    grid[2, :] = [1, 2, 3]
    I = oracle_mod.Instance(grid)
    assert I.nv == 6
    S, steps = I.repair(np.array([3, 3, 1, 2, 1, 2], dtype=np.uint8))
    assert steps == 2 and S.tolist() == [0, 3, 1, 0, 1, 2]


@pytest.mark.parametrize("k", range(4))
def test_partialcol_stays_legal(oracle_mod, k):
    I = oracle_mod.Instance(small_instances()[k])
    P = I.init_population(3, 5)
    for i in range(3):
        start, _ = I.repair(P[i])
        S, fbest, st = I.tabu_walk(start, i, 1, 3, 400, 3, debug=1)
        f, c = count_f_c(I.grid, I.vertices(), S)
        assert c == 0 and f == fbest
        assert fbest <= count_f_c(I.grid, I.vertices(), start)[0]
    with pytest.raises(oracle_mod.OracleError):               # illegal start refused
        bad = I.init_population(1, 1)[0]
        if count_f_c(I.grid, I.vertices(), bad)[1] > 0:
            I.tabu_walk(bad, 0, 0, 3, 10, 1)
        else:
            raise oracle_mod.OracleError("start was legal")
