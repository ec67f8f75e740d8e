"""Pins of the whole oracle run (Alg. 2): the worked example, brute-force optima
for orders n <= 5, completable instances and output validity."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _plse_brute import is_partial_latin, plse_optimum
from test_oracle_instance import read_golden


def check_output(I, grid, res):
    g = res["best_grid"]
    assert is_partial_latin(g)
    assert np.all(g[grid != 0] == grid[grid != 0])               # prefilled kept
    assert res["score"] == int((g != 0).sum()) <= I.ub


def test_n3_example_solved(oracle_mod):
    grid, facts = read_golden()
    I = oracle_mod.Instance(grid)
    res = I.solve(8, 5, 50, 1)
    check_output(I, grid, res)
    assert res["score"] == facts["optimum"][0] == plse_optimum(grid)
    assert res["generations"] == 1          # the bound is reached: optimal stop


def tiny_cases():
    cases = []
    for s in range(8):
        n = 4 + s % 2
        if s % 3 == 0:
            cases.append(inputs.cyclic_delete(n, 0.35, 100 + s)[0])
        else:
            cases.append(inputs.random_insertion(n, 0.45 + 0.05 * (s % 4), 100 + s))
    return cases


@pytest.mark.parametrize("k", range(8))
def test_reaches_brute_force_optimum(oracle_mod, k):
    grid = tiny_cases()[k]
    I = oracle_mod.Instance(grid)
    opt = plse_optimum(grid)
    assert opt <= I.ub
    res = I.solve(16, 10, 200, 1 + k)
    check_output(I, grid, res)
    assert res["score"] == opt


@pytest.mark.parametrize("seed", [0, 1])
def test_completable_instances_completed(oracle_mod, seed):
    grid, witness = inputs.cyclic_delete(8, 0.3, seed)
    I = oracle_mod.Instance(grid)
    res = I.solve(16, 10, 400, 1)
    check_output(I, grid, res)
    assert res["score"] == 64


def test_multi_generation_run_is_deterministic(oracle_mod):
    # an instance that does not close in one generation exercises distances,
    # Alg. 4, matching and AUX; the run is a function of (instance, p, seed)
    grid = inputs.random_insertion(11, 0.7, 7)
    I = oracle_mod.Instance(grid)
    a = I.solve(12, 6, 60, 3)
    b = I.solve(12, 6, 60, 3)
    check_output(I, grid, a)
    assert a["score"] == b["score"] and np.array_equal(a["best_grid"], b["best_grid"])
    assert np.array_equal(a["final_pop"], b["final_pop"])
    assert np.all(np.diff(a["trace"]) <= 0)                    # f* never worsens
    assert a["generations"] >= 2


def test_tiny_workload_runs(oracle_mod):
    I = oracle_mod.Instance(inputs.tiny_n10())
    res = I.solve(64, 20, 2000, 1)
    check_output(I, inputs.tiny_n10(), res)
    assert res["score"] == 100                                 # completable (cyclic)


def test_empty_reduced_graph(oracle_mod):
    _, L = inputs.cyclic_delete(5, 1.0, 1)
    I = oracle_mod.Instance(L)
    assert I.nv == 0
    res = I.solve(4, 3, 10, 1)
    assert res["score"] == 25 and res["generations"] == 0
