"""Whole-run parity (Alg. 2) of plse_solve against the oracle: best grid, score,
generations executed and the summed work counters of every tabu walk, which
pin the whole trajectory of every walk of every generation."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _plse_brute import is_partial_latin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


def compare(plse, oracle_mod, grid, pop, gens, iters, seed, gpu_params=None, oracle_params=None):
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    if gpu_params is not None:
        G.set_params(gpu_params)
    res = G.solve(pop, gens, iters, seed, with_stats=True)
    ref = I.solve(pop, gens, iters, seed, params=oracle_params)
    assert res["score"] == ref["score"]
    assert np.array_equal(res["best_grid"], ref["best_grid"])
    assert res["generations"] == ref["generations"]
    assert res["walks"] == ref["stats"]
    g = res["best_grid"]
    assert is_partial_latin(g) and np.all(g[grid != 0] == grid[grid != 0])
    assert res["score"] == int((g != 0).sum()) <= I.ub
    return res, ref


def test_tiny_workload_n10_p64(plse, oracle_mod):
    # n = 10 cyclic instance (seed 0, keep 0.4), p = 64, 2000 iterations, 20 generations, seed 1
    res, ref = compare(plse, oracle_mod, inputs.tiny_n10(), 64, 20, 2000, 1)
    assert res["score"] == 100


@pytest.mark.parametrize("k", range(4))
def test_multi_generation_runs(plse, oracle_mod, k):
    # over-constrained instances that keep Alg. 4, matching and AUX busy
    grids = [inputs.random_insertion(11, 0.7, 7), inputs.random_insertion(16, 0.75, 8),
             inputs.random_insertion(20, 0.65, 9), inputs.random_insertion(14, 0.8, 10)]
    res, ref = compare(plse, oracle_mod, grids[k], 24 + 8 * k, 8, 150, 3 + k)
    assert ref["generations"] >= 2


def test_population_of_two_and_odd_sizes(plse, oracle_mod):
    compare(plse, oracle_mod, inputs.random_insertion(9, 0.7, 2), 2, 5, 60, 4)
    compare(plse, oracle_mod, inputs.random_insertion(13, 0.7, 2), 131, 3, 80, 5)


def test_partial_mpma_variant(plse, oracle_mod):
    grid = inputs.random_insertion(18, 0.8, 4)
    compare(plse, oracle_mod, grid, 32, 6, 200, 6,
            gpu_params=plse.default_params(mode=plse.MODE_PARTIALCOL),
            oracle_params=oracle_mod.default_params(mode=1))


@pytest.mark.parametrize("r, oracle_mode", [(0.8, 1), (0.85, 1), (0.79, 0), (0.5, 0)])
def test_auto_mode_follows_the_fill_ratio(plse, oracle_mod, r, oracle_mode):
    # Sec. 3.7: Partial-MPMA on instances with at least 80% of the cells prefilled
    grid = inputs.random_insertion(20, r, 21)
    assert (5 * int((grid != 0).sum()) >= 4 * 400) == (oracle_mode == 1)
    compare(plse, oracle_mod, grid, 24, 4, 150, 8,
            gpu_params=plse.default_params(mode=plse.MODE_AUTO),
            oracle_params=oracle_mod.default_params(mode=oracle_mode))


@pytest.mark.parametrize("variant", ["ux", "random"])
def test_ablation_variants(plse, oracle_mod, variant):
    grid = inputs.random_insertion(15, 0.7, 5)
    kw = {"crossover": 1} if variant == "ux" else {"matching": 1}
    compare(plse, oracle_mod, grid, 30, 6, 120, 7,
            gpu_params=plse.default_params(**kw), oracle_params=oracle_mod.default_params(**kw))


def test_small_tested_cap(plse, oracle_mod):
    grid = inputs.random_insertion(12, 0.72, 6)
    compare(plse, oracle_mod, grid, 6, 12, 50, 8,
            gpu_params=plse.default_params(tested_cap=2),
            oracle_params=oracle_mod.default_params(tested_cap=2))


def test_edge_instances(plse, oracle_mod):
    n3 = np.array([[1, 0, 0], [2, 0, 0], [0, 0, 3]], dtype=np.int8)
    res, ref = compare(plse, oracle_mod, n3, 8, 5, 50, 1)
    assert res["score"] == 7 and res["generations"] == 1
    _, L = inputs.cyclic_delete(6, 1.0, 1)
    G = plse.Instance(L)                                  # no reduced vertex at all
    out = G.solve(4, 3, 10, 1, with_stats=True)
    assert out["score"] == 36 and out["generations"] == 0
    assert np.array_equal(out["best_grid"], L)


def test_resumable_run_matches_solve(plse, oracle_mod):
    grid = inputs.random_insertion(16, 0.75, 8)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    ref = I.solve(40, 6, 120, 9)
    G.run_begin(40, 6, 120, 9)
    for _ in range(6):
        if G.run_step(1):
            break
    res = G.run_result(trace=True)
    assert res["score"] == ref["score"] and np.array_equal(res["best_grid"], ref["best_grid"])
    assert res["generations"] == ref["generations"] and res["walks"] == ref["stats"]
    assert res["trace"].tolist() == ref["trace"].tolist()


def test_no_stop_at_bound_keeps_generating(plse, oracle_mod):
    # the bound is reached in generation 1; with the stop disabled the run goes on
    grid = inputs.tiny_n10()
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    ref = I.solve(32, 5, 300, 2)
    G.set_params(plse.default_params(stop_at_bound=0))
    res = G.solve(32, 5, 300, 2, with_stats=True)
    assert res["generations"] == 5 and ref["generations"] == 1
    assert res["score"] == ref["score"] == 100
    g = res["best_grid"]
    assert is_partial_latin(g) and int((g != 0).sum()) == 100


def test_whole_run_at_the_maximum_order(plse, oracle_mod):
    # n = 127, the largest order accepted: every step of the generation at four
    # colour words, whole-run parity over three generations
    grid = inputs.random_insertion(127, 0.85, 227)
    res, ref = compare(plse, oracle_mod, grid, 8, 3, 400, 5)
    assert res["generations"] >= 1
