"""GPU-vs-oracle parity of population initialisation and the tabu local search
(Alg. 3 phases 1 and 2, PartialCol, greedy repair), called through the C ABI.
Integer work: every comparison is bit-exact (colourings, best F values and the
per-walk work counters)."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _gpu import dev, empty, host

pytestmark = pytest.mark.gpu

FIELDS = ["iterations", "moves", "cand", "pairs", "deg", "improvements", "uncolored"]


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


def cases():
    return {
        "tiny_n10": inputs.tiny_n10(),
        "ri_n7_r05": inputs.random_insertion(7, 0.5, 2),
        "cyc_n9_r05": inputs.cyclic_delete(9, 0.5, 4)[0],
        "ri_n16_r06": inputs.random_insertion(16, 0.6, 11),
        "ri_n30_r07": inputs.random_insertion(30, 0.7, 12),
        "cyc_n33_r03": inputs.cyclic_delete(33, 0.3, 13)[0],
        "ri_n40_r05": inputs.random_insertion(40, 0.5, 14),
        "cyc_n70_r06": inputs.cyclic_delete(70, 0.6, 15)[0],
        "ri_n100_r08": inputs.random_insertion(100, 0.8, 16),
    }


def run_gpu_ls(plse, G, P, ind0, gen, iters, seed, flags):
    import torch
    count = P.shape[0]
    S_in = dev(P)
    S_out = empty(P.shape, torch.uint8)
    f = empty((count,), torch.int32)
    F = empty((count,), torch.int64)
    st = empty((count, 7), torch.int64)
    G.local_search(S_in, S_out, count, ind0, gen, iters, seed, flags, f, F, st)
    G.sync()
    return host(S_out), host(f), host(F), host(st)


def oracle_ls(I, S, ind, gen, iters, seed, flags, prm=None):
    st = {k: 0 for k in FIELDS}
    F = 0

    def add(s):
        for k in FIELDS:
            st[k] += s[k]
    if flags & 8:
        if flags & 4:
            S, _ = I.repair(S)
        S, F, s = I.tabu_walk(S, ind, gen, 3, iters, seed, params=prm)
        add(s)
    else:
        if flags & 1:
            S, F, s = I.tabu_walk(S, ind, gen, 1, iters, seed, params=prm)
            add(s)
        if flags & 2:
            it2 = (prm.phase2_iter_per_v if prm else 2) * I.nv
            S, F, s = I.tabu_walk(S, ind, gen, 2, it2, seed, params=prm)
            add(s)
        if flags & 4:
            S, _ = I.repair(S)
    return S, F, st


@pytest.mark.parametrize("name", list(cases()))
def test_init_population_bit_exact(plse, oracle_mod, name):
    import torch
    grid = cases()[name]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    assert (G.nv, G.l, G.ub) == (I.nv, I.l, I.ub)
    pop = 37
    out = empty((pop, G.nv), torch.uint8)
    G.init_population(pop, 12345, out)
    assert np.array_equal(host(out), I.init_population(pop, 12345))


@pytest.mark.parametrize("name", ["tiny_n10", "ri_n7_r05", "cyc_n9_r05", "ri_n16_r06", "ri_n30_r07",
                                  "cyc_n33_r03", "ri_n40_r05"])
def test_plits_two_phase_repair_bit_exact(plse, oracle_mod, name):
    grid = cases()[name]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    count = 40
    iters = min(4 * I.nv, 1500)
    P = I.init_population(count, 7)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    S, f, F, st = run_gpu_ls(plse, G, P, 3, 2, iters, 99, flags)
    for w in range(count):
        So, Fo, sto = oracle_ls(I, P[w], 3 + w, 2, iters, 99, flags)
        assert np.array_equal(S[w], So), (name, w)
        assert F[w] == Fo
        assert f[w] == int((So == 0).sum())
        assert st[w].tolist() == [sto[k] for k in FIELDS], (name, w)


@pytest.mark.parametrize("name", ["tiny_n10", "ri_n16_r06", "ri_n30_r07", "cyc_n70_r06", "ri_n100_r08"])
def test_phase1_only_bit_exact(plse, oracle_mod, name):
    grid = cases()[name]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    count = 6
    iters = min(2 * I.nv, 3000)
    P = I.init_population(count, 1)
    S, f, F, st = run_gpu_ls(plse, G, P, 0, 0, iters, 5, plse.LS_PHASE1)
    for w in range(count):
        So, Fo, sto = oracle_ls(I, P[w], w, 0, iters, 5, plse.LS_PHASE1)
        assert np.array_equal(S[w], So), (name, w)
        assert F[w] == Fo and st[w].tolist() == [sto[k] for k in FIELDS]


def test_long_walk_crosses_clock_rebase(plse, oracle_mod):
    # > 49152 iterations: the relative tabu clock is rebased at least once
    grid = inputs.random_insertion(12, 0.7, 21)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    P = I.init_population(3, 2)
    S, f, F, st = run_gpu_ls(plse, G, P, 0, 1, 70000, 8, plse.LS_PHASE1)
    for w in range(3):
        So, Fo, sto = oracle_ls(I, P[w], w, 1, 70000, 8, plse.LS_PHASE1)
        assert np.array_equal(S[w], So) and F[w] == Fo
        assert st[w].tolist() == [sto[k] for k in FIELDS]


@pytest.mark.parametrize("name", ["ri_n7_r05", "ri_n16_r06", "ri_n30_r07", "ri_n40_r05", "ri_n100_r08"])
def test_partialcol_bit_exact(plse, oracle_mod, name):
    grid = cases()[name]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    count = 24
    iters = min(3 * I.nv, 2000)
    P = I.init_population(count, 3)
    flags = plse.LS_REPAIR | plse.LS_PARTIALCOL
    S, f, F, st = run_gpu_ls(plse, G, P, 0, 4, iters, 17, flags)
    for w in range(count):
        So, Fo, sto = oracle_ls(I, P[w], w, 4, iters, 17, flags)
        assert np.array_equal(S[w], So), (name, w)
        assert F[w] == Fo and st[w].tolist() == [sto[k] for k in FIELDS]


def test_repair_only_bit_exact(plse, oracle_mod):
    grid = inputs.random_insertion(25, 0.4, 3)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    P = I.init_population(50, 4)
    S, f, F, st = run_gpu_ls(plse, G, P, 0, 0, 0, 1, plse.LS_REPAIR)
    for w in range(50):
        assert np.array_equal(S[w], I.repair(P[w])[0])


def test_aliasing_and_uneven_params(plse, oracle_mod):
    import torch
    grid = inputs.random_insertion(20, 0.55, 5)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    prm = plse.default_params(alpha_num=3, alpha_den=4, tenure_rand=7, phase2_iter_per_v=1)
    G.set_params(prm)
    oprm = oracle_mod.default_params(alpha_num=3, alpha_den=4, tenure_rand=7, phase2_iter_per_v=1)
    P = I.init_population(8, 9)
    buf = dev(P)
    G.local_search(buf, buf, 8, 100, 7, 500, 3, plse.LS_PHASE1 | plse.LS_PHASE2)
    G.sync()
    S = host(buf)
    for w in range(8):
        So, _, _ = oracle_ls(I, P[w], 100 + w, 7, 500, 3, 3, prm=oprm)
        assert np.array_equal(S[w], So)


# (threads per walk, colouring placement: 1 shared memory, 2 global memory)
LAUNCHES = [(16, 1), (16, 2), (32, 1), (32, 2), (64, 0), (128, 0), (256, 0)]


@pytest.mark.parametrize("launch", LAUNCHES)
@pytest.mark.parametrize("name", ["ri_n16_r06", "cyc_n33_r03", "cyc_n70_r06", "ri_n100_r08"])
def test_launch_shape_does_not_change_results(plse, oracle_mod, name, launch):
    grid = cases()[name]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    lanes, place = launch
    G.set_launch(lanes, 0, place)
    count = 12
    iters = min(2 * I.nv, 2500)
    P = I.init_population(count, 13)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    S, f, F, st = run_gpu_ls(plse, G, P, 5, 9, iters, 31, flags)
    for w in range(count):
        So, Fo, sto = oracle_ls(I, P[w], 5 + w, 9, iters, 31, flags)
        assert np.array_equal(S[w], So), (name, launch, w)
        assert F[w] == Fo and st[w].tolist() == [sto[k] for k in FIELDS]
    # PartialCol with the same launch shape
    S, f, F, st = run_gpu_ls(plse, G, P, 5, 9, iters, 31, plse.LS_REPAIR | plse.LS_PARTIALCOL)
    for w in range(0, count, 3):
        So, Fo, sto = oracle_ls(I, P[w], 5 + w, 9, iters, 31, plse.LS_REPAIR | plse.LS_PARTIALCOL)
        assert np.array_equal(S[w], So) and F[w] == Fo


# Orders on both sides of each 32-colour-word boundary (colours 0..n take
# ceil((n + 1) / 32) words: n = 31 | 32, 63 | 64, 95 | 96) and the largest order
# the library accepts (127), where a walk's colour words and its launch shape
# (threads per block, registers, walks per SM) change.
BOUNDARY_ORDERS = [(31, 0.6), (32, 0.6), (63, 0.7), (64, 0.7), (95, 0.8), (96, 0.8), (127, 0.85)]


@pytest.mark.parametrize("n,r", BOUNDARY_ORDERS)
def test_colour_word_boundaries_and_maximum_order(plse, oracle_mod, n, r):
    import torch
    grid = inputs.random_insertion(n, r, 100 + n)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    assert (G.nv, G.l, G.ub) == (I.nv, I.l, I.ub)
    count = 12
    P = I.init_population(count, 7)
    out = empty((count, G.nv), torch.uint8)
    G.init_population(count, 7, out)
    assert np.array_equal(host(out), P)
    iters = min(2 * I.nv, 1200)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    S, f, F, st = run_gpu_ls(plse, G, P, 1, 4, iters, 3, flags)
    for w in range(count):
        So, Fo, sto = oracle_ls(I, P[w], 1 + w, 4, iters, 3, flags)
        assert np.array_equal(S[w], So), (n, w)
        assert F[w] == Fo and f[w] == int((So == 0).sum())
        assert st[w].tolist() == [sto[k] for k in FIELDS], (n, w)
    if r >= 0.8:                                     # PartialCol (Sec. 3.7) at the same orders
        flags = plse.LS_REPAIR | plse.LS_PARTIALCOL
        S, f, F, st = run_gpu_ls(plse, G, P, 1, 4, iters, 3, flags)
        for w in range(count):
            So, Fo, sto = oracle_ls(I, P[w], 1 + w, 4, iters, 3, flags)
            assert np.array_equal(S[w], So), (n, w)
            assert F[w] == Fo
            assert st[w].tolist() == [sto[k] for k in FIELDS], (n, w)


def test_empty_inputs_are_no_ops(plse, oracle_mod):
    # zero walks, an empty population and zero-row distance blocks succeed and
    # write nothing (output buffers keep a sentinel)
    import torch
    grid = cases()["ri_n16_r06"]
    G = plse.Instance(grid)
    nv = G.nv
    S = torch.full((4, nv), 7, dtype=torch.uint8, device="cuda")
    out = torch.full((4, nv), 9, dtype=torch.uint8, device="cuda")
    f = torch.full((4,), -5, dtype=torch.int32, device="cuda")
    D = torch.full((4, 4), -3, dtype=torch.int32, device="cuda")
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    G.local_search(S, out, 0, 0, 0, 100, 1, flags, f)
    G.local_search_noalloc(S, out, 0, 0, 0, 100, 1, flags, f)
    G.init_population(0, 1, out)
    G.distances(S, 0, S, 4, D)
    G.distances(S, 4, S, 0, D)
    G.sync()
    assert bool((out == 9).all()) and bool((f == -5).all()) and bool((D == -3).all())
    assert bool((S == 7).all())
