"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: one generation's local search of a whole population (p = 16384
at n = 70, p = 8192 at n = 50) in a single launch, compared with the oracle walk
by walk on sampled individuals (bit-exact colourings, best F and work
counters), plus properties every output must have (legal colourings, f equal
to the number of uncoloured vertices).  Alg. 4 at p = 16384 is checked through
properties that hold at any size: p distinct members, elitism, spacing of the
accepted members and the fill rule."""
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


def oracle_generation(I, S, ind, gen, iters, seed):
    """Phase 1 (iters), phase 2 (2|V|), repair, as one benchmark generation."""
    st = {k: 0 for k in FIELDS}
    S, F, s1 = I.tabu_walk(S, ind, gen, 1, iters, seed)
    S, F, s2 = I.tabu_walk(S, ind, gen, 2, 2 * I.nv, seed)
    S, _ = I.repair(S)
    for s in (s1, s2):
        for k in FIELDS:
            st[k] += s[k]
    return S, F, st


def conflicts(I, grid, S):
    """Conflicting edges of colouring S written into the grid (numpy, no oracle)."""
    n = grid.shape[0]
    g = grid.astype(np.int32).copy().reshape(-1)
    g[I.vertices()] = S
    g = g.reshape(n, n)
    c = 0
    for line in list(g) + list(g.T):
        vals = line[line > 0]
        c += len(vals) - len(np.unique(vals))
    return c


@pytest.mark.parametrize("grid_name, pop, samples", [
    ("n70_r0.3", 16384, (0, 4097, 12345, 16383)),
    ("n70_r0.7", 16384, (1, 8191, 16382)),
    ("n50_r0.5", 8192, (0, 5000, 8191)),
])
def test_full_population_generation_sampled(plse, oracle_mod, grid_name, pop, samples):
    import torch
    grid = {"n70_r0.3": lambda: inputs.n70(0.3), "n70_r0.7": lambda: inputs.n70(0.7),
            "n50_r0.5": inputs.n50_r05}[grid_name]()
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    iters = 10 * G.nv
    P = empty((pop, G.nv), torch.uint8)
    G.init_population(pop, 1, P)                     # the run's P_0 (and S^O of generation 0)
    out = empty((pop, G.nv), torch.uint8)
    f = empty((pop,), torch.int32)
    F = empty((pop,), torch.int64)
    st = empty((pop, 7), torch.int64)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    G.local_search(P, out, pop, 0, 0, iters, 1, flags, f, F, st)
    G.sync()
    P0, S, f, F, st = host(P), host(out), host(f), host(F), host(st)
    assert np.array_equal(P0[list(samples)], I.init_population(pop, 1)[list(samples)])
    for w in samples:
        So, Fo, sto = oracle_generation(I, P0[w], w, 0, iters, 1)
        assert np.array_equal(S[w], So), (grid_name, w)
        assert F[w] == Fo
        assert st[w].tolist() == [sto[k] for k in FIELDS], (grid_name, w)
    # every output: f = uncoloured count; a random sample is legal (repair)
    assert np.array_equal(f, (S == 0).sum(axis=1))
    rng = np.random.default_rng(pop)
    for w in rng.choice(pop, size=64, replace=False):
        assert conflicts(I, grid, S[w]) == 0


def test_full_population_update_properties(plse, oracle_mod):
    import torch
    grid = inputs.n70(0.5)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    p = 16384
    Pall = empty((2 * p, G.nv), torch.uint8)
    G.init_population(2 * p, 3, Pall)
    # offspring: the first half's local-search results give legal colourings
    G.local_search(Pall[p:], Pall[p:], p, 0, 0, 2 * G.nv, 5, plse.LS_PHASE1 | plse.LS_REPAIR)
    A = host(Pall)
    e = np.zeros(2 * p, dtype=np.int64)
    e[:p] = 10**9                                    # P_t ranked after the legal offspring
    e[p:] = (A[p:] == 0).sum(axis=1)
    sel = empty((p,), torch.int32)
    filled = empty((1,), torch.int32)
    G.pop_update(p, Pall, dev(e), sel, filled)
    sel, filled = host(sel), int(host(filled)[0])
    assert len(np.unique(sel)) == p and sel.min() >= 0 and sel.max() < 2 * p
    assert e[sel].min() == e.min()                                    # elitism
    acc = sel[: p - filled]
    # accepted members are pairwise farther than |V| / 10 (sampled pairs)
    rng = np.random.default_rng(11)
    idx = rng.choice(len(acc), size=min(96, len(acc)), replace=False)
    D = I.distances(A[acc[idx]], A[acc[idx]])
    off = ~np.eye(len(idx), dtype=bool)
    assert (10 * D[off] > I.nv).all()
    # the accepted list is in rank order (e, then index)
    key = e[acc] * (2 * p) + acc
    assert (np.diff(key) > 0).all()


@pytest.mark.parametrize("r, samples", [(0.3, (3, 7777, 16380)), (0.7, (0, 9001, 16383))])
def test_steady_state_generation_of_the_benchmark(plse, oracle_mod, r, samples):
    """The launch the benchmark times: generation 3 of a run at n = 70 and
    p = 16384, whose walks start from AUX offspring of legal parents (Alg. 2,
    Alg. 5).  Three generations run through the resumable run API; its offspring
    S^O then go through plse_local_search with the run's own arguments (ind0 0,
    generation 3, 10|V| phase-1 iterations, seed 1), and sampled walks are
    compared with the oracle bit for bit."""
    import torch
    grid = inputs.n70(r)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    G.set_params(plse.default_params(stop_at_bound=0))
    pop, iters, seed = 16384, 10 * G.nv, 1
    G.run_begin(pop, 4, iters, seed)
    G.run_step(3)
    SO = G.run_population(1, out=empty((pop, G.nv), torch.uint8))
    out = empty((pop, G.nv), torch.uint8)
    F = empty((pop,), torch.int64)
    st = empty((pop, 7), torch.int64)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    G.local_search(SO, out, pop, 0, 3, iters, seed, flags, None, F, st)
    G.sync()
    S0, S, F, st = host(SO), host(out), host(F), host(st)
    # steady state: the parents were legal, so an offspring is far from random
    assert all(conflicts(I, grid, S0[w]) < G.nv // 4 for w in samples)
    for w in samples:
        So, Fo, sto = oracle_generation(I, S0[w], w, 3, iters, seed)
        assert np.array_equal(S[w], So), (r, w)
        assert F[w] == Fo
        assert st[w].tolist() == [sto[k] for k in FIELDS], (r, w)
    # the run's own fourth generation consumed the same offspring
    G.run_step(1)
    res = G.run_result()
    assert res["generations"] == 4
    G.close()


def test_pop_update_past_sixteen_chunks_bit_exact(plse, oracle_mod):
    """Alg. 4 over 2p = 4096 candidates (32 chunks of 128): P_t of a run after
    two generations and the legal local-search results of its offspring, scored
    e = f + |V| c, against the oracle on its own 4096 x 4096 distance matrix."""
    import torch
    grid = inputs.random_insertion(30, 0.5, 2024)
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    G.set_params(plse.default_params(stop_at_bound=0))
    p = 2048
    G.run_begin(p, 3, 4 * G.nv, 7)
    G.run_step(2)
    Pt = G.run_population(0)
    SO = G.run_population(1)
    Pall = np.concatenate([Pt, SO])
    buf = dev(Pall)
    G.local_search(buf[p:], buf[p:], p, 0, 2, 4 * G.nv, 7,
                   plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR)
    A = host(buf)
    e = np.array([I.eval(A[k])[1] + G.nv * I.eval(A[k])[2] for k in range(2 * p)], dtype=np.int64)
    sel_o, filled_o = I.pop_update(e, I.distances(A, A))
    sel = empty((p,), torch.int32)
    filled = empty((1,), torch.int32)
    G.pop_update(p, buf, dev(e), sel, filled)
    assert np.array_equal(host(sel), sel_o)
    assert int(host(filled)[0]) == filled_o
    G.close()
