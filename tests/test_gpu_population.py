"""GPU-vs-oracle parity of the population steps called through the C ABI:
Hamming distances (Sec. 3.4), the population update (Alg. 4), parent matching
(Sec. 3.5.1) and AUX / UX crossover (Eq. 10, Alg. 5).  All bit-exact."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _gpu import dev, empty, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


GRIDS = {
    "n3": np.array([[1, 0, 0], [2, 0, 0], [0, 0, 3]], dtype=np.int8),
    "n10": inputs.tiny_n10(),
    "n23_r05": inputs.random_insertion(23, 0.5, 31),
    "n70_r07": inputs.random_insertion(70, 0.7, 32),
    "n127_r085": inputs.random_insertion(127, 0.85, 33),
}


def clustered_population(I, count, seed, frac=0.15):
    """Random colourings, half of them near a few centres, so Alg. 4 rejects."""
    rng = np.random.default_rng(seed)
    P = I.init_population(count, seed)
    for q in range(count // 2, count):
        base = P[int(rng.integers(4))].copy()
        k = int(rng.integers(0, max(1, int(I.nv * frac))))
        idx = rng.choice(I.nv, size=k, replace=False)
        base[idx] = P[q][idx]
        P[q] = base
    return P


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("na,nb", [(1, 1), (37, 130), (64, 64), (129, 3)])
def test_distances_bit_exact(plse, oracle_mod, name, na, nb):
    import torch
    G, I = plse.Instance(GRIDS[name]), oracle_mod.Instance(GRIDS[name])
    A = I.init_population(na, 1)
    B = clustered_population(I, nb, 2) if nb > 3 else I.init_population(nb, 2)
    D = empty((na, nb), torch.int32)
    G.distances(dev(A), na, dev(B), nb, D)
    assert np.array_equal(host(D), I.distances(A, B))


@pytest.mark.parametrize("name", ["n10", "n23_r05", "n70_r07"])
@pytest.mark.parametrize("p", [3, 40, 200, 700])
def test_pop_update_bit_exact(plse, oracle_mod, name, p):
    import torch
    G, I = plse.Instance(GRIDS[name]), oracle_mod.Instance(GRIDS[name])
    Pall = clustered_population(I, 2 * p, p, frac=0.08)
    rng = np.random.default_rng(p)
    e = rng.integers(0, 5, size=2 * p).astype(np.int64)
    e[: p // 3] += 10**9                      # a block of illegal-looking scores
    sel_o, filled_o = I.pop_update(e, I.distances(Pall, Pall))
    sel = empty((p,), torch.int32)
    filled = empty((1,), torch.int32)
    G.pop_update(p, dev(Pall), dev(e), sel, filled)
    assert np.array_equal(host(sel), sel_o)
    assert int(host(filled)[0]) == filled_o


def test_pop_update_fill_rule(plse, oracle_mod):
    import torch
    I = oracle_mod.Instance(GRIDS["n23_r05"])
    G = plse.Instance(GRIDS["n23_r05"])
    p = 150
    Pall = np.repeat(I.init_population(3, 5), 100, axis=0)          # 3 distinct colourings
    e = np.zeros(2 * p, dtype=np.int64)
    sel_o, filled_o = I.pop_update(e, I.distances(Pall, Pall))
    sel = empty((p,), torch.int32)
    filled = empty((1,), torch.int32)
    G.pop_update(p, dev(Pall), dev(e), sel, filled)
    assert filled_o == p - 3
    assert np.array_equal(host(sel), sel_o) and int(host(filled)[0]) == filled_o


@pytest.mark.parametrize("name", ["n3", "n10", "n23_r05", "n70_r07"])
@pytest.mark.parametrize("p", [2, 5, 64, 333])
def test_matching_bit_exact(plse, oracle_mod, name, p):
    import torch
    G, I = plse.Instance(GRIDS[name]), oracle_mod.Instance(GRIDS[name])
    P = clustered_population(I, p, 7 + p)
    rng = np.random.default_rng(p)
    uid = rng.permutation(10 * p)[:p].astype(np.uint32)
    cap = 64
    tested = np.zeros((p, cap), dtype=np.uint32)
    tcount = np.zeros(p, dtype=np.int32)
    for i in range(p):
        k = int(rng.integers(0, min(cap, p) + 1)) if i % 7 == 0 else int(rng.integers(0, 4))
        k = min(k, cap)
        if k:
            tested[i, :k] = rng.choice(uid, size=k, replace=True)
            tcount[i] = k
    tcount[0] = cap                                     # a full list: oldest entry dropped
    tested[0] = rng.choice(uid, size=cap, replace=True)
    D = I.distances(P, P)
    part_o, tested_o, tcount_o = I.matching(D, uid, tested, tcount, 3, 9)
    t_d, c_d = dev(tested), dev(tcount)
    partner = empty((p,), torch.int32)
    dist = empty((p,), torch.int32)
    G.matching(p, dev(P), dev(uid), t_d, c_d, 3, 9, partner, dist)
    assert np.array_equal(host(partner), part_o)
    assert np.array_equal(host(dist), D[np.arange(p), part_o])
    assert np.array_equal(host(c_d), tcount_o)
    got_t = host(t_d)
    for i in range(p):
        assert np.array_equal(got_t[i, :tcount_o[i]], tested_o[i, :tcount_o[i]])


def test_random_matching_bit_exact(plse, oracle_mod):
    import torch
    grid = GRIDS["n23_r05"]
    G, I = plse.Instance(grid), oracle_mod.Instance(grid)
    G.set_params(plse.default_params(matching=plse.MATCH_RANDOM))
    oprm = oracle_mod.default_params(matching=1)
    p = 97
    P = I.init_population(p, 4)
    D = I.distances(P, P)
    z = np.zeros((p, 64), np.uint32)
    part_o, _, _ = I.matching(D, np.arange(p, dtype=np.uint32), z, np.zeros(p, np.int32), 5, 11, params=oprm)
    partner = empty((p,), torch.int32)
    dist = empty((p,), torch.int32)
    G.matching(p, dev(P), dev(np.arange(p, dtype=np.uint32)), dev(z), dev(np.zeros(p, np.int32)), 5, 11,
               partner, dist)
    assert np.array_equal(host(partner), part_o)
    assert np.array_equal(host(dist), D[np.arange(p), part_o])


@pytest.mark.parametrize("name", list(GRIDS))
@pytest.mark.parametrize("ux", [0, 1])
def test_crossover_bit_exact(plse, oracle_mod, name, ux):
    import torch
    G, I = plse.Instance(GRIDS[name]), oracle_mod.Instance(GRIDS[name])
    if ux:
        G.set_params(plse.default_params(crossover=plse.XOVER_UX))
    oprm = oracle_mod.default_params(crossover=ux)
    p = 75
    P = clustered_population(I, p, 3, frac=0.03)
    P[5] = P[6]                                         # D = 0 pair
    partner = np.array([(i * 7 + 1) % p for i in range(p)], dtype=np.int32)
    partner[5] = 6
    D = I.distances(P, P)
    O_o = I.crossover(P, partner, D, 2, 21, params=oprm)
    O = empty((p, G.nv), torch.uint8)
    G.crossover(p, dev(P), dev(partner), dev(D[np.arange(p), partner].astype(np.int32)), 2, 21, O)
    assert np.array_equal(host(O), O_o)
