"""Pins of the oracle's population steps: Hamming distance (Sec. 3.4), the
population update (Alg. 4), parent matching (Sec. 3.5.1) and AUX/UX crossover
(Sec. 3.5.2, Eq. 10, Alg. 5)."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs


@pytest.fixture(scope="module")
def inst(oracle_mod):
    return oracle_mod.Instance(inputs.random_insertion(14, 0.35, 8))


def test_distance_properties(oracle_mod, inst):
    P = inst.init_population(24, 3)
    D = inst.distances(P, P)
    assert np.all(np.diag(D) == 0) and np.array_equal(D, D.T)
    # triangle inequality D(a, c) <= D(a, b) + D(b, c)
    for a in range(24):
        assert np.all(D[a][None, :] <= D[a][:, None] + D)
    # perturbing exactly k vertices gives distance k
    rng = np.random.default_rng(1)
    dom = inst.domains()
    for k in (0, 1, 7, inst.nv):
        Q = P[0].copy()
        for v in rng.choice(inst.nv, size=k, replace=False):
            opts = [c for c in range(inst.n + 1) if dom[v, c] and c != Q[v]]
            Q[v] = opts[int(rng.integers(len(opts)))]
        assert inst.distances(P[:1], Q[None])[0, 0] == k


def greedy_is_consistent(sel, e, D, nv, gamma, p):
    """The Alg. 4 outcome is characterised without replaying it: walking P_all in
    (e, index) order, a candidate is accepted iff every member accepted before it
    is farther than |V|/gamma; accepted members appear in that order."""
    order = sorted(range(len(e)), key=lambda k: (e[k], k))
    rank = {k: q for q, k in enumerate(order)}
    acc = list(sel)
    assert [rank[k] for k in acc] == sorted(rank[k] for k in acc)
    last = rank[acc[-1]]
    accepted_before = []
    for k in order[:last + 1]:
        ok = all(gamma * D[k, a] > nv for a in accepted_before) or not accepted_before
        assert (k in set(acc)) == ok, k
        if ok:
            accepted_before.append(k)
    assert accepted_before == acc


@pytest.mark.parametrize("seed", range(4))
def test_pop_update_greedy_spacing(oracle_mod, inst, seed):
    p = 40
    rng = np.random.default_rng(seed)
    P = inst.init_population(2 * p, seed)
    # cluster half of the candidates around a few centres so spacing bites
    for q in range(p, 2 * p):
        base = P[int(rng.integers(3))].copy()
        idx = rng.choice(inst.nv, size=int(rng.integers(0, inst.nv // 6)), replace=False)
        base[idx] = P[q][idx]
        P[q] = base
    e = rng.integers(0, 6, size=2 * p).astype(np.int64)
    D = inst.distances(P, P)
    sel, filled = inst.pop_update(e, D)
    assert len(set(sel.tolist())) == p
    assert sel[0] == min(range(2 * p), key=lambda k: (e[k], k))   # elitism
    nacc = p - filled
    greedy_is_consistent(sel[:nacc].tolist(), e, D, inst.nv, 10, p)
    acc = sel[:nacc]
    sub = D[np.ix_(acc, acc)] + np.eye(nacc, dtype=np.int64) * 10**9
    assert np.all(10 * sub > inst.nv)                               # spacing D > |V|/10
    if filled:
        # fill rule: the remaining places go to rejected candidates in rank order
        order = sorted(range(2 * p), key=lambda k: (e[k], k))
        rejected = [k for k in order if k not in set(acc.tolist())]
        assert sel[nacc:].tolist() == rejected[:filled]


def test_pop_update_fill_rule(oracle_mod, inst):
    # identical candidates: only one can be accepted, the rest come from the fill rule
    p = 6
    P = np.repeat(inst.init_population(1, 2), 2 * p, axis=0)
    e = np.arange(2 * p, dtype=np.int64)[::-1].copy()
    sel, filled = inst.pop_update(e, inst.distances(P, P))
    assert filled == p - 1 and sel.tolist() == list(range(2 * p - 1, p - 1, -1))


def test_matching_nearest_untested(oracle_mod, inst):
    p = 30
    P = inst.init_population(p, 5)
    D = inst.distances(P, P)
    uid = np.arange(100, 100 + p, dtype=np.uint32)
    cap = 64
    tested = np.zeros((p, cap), dtype=np.uint32)
    tcount = np.zeros(p, dtype=np.int32)
    rng = np.random.default_rng(0)
    for i in range(p):                                 # some partners already tested
        k = int(rng.integers(0, 4))
        tested[i, :k] = rng.choice(uid, size=k, replace=False)
        tcount[i] = k
    partner, t2, c2 = inst.matching(D, uid, tested, tcount, 0, 1)
    for i in range(p):
        allowed = [j for j in range(p) if j != i and uid[j] not in set(tested[i, :tcount[i]].tolist())]
        best = min(allowed, key=lambda j: (D[i, j], j))
        assert partner[i] == best
        assert c2[i] == tcount[i] + 1 and t2[i, tcount[i]] == uid[best]
    # calling again with the updated lists moves every member to its next-nearest
    partner2, _, _ = inst.matching(D, uid, t2, c2, 1, 1)
    assert np.all(partner2 != partner)


def test_matching_all_tested_and_list_cap(oracle_mod, inst):
    p = 4
    P = inst.init_population(p, 6)
    D = inst.distances(P, P)
    uid = np.arange(p, dtype=np.uint32)
    prm = oracle_mod.default_params(tested_cap=3)
    tested = np.tile(uid, (p, 1))[:, :3].copy()
    tcount = np.full(p, 3, dtype=np.int32)
    tested[0] = [1, 2, 3]                              # member 0 has tested everyone
    partner, t2, c2 = inst.matching(D, uid, tested, tcount, 0, 1, params=prm)
    assert partner[0] == min([1, 2, 3], key=lambda j: (D[0, j], j))
    assert c2[0] == 3 and t2[0].tolist() == [2, 3, uid[partner[0]]]   # oldest dropped


def test_random_matching_is_uniform(oracle_mod, inst):
    p = 9
    P = inst.init_population(p, 1)
    D = inst.distances(P, P)
    prm = oracle_mod.default_params(matching=1)
    z = np.zeros((p, 64), dtype=np.uint32)
    hits = np.zeros((p, p))
    for g in range(400):
        partner, _, _ = inst.matching(D, np.arange(p, dtype=np.uint32), z, np.zeros(p, np.int32), g, 3, params=prm)
        assert np.all(partner != np.arange(p))
        hits[np.arange(p), partner] += 1
    expected = 400 / (p - 1)
    off = hits[~np.eye(p, dtype=bool)]
    assert float(((off - expected) ** 2 / expected).sum()) < 2 * p * (p - 1)


def test_aux_closed_forms(oracle_mod):
    # Sec. 3.5.2: E[D(S_i, S_O)] = |V|/beta, E[D(S_j, S_O)] = D_ij - |V|/beta;
    # each vertex is an independent coin with p_ij = 1 - |V|/(beta D_ij)
    I = oracle_mod.Instance(np.zeros((12, 12), dtype=np.int8))
    nv = I.nv
    p = 400
    A = I.init_population(p, 11)
    Dfull = I.distances(A, A)
    partner = np.array([(i + 1) % p for i in range(p)], dtype=np.int32)
    O = I.crossover(A, partner, Dfull, 0, 5)
    dij = Dfull[np.arange(p), partner].astype(float)
    d_i = I.distances(A, O)[np.arange(p), np.arange(p)].astype(float)
    d_j = np.array([I.distances(A[partner[i]][None], O[i][None])[0, 0] for i in range(p)], float)
    beta = 20.0
    q = nv / (beta * dij)                                     # P(vertex from S_j)
    mean_i = (q * dij).sum()                                  # = p * |V| / beta exactly
    var_i = (dij * q * (1 - q)).sum()
    assert abs(mean_i - p * nv / beta) < 1e-6
    assert abs(d_i.sum() - mean_i) < 5 * np.sqrt(var_i)
    assert abs(d_j.sum() - (dij - nv / beta).sum()) < 5 * np.sqrt(var_i)
    # vertices where the parents agree are copied, others come from either parent
    for i in range(0, p, 37):
        j = partner[i]
        agree = A[i] == A[j]
        assert np.all(O[i][agree] == A[i][agree])
        assert np.all((O[i] == A[i]) | (O[i] == A[j]))


def test_ux_is_half_half(oracle_mod):
    I = oracle_mod.Instance(np.zeros((12, 12), dtype=np.int8))
    p = 200
    A = I.init_population(p, 2)
    D = I.distances(A, A)
    partner = np.array([(i + 3) % p for i in range(p)], dtype=np.int32)
    O = I.crossover(A, partner, D, 1, 9, params=oracle_mod.default_params(crossover=1))
    dij = D[np.arange(p), partner].astype(float)
    d_i = np.array([(O[i] != A[i]).sum() for i in range(p)], float)
    assert abs(d_i.sum() - dij.sum() / 2) < 5 * np.sqrt(dij.sum() / 4)


def test_aux_degenerate_distances(oracle_mod):
    I = oracle_mod.Instance(np.zeros((6, 6), dtype=np.int8))
    A = I.init_population(2, 1)
    same = np.stack([A[0], A[0]])
    D0 = np.zeros((2, 2), dtype=np.int32)
    O = I.crossover(same, np.array([1, 0], np.int32), D0, 0, 1)
    assert np.array_equal(O, same)                                  # D = 0: copy
    # beta * D <= |V| (possible only after the fill rule): p_ij clamps at 0 -> S_j
    B = np.stack([A[0], A[0]])
    B[1, 0] = (B[0, 0] % 6) + 1
    D1 = I.distances(B, B)
    assert 20 * D1[0, 1] <= I.nv
    O = I.crossover(B, np.array([1, 0], np.int32), D1, 0, 1)
    assert np.array_equal(O[0], B[1]) and np.array_equal(O[1], B[0])
