"""Pin of the oracle's tabu rule at every iteration (Sec. 3.3, Alg. 3; Sec. 3.7).

The oracle records the move it chose at each iteration.  This file replays the
walk with its own state, written from the paper's text and nothing else:

* the colouring's f and c (Eq. 1-4) and the conflicting set C(S) are counted
  from scratch over all pairs of cells that share a row or a column;
* the domains D(v) are re-derived from the grid (symbols absent from the row
  and the column, plus 0);
* the candidate moves are N0 u Nc (Sec. 3.3): an uncoloured vertex takes a
  colour of D(v)\\{0}; a conflicting vertex takes any other colour of D(v),
  0 included;
* the tabu list is a dictionary of expiries: moving v away from colour i at
  iteration t makes (v, i) tabu for the next T iterations, with
  T = L + floor(alpha * (|V0| + |C(S)|)) counted after the move, L uniform in
  [0, 9] from the walk's Philox draw (the Philox stream is pinned separately
  against cuRAND's host generator);
* a tabu move is admissible only if it leads below the best F of the walk so
  far (aspiration, Sec. 3.3);
* the chosen move minimises (2dF, (v - r) mod |V|, j) among admissible moves.

At each iteration the checker asserts that the oracle's move is admissible and
that no admissible move has a smaller key, or, where the oracle made no move,
that no move was admissible.  PartialCol (Sec. 3.7, the cited legal-space
search): moves colour an uncoloured vertex and uncolour its neighbours of that
colour; the uncoloured neighbours' (u, j) become tabu for L + floor(alpha*|V0|)
iterations; aspiration against the best f of the walk.
"""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _plse_brute import count_f_c

TABU_PURPOSE = 2
ALPHA_NUM, ALPHA_DEN, L_RANGE = 6, 10, 10     # Table 1: alpha = 0.6, L in [0, 9]


class Scratch:
    """From-scratch evaluation of colourings of one instance (Eq. 1-4)."""

    def __init__(self, grid, cells):
        self.grid = np.asarray(grid)
        self.n = self.grid.shape[0]
        self.cells = np.asarray(cells)
        rows, cols = self.cells // self.n, self.cells % self.n
        self.adj = (rows[:, None] == rows[None, :]) | (cols[:, None] == cols[None, :])
        np.fill_diagonal(self.adj, False)
        self.dom = []
        for r, c in zip(rows, cols):
            used = set(self.grid[r, :].tolist()) | set(self.grid[:, c].tolist())
            self.dom.append([0] + [k for k in range(1, self.n + 1) if k not in used])

    def f_c(self, M):
        """f and c of each row of M (a batch of colourings)."""
        M = np.atleast_2d(M).astype(np.int64)
        same = (M[:, :, None] == M[:, None, :]) & (M[:, :, None] != 0) & self.adj[None]
        return (M == 0).sum(1), same.sum((1, 2)) // 2

    def conflicting(self, S):
        """C(S): coloured vertices with a neighbour of the same colour."""
        S = np.asarray(S, dtype=np.int64)
        return (S != 0) & ((S[:, None] == S[None, :]) & self.adj).any(1)


def draw(oracle_mod, t, ind, gen, phase, seed, nv):
    u = oracle_mod.philox4x32_10([t, ind, (gen << 8) | (TABU_PURPOSE << 4) | phase, 0],
                                 [seed & 0xFFFFFFFF, seed >> 32])
    return (int(u[0]) * L_RANGE) >> 32, (int(u[1]) * nv) >> 32


def replay_plits(oracle_mod, I, X, S0, ind, gen, phase, seed, trace, events):
    """Replays a PLITS walk (Alg. 3) and checks every recorded choice."""
    nv = I.nv
    phi2 = 1 if phase == 1 else 2 * nv
    S = np.array(S0, dtype=np.int64)
    f, c = (int(x[0]) for x in X.f_c(S))
    F2 = 2 * f + phi2 * c
    F2best, best = F2, S.copy()
    expiry = {}
    for t, (v_ch, i_ch, j_ch) in enumerate(trace, start=1):
        V0 = S == 0
        cand = np.nonzero(V0 | X.conflicting(S))[0]
        assert len(cand) > 0, "the walk went on with no candidate (Sec. 3.3)"
        L, r = draw(oracle_mod, t, ind, gen, phase, seed, nv)
        moves = [(v, j) for v in cand for j in X.dom[v]
                 if j != S[v] and not (S[v] == 0 and j == 0)]
        M = np.repeat(S[None], len(moves), 0)
        for q, (v, j) in enumerate(moves):
            M[q, v] = j
        fm, cm = X.f_c(M)
        F2m = 2 * fm + phi2 * cm
        admissible = []
        for q, (v, j) in enumerate(moves):
            tabu = expiry.get((v, j), 0) >= t
            if not tabu or F2m[q] < F2best:
                admissible.append(((int(F2m[q]) - F2, (v - r) % nv, j), v, j, tabu))
        if v_ch < 0:
            assert not admissible, "t=%d: no move made although %s was admissible" % (t, admissible[0])
            events["all_tabu"] += 1
            continue
        assert i_ch == S[v_ch], "t=%d: recorded colour before the move is not S(v)" % t
        chosen = [a for a in admissible if a[1] == v_ch and a[2] == j_ch]
        assert chosen, "t=%d: move (%d, %d->%d) is tabu and does not aspirate" % (t, v_ch, i_ch, j_ch)
        assert chosen[0][0] == min(a[0] for a in admissible), "t=%d: a better admissible move exists" % t
        if chosen[0][3]:
            events["aspiration"] += 1
        S[v_ch] = j_ch
        f, c = (int(x[0]) for x in X.f_c(S))
        F2 = 2 * f + phi2 * c
        k = f + int(X.conflicting(S).sum())             # after the move
        expiry[(v_ch, i_ch)] = t + L + (ALPHA_NUM * k) // ALPHA_DEN
        if F2 < F2best:
            F2best, best = F2, S.copy()
    events["iterations"] += len(trace)
    return best, F2best


def replay_partialcol(oracle_mod, I, X, S0, ind, gen, seed, trace, events):
    """Replays a PartialCol walk (Sec. 3.7) and checks every recorded choice."""
    nv = I.nv
    S = np.array(S0, dtype=np.int64)
    f, c = (int(x[0]) for x in X.f_c(S))
    assert c == 0
    fbest, best = f, S.copy()
    expiry = {}
    for t, (v_ch, i_ch, j_ch) in enumerate(trace, start=1):
        cand = np.nonzero(S == 0)[0]
        assert len(cand) > 0
        L, r = draw(oracle_mod, t, ind, gen, 3, seed, nv)
        moves = [(v, j) for v in cand for j in X.dom[v] if j != 0]
        M = np.repeat(S[None], len(moves), 0)
        for q, (v, j) in enumerate(moves):
            M[q, (X.adj[v]) & (S == j)] = 0             # neighbours of colour j lose it
            M[q, v] = j
        fm, cm = X.f_c(M)
        assert np.all(cm == 0), "a PartialCol move left a conflict"
        admissible = []
        for q, (v, j) in enumerate(moves):
            tabu = expiry.get((v, j), 0) >= t
            if not tabu or fm[q] < fbest:
                admissible.append(((int(fm[q]) - f, (v - r) % nv, j), v, j, tabu, q))
        if v_ch < 0:
            assert not admissible, "t=%d: no move made although one was admissible" % t
            events["all_tabu"] += 1
            continue
        assert i_ch == 0 and S[v_ch] == 0
        chosen = [a for a in admissible if a[1] == v_ch and a[2] == j_ch]
        assert chosen, "t=%d: move (%d -> %d) is tabu and does not aspirate" % (t, v_ch, j_ch)
        assert chosen[0][0] == min(a[0] for a in admissible), "t=%d: a better admissible move exists" % t
        if chosen[0][3]:
            events["aspiration"] += 1
        unc = np.nonzero(X.adj[v_ch] & (S == j_ch))[0]
        S = M[chosen[0][4]].copy()
        f = int((S == 0).sum())
        for u in unc:
            expiry[(int(u), j_ch)] = t + L + (ALPHA_NUM * f) // ALPHA_DEN
        if f < fbest:
            fbest, best = f, S.copy()
    events["iterations"] += len(trace)
    return best, fbest


# small instances of both constructions: n = 6..12, sparse and dense
CASES = [("cyc", 6, 0.3, 1), ("ins", 7, 0.5, 2), ("ins", 8, 0.7, 3), ("cyc", 9, 0.5, 4),
         ("ins", 10, 0.6, 5), ("cyc", 12, 0.75, 6), ("ins", 6, 0.6, 7), ("ins", 12, 0.8, 8)]


def make(case):
    kind, n, r, seed = case
    return inputs.cyclic_delete(n, r, seed)[0] if kind == "cyc" else inputs.random_insertion(n, r, seed)


EVENTS = {"aspiration": 0, "all_tabu": 0, "iterations": 0,
          "pc_aspiration": 0, "pc_all_tabu": 0, "pc_iterations": 0}


def test_scratch_evaluator_agrees_with_pairwise_count(oracle_mod):
    # the vectorised from-scratch f and c equal the plain pairwise count
    I = oracle_mod.Instance(make(CASES[3]))
    X = Scratch(I.grid, I.vertices())
    P = I.init_population(5, 3)
    fs, cs = X.f_c(P)
    for k in range(5):
        assert (int(fs[k]), int(cs[k])) == count_f_c(I.grid, I.vertices(), P[k])
    dom = I.domains()
    for v in range(I.nv):
        assert X.dom[v] == [j for j in range(I.n + 1) if dom[v, j]]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("phase", [1, 2])
def test_plits_every_move_obeys_the_tabu_rule(oracle_mod, case, phase):
    I = oracle_mod.Instance(make(case))
    X = Scratch(I.grid, I.vertices())
    iters = 300 if phase == 1 else 2 * I.nv
    P = I.init_population(3, 17)
    for ind in range(3):
        gen, seed = 2 + ind, 40 + case[3]
        S, F2, st, trace = I.tabu_walk_traced(P[ind], ind, gen, phase, iters, seed)
        ev = {"aspiration": 0, "all_tabu": 0, "iterations": 0}
        best, F2best = replay_plits(oracle_mod, I, X, P[ind], ind, gen, phase, seed, trace, ev)
        assert F2 == F2best and np.array_equal(S, best)
        assert st["moves"] == st["iterations"] - ev["all_tabu"]
        for k in ev:
            EVENTS[k] += ev[k]


@pytest.mark.parametrize("case", CASES)
def test_partialcol_every_move_obeys_the_tabu_rule(oracle_mod, case):
    I = oracle_mod.Instance(make(case))
    X = Scratch(I.grid, I.vertices())
    P = I.init_population(3, 23)
    for ind in range(3):
        start, _ = I.repair(P[ind])
        gen, seed = 1 + ind, 70 + case[3]
        S, fb, st, trace = I.tabu_walk_traced(start, ind, gen, 3, 300, seed)
        ev = {"aspiration": 0, "all_tabu": 0, "iterations": 0}
        best, fbest = replay_partialcol(oracle_mod, I, X, start, ind, gen, seed, trace, ev)
        assert fb == fbest and np.array_equal(S, best)
        for k in ev:
            EVENTS["pc_" + k] += ev[k]


def test_aspiration_and_all_tabu_iterations_were_exercised():
    # the replays above met both special cases of the rule: a tabu move taken
    # because it beats the walk's best, and an iteration where every move is
    # tabu and none aspirates (no move is made)
    if EVENTS["iterations"] == 0:
        pytest.skip("run with the replay tests")
    assert EVENTS["aspiration"] > 0, EVENTS
    assert EVENTS["all_tabu"] > 0, EVENTS
    assert EVENTS["pc_iterations"] > 0, EVENTS
    assert EVENTS["pc_aspiration"] > 0, EVENTS
    assert EVENTS["pc_all_tabu"] > 0, EVENTS
