"""Python handle on the plain CPU oracle of the MPMA hot path (arXiv 2103.10453).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only users.  The product path (the CUDA
library and ``paper_2103_10453_gb300``) never imports this package, and this
package imports nothing from it.

The oracle itself is plain C (``plse_oracle.c``), compiled with gcc on first use
into ``liboracle_plse.so`` next to this file.  Every function restates one
passage of the paper; see the header comments for the citation of each and for
the readings taken where the paper is silent.  Parity pins live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plse_oracle.c")
_HDR = os.path.join(_HERE, "plse_oracle.h")
_LIB = os.path.join(_HERE, "liboracle_plse.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: it must build on x86 and Arm)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
        if force or stale:
            tmp = _LIB + ".tmp.%d" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-Wall", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    """Mirror of ``or_params`` (Table 1 and Sec. 3.3 of the paper)."""
    _fields_ = [(name, C.c_int32) for name in (
        "alpha_num", "alpha_den", "tenure_rand", "phase1_phi2", "phase2_phi2_per_v",
        "phase2_iter_per_v", "spacing_gamma", "beta", "mode", "matching",
        "crossover", "tested_cap")]


class Stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in (
        "iterations", "moves", "cand", "pairs", "deg", "improvements", "uncolored")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER
        u8p, i8p, i32p, u32p, i64p = (P(C.c_uint8), P(C.c_int8), P(C.c_int32),
                                      P(C.c_uint32), P(C.c_int64))
        lib.or_default_params.argtypes = [P(Params)]
        lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.or_create.restype = C.c_void_p
        lib.or_create.argtypes = [C.c_int32, i8p, i32p]
        lib.or_destroy.argtypes = [C.c_void_p]
        lib.or_info.argtypes = [C.c_void_p, i32p, i32p, i32p, i32p, i32p]
        lib.or_vertices.argtypes = [C.c_void_p, i32p]
        lib.or_domains.argtypes = [C.c_void_p, u8p]
        lib.or_num_edges.restype = C.c_int64
        lib.or_num_edges.argtypes = [C.c_void_p]
        lib.or_eval.restype = C.c_int64
        lib.or_eval.argtypes = [C.c_void_p, u8p, C.c_int32, i64p, i64p]
        lib.or_gamma.argtypes = [C.c_void_p, u8p, i32p]
        lib.or_num_conflicting.restype = C.c_int64
        lib.or_num_conflicting.argtypes = [C.c_void_p, u8p]
        lib.or_init_population.argtypes = [C.c_void_p, C.c_int32, C.c_uint64, u8p]
        lib.or_tabu_walk.restype = C.c_int64
        lib.or_tabu_walk.argtypes = [C.c_void_p, P(Params), u8p, C.c_int32, C.c_int32,
                                     C.c_int32, C.c_int64, C.c_uint64, C.c_int32, P(Stats)]
        lib.or_tabu_walk_traced.restype = C.c_int64
        lib.or_tabu_walk_traced.argtypes = [C.c_void_p, P(Params), u8p, C.c_int32, C.c_int32,
                                            C.c_int32, C.c_int64, C.c_uint64, C.c_int32,
                                            P(Stats), i32p]
        lib.or_repair.restype = C.c_int32
        lib.or_repair.argtypes = [C.c_void_p, u8p]
        lib.or_distances.argtypes = [C.c_void_p, u8p, C.c_int32, u8p, C.c_int32, i32p]
        lib.or_pop_update.restype = C.c_int32
        lib.or_pop_update.argtypes = [C.c_void_p, P(Params), C.c_int32, i64p, i32p, i32p]
        lib.or_matching.argtypes = [C.c_void_p, P(Params), C.c_int32, i32p, u32p, u32p,
                                    i32p, C.c_int32, C.c_uint64, i32p]
        lib.or_crossover.argtypes = [C.c_void_p, P(Params), C.c_int32, u8p, i32p, i32p,
                                     C.c_int32, C.c_uint64, u8p]
        lib.or_solve.restype = C.c_int32
        lib.or_solve.argtypes = [C.c_void_p, P(Params), C.c_int32, C.c_int32, C.c_int64,
                                 C.c_uint64, i8p, i32p, i32p, P(Stats), u8p]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(ct))


def default_params(**overrides) -> Params:
    p = Params()
    _load().or_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, int(v))
    return p


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for counter ``ctr`` (4 words) and key ``key`` (2 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


class OracleError(ValueError):
    pass


class Instance:
    """A PLSE instance reduced by Alg. 1 (oracle side)."""

    def __init__(self, grid: np.ndarray):
        grid = np.ascontiguousarray(grid, dtype=np.int8)
        assert grid.ndim == 2 and grid.shape[0] == grid.shape[1]
        self.lib = _load()
        err = C.c_int32(0)
        self.h = self.lib.or_create(grid.shape[0], _ptr(grid, C.c_int8), C.byref(err))
        if not self.h:
            raise OracleError("invalid grid (code %d)" % err.value)
        vals = [C.c_int32() for _ in range(5)]
        self.lib.or_info(self.h, *[C.byref(v) for v in vals])
        self.n, self.nv, self.l, self.ub, self.nfixed = (v.value for v in vals)
        self.grid = grid.copy()

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.or_destroy(h)
            self.h = None

    # -- graph -------------------------------------------------------------
    def vertices(self) -> np.ndarray:
        out = np.zeros(self.nv, dtype=np.int32)
        self.lib.or_vertices(self.h, _ptr(out, C.c_int32))
        return out

    def domains(self) -> np.ndarray:
        out = np.zeros((self.nv, self.n + 1), dtype=np.uint8)
        self.lib.or_domains(self.h, _ptr(out, C.c_uint8))
        return out

    def num_edges(self) -> int:
        return int(self.lib.or_num_edges(self.h))

    # -- evaluation ----------------------------------------------------------
    def eval(self, S: np.ndarray, phi2: int = 0):
        S = np.ascontiguousarray(S, dtype=np.uint8)
        f, c = C.c_int64(), C.c_int64()
        F2 = self.lib.or_eval(self.h, _ptr(S, C.c_uint8), phi2, C.byref(f), C.byref(c))
        return int(F2), int(f.value), int(c.value)

    def gamma(self, S: np.ndarray) -> np.ndarray:
        S = np.ascontiguousarray(S, dtype=np.uint8)
        out = np.zeros((self.nv, self.n + 1), dtype=np.int32)
        self.lib.or_gamma(self.h, _ptr(S, C.c_uint8), _ptr(out, C.c_int32))
        return out

    def num_conflicting(self, S: np.ndarray) -> int:
        S = np.ascontiguousarray(S, dtype=np.uint8)
        return int(self.lib.or_num_conflicting(self.h, _ptr(S, C.c_uint8)))

    # -- method steps --------------------------------------------------------
    def init_population(self, p: int, seed: int) -> np.ndarray:
        P = np.zeros((p, self.nv), dtype=np.uint8)
        self.lib.or_init_population(self.h, p, seed, _ptr(P, C.c_uint8))
        return P

    def tabu_walk(self, S, ind, gen, phase, iters, seed, params=None, debug=0):
        """Alg. 3 on a copy of ``S``; returns (best colouring, best F2 or f, stats)."""
        params = params or default_params()
        S = np.array(S, dtype=np.uint8, copy=True, order="C")
        st = Stats()
        r = self.lib.or_tabu_walk(self.h, C.byref(params), _ptr(S, C.c_uint8), ind, gen,
                                  phase, int(iters), seed, debug, C.byref(st))
        if r < 0:
            raise OracleError("walk self-check failed or start colouring illegal")
        return S, int(r), st.as_dict()

    def tabu_walk_traced(self, S, ind, gen, phase, iters, seed, params=None):
        """Alg. 3 as ``tabu_walk``, also returning the move chosen at each
        iteration executed: an int32 array [iterations, 3] of (v, colour before,
        colour after), (-1, -1, -1) where no move was admissible."""
        params = params or default_params()
        S = np.array(S, dtype=np.uint8, copy=True, order="C")
        st = Stats()
        trace = np.full((max(int(iters), 1), 3), -2, dtype=np.int32)
        r = self.lib.or_tabu_walk_traced(self.h, C.byref(params), _ptr(S, C.c_uint8), ind, gen,
                                         phase, int(iters), seed, 0, C.byref(st),
                                         _ptr(trace, C.c_int32))
        if r < 0:
            raise OracleError("start colouring illegal")
        stats = st.as_dict()
        return S, int(r), stats, trace[:stats["iterations"]].copy()

    def repair(self, S):
        S = np.array(S, dtype=np.uint8, copy=True, order="C")
        steps = self.lib.or_repair(self.h, _ptr(S, C.c_uint8))
        return S, int(steps)

    def distances(self, A, B) -> np.ndarray:
        A = np.ascontiguousarray(A, dtype=np.uint8).reshape(-1, self.nv)
        B = np.ascontiguousarray(B, dtype=np.uint8).reshape(-1, self.nv)
        D = np.zeros((A.shape[0], B.shape[0]), dtype=np.int32)
        self.lib.or_distances(self.h, _ptr(A, C.c_uint8), A.shape[0], _ptr(B, C.c_uint8),
                              B.shape[0], _ptr(D, C.c_int32))
        return D

    def pop_update(self, e, Dall, params=None):
        params = params or default_params()
        e = np.ascontiguousarray(e, dtype=np.int64)
        Dall = np.ascontiguousarray(Dall, dtype=np.int32)
        p = e.shape[0] // 2
        sel = np.zeros(p, dtype=np.int32)
        filled = self.lib.or_pop_update(self.h, C.byref(params), p, _ptr(e, C.c_int64),
                                        _ptr(Dall, C.c_int32), _ptr(sel, C.c_int32))
        return sel, int(filled)

    def matching(self, D, uid, tested, tcount, gen, seed, params=None):
        params = params or default_params()
        D = np.ascontiguousarray(D, dtype=np.int32)
        uid = np.ascontiguousarray(uid, dtype=np.uint32)
        tested = np.array(tested, dtype=np.uint32, copy=True, order="C")
        tcount = np.array(tcount, dtype=np.int32, copy=True, order="C")
        p = D.shape[0]
        partner = np.zeros(p, dtype=np.int32)
        self.lib.or_matching(self.h, C.byref(params), p, _ptr(D, C.c_int32),
                             _ptr(uid, C.c_uint32), _ptr(tested, C.c_uint32),
                             _ptr(tcount, C.c_int32), gen, seed, _ptr(partner, C.c_int32))
        return partner, tested, tcount

    def crossover(self, P, partner, D, gen, seed, params=None):
        params = params or default_params()
        P = np.ascontiguousarray(P, dtype=np.uint8)
        partner = np.ascontiguousarray(partner, dtype=np.int32)
        D = np.ascontiguousarray(D, dtype=np.int32)
        O = np.zeros_like(P)
        self.lib.or_crossover(self.h, C.byref(params), P.shape[0], _ptr(P, C.c_uint8),
                              _ptr(partner, C.c_int32), _ptr(D, C.c_int32), gen, seed,
                              _ptr(O, C.c_uint8))
        return O

    def solve(self, pop, generations, iters, seed, params=None):
        """Alg. 2.  Returns dict(best_grid, score, trace, generations, stats, final_pop)."""
        params = params or default_params()
        grid = np.zeros((self.n, self.n), dtype=np.int8)
        score = C.c_int32()
        trace = np.full(max(generations, 1), -1, dtype=np.int32)
        st = Stats()
        final = np.zeros((pop, max(self.nv, 1)), dtype=np.uint8)
        g = self.lib.or_solve(self.h, C.byref(params), pop, generations, int(iters), seed,
                              _ptr(grid, C.c_int8), C.byref(score), _ptr(trace, C.c_int32),
                              C.byref(st), _ptr(final, C.c_uint8))
        return {"best_grid": grid, "score": int(score.value), "trace": trace[:g],
                "generations": int(g), "stats": st.as_dict(), "final_pop": final[:, :self.nv]}
