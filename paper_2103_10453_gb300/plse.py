"""Thin ctypes binding of libplse.so (the C ABI in include/plse.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their ``data_ptr()`` is passed
through); streams are torch streams (``torch.cuda.current_stream()`` by
default).  If the library or a GPU is missing, calls raise ``PlseError``: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libplse.so")

PLSE_OK, PLSE_EINVAL, PLSE_ENOMEM, PLSE_ECUDA = 0, -1, -2, -3
PLSE_EBUSY, PLSE_ECANCELLED, PLSE_ENOTSUP, PLSE_ECHECK = -4, -5, -6, -7
PLSE_PENDING = 1
LS_PHASE1, LS_PHASE2, LS_REPAIR, LS_PARTIALCOL = 1, 2, 4, 8
MODE_PLITS, MODE_PARTIALCOL, MODE_AUTO = 0, 1, 2
MATCH_NEAREST, MATCH_RANDOM = 0, 1
XOVER_AUX, XOVER_UX = 0, 1


class PlseError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__("%s (%d)%s" % (_strerror(code), code, (": " + msg) if msg else ""))
        self.code = code


class Params(C.Structure):
    _fields_ = [(name, C.c_int32) for name in (
        "alpha_num", "alpha_den", "tenure_rand", "phase1_phi2", "phase2_phi2_per_v",
        "phase2_iter_per_v", "spacing_gamma", "beta", "mode", "matching", "crossover",
        "tested_cap", "stop_at_bound")]


class WalkStats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in (
        "iterations", "moves", "cand", "pairs", "deg", "improvements", "uncolored")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


WALK_STATS_FIELDS = [k for k, _ in WalkStats._fields_]


class SolveStats(C.Structure):
    _fields_ = [("generations", C.c_int32), ("best_f", C.c_int32), ("walks", WalkStats),
                ("ms_total", C.c_double), ("ms_local_search", C.c_double), ("launches", C.c_int64)]


class Job(C.Structure):
    _fields_ = [("pop", C.c_int32), ("generations", C.c_int32), ("iters", C.c_int64), ("seed", C.c_uint64)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("best_score", C.c_int32), ("stats", SolveStats),
                ("ms_queue", C.c_double), ("ms_wall", C.c_double), ("detail", C.c_char * 128),
                ("mem_bytes", C.c_int64)]

    def as_dict(self):
        st = self.stats
        return {"status": int(self.status), "score": int(self.best_score),
                "generations": int(st.generations), "best_f": int(st.best_f),
                "walks": st.walks.as_dict(), "ms_total": float(st.ms_total),
                "ms_local_search": float(st.ms_local_search), "launches": int(st.launches),
                "ms_queue": float(self.ms_queue), "ms_wall": float(self.ms_wall),
                "detail": self.detail.decode(errors="replace"), "mem_bytes": int(self.mem_bytes)}


_lib = None

# exported C symbols and their (restype, argtypes)
_vp, _i32, _i64, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
SIGNATURES = {
    "plse_create": (C.c_int, [C.c_int, _vp, C.POINTER(_vp)]),
    "plse_destroy": (None, [_vp]),
    "plse_strerror": (C.c_char_p, [C.c_int]),
    "plse_last_error_detail": (C.c_int, [_vp, C.c_char_p, C.c_size_t]),
    "plse_info": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "plse_sync": (C.c_int, [_vp, _vp]),
    "plse_smem_bandwidth": (C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "plse_autotune": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "plse_workspace_size": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "plse_bind_workspace": (C.c_int, [_vp, _vp, C.c_size_t]),
    "plse_set_launch": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "plse_run_timeline": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.POINTER(C.c_float)]),
    "plse_default_params": (None, [C.POINTER(Params)]),
    "plse_set_params": (C.c_int, [_vp, C.POINTER(Params)]),
    "plse_get_params": (C.c_int, [_vp, C.POINTER(Params)]),
    "plse_solve": (C.c_int, [_vp, C.c_int, C.c_int, _i64, _u64, _vp, C.POINTER(C.c_int)]),
    "plse_solve_ex": (C.c_int, [_vp, C.c_int, C.c_int, _i64, _u64, _vp, _vp, C.POINTER(C.c_int),
                                C.POINTER(SolveStats)]),
    "plse_run_begin": (C.c_int, [_vp, C.c_int, C.c_int, _i64, _u64, _vp]),
    "plse_run_step": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(C.c_int)]),
    "plse_run_result": (C.c_int, [_vp, _vp, _vp, C.POINTER(C.c_int), C.POINTER(SolveStats), _vp]),
    "plse_run_issue": (C.c_int, [_vp, _vp, C.POINTER(C.c_int)]),
    "plse_run_population": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "plse_run_query": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "plse_solve_batch": (C.c_int, [C.POINTER(_vp), C.POINTER(Job), C.c_int, C.c_int, C.POINTER(_vp),
                                   C.POINTER(Result)]),
    "plse_server_create": (C.c_int, [C.c_int, C.c_int, C.c_size_t, C.POINTER(_vp)]),
    "plse_server_memory": (C.c_int, [_vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                     C.POINTER(C.c_size_t), C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "plse_server_submit": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(Job), C.POINTER(Params),
                                     C.POINTER(C.c_int64)]),
    "plse_server_poll": (C.c_int, [_vp, C.c_int64, C.c_int, _vp, C.POINTER(Result)]),
    "plse_server_cancel": (C.c_int, [_vp, C.c_int64]),
    "plse_server_pending": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "plse_server_set_launch": (C.c_int, [_vp, C.c_int, C.c_int, C.c_int]),
    "plse_server_destroy": (None, [_vp]),
    "plse_init_population": (C.c_int, [_vp, C.c_int, _u64, _vp, _vp]),
    "plse_local_search": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _i64, _u64, C.c_int,
                                    _vp, _vp, _vp, _vp]),
    "plse_local_search_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, C.c_int, _i64, _u64,
                                            C.c_int, _vp, _vp, _vp, _vp]),
    "plse_distances": (C.c_int, [_vp, _vp, C.c_int, _vp, C.c_int, _vp, _vp]),
    "plse_pop_update": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, _vp]),
    "plse_matching": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, _vp, C.c_int, _u64, _vp, _vp, _vp]),
    "plse_crossover": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int, _u64, _vp, _vp]),
}


def load(path: str = LIB_PATH):
    """Opens libplse.so (built by ``paper_2103_10453_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise PlseError(PLSE_ENOTSUP, "libplse.so not built (run __graft_entry__.build())")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _strerror(code):
    try:
        return load().plse_strerror(code).decode()
    except Exception:
        return "error"


def default_params(**overrides) -> Params:
    p = Params()
    load().plse_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, int(v))
    return p


def _dptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise PlseError(PLSE_EINVAL, "expected a CUDA tensor")
    if not t.is_contiguous():
        raise PlseError(PLSE_EINVAL, "expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Instance:
    """A PLSE instance on the GPU (``plse_create``)."""

    def __init__(self, grid):
        grid = np.ascontiguousarray(grid, dtype=np.int8)
        if grid.ndim != 2 or grid.shape[0] != grid.shape[1]:
            raise PlseError(PLSE_EINVAL, "grid must be square")
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.plse_create(grid.shape[0], grid.ctypes.data, C.byref(h))
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_create")
        self.h = h
        nv, l, ub = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.plse_info(self.h, C.byref(nv), C.byref(l), C.byref(ub)))
        self.n, self.nv, self.l, self.ub = grid.shape[0], nv.value, l.value, ub.value
        self.grid = grid.copy()

    def close(self):
        if getattr(self, "h", None):
            self.lib.plse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != PLSE_OK:
            buf = C.create_string_buffer(512)
            if getattr(self, "h", None):
                self.lib.plse_last_error_detail(self.h, buf, 512)
            raise PlseError(rc, buf.value.decode())

    # ---- parameters ------------------------------------------------------
    def set_params(self, params: Params):
        self._check(self.lib.plse_set_params(self.h, C.byref(params)))

    def get_params(self) -> Params:
        p = Params()
        self._check(self.lib.plse_get_params(self.h, C.byref(p)))
        return p

    def set_launch(self, ls_lanes: int = 0, ls_walks: int = 0, ls_colourings: int = 0):
        """Threads per walk, walks per block and colouring placement of the
        local-search kernel (results do not depend on them)."""
        self._check(self.lib.plse_set_launch(self.h, ls_lanes, ls_walks, ls_colourings))

    def sync(self, stream=None):
        self._check(self.lib.plse_sync(self.h, _stream(stream)))

    def autotune(self, pop: int, probe_iters: int = 200):
        """Times probe launches and applies the fastest local-search launch knobs
        for runs of ``pop`` individuals (plse_autotune); returns
        (lanes, walks, colourings, probe moves/s)."""
        l, w, c, r = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        self._check(self.lib.plse_autotune(self.h, pop, probe_iters, C.byref(l), C.byref(w), C.byref(c),
                                           C.byref(r)))
        return l.value, w.value, c.value, r.value

    # ---- caller-supplied device memory ------------------------------------
    def workspace_size(self, pop: int, max_generations: int) -> int:
        """Device bytes a run of ``pop`` individuals and ``max_generations``
        generations takes (plse_workspace_size)."""
        out = C.c_size_t(0)
        self._check(self.lib.plse_workspace_size(self.h, pop, max_generations, C.byref(out)))
        return int(out.value)

    def bind_workspace(self, buf=None, nbytes=None):
        """Carves the handle's run and scratch buffers out of ``buf`` (a CUDA
        tensor, kept alive by the caller) instead of the library's pool; None
        unbinds (plse_bind_workspace)."""
        if buf is None:
            self._check(self.lib.plse_bind_workspace(self.h, None, 0))
            return
        nbytes = buf.numel() * buf.element_size() if nbytes is None else nbytes
        self._check(self.lib.plse_bind_workspace(self.h, C.c_void_p(buf.data_ptr()), nbytes))

    # ---- whole solve -----------------------------------------------------
    def solve(self, pop, generations, iters, seed, stream=None, with_stats=False):
        grid = np.zeros((self.n, self.n), dtype=np.int8)
        score = C.c_int()
        st = SolveStats()
        self._check(self.lib.plse_solve_ex(self.h, pop, generations, int(iters), seed,
                                           _stream(stream), grid.ctypes.data, C.byref(score),
                                           C.byref(st)))
        out = {"best_grid": grid, "score": int(score.value)}
        if with_stats:
            out.update(generations=int(st.generations), best_f=int(st.best_f),
                       walks=st.walks.as_dict(), ms_total=float(st.ms_total),
                       ms_local_search=float(st.ms_local_search), launches=int(st.launches))
        return out

    # ---- resumable run ---------------------------------------------------
    def run_begin(self, pop, max_generations, iters, seed, stream=None):
        self._check(self.lib.plse_run_begin(self.h, pop, max_generations, int(iters), seed, _stream(stream)))
        self._run_pop = pop

    def run_step(self, generations=1, stream=None) -> bool:
        done = C.c_int()
        self._check(self.lib.plse_run_step(self.h, generations, _stream(stream), C.byref(done)))
        return bool(done.value)

    def run_population(self, which=1, out=None, stream=None):
        """The run's population P_t (which=0) or its next offspring S^O (which=1)
        as a host array [pop, nv], or copied into the CUDA tensor ``out``."""
        pop = self._run_pop
        if out is None:
            buf = np.zeros((pop, max(self.nv, 1)), dtype=np.uint8)
            self._check(self.lib.plse_run_population(self.h, which, buf.ctypes.data, _stream(stream)))
            return buf[:, :self.nv]
        self._check(self.lib.plse_run_population(self.h, which, C.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def run_issue(self, stream=None) -> bool:
        """Enqueues the run's next generation without waiting (plse_run_issue)."""
        issued = C.c_int()
        self._check(self.lib.plse_run_issue(self.h, _stream(stream), C.byref(issued)))
        return bool(issued.value)

    def run_query(self):
        """(done, completed generations, generations in flight), never waits."""
        done, gens, inflight = C.c_int(), C.c_int(), C.c_int()
        self._check(self.lib.plse_run_query(self.h, C.byref(done), C.byref(gens), C.byref(inflight)))
        return bool(done.value), int(gens.value), int(inflight.value)

    def run_timeline(self, ref_event, first, count):
        """plse_run_timeline: [count, 2] float array, start and end (ms after the
        completed torch.cuda.Event ``ref_event``) of the local-search launches of
        generations first .. first+count-1."""
        out = np.zeros((max(count, 1), 2), dtype=np.float32)
        self._check(self.lib.plse_run_timeline(self.h, C.c_void_p(ref_event.cuda_event), first, count,
                                               out.ctypes.data_as(C.POINTER(C.c_float))))
        return out[:count]

    def run_result(self, stream=None, trace=False):
        grid = np.zeros((self.n, self.n), dtype=np.int8)
        score = C.c_int()
        st = SolveStats()
        tr = np.zeros(65535, dtype=np.int32) if trace else None
        self._check(self.lib.plse_run_result(self.h, _stream(stream), grid.ctypes.data, C.byref(score),
                                             C.byref(st), tr.ctypes.data if trace else None))
        out = {"best_grid": grid, "score": int(score.value), "generations": int(st.generations),
               "best_f": int(st.best_f), "walks": st.walks.as_dict(), "ms_total": float(st.ms_total),
               "ms_local_search": float(st.ms_local_search), "launches": int(st.launches)}
        if trace:
            out["trace"] = tr[:st.generations].copy()
        return out

    # ---- steps (device tensors) ------------------------------------------
    def init_population(self, pop, seed, out, stream=None):
        self._check(self.lib.plse_init_population(self.h, pop, seed, _dptr(out), _stream(stream)))
        return out

    def local_search(self, S_in, S_out, count, ind0, gen, iters, seed, flags,
                     f_out=None, F_out=None, stats=None, stream=None):
        self._check(self.lib.plse_local_search(
            self.h, _dptr(S_in), _dptr(S_out), count, ind0, gen, int(iters), seed, flags,
            _dptr(f_out), _dptr(F_out), _dptr(stats), _stream(stream)))

    def local_search_noalloc(self, S_in, S_out, count, ind0, gen, iters, seed, flags,
                             f_out=None, F_out=None, stats=None, stream=None):
        """As local_search, with the library's fixed scratch array instead of
        device memory allocated at call time (for callers that cannot allocate)."""
        self._check(self.lib.plse_local_search_noalloc(
            self.h, _dptr(S_in), _dptr(S_out), count, ind0, gen, int(iters), seed, flags,
            _dptr(f_out), _dptr(F_out), _dptr(stats), _stream(stream)))

    def distances(self, A, na, B, nb, D, stream=None):
        self._check(self.lib.plse_distances(self.h, _dptr(A), na, _dptr(B), nb, _dptr(D),
                                            _stream(stream)))

    def pop_update(self, p, Pall, e, sel, filled=None, stream=None):
        self._check(self.lib.plse_pop_update(self.h, p, _dptr(Pall), _dptr(e), _dptr(sel),
                                             _dptr(filled), _stream(stream)))

    def matching(self, p, P, uid, tested, tcount, gen, seed, partner, dist, stream=None):
        self._check(self.lib.plse_matching(self.h, p, _dptr(P), _dptr(uid), _dptr(tested),
                                           _dptr(tcount), gen, seed, _dptr(partner), _dptr(dist),
                                           _stream(stream)))

    def crossover(self, p, P, partner, dist, gen, seed, O, stream=None):
        self._check(self.lib.plse_crossover(self.h, p, _dptr(P), _dptr(partner), _dptr(dist),
                                            gen, seed, _dptr(O), _stream(stream)))


def _job(pop, generations, iters, seed):
    return Job(int(pop), int(generations), int(iters), int(seed))


def smem_bandwidth(iters=4096):
    """Measured shared-memory load bandwidth of the current device in bytes/s
    (plse_smem_bandwidth) and the probe's milliseconds."""
    lib = load()
    bw, ms = C.c_double(), C.c_double()
    rc = lib.plse_smem_bandwidth(int(iters), C.byref(bw), C.byref(ms))
    if rc != PLSE_OK:
        raise PlseError(rc, "plse_smem_bandwidth")
    return bw.value, ms.value


PLSE_BATCH_LOCKSTEP = -1


def solve_batch(instances, jobs, max_inflight=0, lockstep=False):
    """plse_solve_batch: job i = (pop, generations, iters, seed) on instances[i];
    lockstep=True asks for one multi-instance local-search launch per generation
    (max_inflight = PLSE_BATCH_LOCKSTEP).  Returns (list of result dicts with
    'best_grid', first error code)."""
    if lockstep:
        max_inflight = PLSE_BATCH_LOCKSTEP
    count = len(instances)
    lib = load()
    hs = (_vp * count)(*[inst.h for inst in instances])
    js = (Job * count)(*[_job(*j) for j in jobs])
    grids = [np.zeros((inst.n, inst.n), dtype=np.int8) for inst in instances]
    gp = (_vp * count)(*[g.ctypes.data for g in grids])
    res = (Result * count)()
    rc = lib.plse_solve_batch(hs, js, count, max_inflight, gp, res)
    out = []
    for i in range(count):
        d = res[i].as_dict()
        d["best_grid"] = grids[i]
        out.append(d)
    return out, rc


class Server:
    """plse_server_*: requests admitted into at most `max_inflight` concurrent
    runs on the current device while their device memory fits `mem_budget`
    bytes (0: 90% of the free memory at creation), served by the library's own
    host thread."""

    def __init__(self, max_inflight=8, max_queue=1024, mem_budget=0):
        self.lib = load()
        h = C.c_void_p()
        rc = self.lib.plse_server_create(max_inflight, max_queue, int(mem_budget), C.byref(h))
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_create")
        self.h = h
        self.sizes = {}

    def submit(self, grid, pop, generations, iters, seed, params=None):
        """Returns a ticket, or raises PlseError(PLSE_EBUSY) when the queue is full."""
        grid = np.ascontiguousarray(grid, dtype=np.int8)
        t = C.c_int64()
        job = _job(pop, generations, iters, seed)
        rc = self.lib.plse_server_submit(self.h, grid.shape[0], grid.ctypes.data, C.byref(job),
                                         C.byref(params) if params is not None else None, C.byref(t))
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_submit")
        self.sizes[t.value] = grid.shape[0]
        return t.value

    def poll(self, ticket, wait_ms=0):
        """None while pending, else the result dict (with 'best_grid')."""
        n = self.sizes.get(ticket, 1)
        grid = np.zeros((n, n), dtype=np.int8)
        res = Result()
        rc = self.lib.plse_server_poll(self.h, ticket, int(wait_ms), grid.ctypes.data, C.byref(res))
        if rc == PLSE_PENDING:
            return None
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_poll")
        self.sizes.pop(ticket, None)
        d = res.as_dict()
        d["best_grid"] = grid
        return d

    def memory(self):
        """Admission by device memory: budget, bytes held now, peak bytes held,
        peak concurrent runs, admissions that waited for memory."""
        b, u, pk = C.c_size_t(), C.c_size_t(), C.c_size_t()
        pr, w = C.c_int(), C.c_int64()
        rc = self.lib.plse_server_memory(self.h, C.byref(b), C.byref(u), C.byref(pk), C.byref(pr), C.byref(w))
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_memory")
        return {"budget": b.value, "in_use": u.value, "peak": pk.value, "peak_running": pr.value,
                "waited_for_memory": w.value}

    def cancel(self, ticket):
        rc = self.lib.plse_server_cancel(self.h, ticket)
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_cancel")

    def set_launch(self, ls_lanes=0, ls_walks=0, ls_colourings=0):
        rc = self.lib.plse_server_set_launch(self.h, ls_lanes, ls_walks, ls_colourings)
        if rc != PLSE_OK:
            raise PlseError(rc, "plse_server_set_launch")

    def pending(self):
        q, c = C.c_int(), C.c_int()
        self.lib.plse_server_pending(self.h, C.byref(q), C.byref(c))
        return int(q.value), int(c.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.plse_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
