/*
 * plse.h -- C ABI of the GB300 (sm_103a) hot path of MPMA, the massively
 * parallel memetic algorithm for partial Latin square extension (PLSE) of
 * Goudet & Hao, arXiv 2103.10453.
 *
 * All compute runs in hand-written CUDA kernels inside libplse.so.  Signatures
 * use plain pointers and sizes only.  Unless stated otherwise:
 *   - "host" buffers are caller-owned CPU memory, read or written before the
 *     call returns;
 *   - "device" buffers are caller-owned GPU memory on the current device
 *     (e.g. torch tensors), accessed in stream order on `stream`;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *     calls taking a stream are asynchronous with respect to the host;
 *   - every call returns PLSE_OK (0) or a negative PLSE_E* code, and on error
 *     leaves outputs unspecified; plse_last_error_detail() explains the last
 *     error of a handle.
 *
 * Colourings are uint8 arrays [count][nv] (row-major by individual) over the
 * reduced vertices of the instance, in row-major cell order; colour 0 means
 * "uncoloured", colour k in 1..n means symbol k (Sec. 2.1).
 * Random numbers are Philox4x32-10 blocks keyed by `seed` with the counter
 * (iteration or vertex block, individual, generation<<8 | purpose<<4 | phase, 0),
 * so every result is a deterministic function of its arguments.
 */
#ifndef PLSE_H
#define PLSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes --------------------------------------------------------- */
#define PLSE_OK          0
#define PLSE_EINVAL     -1   /* invalid argument or invalid grid               */
#define PLSE_ENOMEM     -2   /* host or device allocation failed               */
#define PLSE_ECUDA      -3   /* CUDA runtime error                             */
#define PLSE_EBUSY      -4   /* admission refused (request queue full)         */
#define PLSE_ECANCELLED -5   /* cancelled through plse_server_cancel           */
#define PLSE_ENOTSUP    -6   /* parameter combination not supported            */
#define PLSE_ECHECK     -7   /* a device-side bound check failed               */
#define PLSE_PENDING     1   /* plse_server_poll: the request is not complete  */

typedef struct plse_instance *plse_handle;

/* Algorithm parameters: Table 1 of the paper and Sec. 3.3, as integers. */
typedef struct {
    int32_t alpha_num, alpha_den;  /* tabu tenure factor alpha = 6/10            */
    int32_t tenure_rand;           /* L uniform in [0, tenure_rand) = [0, 9]     */
    int32_t phase1_phi2;           /* 2*phi of phase 1 (phi = 0.5 -> 1)          */
    int32_t phase2_phi2_per_v;     /* 2*phi of phase 2 per |V| (phi = |V| -> 2)  */
    int32_t phase2_iter_per_v;     /* phase-2 iterations per |V| (2); at most    */
                                   /* 2^30 iterations in all (else PLSE_ENOTSUP) */
    int32_t spacing_gamma;         /* Alg. 4 spacing D > |V|/gamma (10)          */
    int32_t beta;                  /* AUX parameter beta (20)                    */
    int32_t mode;                  /* PLSE_MODE_PLITS, _PARTIALCOL or _AUTO      */
    int32_t matching;              /* PLSE_MATCH_NEAREST or PLSE_MATCH_RANDOM    */
    int32_t crossover;             /* PLSE_XOVER_AUX or PLSE_XOVER_UX            */
    int32_t tested_cap;            /* tested-partner list capacity, 1..256 (64)  */
    int32_t stop_at_bound;         /* 1: stop once f(S*) reaches the bound (Sec. 3.2);
                                      0: keep running the requested generations   */
} plse_params;

#define PLSE_MODE_PLITS       0    /* two-phase tabu search, Sec. 3.3            */
#define PLSE_MODE_PARTIALCOL  1    /* Partial-MPMA local search, Sec. 3.7        */
#define PLSE_MODE_AUTO        2    /* Partial-MPMA when at least 80% of the cells
                                      are prefilled (Sec. 3.7), else PLITS        */
#define PLSE_MATCH_NEAREST    0    /* nearest untested partner, Sec. 3.5.1       */
#define PLSE_MATCH_RANDOM     1    /* random partner (ablation of Sec. 5.3)      */
#define PLSE_XOVER_AUX        0    /* asymmetric uniform crossover, Eq. 10       */
#define PLSE_XOVER_UX         1    /* uniform crossover, p_ij = 1/2              */

/* Work counters of tabu walks (identical to the CPU oracle's on the same
 * trajectory): iterations executed, moves applied, sum of |V0 u C(S)| over
 * iterations, sum of scanned (v, j) pairs, sum of deg(v*) over moves,
 * strict improvements of the walk's best, neighbours uncoloured (PartialCol). */
typedef struct {
    int64_t iterations, moves, cand, pairs, deg, improvements, uncolored;
} plse_walk_stats;

typedef struct {
    int32_t generations;      /* generations executed (early stop at the bound) */
    int32_t best_f;           /* f(S*): uncoloured reduced vertices of S*       */
    plse_walk_stats walks;    /* summed over every walk of the run              */
    double  ms_total;         /* device time of the whole run (CUDA events)     */
    double  ms_local_search;  /* device time of the local-search launches       */
    int64_t launches;         /* kernels launched by the run                    */
} plse_solve_stats;

/* ---- instance -------------------------------------------------------------
 * plse_create -- Sec. 2.1-2.2, Alg. 1.  `grid`: host int8 [n*n], row-major,
 * 0 = empty cell, 1..n = prefilled symbol; copied, so the caller may free it on
 * return.  Validates 1 <= n <= 127, symbols in 0..n and no symbol twice in a
 * row or a column (partial Latin square, Sec. 1); PLSE_EINVAL otherwise.
 * Builds the reduced graph (empty cells with D(v) != {0}), the domains D(v),
 * l and the bound, and uploads them to the current device.  *out is written
 * only on success.  The handle is not thread-safe: one host thread at a time. */
int  plse_create(int n, const int8_t *grid, plse_handle *out);
/* Frees every host and device resource of `h`; NULL is accepted.  Device memory
 * goes back to the library's stream-ordered pool after the last work enqueued
 * for `h` (on any stream) has run; the call waits only for a run's generations
 * in flight, never for the whole device. */
void plse_destroy(plse_handle h);
/* Static description of an error code; never NULL. */
const char *plse_strerror(int code);
/* Copies the last error message of `h` (NUL-terminated, truncated to len). */
int  plse_last_error_detail(plse_handle h, char *buf, size_t len);
/* |V| (reduced vertices), l (cells removed by Alg. 1 because D = {0}) and the
 * upper bound n^2 - l, or n^2 - 2 when l = 1 (Sec. 2.2).  NULL outputs skipped. */
int  plse_info(plse_handle h, int *nv, int *l, int *ub);

/* Waits for `stream`, then reports PLSE_ECHECK (and clears the condition) if a
 * kernel of an earlier call on `h` failed one of its device-side consistency
 * checks; PLSE_OK otherwise. */
int  plse_sync(plse_handle h, void *stream);

/* ---- parameters ---------------------------------------------------------- */
/* Table 1 defaults: alpha 6/10, L in [0,9], phi 0.5 then |V| for 2|V|
 * iterations, gamma 10, beta 20, PLITS, nearest matching, AUX, 64 partners. */
void plse_default_params(plse_params *p);
int  plse_set_params(plse_handle h, const plse_params *p);
int  plse_get_params(plse_handle h, plse_params *p);

/* Launch knobs of the local-search kernel; they never change results.
 * ls_lanes: threads per walk, 16 (two walks share a warp), 32, 64, 128 or 256;
 * 0 = automatic.  ls_walks: cap on concurrent walks per block (0 = as many as
 * fit).  ls_colourings: where a walk's current colouring lives, 1 = shared
 * memory, 2 = global memory (frees shared memory for more walks), 0 =
 * automatic (shared memory unless that would cut the walks per block). */
int  plse_set_launch(plse_handle h, int ls_lanes, int ls_walks, int ls_colourings);

/* plse_autotune -- picks the launch knobs above for runs of `pop` individuals
 * on this handle's instance by timing short probe launches of the local search
 * (`probe_iters` phase-1 iterations on `pop` colourings, several candidate
 * shapes: threads per walk, walks per block, colouring placement), applies the
 * fastest to the handle and reports it (each output may be NULL; moves_per_s is
 * the probe's rate).  The choice is cached for the process per device, n, |V|
 * and pop, so later calls for the same shape return at once.  Results of every
 * call never depend on the knobs.  Uses device memory for two probe
 * populations (from the handle's allocator: its bound workspace, if any) and
 * waits for the device. */
int  plse_autotune(plse_handle h, int pop, int probe_iters, int *lanes, int *walks, int *colourings,
                   double *moves_per_s);

/* ---- caller-supplied device memory -------------------------------------------
 * plse_workspace_size: device bytes that a run of `pop` individuals and up to
 * `max_generations` generations (plse_run_begin / plse_solve) takes for its
 * population buffers, Alg. 4 scratch and local-search scratch, under the
 * handle's current parameters and launch knobs (0 for an instance with no
 * vertex left to colour).
 * plse_bind_workspace: from now on the handle carves those buffers (and the
 * scratch of the step entry points) out of the device range
 * [dev_ptr, dev_ptr + bytes) instead of the library's pool; e.g. a torch
 * tensor's memory.  The range is caller-owned: it must start on a 256-byte
 * boundary, be memory of the handle's device, and stay valid until it is
 * unbound, another is bound or the handle is destroyed.  The call waits for the
 * handle's work, releases its current buffers and discards its current run
 * (begin a new one).  Pieces are never returned to the range one by one: a
 * later call that needs more than is left (a larger run, more step scratch)
 * fails with PLSE_ENOMEM.  dev_ptr = NULL unbinds (buffers come from the pool
 * again).  The instance image uploaded by plse_create stays in the pool.
 * Results do not depend on where the memory comes from. */
int  plse_workspace_size(plse_handle h, int pop, int max_generations, size_t *bytes);
int  plse_bind_workspace(plse_handle h, void *dev_ptr, size_t bytes);

/* ---- whole solve (Alg. 2) ---------------------------------------------------
 * Runs `generations` generations of MPMA with population `pop` (2..65535) and
 * `iters` phase-1 tabu iterations (nbIter_TS of Sec. 3.3; phase 2 uses
 * phase2_iter_per_v*|V|), stopping early once the bound is reached (Sec. 3.2).
 * `best_grid`: host int8 [n*n] output = prefilled symbols + the best legal
 * colouring S* (0 for uncoloured and removed cells).  `best_score` = number of
 * filled cells = n^2 - l - f(S*).  Blocks until done.  Deterministic in
 * (instance, params, pop, generations, iters, seed). */
int  plse_solve(plse_handle h, int pop, int generations, int64_t iters, uint64_t seed,
                int8_t *best_grid, int *best_score);
/* As plse_solve, enqueued on `stream` (the call still blocks until the result is
 * on the host) and returning device-timed statistics in *stats (may be NULL). */
int  plse_solve_ex(plse_handle h, int pop, int generations, int64_t iters, uint64_t seed,
                   void *stream, int8_t *best_grid, int *best_score,
                   plse_solve_stats *stats);

/* ---- resumable run: the population stays resident on the device ----------
 * plse_run_begin initialises a run of Alg. 2 (population P_0, S* empty) with
 * room for `max_generations`; plse_run_step executes up to `generations` more
 * generations on `stream` (blocking; *done (may be NULL) is set once the run has
 * stopped at the bound or used its generations); plse_run_result copies the
 * best grid, score and statistics of the run so far.  plse_solve is
 * begin + step + result.  One run per handle at a time; a new begin discards
 * the previous run.  Every call of a run takes the stream given to
 * plse_run_begin (plse_run_step returns PLSE_EINVAL for another one). */
int  plse_run_begin(plse_handle h, int pop, int max_generations, int64_t iters, uint64_t seed,
                    void *stream);
int  plse_run_step(plse_handle h, int generations, void *stream, int *done);
int  plse_run_result(plse_handle h, void *stream, int8_t *best_grid, int *best_score,
                     plse_solve_stats *stats, int32_t *trace);

/* plse_run_population -- copies the run's current population P_t
 * (which = PLSE_RUN_POPULATION) or the offspring S^O that the next generation's
 * local search starts from (PLSE_RUN_OFFSPRING) into dst (device or host
 * uint8 [pop*nv]); waits for the run's generations in flight and for the copy.
 * The next generation (index = generations completed) runs plse_local_search
 * on S^O with ind0 = 0, gen = that index and the run's iters and seed. */
#define PLSE_RUN_POPULATION 0
#define PLSE_RUN_OFFSPRING  1
int  plse_run_population(plse_handle h, int which, uint8_t *dst, void *stream);

/* Non-blocking form of plse_run_step, for callers that drive several runs from
 * one host thread (each run on its own stream, so their kernels overlap).
 * plse_run_issue enqueues the run's next generation on `stream` (which must be
 * the stream given to plse_run_begin; PLSE_EINVAL otherwise) without waiting
 * for anything, unless the run has finished, has enqueued all its generations
 * or already has two generations in flight; *issued (may be NULL) says whether
 * it did.  plse_run_query never waits: it takes note of completed generations
 * and reports *done = 1 once the run has finished (bound reached or
 * generations used) and nothing of it is in flight, *generations = completed
 * generations and *in_flight = enqueued but not yet completed (each may be
 * NULL).  A generation enqueued before the host saw the stop returns at entry
 * in every kernel, so results equal those of plse_run_step.  plse_run_result
 * and plse_destroy wait for the generations in flight. */
int  plse_run_issue(plse_handle h, void *stream, int *issued);
int  plse_run_query(plse_handle h, int *done, int *generations, int *in_flight);

/* plse_run_timeline -- when each local-search launch of the run ran: for the
 * completed generations first .. first+count-1 (counted from plse_run_begin),
 * ls_start_end[2k], ls_start_end[2k+1] = start and end of generation
 * first+k's local-search launch, in milliseconds after `ref_event` (a
 * cudaEvent_t with timing that the caller recorded on the run's device before
 * calling plse_run_begin, and that has completed).  Lets a caller that
 * runs several runs at once measure the time during which any local search ran.
 * Waits for the run's enqueued generations; PLSE_EINVAL if a generation in the
 * range has not run or the event has not completed. */
int  plse_run_timeline(plse_handle h, void *ref_event, int first, int count, float *ls_start_end);

/* ---- many jobs at once ------------------------------------------------------
 * A job is one plse_solve: population, generations, phase-1 iterations, seed. */
typedef struct {
    int32_t  pop;             /* 2..65535                                       */
    int32_t  generations;     /* 0..65534                                       */
    int64_t  iters;           /* phase-1 tabu iterations, 0..2^30               */
    uint64_t seed;
} plse_job;

typedef struct {
    int32_t status;           /* PLSE_OK, or the job's own negative code        */
    int32_t best_score;       /* as plse_solve                                  */
    plse_solve_stats stats;   /* as plse_solve_ex                               */
    double  ms_queue;         /* host wall time from submission to the start    */
    double  ms_wall;          /* host wall time from submission to completion   */
    char    detail[128];      /* message of the job's error ("" on success)     */
    int64_t mem_bytes;        /* server: device bytes the request was admitted
                                 with (instance image + plse_workspace_size)    */
} plse_result;

/* plse_solve_batch -- runs job i on handle hs[i] (with that handle's
 * parameters).  Two ways to share the device:
 *   concurrent: up to `max_inflight` runs at a time (0 = 16), each on its own
 *     stream, each advancing at its own pace, their kernels overlapping on the
 *     current device; jobs naming the same handle run one after another;
 *   lockstep (max_inflight = PLSE_BATCH_LOCKSTEP, a handle per job): all runs
 *     advance one generation at a time, and the local searches of a generation
 *     run as one persistent launch per colour-word class (orders n below 32, 64,
 *     96, 128) whose walk groups take the runs' walks in turn, so one run's tail
 *     is filled with the next run's walks; the rest of each generation runs on
 *     the run's own stream.  A class whose first handle has automatic launch
 *     knobs gets them from plse_autotune on its largest instance (the handles
 *     keep them).  Every generation waits for the slowest run.
 * max_inflight = 0 means concurrent with 16 runs.  Runs of a batch (and of the
 * request server) share the device, so their Alg. 4 uses one kernel pair per
 * chunk of 128 candidates instead of the single cooperative launch of a run
 * alone, which would wait for every other run's kernels to leave the device.
 * best_grids (may be NULL, entries may be NULL): host int8
 * [n_i*n_i] outputs as plse_solve.  results: host [count].  Every job's result
 * equals that of plse_solve with the same arguments.  Blocks until every job is
 * done; returns the first job error (in index order) or PLSE_OK;
 * results[i].status holds each job's own code. */
#define PLSE_BATCH_LOCKSTEP (-1)
int  plse_solve_batch(plse_handle *hs, const plse_job *jobs, int count, int max_inflight,
                      int8_t *const *best_grids, plse_result *results);

/* Request server: a host thread of the library that admits submitted requests
 * (grid + job + parameters) into at most `max_inflight` concurrent runs on the
 * device that is current at plse_server_create, in arrival order, and keeps
 * each result until it is polled.  Admission is by device memory: the request
 * at the head of the queue has its handle built (host work and the small
 * instance upload), its footprint computed (instance image + plse_workspace_size
 * of its run), and starts once a run slot is free and the footprint fits in
 * `mem_budget` minus the footprints of the runs in progress (0 = 90% of the
 * device memory free at creation); a run's bytes return to the budget when it
 * completes.  A request whose footprint alone exceeds the budget completes with
 * PLSE_ENOMEM.  Per-request results are identical to plse_solve of the same
 * request alone (the job's size never depends on load).
 *   submit: copies `grid` (n*n) and `params` (NULL = defaults); returns a
 *     ticket, or PLSE_EBUSY when `max_queue` requests already wait (admission
 *     refused; nothing is queued), PLSE_EINVAL for a malformed request (grids
 *     are validated at admission: a bad one completes with PLSE_EINVAL).
 *   poll: waits up to wait_ms (0 = not at all, -1 = until done); PLSE_PENDING
 *     if the request is not complete, else PLSE_OK with *out and best_grid
 *     (host n*n, may be NULL) written and the ticket released; PLSE_EINVAL for
 *     an unknown or released ticket.
 *   cancel: a waiting request completes with PLSE_ECANCELLED without running;
 *     a running one stops enqueueing generations and completes with
 *     PLSE_ECANCELLED and its best so far once its generations in flight end.
 *   pending: requests waiting for admission and results not yet polled.
 *   memory: the budget, bytes held by running requests now, the peak of that,
 *     the peak number of concurrent runs, and how many admissions had to wait
 *     for memory (each output may be NULL).
 *   destroy: cancels what is waiting or running, joins the threads, frees all.
 * Every call except destroy may come from any host thread at any time; destroy
 * must not overlap another call on the same server. */
typedef struct plse_server_s *plse_server;
int  plse_server_create(int max_inflight, int max_queue, size_t mem_budget, plse_server *out);
int  plse_server_submit(plse_server s, int n, const int8_t *grid, const plse_job *job,
                        const plse_params *params, int64_t *ticket);
int  plse_server_poll(plse_server s, int64_t ticket, int wait_ms, int8_t *best_grid,
                      plse_result *out);
int  plse_server_cancel(plse_server s, int64_t ticket);
int  plse_server_pending(plse_server s, int *queued, int *completed);
int  plse_server_memory(plse_server s, size_t *budget, size_t *in_use, size_t *peak, int *peak_running,
                        int64_t *waited);
/* Launch knobs (as plse_set_launch) for the handles of requests admitted from
 * now on; they never change results. */
int  plse_server_set_launch(plse_server s, int ls_lanes, int ls_walks, int ls_colourings);
void plse_server_destroy(plse_server s);

/* ---- step entry points (device buffers, asynchronous on `stream`) ---------
 * plse_init_population -- Sec. 3.2: P[i][v] uniform over D(v)\{0}, individual
 * index i for i < pop.  P: device uint8 [pop*nv]. */
int  plse_init_population(plse_handle h, int pop, uint64_t seed, uint8_t *P, void *stream);

/* plse_local_search -- Alg. 3 on `count` colourings.  S_in / S_out: device
 * uint8 [count*nv] (may alias).  Walk w uses individual index ind0 + w and
 * generation `gen` for its Philox draws.  flags: PLSE_LS_PHASE1 runs
 * `iters` iterations with phi = 0.5 (Sec. 3.3); PLSE_LS_PHASE2 then runs
 * phase2_iter_per_v*|V| iterations with phi = |V| from the phase-1 best;
 * PLSE_LS_REPAIR then applies the greedy conflict removal of Sec. 3.7;
 * PLSE_LS_PARTIALCOL (alone or with REPAIR first) runs the PartialCol tabu
 * search of Sec. 3.7 for `iters` iterations on a legal colouring.
 * Outputs: S_out = best colouring (S'*); f_out (device int32 [count] or NULL)
 * = uncoloured vertices of S_out; F_out (device int64 [count] or NULL) = best
 * value of the last phase run (2F for PLITS, f for PartialCol); stats (device
 * plse_walk_stats [count] or NULL) = per-walk counters summed over phases.
 * PLSE_ECHECK if a walk's device bound check failed (the walk's output is then
 * unspecified).  Uses internal device scratch (tabu overflow tables). */
#define PLSE_LS_PHASE1      1
#define PLSE_LS_PHASE2      2
#define PLSE_LS_REPAIR      4
#define PLSE_LS_PARTIALCOL  8
int  plse_local_search(plse_handle h, const uint8_t *S_in, uint8_t *S_out, int count,
                       int ind0, int gen, int64_t iters, uint64_t seed, int flags,
                       int32_t *f_out, int64_t *F_out, plse_walk_stats *stats, void *stream);

/* plse_local_search_noalloc -- plse_local_search for callers that cannot
 * allocate device memory at call time (an application whose device memory is
 * reserved up front by its own pool allocator, or a latency-critical loop that
 * must not pay the implicit device-wide synchronisation of cudaMalloc/cudaFree).
 * The paper has no counterpart: this is a deployment variant only.  Same
 * arguments, outputs and results as plse_local_search; it calls no cudaMalloc,
 * cudaFree or allocating routine.  Its scratch is a fixed 16 MiB array inside
 * the library on every GPU that loads it (held until exit).  Each concurrent
 * walk needs 4*|V|*n1p + 10*|V| + 4*n*n1p + 64*n*cw + 4 bytes of it
 * (n1p = n + 1 rounded up to a multiple of 4, cw = 32-colour words of n + 1
 * colours), so fewer walks run at once than in plse_local_search on large
 * instances (15 at n = 70, r = 0.3), with the same results.  PLSE_ENOTSUP if
 * not even one walk fits.  The first call on a device looks up the array's
 * device address (with that device current); make that first call before any
 * stream capture.  Calls share the array: each clears the part it uses, and
 * calls whose work overlaps on the GPU (e.g. on two streams) race.  A failed
 * device-side check is reported as PLSE_ECHECK by plse_sync on the calling
 * handle, as for plse_local_search, provided that no later call of this entry
 * point (which clears the flag) was made first. */
int  plse_local_search_noalloc(plse_handle h, const uint8_t *S_in, uint8_t *S_out, int count,
                               int ind0, int gen, int64_t iters, uint64_t seed, int flags,
                               int32_t *f_out, int64_t *F_out, plse_walk_stats *stats,
                               void *stream);

/* plse_distances -- Sec. 3.4, Eq. 9: D[a*nb + b] = #v with A_a(v) != B_b(v).
 * A: device uint8 [na*nv], B: device uint8 [nb*nv], D: device int32 [na*nb]. */
int  plse_distances(plse_handle h, const uint8_t *A, int na, const uint8_t *B, int nb,
                    int32_t *D, void *stream);

/* plse_pop_update -- Alg. 4 over P_all = Pall[0..2p-1] (P_t first, then P'):
 * ranks by (e, index), accepts greedily with spacing gamma*min D > |V|, fills
 * from rejected candidates in rank order if P_all runs out.  Pall: device
 * uint8 [2p*nv]; e: device int64 [2p] (ranking score, e.g. f + |V|*c);
 * sel: device int32 [p] receives the chosen indices in acceptance order;
 * filled (device int32 [1] or NULL): places taken by the fill rule.
 * Distances are computed on the fly; nothing p x p is materialised. */
int  plse_pop_update(plse_handle h, int p, const uint8_t *Pall, const int64_t *e,
                     int32_t *sel, int32_t *filled, void *stream);

/* plse_matching -- Sec. 3.5.1 / Alg. 5: partner[i] = nearest j != i (Hamming)
 * whose uid is not in i's tested list (lowest index on ties; plain nearest if
 * every partner was tested), or a random j != i with PLSE_MATCH_RANDOM.
 * P: device uint8 [p*nv]; uid: device uint32 [p]; tested: device uint32
 * [p*tested_cap] and tcount: device int32 [p] (updated in place: the partner's
 * uid is appended, the oldest entry dropped when full; untouched for random
 * matching); partner, dist: device int32 [p] (dist = D(i, partner)). */
int  plse_matching(plse_handle h, int p, const uint8_t *P, const uint32_t *uid,
                   uint32_t *tested, int32_t *tcount, int gen, uint64_t seed,
                   int32_t *partner, int32_t *dist, void *stream);

/* plse_crossover -- Eq. 10 / Alg. 5: O[i](v) = P[i](v) with probability
 * p_ij = 1 - |V|/(beta*dist[i]) (clamped at 0; 1/2 for UX), else
 * P[partner[i]](v).  P, O: device uint8 [p*nv] (must not alias);
 * partner, dist: device int32 [p]. */
int  plse_crossover(plse_handle h, int p, const uint8_t *P, const int32_t *partner,
                    const int32_t *dist, int gen, uint64_t seed, uint8_t *O, void *stream);

/* ---- diagnostics -------------------------------------------------------------
 * plse_smem_bandwidth -- measures the shared-memory load bandwidth of the
 * current device (conflict-free 16-byte loads by two blocks of 1024 threads per
 * SM, `iters` rounds of four loads per thread, timed by CUDA events); writes
 * bytes/s (and the kernel's milliseconds, may be NULL).  The peak against which
 * the local search's byte rate is reported; the paper has no counterpart. */
int  plse_smem_bandwidth(int iters, double *bytes_per_s, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* PLSE_H */
