// plse_handle.cuh -- host-side state behind a plse_handle (library-internal).
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include "plse_internal.cuh"
#include "plse_pop.cuh"

namespace plse {

struct SolverState;   // generation-loop buffers (solve.cu)

// device scratch of the local search, grown on demand and reused across calls
struct Workspace {
    uint32_t *G = nullptr;          // evicted tabu expiries, one table per walk slot
    size_t G_cap = 0;
    uint2 *TC = nullptr;            // two-entry tabu caches, one array per walk slot
    size_t TC_cap = 0;
    uint16_t *LIST = nullptr;       // candidate lists, one array per walk slot
    size_t LIST_cap = 0;
    uint16_t *XR = nullptr;         // member-id XOR tables, one per walk slot
    size_t XR_cap = 0;
    uint32_t *HP = nullptr;         // colour-count planes 2..6, one set per walk slot
    size_t HP_cap = 0;
    uint8_t *SW = nullptr;          // current colourings kept in global memory, one per walk slot
    size_t SW_cap = 0;
    uint32_t *slot_clock = nullptr; // per-slot clock
    size_t clock_cap = 0;
    int *counters = nullptr;        // [0] walk counter, [1] error flag, [2..] spare
    size_t counters_cap = 0;
};

// one resumable run of Alg. 2 (plse_run_begin / plse_run_step / plse_run_result)
struct Session {
    int active = 0, finished = 0;
    int pop = 0, max_gens = 0, gen = 0, cur = 0;
    int issued = 0;     // generations enqueued on the device
    int polled = 0;     // enqueued generations whose completion the host has seen
    int64_t iters = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    double ms_ls = 0;
    long long launches = 0;
    std::vector<float> ls_iv;   // per completed generation: local-search start, end (ms after run begin)
};

}  // namespace plse

struct plse_instance {
    int n = 0, nv = 0, l = 0, ub = 0, nfixed = 0;
    int device = 0;
    std::vector<int8_t> grid;
    std::vector<int32_t> cell;       // row-major cell of each reduced vertex
    std::vector<uint16_t> rc;
    std::vector<uint4> dom;
    std::vector<uint8_t> ndom;
    std::vector<int32_t> row_ptr, col_ptr;
    std::vector<uint16_t> row_v, col_v;
    std::vector<uint4> allow_row, allow_col;
    int ls_lanes = 0;                  // threads per walk of the local search (0 = automatic)
    int ls_walks = 0;                  // cap on concurrent walks per block (0 = fill shared memory)
    int ls_splace = 0;                 // colourings: 0 automatic, 1 shared memory, 2 global memory
    uint32_t alpha_recip = 0;          // reciprocal of alpha_den for the tenure (0: divide)
    plse_params params{};
    void *inst_mem = nullptr;        // one device allocation holding the DevInst arrays
    size_t inst_bytes = 0;
    plse::DevInst di{};
    plse::Workspace ws;
    plse::SolverState *solver = nullptr;
    plse::Session session;
    uint32_t *step_planes = nullptr;   // bit planes for the population step entry points
    size_t step_planes_cap = 0;
    plse::PopScratch step_ps;          // Alg. 4 scratch for plse_pop_update
    char *arena = nullptr;             // caller-bound device range (plse_bind_workspace), or null
    size_t arena_size = 0, arena_used = 0;
    int *noalloc_flag = nullptr;       // check flag of the last plse_local_search_noalloc call (in
                                       // the library's fixed scratch array), read by plse_sync
    cudaEvent_t done_ev = nullptr;     // recorded after the handle's latest enqueued work
    bool done_recorded = false;
    std::string err;
};

namespace plse {
int fail(plse_instance *h, int code, const char *fmt, ...);
int cuda_fail(plse_instance *h, cudaError_t e, const char *where);
int max_tenure(const plse_instance *h);
uint32_t tenure_reciprocal(int alpha_num, int alpha_den, int nv);
// per-slot strides of a launch's scratch for one instance alone
void set_ls_strides(const DevInst &I, LSArgs &a);
// arguments of a local-search launch on the handle's current workspace
LSArgs ls_args(plse_instance *h, const uint8_t *S_in, uint8_t *S_out, int count, int ind0, int gen, int64_t iters,
               uint64_t seed, int flags, int32_t *f_out, int64_t *F_out, plse_walk_stats *stats, const int *skip);
int ensure_ls_workspace(plse_instance *h, int slots, cudaStream_t st);
// the walk counter and the device check flag (read by plse_sync), allocated once
int ensure_counters(plse_instance *h, cudaStream_t st);
int enqueue_local_search(plse_instance *h, const uint8_t *S_in, uint8_t *S_out, int count, int ind0,
                         int gen, int64_t iters, uint64_t seed, int flags, int32_t *f_out,
                         int64_t *F_out, plse_walk_stats *stats, cudaStream_t st,
                         const int *skip = nullptr);
void release_solver(plse_instance *h, cudaStream_t st);

// device memory of handles (stream-ordered pool) and pinned flag slots (devmem.cu)
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t st);
void dev_free(void *p, cudaStream_t st);
// a handle's run and scratch buffers: carved from its bound workspace if it has
// one (256-byte aligned pieces, freed only as a whole), else from the pool
constexpr size_t kWsAlign = 256;
inline size_t ws_align(size_t bytes) { return (bytes + kWsAlign - 1) & ~(kWsAlign - 1); }
cudaError_t h_malloc(plse_instance *h, void **p, size_t bytes, cudaStream_t st);
void h_free(plse_instance *h, void *p, cudaStream_t st);
size_t solver_bytes(const plse_instance *h, int p, int gens);
size_t ls_workspace_bytes(const plse_instance *h, int slots);
void release_ls_workspace(plse_instance *h, cudaStream_t st);
int *pinned_slot_get();          // 16 bytes of pinned host memory, zeroed
void pinned_slot_put(int *slot);

// Orders work enqueued on st after the handle's earlier work (any stream) and
// records the handle's event after it; one per call that enqueues work.
struct StreamScope {
    plse_instance *h;
    cudaStream_t st;
    StreamScope(plse_instance *h, cudaStream_t st);
    ~StreamScope();
    StreamScope(const StreamScope &) = delete;
    StreamScope &operator=(const StreamScope &) = delete;
};

// resumable run of Alg. 2 (solve.cu).  run_issue enqueues one more generation
// when fewer than two are in flight (never waits); run_poll consumes completed
// generations (wait = block until every enqueued one completed); run_drain is
// run_poll(wait) when anything is in flight.
int run_begin(plse_instance *h, int pop, int max_generations, int64_t iters, uint64_t seed, cudaStream_t st);
int run_issue(plse_instance *h, int *issued);
int run_poll(plse_instance *h, bool wait);
int run_drain(plse_instance *h);
int run_step(plse_instance *h, int generations, cudaStream_t st, int *done_out);
// one generation of a run split around a local search launched by the caller
// (several runs' generations in one multi-instance launch): head fills the
// launch's arguments (the caller supplies the walk-slot scratch) and records the
// generation's start event (*ready) on the run's stream; tail, after the caller's
// launch (event ls_done), enqueues the rest of the generation on the run's
// stream.  A run with nothing left to issue (finished, generations used) is
// refused by head with PLSE_ENOTSUP.
int generation_head(plse_instance *h, LSArgs &a, cudaEvent_t *ready);
int generation_tail(plse_instance *h, cudaEvent_t ls_done);
int run_result(plse_instance *h, cudaStream_t st, int8_t *best_grid, int *best_score, plse_solve_stats *stats,
               int32_t *trace_out);
}  // namespace plse
