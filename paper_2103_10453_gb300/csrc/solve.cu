// solve.cu -- the generation loop of MPMA (Alg. 2) on one GPU, its bookkeeping
// kernels (initial evaluation, best-solution update, population gather) and the
// population-level step entry points of the C ABI.
//
// Per generation, all on one stream and all on the device:
//   local search of the offspring S^O -> P'          (Alg. 3 twice + repair)
//   best update S* / f*, optimality flag              (Alg. 2)
//   bit planes of P', Alg. 4 over P_t u P' -> P_{t+1} (distances on the fly)
//   gather P_{t+1} (colourings, planes, scores, uids, tested lists)
//   matching + AUX -> next S^O                        (Alg. 5)
// Once the bound is reached every later kernel of the run returns at entry, so
// the host only reads the 4-byte flag once per generation.
#include <algorithm>
#include <climits>
#include <cstring>

#include "plse_handle.cuh"
#include "plse_pop.cuh"

namespace plse {

// generations of one run that may be enqueued before the host has seen the
// first of them complete
constexpr int kGenDepth = 2;

struct Ctrl {
    int fstar;      // f(S*)
    int done;       // bound reached: later kernels return at entry
    int gens;       // generations executed
    int pad;
    long long stats[7];   // summed plse_walk_stats of every walk
};

struct SolverState {
    int cap_p = 0, cap_gens = 0;
    uint8_t *Pall[2] = {nullptr, nullptr};   // [2p][nv]: P_t then P'
    uint32_t *planes[2] = {nullptr, nullptr};// [2p][nw*nb]
    int64_t *e[2] = {nullptr, nullptr};      // [2p]
    uint32_t *uid[2] = {nullptr, nullptr};   // [p]
    uint32_t *tested[2] = {nullptr, nullptr};// [p][cap]
    int32_t *tcount[2] = {nullptr, nullptr}; // [p]
    int tested_cap = 0;
    uint8_t *SO = nullptr;                   // [p][nv] offspring
    int32_t *fprime = nullptr, *sel = nullptr, *partner = nullptr, *dist = nullptr;
    plse_walk_stats *wstats = nullptr;
    PopScratch ps;
    Ctrl *ctrl = nullptr;
    uint8_t *Sstar = nullptr;
    int32_t *trace = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // per in-flight generation: local search begin / end, flag copied to the host
    cudaEvent_t gev[kGenDepth][3] = {};
    int *hflag = nullptr;                    // pinned host [kGenDepth][2]: f*, done
};

namespace {

constexpr unsigned FULL = 0xffffffffu;

// f and c of each colouring (Eq. 1, 3), ranking score e = f + |V| c (one warp each)
__global__ void __launch_bounds__(32) eval_kernel(const DevInst I, const uint8_t *P, int count, int64_t *e)
{
    extern __shared__ __align__(16) uint8_t cnt[];   // R then K, n x n1p each
    const int lane = threadIdx.x;
    for (int x = blockIdx.x; x < count; x += gridDim.x) {
        const uint8_t *S = P + (size_t)x * I.nv;
        uint32_t *w32 = reinterpret_cast<uint32_t *>(cnt);
        for (int q = lane; q < (2 * I.n * I.n1p) / 4; q += 32) w32[q] = 0u;
        __syncwarp();
        for (int r = lane; r < I.n; r += 32) {
            for (int q = I.row_ptr[r]; q < I.row_ptr[r + 1]; ++q) {
                const int k = S[I.row_v[q]];
                if (k) cnt[r * I.n1p + k] += 1;
            }
            for (int q = I.col_ptr[r]; q < I.col_ptr[r + 1]; ++q) {
                const int k = S[I.col_v[q]];
                if (k) cnt[I.n * I.n1p + r * I.n1p + k] += 1;
            }
        }
        __syncwarp();
        long long c = 0;
        for (int q = lane; q < 2 * I.n * I.n1p; q += 32) c += cnt[q] * (cnt[q] - 1) / 2;
        int f = 0;
        for (int v = lane; v < I.nv; v += 32) f += S[v] == 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(FULL, c, o);
            f += __shfl_xor_sync(FULL, f, o);
        }
        if (lane == 0) e[x] = (int64_t)f + (int64_t)I.nv * c;
        __syncwarp();
    }
}

// Alg. 2: S'* = argmin f over the (legal) offspring, S* replaced if strictly better
__global__ void __launch_bounds__(1024) best_kernel(int p, int nv, int ftarget, int gen, int stop_at_bound,
                                                    const int32_t *fprime, const uint8_t *Pp,
                                                    const plse_walk_stats *ws, int64_t *e_p,
                                                    Ctrl *ctrl, uint8_t *Sstar, int32_t *trace)
{
    if (stop_at_bound && ctrl->done) return;
    __shared__ uint32_t skey[32];
    __shared__ long long sst[7][32];
    uint32_t key = 0xffffffffu;
    long long st[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < p; i += blockDim.x) {
        const int f = fprime[i];
        e_p[i] = f;                       // legal after repair / PartialCol: e = f
        key = min(key, ((uint32_t)f << 16) | (uint32_t)i);
        const long long *s = reinterpret_cast<const long long *>(ws + i);
#pragma unroll
        for (int k = 0; k < 7; ++k) st[k] += s[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        key = min(key, __shfl_xor_sync(FULL, key, o));
#pragma unroll
        for (int k = 0; k < 7; ++k) st[k] += __shfl_xor_sync(FULL, st[k], o);
    }
    if (lane == 0) {
        skey[wid] = key;
#pragma unroll
        for (int k = 0; k < 7; ++k) sst[k][wid] = st[k];
    }
    __syncthreads();
    __shared__ int s_best, s_take;
    if (threadIdx.x == 0) {
        uint32_t kmin = 0xffffffffu;
        const int nw = (blockDim.x + 31) / 32;
        for (int q = 0; q < nw; ++q) kmin = min(kmin, skey[q]);
        for (int k = 0; k < 7; ++k) {
            long long t = 0;
            for (int q = 0; q < nw; ++q) t += sst[k][q];
            ctrl->stats[k] += t;
        }
        const int fb = (int)(kmin >> 16);
        s_best = (int)(kmin & 0xffffu);
        s_take = fb < ctrl->fstar;
        if (s_take) ctrl->fstar = fb;
        trace[gen] = ctrl->fstar;
        ctrl->gens = gen + 1;
        if (ctrl->fstar <= ftarget) ctrl->done = 1;
    }
    __syncthreads();
    if (s_take)
        for (int v = threadIdx.x; v < nv; v += blockDim.x) Sstar[v] = Pp[(size_t)s_best * nv + v];
}

// P_{t+1}[q] = P_all[sel[q]] with its planes, score, uid and tested list (warp per q)
__global__ void gather_kernel(const DevInst I, int p, int gen, const int32_t *sel,
                              const uint8_t *Pall, const uint32_t *planes, const int64_t *e,
                              const uint32_t *uid, const uint32_t *tested, const int32_t *tcount,
                              int cap, uint8_t *Pn, uint32_t *planesn, int64_t *en, uint32_t *uidn,
                              uint32_t *testedn, int32_t *tcountn, const int *skip)
{
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= p) return;
    const int s = sel[q];
    const uint8_t *src = Pall + (size_t)s * I.nv;
    uint8_t *dst = Pn + (size_t)q * I.nv;
    for (int v = lane; v < I.nv; v += 32) dst[v] = src[v];
    const size_t stride = (size_t)I.nw * I.nb;
    for (size_t k = lane; k < stride; k += 32) planesn[(size_t)q * stride + k] = planes[(size_t)s * stride + k];
    if (s < p) {
        const int c = tcount[s];
        for (int k = lane; k < c; k += 32) testedn[(size_t)q * cap + k] = tested[(size_t)s * cap + k];
        if (lane == 0) { tcountn[q] = c; uidn[q] = uid[s]; }
    } else if (lane == 0) {
        tcountn[q] = 0;
        uidn[q] = ((uint32_t)(gen + 1) << 16) | (uint32_t)(s - p);   // uid of a new member
    }
    if (lane == 0) en[q] = e[s];
}

__global__ void init_ids_kernel(int p, uint32_t *uid, int32_t *tcount)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < p) { uid[i] = (uint32_t)i; tcount[i] = 0; }
}

__global__ void init_ctrl_kernel(Ctrl *ctrl, int nv, int ftarget)
{
    ctrl->fstar = nv;
    ctrl->done = nv <= ftarget;
    ctrl->gens = 0;
    for (int k = 0; k < 7; ++k) ctrl->stats[k] = 0;
}

template <typename T>
int dalloc(plse_instance *h, T *&p, size_t n, cudaStream_t st)
{
    if (p) { h_free(h, p, st); p = nullptr; }
    if (n == 0) n = 1;
    void *q = nullptr;
    cudaError_t e = h_malloc(h, &q, n * sizeof(T), st);
    if (e != cudaSuccess) return fail(h, PLSE_ENOMEM, "solver allocation: %s", cudaGetErrorString(e));
    p = static_cast<T *>(q);
    return PLSE_OK;
}

static_assert(2 * kGenDepth <= 4, "the host flag slot holds two generations");

}  // namespace

void free_pop_scratch(plse_instance *h, PopScratch &ps, cudaStream_t st);

namespace {

// device buffers, events and the pinned flag slot of a solver state
void free_solver_state(plse_instance *h, SolverState *s, cudaStream_t st)
{
    for (int k = 0; k < 2; ++k) {
        h_free(h, s->Pall[k], st); h_free(h, s->planes[k], st); h_free(h, s->e[k], st);
        h_free(h, s->uid[k], st); h_free(h, s->tested[k], st); h_free(h, s->tcount[k], st);
    }
    h_free(h, s->SO, st); h_free(h, s->fprime, st); h_free(h, s->sel, st); h_free(h, s->partner, st);
    h_free(h, s->dist, st); h_free(h, s->wstats, st); h_free(h, s->ctrl, st); h_free(h, s->Sstar, st);
    h_free(h, s->trace, st);
    free_pop_scratch(h, s->ps, st);
    for (auto &ev : s->ev) if (ev) cudaEventDestroy(ev);
    for (auto &g : s->gev)
        for (auto &ev : g) if (ev) cudaEventDestroy(ev);
    pinned_slot_put(s->hflag);
    delete s;
}

}  // namespace

int ensure_pop_scratch(plse_instance *h, PopScratch &ps, int p, cudaStream_t st)
{
    if (p <= ps.cap_p) return PLSE_OK;
    const int m = 2 * p, nchunks = (m + kChunk - 1) / kChunk;
    int rc;
    if ((rc = dalloc(h, ps.order, m, st)) || (rc = dalloc(h, ps.mind, m, st)) || (rc = dalloc(h, ps.acc, p, st)) ||
        (rc = dalloc(h, ps.rej, m, st)) || (rc = dalloc(h, ps.Dloc, (size_t)nchunks * kChunk * kChunk, st)) ||
        (rc = dalloc(h, ps.sel_state, 1, st)) || (rc = dalloc(h, ps.flow, sel_flow_ints(nchunks), st)))
        return rc;
    ps.cap_p = p;
    return PLSE_OK;
}

void free_pop_scratch(plse_instance *h, PopScratch &ps, cudaStream_t st)
{
    h_free(h, ps.order, st); h_free(h, ps.mind, st); h_free(h, ps.acc, st); h_free(h, ps.rej, st);
    h_free(h, ps.Dloc, st); h_free(h, ps.sel_state, st); h_free(h, ps.flow, st);
    ps = PopScratch();
}

void release_solver(plse_instance *h, cudaStream_t st)
{
    if (h->solver) free_solver_state(h, h->solver, st);
    h->solver = nullptr;
    // step scratch
    h_free(h, h->step_planes, st);
    h->step_planes = nullptr;
    h->step_planes_cap = 0;
    free_pop_scratch(h, h->step_ps, st);
}

// Device bytes ensure_solver takes for a run of p individuals and `gens`
// generations, each buffer rounded up as the bound-workspace allocator does.
size_t solver_bytes(const plse_instance *h, int p, int gens)
{
    const DevInst &I = h->di;
    const size_t PV = (size_t)p * I.nv, stride = (size_t)I.nw * I.nb, cap = (size_t)h->params.tested_cap;
    auto a = [](size_t bytes) { return ws_align(bytes ? bytes : 1); };
    size_t t = 0;
    for (int k = 0; k < 2; ++k)
        t += a(2 * PV) + a(4 * 2 * (size_t)p * stride) + a(8 * 2 * (size_t)p) + a(4 * (size_t)p) +
             a(4 * (size_t)p * cap) + a(4 * (size_t)p);
    t += a(PV) + 4 * a(4 * (size_t)p) + a(sizeof(plse_walk_stats) * (size_t)p) + a(sizeof(Ctrl)) +
         a((size_t)I.nv) + a(4 * (size_t)gens);
    const int m = 2 * p, nchunks = (m + kChunk - 1) / kChunk;
    t += a(4 * (size_t)m) + a(4 * (size_t)m) + a(4 * (size_t)p) + a(4 * (size_t)m) +
         a(2 * (size_t)nchunks * kChunk * kChunk) + a(sizeof(SelState)) + a(4 * sel_flow_ints(nchunks));
    return t;
}

static int ensure_solver(plse_instance *h, int p, int gens, cudaStream_t st)
{
    SolverState *s = h->solver;
    const int cap = h->params.tested_cap;
    if (s && s->cap_p >= p && s->cap_gens >= gens && s->tested_cap == cap) return PLSE_OK;
    if (s) {
        // keep the step scratch, rebuild the solver buffers
        free_solver_state(h, s, st);
        h->solver = nullptr;
    }
    s = new SolverState();
    h->solver = s;
    const DevInst &I = h->di;
    const size_t PV = (size_t)p * I.nv, stride = (size_t)I.nw * I.nb;
    int rc;
    for (int k = 0; k < 2; ++k) {
        if ((rc = dalloc(h, s->Pall[k], 2 * PV, st)) || (rc = dalloc(h, s->planes[k], 2 * (size_t)p * stride, st)) ||
            (rc = dalloc(h, s->e[k], 2 * (size_t)p, st)) || (rc = dalloc(h, s->uid[k], (size_t)p, st)) ||
            (rc = dalloc(h, s->tested[k], (size_t)p * cap, st)) || (rc = dalloc(h, s->tcount[k], (size_t)p, st)))
            return rc;
    }
    if ((rc = dalloc(h, s->SO, PV, st)) || (rc = dalloc(h, s->fprime, (size_t)p, st)) ||
        (rc = dalloc(h, s->sel, (size_t)p, st)) || (rc = dalloc(h, s->partner, (size_t)p, st)) ||
        (rc = dalloc(h, s->dist, (size_t)p, st)) || (rc = dalloc(h, s->wstats, (size_t)p, st)) ||
        (rc = dalloc(h, s->ctrl, 1, st)) || (rc = dalloc(h, s->Sstar, (size_t)I.nv, st)) ||
        (rc = dalloc(h, s->trace, (size_t)gens, st)))
        return rc;
    if ((rc = ensure_pop_scratch(h, s->ps, p, st))) return rc;
    for (auto &ev : s->ev)
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(h, PLSE_ECUDA, "event create");
    for (auto &g : s->gev)
        for (auto &ev : g)
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(h, PLSE_ECUDA, "event create");
    s->hflag = pinned_slot_get();
    if (!s->hflag) return fail(h, PLSE_ENOMEM, "pinned host allocation");
    s->cap_p = p;
    s->cap_gens = gens;
    s->tested_cap = cap;
    return PLSE_OK;
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);       \
    } while (0)

int run_begin(plse_instance *h, int pop, int max_generations, int64_t iters, uint64_t seed, cudaStream_t st)
{
    if (pop < 2 || pop > 65535 || max_generations < 0 || max_generations > 65534 || iters < 0 ||
        iters > (1ll << 30))
        return fail(h, PLSE_EINVAL, "plse_run_begin: invalid argument");
    Session &se = h->session;
    int rc = run_drain(h);
    if (rc) return rc;
    StreamScope scope(h, st);
    se = Session();
    se.pop = pop;
    se.iters = iters;
    se.seed = seed;
    se.max_gens = max_generations;
    se.stream = st;
    se.active = 1;
    const int nv = h->nv;
    const int ftarget = h->l == 1 ? 1 : 0;
    se.finished = (nv == 0 || nv <= ftarget || max_generations == 0);
    if (se.finished) return PLSE_OK;
    rc = ensure_solver(h, pop, max_generations, st);
    if (rc) return rc;
    SolverState *s = h->solver;
    const DevInst &I = h->di;
    const int p = pop;
    const size_t PV = (size_t)p * nv;
    CK(cudaEventRecord(s->ev[0], st));
    // P_0, its scores, planes, ids; S^O = P_0; S* = empty colouring, f* = |V|
    CK(launch_init_population(I, p, seed, s->Pall[0], st));
    const size_t cnt_smem = 2 * (size_t)I.n * I.n1p;
    eval_kernel<<<std::min(p, 65535), 32, cnt_smem, st>>>(I, s->Pall[0], p, s->e[0]);
    CK(cudaGetLastError());
    CK(launch_planes(I, s->Pall[0], p, s->planes[0], st));
    init_ids_kernel<<<(p + 255) / 256, 256, 0, st>>>(p, s->uid[0], s->tcount[0]);
    init_ctrl_kernel<<<1, 1, 0, st>>>(s->ctrl, nv, ftarget);
    CK(cudaMemsetAsync(s->Sstar, 0, (size_t)nv, st));
    CK(cudaMemcpyAsync(s->SO, s->Pall[0], PV, cudaMemcpyDeviceToDevice, st));
    CK(cudaGetLastError());
    se.launches += 6;
    se.cur = 0;
    se.gen = 0;
    return PLSE_OK;
}

// Local search of the run: Partial-MPMA (greedy repair of each offspring, then
// PartialCol) or the two-phase PLITS walk.  The automatic policy follows
// Sec. 3.7: Partial-MPMA on highly constrained instances, r >= 0.8 of the cells
// prefilled (exact integer test 5 * prefilled >= 4 * n^2).
static bool partial_mpma(const plse_instance *h)
{
    const int mode = h->params.mode;
    if (mode == PLSE_MODE_AUTO) return 5LL * h->nfixed >= 4LL * h->n * h->n;
    return mode == PLSE_MODE_PARTIALCOL;
}

// Enqueues generation se.issued of the run on its stream without waiting for
// anything: local search, best update, an 8-byte copy of (f*, done) to pinned
// host memory, then Alg. 4, gather, matching and crossover.  If the bound is
// reached in this or an earlier generation, every later kernel returns at
// entry, so generations enqueued past the stop leave no trace in the results.
struct GenPlan {
    int p, g, cur, nxt, slot, flags;
    size_t PV;
    const int *skip;
    uint8_t *Pp;
};

static GenPlan plan_generation(plse_instance *h)
{
    Session &se = h->session;
    SolverState *s = h->solver;
    const plse_params &prm = h->params;
    GenPlan q;
    q.p = se.pop;
    q.g = se.issued;
    q.cur = se.cur;
    q.nxt = q.cur ^ 1;
    q.slot = q.g % kGenDepth;
    q.PV = (size_t)q.p * h->nv;
    q.skip = prm.stop_at_bound ? &s->ctrl->done : nullptr;
    q.flags = partial_mpma(h) ? (PLSE_LS_REPAIR | PLSE_LS_PARTIALCOL)
                              : (PLSE_LS_PHASE1 | PLSE_LS_PHASE2 | PLSE_LS_REPAIR);
    q.Pp = s->Pall[q.cur] + q.PV;
    return q;
}

// the generation after its local search: best update, Alg. 4, matching, AUX
static int issue_generation_rest(plse_instance *h, const GenPlan &q)
{
    Session &se = h->session;
    SolverState *s = h->solver;
    const cudaStream_t st = se.stream;
    const DevInst &I = h->di;
    const plse_params &prm = h->params;
    const int nv = h->nv, ftarget = h->l == 1 ? 1 : 0;
    const int p = q.p, g = q.g, cur = q.cur, nxt = q.nxt, cap = prm.tested_cap;
    const size_t stride = (size_t)I.nw * I.nb;
    const int *skip = q.skip;
    CK(cudaEventRecord(s->gev[q.slot][1], st));
    best_kernel<<<1, 1024, 0, st>>>(p, nv, ftarget, g, prm.stop_at_bound, s->fprime, q.Pp, s->wstats,
                                    s->e[cur] + p, s->ctrl, s->Sstar, s->trace);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(s->hflag + 2 * q.slot, s->ctrl, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(s->gev[q.slot][2], st));
    CK(launch_planes(I, q.Pp, p, s->planes[cur] + (size_t)p * stride, st));
    s->ps.error_flag = h->ws.counters ? h->ws.counters + 1 : nullptr;
    long long sel_kernels = 0;
    CK(launch_pop_update(I, p, s->planes[cur], s->e[cur], prm.spacing_gamma, s->ps, s->sel, nullptr, skip, st,
                         &sel_kernels));
    gather_kernel<<<(p * 32 + 255) / 256, 256, 0, st>>>(
        I, p, g, s->sel, s->Pall[cur], s->planes[cur], s->e[cur], s->uid[cur], s->tested[cur], s->tcount[cur],
        cap, s->Pall[nxt], s->planes[nxt], s->e[nxt], s->uid[nxt], s->tested[nxt], s->tcount[nxt], skip);
    CK(cudaGetLastError());
    CK(launch_matching(I, p, s->planes[nxt], s->uid[nxt], s->tested[nxt], s->tcount[nxt], cap,
                       prm.matching == PLSE_MATCH_RANDOM, g, se.seed, s->partner, s->dist, skip, st));
    CK(launch_crossover(I, p, s->Pall[nxt], s->partner, s->dist, g, se.seed, prm.beta,
                        prm.crossover == PLSE_XOVER_UX, s->SO, skip, st));
    se.launches += 3 + sel_kernels + 3;
    se.cur = nxt;
    se.issued = g + 1;
    return PLSE_OK;
}

// Enqueues generation se.issued on the run's stream.  Every kernel returns at
// entry once the bound is reached (the skip flag), so generations enqueued past
// the stop leave no trace in the results.
static int issue_generation(plse_instance *h)
{
    Session &se = h->session;
    SolverState *s = h->solver;
    const cudaStream_t st = se.stream;
    const GenPlan q = plan_generation(h);
    StreamScope scope(h, st);
    CK(cudaEventRecord(s->gev[q.slot][0], st));
    int rc = enqueue_local_search(h, s->SO, q.Pp, q.p, 0, q.g, se.iters, se.seed, q.flags, s->fprime, nullptr,
                                  s->wstats, st, q.skip);
    if (rc) return rc;
    return issue_generation_rest(h, q);
}

int generation_head(plse_instance *h, LSArgs &a, cudaEvent_t *ready)
{
    Session &se = h->session;
    if (!se.active || se.finished || se.issued >= se.max_gens || !h->solver)
        return fail(h, PLSE_ENOTSUP, "no generation to issue");
    SolverState *s = h->solver;
    const cudaStream_t st = se.stream;
    const GenPlan q = plan_generation(h);
    StreamScope scope(h, st);
    int rc = ensure_counters(h, st);
    if (rc) return rc;
    a = ls_args(h, s->SO, q.Pp, q.p, 0, q.g, se.iters, se.seed, q.flags, s->fprime, nullptr, s->wstats, q.skip);
    CK(cudaMemsetAsync(a.work_counter, 0, sizeof(int), st));
    CK(cudaEventRecord(s->gev[q.slot][0], st));
    *ready = s->gev[q.slot][0];
    return PLSE_OK;
}

int generation_tail(plse_instance *h, cudaEvent_t ls_done)
{
    Session &se = h->session;
    const cudaStream_t st = se.stream;
    const GenPlan q = plan_generation(h);
    StreamScope scope(h, st);
    CK(cudaStreamWaitEvent(st, ls_done, 0));
    return issue_generation_rest(h, q);
}

int run_issue(plse_instance *h, int *issued)
{
    Session &se = h->session;
    if (issued) *issued = 0;
    if (!se.active) return fail(h, PLSE_EINVAL, "plse_run_issue: no run in progress");
    if (se.finished || se.issued >= se.max_gens || se.issued - se.polled >= kGenDepth) return PLSE_OK;
    const int rc = issue_generation(h);
    if (!rc && issued) *issued = 1;
    return rc;
}

int run_poll(plse_instance *h, bool wait)
{
    Session &se = h->session;
    SolverState *s = h->solver;
    while (se.polled < se.issued) {
        const int slot = se.polled % kGenDepth;
        if (wait) {
            CK(cudaEventSynchronize(s->gev[slot][2]));
        } else {
            const cudaError_t q = cudaEventQuery(s->gev[slot][2]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return cuda_fail(h, q, "plse_run_query");
        }
        ++se.polled;
        if (se.finished) continue;   // enqueued past the stop: skipped on the device
        float ms = 0, t0 = 0, t1 = 0;
        CK(cudaEventElapsedTime(&ms, s->gev[slot][0], s->gev[slot][1]));
        CK(cudaEventElapsedTime(&t0, s->ev[0], s->gev[slot][0]));
        CK(cudaEventElapsedTime(&t1, s->ev[0], s->gev[slot][1]));
        se.ms_ls += ms;
        se.ls_iv.push_back(t0);
        se.ls_iv.push_back(t1);
        se.gen += 1;
        if ((h->params.stop_at_bound && s->hflag[2 * slot + 1]) || se.gen >= se.max_gens) se.finished = 1;
    }
    if (se.gen >= se.max_gens) se.finished = 1;
    return PLSE_OK;
}

int run_drain(plse_instance *h)
{
    Session &se = h->session;
    if (!se.active || se.polled >= se.issued) return PLSE_OK;
    return run_poll(h, true);
}

int run_step(plse_instance *h, int generations, cudaStream_t st, int *done_out)
{
    Session &se = h->session;
    if (!se.active) return fail(h, PLSE_EINVAL, "plse_run_step: no run in progress");
    if (generations < 0) return fail(h, PLSE_EINVAL, "plse_run_step: invalid argument");
    if (st != se.stream) return fail(h, PLSE_EINVAL, "plse_run_step: not the stream of plse_run_begin");
    int rc = run_poll(h, false);
    if (rc) return rc;
    const long long target = std::min<long long>((long long)se.issued + generations, se.max_gens);
    while (!se.finished && se.issued < target) {
        if (se.issued - se.polled < kGenDepth) {
            if ((rc = issue_generation(h))) return rc;
        } else if ((rc = run_poll(h, true))) {
            return rc;
        }
    }
    // blocking call: everything it enqueued has completed when it returns
    if ((rc = run_drain(h))) return rc;
    if (done_out) *done_out = se.finished;
    return PLSE_OK;
}

int run_result(plse_instance *h, cudaStream_t st, int8_t *best_grid, int *best_score, plse_solve_stats *stats,
               int32_t *trace_out)
{
    Session &se = h->session;
    if (!se.active) return fail(h, PLSE_EINVAL, "plse_run_result: no run in progress");
    int rc = run_drain(h);
    if (rc) return rc;
    const int nv = h->nv, n = h->n;
    int fstar = nv, gens_done = 0;
    std::vector<uint8_t> Sstar_h((size_t)nv, 0);
    double ms_total = 0;
    long long wst[7] = {0, 0, 0, 0, 0, 0, 0};
    if (h->solver && se.gen > 0) {
        SolverState *s = h->solver;
        StreamScope scope(h, st);
        CK(cudaEventRecord(s->ev[3], st));
        Ctrl hctrl;
        CK(cudaMemcpyAsync(&hctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        if (nv) CK(cudaMemcpyAsync(Sstar_h.data(), s->Sstar, (size_t)nv, cudaMemcpyDeviceToHost, st));
        if (trace_out) CK(cudaMemcpyAsync(trace_out, s->trace, sizeof(int32_t) * se.gen, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        float mt = 0;
        CK(cudaEventElapsedTime(&mt, s->ev[0], s->ev[3]));
        ms_total = mt;
        fstar = hctrl.fstar;
        gens_done = hctrl.gens;
        for (int k = 0; k < 7; ++k) wst[k] = hctrl.stats[k];
        int flag = 0;
        CK(cudaMemcpy(&flag, h->ws.counters + 1, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) {
            cudaMemsetAsync(h->ws.counters + 1, 0, sizeof(int), st);
            cudaStreamSynchronize(st);
            return fail(h, PLSE_ECHECK, "a local-search consistency check failed");
        }
    }
    if (best_grid) {
        memcpy(best_grid, h->grid.data(), (size_t)n * n);
        for (int v = 0; v < nv; ++v) best_grid[h->cell[v]] = (int8_t)Sstar_h[v];
    }
    if (best_score) *best_score = n * n - h->l - fstar;
    if (stats) {
        stats->generations = gens_done;
        stats->best_f = fstar;
        int64_t *w = &stats->walks.iterations;
        for (int k = 0; k < 7; ++k) w[k] = wst[k];
        stats->ms_total = ms_total;
        stats->ms_local_search = se.ms_ls;
        stats->launches = se.launches;
    }
    return PLSE_OK;
}

int run_solve(plse_instance *h, int pop, int generations, int64_t iters, uint64_t seed, cudaStream_t st,
              int8_t *best_grid, int *best_score, plse_solve_stats *stats, int32_t *trace_out)
{
    int rc = run_begin(h, pop, generations, iters, seed, st);
    if (!rc) rc = run_step(h, generations, st, nullptr);
    if (!rc) rc = run_result(h, st, best_grid, best_score, stats, trace_out);
    h->session.active = 0;
    return rc;
}

int ensure_step_planes(plse_instance *h, size_t individuals, cudaStream_t st)
{
    const size_t need = individuals * (size_t)h->di.nw * h->di.nb;
    if (need <= h->step_planes_cap) return PLSE_OK;
    int rc = dalloc(h, h->step_planes, need, st);
    if (rc) return rc;
    h->step_planes_cap = need;
    return PLSE_OK;
}

}  // namespace plse

using namespace plse;

extern "C" {

int plse_solve(plse_handle h, int pop, int generations, int64_t iters, uint64_t seed, int8_t *best_grid,
               int *best_score)
{
    if (!h) return PLSE_EINVAL;
    return run_solve(h, pop, generations, iters, seed, nullptr, best_grid, best_score, nullptr, nullptr);
}

int plse_solve_ex(plse_handle h, int pop, int generations, int64_t iters, uint64_t seed, void *stream,
                  int8_t *best_grid, int *best_score, plse_solve_stats *stats)
{
    if (!h) return PLSE_EINVAL;
    return run_solve(h, pop, generations, iters, seed, (cudaStream_t)stream, best_grid, best_score, stats,
                     nullptr);
}

int plse_run_begin(plse_handle h, int pop, int max_generations, int64_t iters, uint64_t seed, void *stream)
{
    if (!h) return PLSE_EINVAL;
    return run_begin(h, pop, max_generations, iters, seed, (cudaStream_t)stream);
}

int plse_run_step(plse_handle h, int generations, void *stream, int *done)
{
    if (!h) return PLSE_EINVAL;
    return run_step(h, generations, (cudaStream_t)stream, done);
}

int plse_run_issue(plse_handle h, void *stream, int *issued)
{
    if (!h) return PLSE_EINVAL;
    if (h->session.active && (cudaStream_t)stream != h->session.stream)
        return fail(h, PLSE_EINVAL, "plse_run_issue: not the stream of plse_run_begin");
    return run_issue(h, issued);
}

int plse_run_query(plse_handle h, int *done, int *generations, int *in_flight)
{
    if (!h) return PLSE_EINVAL;
    Session &se = h->session;
    if (!se.active) return fail(h, PLSE_EINVAL, "plse_run_query: no run in progress");
    const int rc = run_poll(h, false);
    if (rc) return rc;
    if (done) *done = se.finished && se.polled == se.issued;
    if (generations) *generations = se.gen;
    if (in_flight) *in_flight = se.issued - se.polled;
    return PLSE_OK;
}

int plse_run_population(plse_handle h, int which, uint8_t *dst, void *stream)
{
    if (!h || !dst || (which != PLSE_RUN_POPULATION && which != PLSE_RUN_OFFSPRING)) return PLSE_EINVAL;
    Session &se = h->session;
    if (!se.active || !h->solver) return fail(h, PLSE_EINVAL, "plse_run_population: no run in progress");
    int rc = run_drain(h);
    if (rc) return rc;
    const cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    SolverState *s = h->solver;
    const size_t bytes = (size_t)se.pop * h->nv;
    const uint8_t *src = which == PLSE_RUN_POPULATION ? s->Pall[se.cur] : s->SO;
    if (bytes) CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return PLSE_OK;
}

int plse_run_timeline(plse_handle h, void *ref_event, int first, int count, float *ls_start_end)
{
    if (!h || !ref_event || first < 0 || count < 0 || (count > 0 && !ls_start_end)) return PLSE_EINVAL;
    Session &se = h->session;
    if (!se.active || !h->solver) return fail(h, PLSE_EINVAL, "plse_run_timeline: no run in progress");
    int rc = run_drain(h);
    if (rc) return rc;
    if ((long long)first + count > (long long)se.ls_iv.size() / 2)
        return fail(h, PLSE_EINVAL, "plse_run_timeline: generations not run");
    if (count == 0) return PLSE_OK;
    const cudaEvent_t ref = static_cast<cudaEvent_t>(ref_event);
    const cudaError_t q = cudaEventQuery(ref);
    if (q != cudaSuccess)
        return q == cudaErrorNotReady ? fail(h, PLSE_EINVAL, "plse_run_timeline: reference event not complete")
                                      : cuda_fail(h, q, "plse_run_timeline");
    float off = 0;
    CK(cudaEventElapsedTime(&off, ref, h->solver->ev[0]));
    for (int k = 0; k < 2 * count; ++k) ls_start_end[k] = off + se.ls_iv[2 * (size_t)first + k];
    return PLSE_OK;
}

int plse_run_result(plse_handle h, void *stream, int8_t *best_grid, int *best_score, plse_solve_stats *stats,
                    int32_t *trace)
{
    if (!h) return PLSE_EINVAL;
    return run_result(h, (cudaStream_t)stream, best_grid, best_score, stats, trace);
}

int plse_distances(plse_handle h, const uint8_t *A, int na, const uint8_t *B, int nb, int32_t *D, void *stream)
{
    if (!h || na < 0 || nb < 0) return PLSE_EINVAL;
    if (na == 0 || nb == 0) return PLSE_OK;
    if (!D || (h->nv > 0 && (!A || !B))) return fail(h, PLSE_EINVAL, "plse_distances: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    if (h->nv == 0) {
        CK(cudaMemsetAsync(D, 0, sizeof(int32_t) * (size_t)na * nb, st));
        return PLSE_OK;
    }
    int rc = ensure_step_planes(h, (size_t)na + nb, st);
    if (rc) return rc;
    uint32_t *pa = h->step_planes, *pb = h->step_planes + (size_t)na * h->di.nw * h->di.nb;
    CK(launch_planes(h->di, A, na, pa, st));
    CK(launch_planes(h->di, B, nb, pb, st));
    CK(launch_distance_matrix(h->di, pa, na, pb, nb, D, st));
    return PLSE_OK;
}

int plse_pop_update(plse_handle h, int p, const uint8_t *Pall, const int64_t *e, int32_t *sel, int32_t *filled,
                    void *stream)
{
    if (!h || p < 1 || p > 65535 || !e || !sel || (h->nv > 0 && !Pall))
        return PLSE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    int rc = ensure_step_planes(h, 2 * (size_t)p, st);
    if (rc) return rc;
    if ((rc = ensure_pop_scratch(h, h->step_ps, p, st))) return rc;
    if ((rc = ensure_counters(h, st))) return rc;
    h->step_ps.error_flag = h->ws.counters + 1;
    if (h->nv > 0) CK(launch_planes(h->di, Pall, 2 * p, h->step_planes, st));
    CK(launch_pop_update(h->di, p, h->step_planes, e, h->params.spacing_gamma, h->step_ps, sel, filled,
                         nullptr, st));
    return PLSE_OK;
}

int plse_matching(plse_handle h, int p, const uint8_t *P, const uint32_t *uid, uint32_t *tested,
                  int32_t *tcount, int gen, uint64_t seed, int32_t *partner, int32_t *dist, void *stream)
{
    if (!h || p < 2 || p > 65535 || gen < 0 || gen >= (1 << 24) || !partner || !dist ||
        (h->nv > 0 && !P) || (h->params.matching == PLSE_MATCH_NEAREST && (!uid || !tested || !tcount)))
        return PLSE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    int rc = ensure_step_planes(h, (size_t)p, st);
    if (rc) return rc;
    if (h->nv > 0) CK(launch_planes(h->di, P, p, h->step_planes, st));
    CK(launch_matching(h->di, p, h->step_planes, uid, tested, tcount, h->params.tested_cap,
                       h->params.matching == PLSE_MATCH_RANDOM, gen, seed, partner, dist, nullptr, st));
    return PLSE_OK;
}

int plse_crossover(plse_handle h, int p, const uint8_t *P, const int32_t *partner, const int32_t *dist, int gen,
                   uint64_t seed, uint8_t *O, void *stream)
{
    if (!h || p < 1 || gen < 0 || gen >= (1 << 24) || !partner || !dist || (h->nv > 0 && (!P || !O)) || P == O)
        return PLSE_EINVAL;
    CK(launch_crossover(h->di, p, P, partner, dist, gen, seed, h->params.beta,
                        h->params.crossover == PLSE_XOVER_UX, O, nullptr, (cudaStream_t)stream));
    return PLSE_OK;
}

}  // extern "C"
