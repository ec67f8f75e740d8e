// engine.cu -- many runs of Alg. 2 in flight at once, driven from one host
// thread: plse_solve_batch (a fixed list of jobs) and the plse_server_* request
// server (jobs arriving over time, admitted into a bounded number of slots).
//
// Each running job has its own handle (instance + resident population) and its
// own non-blocking CUDA stream.  The driver loop enqueues generations with
// run_issue (at most two in flight per job) and notes completed ones with
// run_poll, so the host never waits on any one job while others have work, and
// the kernels of different jobs overlap on the GPU: a small population leaves
// most SMs idle during its local search, and the tail of one job's launch is
// filled by another's.  Per-job results are a function of the job alone (its
// instance, parameters, pop, generations, iters and seed), never of the mix,
// because no device state is shared between handles.
//
// The server admits requests in arrival order by device memory: a request's
// footprint (its instance image plus plse_workspace_size of its run) is known
// once its handle is built on the host, and the request at the head of the
// queue starts when a stream slot is free and the footprint fits in the budget
// left by the requests running; the bytes return to the budget when it ends.
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "plse_handle.cuh"

namespace plse {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

bool job_valid(const plse_job &j)
{
    return j.pop >= 2 && j.pop <= 65535 && j.generations >= 0 && j.generations <= 65534 && j.iters >= 0 &&
           j.iters <= (1ll << 30);
}

void note_detail(plse_result &r, const plse_instance *h)
{
    const char *msg = h ? h->err.c_str() : "";
    if (!*msg) msg = plse_strerror(r.status);
    snprintf(r.detail, sizeof(r.detail), "%s", msg);
}

// One job occupying a stream slot.
struct Active {
    plse_instance *h = nullptr;
    cudaStream_t st = nullptr;
    int8_t *grid_out = nullptr;
    plse_result *res = nullptr;
    bool cancel = false;
};

// Advances one running job by what is possible without waiting.  Returns true
// once the job has completed and its result is written.
bool advance(Active &a, bool &progressed)
{
    plse_instance *h = a.h;
    Session &se = h->session;
    int rc = run_poll(h, false);
    if (!rc && !(se.finished || a.cancel)) {
        int issued = 0;
        rc = run_issue(h, &issued);
        progressed |= issued != 0;
    }
    const bool drained = se.polled == se.issued;
    if (rc == PLSE_OK && !((se.finished || a.cancel) && drained)) return false;
    // completed, cancelled (after its generations in flight) or failed
    progressed = true;
    plse_result &r = *a.res;
    r.status = rc;
    if (rc == PLSE_OK) {
        rc = run_result(h, a.st, a.grid_out, &r.best_score, &r.stats, nullptr);
        r.status = rc ? rc : (a.cancel && !se.finished ? PLSE_ECANCELLED : PLSE_OK);
    }
    if (r.status != PLSE_OK) note_detail(r, h);
    // nothing of the job may still run when its handle is released or reused
    cudaStreamSynchronize(a.st);
    se.active = 0;
    return true;
}

// plse_solve_batch when every job has a handle of its own: the runs advance one
// generation at a time, and the local searches of a generation run as one
// persistent multi-instance launch per colour-word class (instances that share a
// kernel), each on a stream of its own; the rest of each run's generation runs
// on the run's stream, overlapping with the other runs'.  Per-run results are
// those of plse_solve: every kernel sees the same arguments as in a run alone.
// Returns PLSE_ENOTSUP (nothing started) when a class has no launch that fits.
int batch_lockstep(plse_instance **hs, const plse_job *jobs, int count, int8_t *const *grids,
                   plse_result *results, Clock::time_point t0)
{
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PLSE_ECUDA;
    // one launch plan per colour-word class, fixed for the whole batch
    constexpr int kClasses = 4;
    std::vector<int> cls(count);
    std::vector<std::vector<int>> members(kClasses);
    for (int i = 0; i < count; ++i) {
        cls[i] = colour_words(hs[i]->n) - 1;
        if (hs[i]->nv > 0 && job_valid(jobs[i])) members[cls[i]].push_back(i);
    }
    LSLaunch plan[kClasses];
    int base[kClasses];                  // first entry of each class in the job tables
    for (int c = 0, b = 0; c < kClasses; ++c) {
        base[c] = b;
        b += (int)members[c].size();
    }
    for (int c = 0; c < kClasses; ++c) {
        if (members[c].empty()) continue;
        std::vector<DevInst> insts;
        for (int i : members[c]) insts.push_back(hs[i]->di);
        plse_instance *h0 = hs[members[c][0]];
        if (!h0->ls_lanes && !h0->ls_walks && !h0->ls_splace) {
            // knobs of the class from its largest instance at its population
            int big = members[c][0];
            for (int i : members[c])
                if (hs[i]->nv > hs[big]->nv) big = i;
            int l = 0, w = 0, pl = 0;
            if (plse_autotune(hs[big], jobs[big].pop, std::min(200, 2 * hs[big]->nv + 1), &l, &w, &pl,
                              nullptr) == PLSE_OK) {
                h0->ls_lanes = l;
                h0->ls_walks = w;
                h0->ls_splace = pl;
            }
        }
        plan[c] = plan_local_search_multi(insts.data(), (int)insts.size(), device, h0->ls_lanes, h0->ls_walks,
                                          h0->ls_splace);
        if (plan[c].blocks <= 0) return PLSE_ENOTSUP;
    }
    std::vector<cudaStream_t> st(count, nullptr), cst(kClasses, nullptr);
    std::vector<cudaEvent_t> cev(kClasses, nullptr);
    LSJob *htab = nullptr, *dtab = nullptr;
    // one scratch set per class, shared by its runs: a walk slot works on one
    // run at a time, so its tables are sized for the class's largest instance
    // (the slot clocks keep the evicted-tabu table valid across runs)
    struct Shared {
        void *buf[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        size_t stride[6] = {0, 0, 0, 0, 0, 0};   // G, TC, LIST, XR, HP, SW elements per slot
    } sh[kClasses];
    int rc = PLSE_OK;
    auto cleanup = [&]() {
        for (auto &q : st) if (q) { cudaStreamSynchronize(q); cudaStreamDestroy(q); }
        for (int c = 0; c < kClasses; ++c) {
            if (cst[c]) cudaStreamSynchronize(cst[c]);
            for (void *p : sh[c].buf)
                if (p) cudaFreeAsync(p, cst[c]);
            if (cst[c]) { cudaStreamSynchronize(cst[c]); cudaStreamDestroy(cst[c]); }
        }
        for (auto &e : cev) if (e) cudaEventDestroy(e);
        if (dtab) cudaFree(dtab);
        if (htab) cudaFreeHost(htab);
    };
    for (auto &q : st)
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess) rc = PLSE_ECUDA;
    for (int c = 0; c < kClasses; ++c)
        if (cudaStreamCreateWithFlags(&cst[c], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&cev[c], cudaEventDisableTiming) != cudaSuccess)
            rc = PLSE_ECUDA;
    if (!rc && (cudaMallocHost(reinterpret_cast<void **>(&htab), sizeof(LSJob) * count) != cudaSuccess ||
                cudaMalloc(reinterpret_cast<void **>(&dtab), sizeof(LSJob) * count) != cudaSuccess))
        rc = PLSE_ENOMEM;
    for (int c = 0; c < kClasses && !rc; ++c) {
        if (members[c].empty()) continue;
        size_t *sd = sh[c].stride;
        for (int i : members[c]) {
            const DevInst &I = hs[i]->di;
            LSArgs x{};
            set_ls_strides(I, x);
            sd[0] = std::max(sd[0], x.g_stride);
            sd[1] = std::max(sd[1], x.tc_stride);
            sd[2] = std::max(sd[2], x.list_stride);
            sd[3] = std::max(sd[3], x.xr_stride);
            sd[4] = std::max(sd[4], x.hp_stride);
            sd[5] = std::max(sd[5], x.sw_stride);
        }
        const size_t slots = (size_t)plan[c].slots();
        const size_t bytes[7] = {4 * slots * sd[0], 8 * slots * sd[1], 2 * slots * sd[2], 2 * slots * sd[3],
                                 4 * slots * sd[4], slots * sd[5], 4 * slots};
        for (int k = 0; k < 7 && !rc; ++k)
            if (dev_malloc(&sh[c].buf[k], bytes[k], cst[c]) != cudaSuccess) rc = PLSE_ENOMEM;
        // evicted-tabu tables and slot clocks start at zero; the rest is rebuilt by every walk
        if (!rc && (cudaMemsetAsync(sh[c].buf[0], 0, bytes[0], cst[c]) != cudaSuccess ||
                    cudaMemsetAsync(sh[c].buf[6], 0, bytes[6], cst[c]) != cudaSuccess))
            rc = PLSE_ECUDA;
    }
    if (rc) {
        cleanup();
        return rc;
    }
    std::vector<char> live(count, 0);
    for (int i = 0; i < count; ++i) {
        plse_result &r = results[i];
        r.ms_queue = ms_between(t0, Clock::now());
        if (!job_valid(jobs[i])) {
            r.status = fail(hs[i], PLSE_EINVAL, "plse_solve_batch: invalid job %d", i);
            note_detail(r, hs[i]);
            continue;
        }
        const int e = run_begin(hs[i], jobs[i].pop, jobs[i].generations, jobs[i].iters, jobs[i].seed, st[i]);
        if (e) {
            r.status = e;
            note_detail(r, hs[i]);
            continue;
        }
        r.status = PLSE_OK;
        live[i] = 1;
    }
    auto can_issue = [&](int i) {
        const Session &se = hs[i]->session;
        return live[i] && se.active && !se.finished && se.issued < se.max_gens && hs[i]->solver;
    };
    for (;;) {
        bool any = false;
        for (int c = 0; c < kClasses; ++c) {
            std::vector<int> idx;
            for (int i : members[c])
                if (can_issue(i)) idx.push_back(i);
            if (idx.empty()) continue;
            any = true;
            std::vector<int> ok;
            for (int i : idx) {
                LSArgs a;
                cudaEvent_t ready = nullptr;
                const int e = generation_head(hs[i], a, &ready);
                if (e) {
                    results[i].status = e;
                    note_detail(results[i], hs[i]);
                    live[i] = 0;
                    continue;
                }
                a.G = static_cast<uint32_t *>(sh[c].buf[0]);
                a.TC = static_cast<uint2 *>(sh[c].buf[1]);
                a.LIST = static_cast<uint16_t *>(sh[c].buf[2]);
                a.XR = static_cast<uint16_t *>(sh[c].buf[3]);
                a.HP = static_cast<uint32_t *>(sh[c].buf[4]);
                a.SW = static_cast<uint8_t *>(sh[c].buf[5]);
                a.slot_clock = static_cast<uint32_t *>(sh[c].buf[6]);
                a.g_stride = sh[c].stride[0];
                a.tc_stride = sh[c].stride[1];
                a.list_stride = sh[c].stride[2];
                a.xr_stride = sh[c].stride[3];
                a.hp_stride = sh[c].stride[4];
                a.sw_stride = sh[c].stride[5];
                htab[base[c] + (int)ok.size()] = LSJob{hs[i]->di, a};
                cudaStreamWaitEvent(cst[c], ready, 0);
                ok.push_back(i);
            }
            if (ok.empty()) continue;
            const int off = base[c];
            cudaError_t e = cudaMemcpyAsync(dtab + off, htab + off, sizeof(LSJob) * ok.size(),
                                            cudaMemcpyHostToDevice, cst[c]);
            if (e == cudaSuccess) e = launch_local_search_multi(dtab + off, (int)ok.size(), plan[c], cst[c]);
            if (e == cudaSuccess) e = cudaEventRecord(cev[c], cst[c]);
            for (int i : ok) {
                const int t = e == cudaSuccess ? generation_tail(hs[i], cev[c]) : cuda_fail(hs[i], e, "batched launch");
                if (t) {
                    results[i].status = t;
                    note_detail(results[i], hs[i]);
                    live[i] = 0;
                }
            }
        }
        if (!any) break;
        // the generation of every run completes before the table is refilled
        for (int i = 0; i < count; ++i) {
            if (!live[i]) continue;
            const int e = run_poll(hs[i], true);
            if (e) {
                results[i].status = e;
                note_detail(results[i], hs[i]);
                live[i] = 0;
            }
        }
    }
    for (int i = 0; i < count; ++i) {
        plse_result &r = results[i];
        if (live[i]) {
            const int e = run_result(hs[i], st[i], grids ? grids[i] : nullptr, &r.best_score, &r.stats, nullptr);
            r.status = e;
            if (e) note_detail(r, hs[i]);
        }
        if (hs[i]->session.active) {
            cudaStreamSynchronize(st[i]);
            hs[i]->session.active = 0;
        }
        r.ms_wall = ms_between(t0, Clock::now());
    }
    cleanup();
    return PLSE_OK;
}

}  // namespace
}  // namespace plse

using namespace plse;

// ============================================================================
// plse_solve_batch
extern "C" int plse_solve_batch(plse_handle *hs, const plse_job *jobs, int count, int max_inflight,
                                int8_t *const *best_grids, plse_result *results)
{
    if (count < 0 || max_inflight < PLSE_BATCH_LOCKSTEP || (count > 0 && (!hs || !jobs || !results)))
        return PLSE_EINVAL;
    if (count == 0) return PLSE_OK;
    for (int i = 0; i < count; ++i)
        if (!hs[i]) return PLSE_EINVAL;
    const auto t0 = Clock::now();
    for (int i = 0; i < count; ++i) {
        memset(&results[i], 0, sizeof(plse_result));
        results[i].status = PLSE_EINVAL;
    }
    // lockstep (max_inflight = PLSE_BATCH_LOCKSTEP, every job on a handle of its
    // own): one multi-instance local-search launch per generation and colour-word
    // class; otherwise concurrent runs, each on a stream of its own.
    bool distinct = max_inflight == PLSE_BATCH_LOCKSTEP;
    if (distinct) {
        std::unordered_set<plse_instance *> seen;
        for (int i = 0; i < count; ++i) distinct = distinct && seen.insert(hs[i]).second;
    }
    if (distinct) {
        const int rc = batch_lockstep(hs, jobs, count, best_grids, results, t0);
        if (rc != PLSE_ENOTSUP) {
            int first = rc;
            for (int i = 0; i < count && !first; ++i) first = results[i].status;
            return first;
        }
    }
    const int slots = std::max(1, std::min(count, max_inflight > 0 ? max_inflight : 16));
    std::vector<cudaStream_t> streams(slots, nullptr);
    for (auto &s : streams)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto &q : streams) if (q) cudaStreamDestroy(q);
            return PLSE_ECUDA;
        }
    std::vector<Active> act(slots);
    std::vector<int> slot_job(slots, -1);
    std::vector<char> started(count, 0);
    std::vector<double> t_start(count, 0.0);
    int next = 0, remaining = count;
    while (remaining > 0) {
        bool progressed = false;
        // admission: jobs in index order; a job whose handle is busy waits for it
        for (int s = 0; s < slots; ++s) {
            if (slot_job[s] >= 0) continue;
            for (int i = next; i < count; ++i) {
                if (started[i]) continue;
                bool busy = false;
                for (int q = 0; q < slots; ++q)
                    if (slot_job[q] >= 0 && hs[slot_job[q]] == hs[i]) busy = true;
                if (busy) continue;
                started[i] = 1;
                progressed = true;
                while (next < count && started[next]) ++next;
                plse_result &r = results[i];
                t_start[i] = ms_between(t0, Clock::now());
                r.ms_queue = t_start[i];
                if (!job_valid(jobs[i])) {
                    r.status = fail(hs[i], PLSE_EINVAL, "plse_solve_batch: invalid job %d", i);
                    note_detail(r, hs[i]);
                    r.ms_wall = ms_between(t0, Clock::now());
                    --remaining;
                    continue;
                }
                const int rc = run_begin(hs[i], jobs[i].pop, jobs[i].generations, jobs[i].iters, jobs[i].seed,
                                         streams[s]);
                if (rc) {
                    r.status = rc;
                    note_detail(r, hs[i]);
                    cudaStreamSynchronize(streams[s]);
                    hs[i]->session.active = 0;
                    r.ms_wall = ms_between(t0, Clock::now());
                    --remaining;
                    continue;
                }
                act[s] = Active{hs[i], streams[s], best_grids ? best_grids[i] : nullptr, &r, false};
                slot_job[s] = i;
                break;
            }
        }
        for (int s = 0; s < slots; ++s) {
            if (slot_job[s] < 0) continue;
            if (advance(act[s], progressed)) {
                results[slot_job[s]].ms_wall = ms_between(t0, Clock::now());
                slot_job[s] = -1;
                --remaining;
            }
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (auto &s : streams) cudaStreamDestroy(s);
    int first = PLSE_OK;
    for (int i = 0; i < count && !first; ++i) first = results[i].status;
    return first;
}

// ============================================================================
// request server
struct plse_server_s {
    struct Request {
        int64_t ticket = 0;
        int n = 0;
        std::vector<int8_t> grid;
        plse_job job{};
        plse_params params{};
        Clock::time_point arrival;
        bool cancel = false;
    };
    struct Done {
        plse_result res{};
        std::vector<int8_t> grid;
    };
    struct Running {
        Request req;
        Active a;
        std::vector<int8_t> grid;
        plse_result res{};
        size_t need = 0;          // bytes counted against the budget while it runs
    };

    int device = 0;
    int max_inflight = 0, max_queue = 0;
    size_t budget = 0, in_use = 0, peak = 0;   // device-memory admission (bytes)
    int64_t waited_for_memory = 0;             // admissions that had to wait for memory
    int running = 0, peak_running = 0;
    int head_pending = 0;                      // a dequeued request waiting for a slot or memory
    int ls_lanes = 0, ls_walks = 0, ls_colourings = 0;   // launch knobs of every request's handle
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> queue;
    std::unordered_map<int64_t, Done> done;
    std::unordered_map<int64_t, bool> cancel_running;   // tickets in slots asked to cancel
    std::unordered_set<int64_t> live;                   // submitted and not yet released by a poll
    int64_t next_ticket = 1;
    bool stop = false;
    std::thread worker, reaper;
    // handles of completed jobs, destroyed off the driver thread
    std::mutex reap_mu;
    std::condition_variable reap_cv;
    std::vector<plse_instance *> reap;
    bool reap_stop = false;

    void finish(Running &r)
    {
        Done d;
        r.res.mem_bytes = (int64_t)r.need;
        d.res = r.res;
        d.res.ms_wall = ms_between(r.req.arrival, Clock::now());
        d.grid = std::move(r.grid);
        {
            std::lock_guard<std::mutex> lk(mu);
            cancel_running.erase(r.req.ticket);
            done.emplace(r.req.ticket, std::move(d));
            if (r.need) {
                in_use -= r.need;
                --running;
                r.need = 0;
            }
        }
        cv_done.notify_all();
        if (r.a.h) {
            std::lock_guard<std::mutex> lk(reap_mu);
            reap.push_back(r.a.h);
            r.a.h = nullptr;
        }
        reap_cv.notify_one();
    }

    void reaper_loop()
    {
        cudaSetDevice(device);
        for (;;) {
            std::vector<plse_instance *> batch;
            {
                std::unique_lock<std::mutex> lk(reap_mu);
                reap_cv.wait(lk, [&] { return reap_stop || !reap.empty(); });
                batch.swap(reap);
                if (batch.empty() && reap_stop) return;
            }
            for (plse_instance *h : batch) plse_destroy(h);
        }
    }

    void worker_loop()
    {
        cudaSetDevice(device);
        std::vector<cudaStream_t> streams(max_inflight, nullptr);
        for (auto &s : streams) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        std::vector<Running> slot(max_inflight);
        std::vector<char> used(max_inflight, 0);
        Running head;                    // next request, handle built, waiting for a slot or memory
        size_t head_need = 0;
        bool head_ready = false, head_waited = false;
        for (;;) {
            bool progressed = false;
            // admission: the request at the head of the queue gets its handle
            // built (host work and the instance upload), then waits until a slot
            // is free and its footprint fits in the memory budget
            for (int s = 0; s < max_inflight; ++s) {
                if (used[s]) continue;
                if (!head_ready) {
                    Request req;
                    {
                        std::unique_lock<std::mutex> lk(mu);
                        int busy = 0;
                        for (char u : used) busy += u;
                        if (queue.empty()) {
                            if (stop) break;
                            if (busy == 0) {
                                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
                                if (queue.empty()) break;
                            } else {
                                break;
                            }
                        }
                        req = std::move(queue.front());
                        queue.pop_front();
                    }
                    progressed = true;
                    head = Running();
                    head.req = std::move(req);
                    if (head.req.cancel) {
                        head.res.ms_queue = ms_between(head.req.arrival, Clock::now());
                        head.res.status = PLSE_ECANCELLED;
                        note_detail(head.res, nullptr);
                        finish(head);
                        continue;
                    }
                    plse_instance *h = nullptr;
                    int rc = plse_create(head.req.n, head.req.grid.data(), &h);
                    if (!rc) rc = plse_set_params(h, &head.req.params);
                    if (!rc) {
                        std::lock_guard<std::mutex> lk(mu);
                        rc = plse_set_launch(h, ls_lanes, ls_walks, ls_colourings);
                    }
                    size_t ws = 0;
                    if (!rc) rc = plse_workspace_size(h, head.req.job.pop, head.req.job.generations, &ws);
                    head.grid.assign((size_t)head.req.n * head.req.n, 0);
                    head.a = Active{h, nullptr, head.grid.data(), &head.res, false};
                    head_need = (h ? h->inst_bytes : 0) + ws;
                    if (!rc && head_need > budget)
                        rc = h ? fail(h, PLSE_ENOMEM, "request needs %zu bytes of device memory, the server's "
                                      "budget is %zu", head_need, budget) : PLSE_ENOMEM;
                    if (rc) {
                        head.res.ms_queue = ms_between(head.req.arrival, Clock::now());
                        head.res.status = rc;
                        note_detail(head.res, h);
                        finish(head);
                        continue;
                    }
                    head_ready = true;
                    std::lock_guard<std::mutex> lk(mu);
                    head_pending = 1;
                }
                bool cancelled = false, fits = false;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    cancelled = stop || cancel_running.count(head.req.ticket) != 0;
                    fits = in_use + head_need <= budget;
                    if (cancelled || fits) head_pending = 0;
                    if (!cancelled && fits) {
                        in_use += head_need;
                        peak = std::max(peak, in_use);
                        ++running;
                        peak_running = std::max(peak_running, running);
                        if (head_waited) ++waited_for_memory;
                    }
                }
                if (cancelled) {
                    head.res.ms_queue = ms_between(head.req.arrival, Clock::now());
                    head.res.status = PLSE_ECANCELLED;
                    note_detail(head.res, nullptr);
                    finish(head);
                    head_ready = head_waited = false;
                    progressed = true;
                    continue;
                }
                if (!fits) {                      // wait for running requests to free memory
                    head_waited = true;
                    break;
                }
                progressed = true;
                Running &r = slot[s];
                r = std::move(head);
                head_ready = head_waited = false;
                r.need = head_need;
                r.res.ms_queue = ms_between(r.req.arrival, Clock::now());
                r.a.st = streams[s];
                r.a.grid_out = r.grid.data();
                r.a.res = &r.res;
                const int rc = run_begin(r.a.h, r.req.job.pop, r.req.job.generations, r.req.job.iters,
                                         r.req.job.seed, streams[s]);
                if (rc) {
                    r.res.status = rc;
                    note_detail(r.res, r.a.h);
                    cudaStreamSynchronize(streams[s]);
                    r.a.h->session.active = 0;
                    finish(r);
                    continue;
                }
                used[s] = 1;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                bool any = head_ready;
                for (char u : used) any |= u != 0;
                if (stop && !any && queue.empty()) break;
                for (int s = 0; s < max_inflight; ++s)
                    if (used[s] && (stop || cancel_running.count(slot[s].req.ticket))) slot[s].a.cancel = true;
            }
            for (int s = 0; s < max_inflight; ++s) {
                if (!used[s]) continue;
                if (advance(slot[s].a, progressed)) {
                    finish(slot[s]);
                    used[s] = 0;
                }
            }
            if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
        for (auto &s : streams) cudaStreamDestroy(s);
    }
};

extern "C" {

int plse_server_create(int max_inflight, int max_queue, size_t mem_budget, plse_server *out)
{
    if (!out || max_inflight < 1 || max_inflight > 256 || max_queue < 0) return PLSE_EINVAL;
    plse_server_s *s = new (std::nothrow) plse_server_s();
    if (!s) return PLSE_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PLSE_ECUDA;
    }
    if (mem_budget == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            delete s;
            return PLSE_ECUDA;
        }
        mem_budget = free_b / 10 * 9;
    }
    s->budget = mem_budget;
    s->max_inflight = max_inflight;
    s->max_queue = max_queue;
    s->worker = std::thread([s] { s->worker_loop(); });
    s->reaper = std::thread([s] { s->reaper_loop(); });
    *out = s;
    return PLSE_OK;
}

int plse_server_submit(plse_server s, int n, const int8_t *grid, const plse_job *job, const plse_params *params,
                       int64_t *ticket)
{
    if (!s || !grid || !job || !ticket || n < 1 || n > kMaxN || !job_valid(*job)) return PLSE_EINVAL;
    plse_server_s::Request r;
    r.n = n;
    r.grid.assign(grid, grid + (size_t)n * n);
    r.job = *job;
    if (params) r.params = *params;
    else plse_default_params(&r.params);
    r.arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return PLSE_EINVAL;
        if ((int)s->queue.size() >= s->max_queue) return PLSE_EBUSY;
        r.ticket = s->next_ticket++;
        *ticket = r.ticket;
        s->live.insert(r.ticket);
        s->queue.push_back(std::move(r));
    }
    s->cv_work.notify_one();
    return PLSE_OK;
}

int plse_server_poll(plse_server s, int64_t ticket, int wait_ms, int8_t *best_grid, plse_result *out)
{
    if (!s) return PLSE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->done.count(ticket) != 0; };
    if (!s->live.count(ticket)) return PLSE_EINVAL;
    if (!ready()) {
        if (wait_ms < 0) s->cv_done.wait(lk, ready);
        else if (wait_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
        if (!ready()) return PLSE_PENDING;
    }
    auto it = s->done.find(ticket);
    if (out) *out = it->second.res;
    if (best_grid && !it->second.grid.empty()) memcpy(best_grid, it->second.grid.data(), it->second.grid.size());
    s->done.erase(it);
    s->live.erase(ticket);
    return PLSE_OK;
}

int plse_server_memory(plse_server s, size_t *budget, size_t *in_use, size_t *peak, int *peak_running,
                       int64_t *waited)
{
    if (!s) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (budget) *budget = s->budget;
    if (in_use) *in_use = s->in_use;
    if (peak) *peak = s->peak;
    if (peak_running) *peak_running = s->peak_running;
    if (waited) *waited = s->waited_for_memory;
    return PLSE_OK;
}

int plse_server_cancel(plse_server s, int64_t ticket)
{
    if (!s) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->live.count(ticket)) return PLSE_EINVAL;
    for (auto &r : s->queue)
        if (r.ticket == ticket) {
            r.cancel = true;
            return PLSE_OK;
        }
    if (s->done.count(ticket)) return PLSE_OK;   // already complete: nothing to cancel
    s->cancel_running[ticket] = true;
    return PLSE_OK;
}

int plse_server_set_launch(plse_server s, int ls_lanes, int ls_walks, int ls_colourings)
{
    if (!s || ls_lanes < 0 || ls_walks < 0 || ls_colourings < 0 || ls_colourings > 2) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->ls_lanes = ls_lanes;
    s->ls_walks = ls_walks;
    s->ls_colourings = ls_colourings;
    return PLSE_OK;
}

int plse_server_pending(plse_server s, int *queued, int *completed)
{
    if (!s) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size() + s->head_pending;
    if (completed) *completed = (int)s->done.size();
    return PLSE_OK;
}

void plse_server_destroy(plse_server s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;                          // running jobs are cancelled by the worker
        for (auto &r : s->queue) r.cancel = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->reap_mu);
        s->reap_stop = true;
    }
    s->reap_cv.notify_all();
    s->reaper.join();
    delete s;
}

}  // extern "C"
