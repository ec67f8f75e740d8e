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

}  // namespace
}  // namespace plse

using namespace plse;

// ============================================================================
// plse_solve_batch
extern "C" int plse_solve_batch(plse_handle *hs, const plse_job *jobs, int count, int max_inflight,
                                int8_t *const *best_grids, plse_result *results)
{
    if (count < 0 || max_inflight < 0 || (count > 0 && (!hs || !jobs || !results))) return PLSE_EINVAL;
    if (count == 0) return PLSE_OK;
    for (int i = 0; i < count; ++i)
        if (!hs[i]) return PLSE_EINVAL;
    const auto t0 = Clock::now();
    for (int i = 0; i < count; ++i) {
        memset(&results[i], 0, sizeof(plse_result));
        results[i].status = PLSE_EINVAL;
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
    };

    int device = 0;
    int max_inflight = 0, max_queue = 0;
    int ls_warps = 0, ls_walks = 0;     // launch knobs applied to every request's handle
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
        d.res = r.res;
        d.res.ms_wall = ms_between(r.req.arrival, Clock::now());
        d.grid = std::move(r.grid);
        {
            std::lock_guard<std::mutex> lk(mu);
            cancel_running.erase(r.req.ticket);
            done.emplace(r.req.ticket, std::move(d));
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
        for (;;) {
            bool progressed = false;
            // admission
            for (int s = 0; s < max_inflight; ++s) {
                if (used[s]) continue;
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
                Running &r = slot[s];
                r = Running();
                r.req = std::move(req);
                r.res.ms_queue = ms_between(r.req.arrival, Clock::now());
                if (r.req.cancel) {
                    r.res.status = PLSE_ECANCELLED;
                    note_detail(r.res, nullptr);
                    finish(r);
                    continue;
                }
                plse_instance *h = nullptr;
                int rc = plse_create(r.req.n, r.req.grid.data(), &h);
                if (!rc) rc = plse_set_params(h, &r.req.params);
                if (!rc) {
                    std::lock_guard<std::mutex> lk(mu);
                    rc = plse_set_launch(h, ls_warps, ls_walks);
                }
                if (!rc) rc = run_begin(h, r.req.job.pop, r.req.job.generations, r.req.job.iters, r.req.job.seed,
                                        streams[s]);
                r.grid.assign((size_t)r.req.n * r.req.n, 0);
                r.a = Active{h, streams[s], r.grid.data(), &r.res, false};
                if (rc) {
                    r.res.status = rc;
                    note_detail(r.res, h);
                    cudaStreamSynchronize(streams[s]);
                    if (h) h->session.active = 0;
                    finish(r);
                    continue;
                }
                used[s] = 1;
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                bool any = false;
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

int plse_server_create(int max_inflight, int max_queue, plse_server *out)
{
    if (!out || max_inflight < 1 || max_inflight > 256 || max_queue < 0) return PLSE_EINVAL;
    plse_server_s *s = new (std::nothrow) plse_server_s();
    if (!s) return PLSE_ENOMEM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return PLSE_ECUDA;
    }
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

int plse_server_set_launch(plse_server s, int ls_warps, int ls_walks)
{
    if (!s || ls_warps < 0 || ls_walks < 0) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->ls_warps = ls_warps;
    s->ls_walks = ls_walks;
    return PLSE_OK;
}

int plse_server_pending(plse_server s, int *queued, int *completed)
{
    if (!s) return PLSE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int)s->queue.size();
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
