// autotune.cu -- picks the launch knobs of a handle's local search (threads per
// walk, walks per block, where a walk's current colouring lives) for a
// population size by timing short probe launches of the real kernel on the
// handle's own instance.  The knobs never change results, only speed (the move
// of every iteration is the minimum of a total order, whatever the split of the
// candidates among threads), so the choice is free to follow the measurement.
// Choices are cached for the process, keyed by device, n, |V| and population.
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "plse_handle.cuh"

namespace plse {
namespace {

struct Choice {
    int lanes, walks, place;
    double rate;
};

std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, Choice> g_tune_cache;

struct ProbeBuffers {
    plse_instance *h;
    cudaStream_t st;
    uint8_t *P = nullptr, *Q = nullptr;
    plse_walk_stats *stats = nullptr;
    ~ProbeBuffers()
    {
        h_free(h, P, st);
        h_free(h, Q, st);
        h_free(h, stats, st);
    }
};

}  // namespace
}  // namespace plse

using namespace plse;

extern "C" int plse_autotune(plse_handle h, int pop, int probe_iters, int *lanes, int *walks, int *colourings,
                             double *moves_per_s)
{
    if (!h || pop < 1 || pop > 65535 || probe_iters < 1 || probe_iters > (1 << 20))
        return h ? fail(h, PLSE_EINVAL, "plse_autotune: invalid argument") : PLSE_EINVAL;
    auto report = [&](const Choice &c) {
        if (lanes) *lanes = c.lanes;
        if (walks) *walks = c.walks;
        if (colourings) *colourings = c.place;
        if (moves_per_s) *moves_per_s = c.rate;
    };
    if (h->nv == 0) {
        report(Choice{0, 0, 0, 0.0});
        return PLSE_OK;
    }
    const auto key = std::make_tuple(h->device, h->n, h->nv, pop);
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            h->ls_lanes = it->second.lanes;
            h->ls_walks = it->second.walks;
            h->ls_splace = it->second.place;
            report(it->second);
            return PLSE_OK;
        }
    }
    int rc = run_drain(h);
    if (rc) return rc;
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return fail(h, PLSE_ECUDA, "plse_autotune: stream");
    const int saved[3] = {h->ls_lanes, h->ls_walks, h->ls_splace};
    Choice best{saved[0], saved[1], saved[2], -1.0};
    {
        ProbeBuffers b;
        b.h = h;
        b.st = st;
        const size_t PV = (size_t)pop * h->nv;
        void *q[3] = {nullptr, nullptr, nullptr};
        if (h_malloc(h, &q[0], PV, st) != cudaSuccess || h_malloc(h, &q[1], PV, st) != cudaSuccess ||
            h_malloc(h, &q[2], sizeof(plse_walk_stats) * (size_t)pop, st) != cudaSuccess) {
            for (void *x : q) h_free(h, x, st);
            cudaStreamDestroy(st);
            return fail(h, PLSE_ENOMEM, "plse_autotune: probe buffers");
        }
        b.P = static_cast<uint8_t *>(q[0]);
        b.Q = static_cast<uint8_t *>(q[1]);
        b.stats = static_cast<plse_walk_stats *>(q[2]);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        std::vector<plse_walk_stats> hs((size_t)pop);
        // probe input: random colourings after one short walk and the repair
        // (closer to the offspring of a running GA than random colourings)
        rc = plse_init_population(h, pop, 0x5eedULL, b.P, st);
        if (!rc) rc = plse_local_search(h, b.P, b.P, pop, 0, 0, probe_iters, 0x5eedULL,
                                        PLSE_LS_PHASE1 | PLSE_LS_REPAIR, nullptr, nullptr, nullptr, st);
        // candidates: (threads per walk, walks per block (0 = as many as fit), colourings)
        const int cand[][3] = {{32, 0, 1}, {32, 0, 2}, {16, 0, 2}, {64, 0, 1}, {32, 8, 1}, {128, 0, 1}};
        std::vector<std::tuple<int, int, int>> seen;
        for (const auto &c : cand) {
            if (rc) break;
            h->ls_lanes = c[0];
            h->ls_walks = c[1];
            h->ls_splace = c[2];
            const LSLaunch L = plan_local_search(h->di, h->device, pop, c[0], c[1], c[2]);
            if (L.blocks <= 0) continue;
            const auto shape = std::make_tuple(L.group, L.walks, L.s_smem);
            bool dup = false;
            for (const auto &s : seen) dup = dup || s == shape;
            if (dup) continue;
            seen.push_back(shape);
            double moves = 0, ms = 0;
            for (int rep = 0; rep < 3 && !rc; ++rep) {       // the first launch is a warm-up
                cudaEventRecord(e0, st);
                rc = plse_local_search(h, b.P, b.Q, pop, 0, 1 + rep, probe_iters, 0x5eedULL, PLSE_LS_PHASE1,
                                       nullptr, nullptr, b.stats, st);
                cudaEventRecord(e1, st);
                if (rc) break;
                if (cudaMemcpyAsync(hs.data(), b.stats, sizeof(plse_walk_stats) * (size_t)pop,
                                    cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = fail(h, PLSE_ECUDA, "plse_autotune: probe");
                    break;
                }
                if (rep == 0) continue;
                float t = 0;
                cudaEventElapsedTime(&t, e0, e1);
                ms += t;
                for (const auto &w : hs) moves += (double)w.moves;
            }
            if (rc) break;
            const double rate = ms > 0 ? moves / (ms * 1e-3) : 0.0;
            if (rate > best.rate) best = Choice{c[0], c[1], c[2], rate};
        }
        if (!rc) rc = plse_sync(h, st);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamSynchronize(st);
    }
    cudaStreamDestroy(st);
    if (rc) {
        h->ls_lanes = saved[0];
        h->ls_walks = saved[1];
        h->ls_splace = saved[2];
        return rc;
    }
    h->ls_lanes = best.lanes;
    h->ls_walks = best.walks;
    h->ls_splace = best.place;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    report(best);
    return PLSE_OK;
}
