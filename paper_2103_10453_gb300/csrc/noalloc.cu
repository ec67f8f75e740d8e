// noalloc.cu -- plse_local_search_noalloc: the tabu local search with its
// device scratch in a fixed, library-owned array instead of memory allocated at
// call time.
//
// Some callers cannot allocate device memory when they call the library: an
// application whose device memory is reserved up front by its own pool
// allocator (cudaMalloc would fail or break its budget), or a latency-critical
// loop that must not hit the implicit device-wide synchronisation of
// cudaMalloc / cudaFree.  This entry point serves them: it calls no cudaMalloc,
// cudaFree or allocating library routine.  Its scratch (the evicted-tabu
// tables, the tabu caches, the candidate lists, the member-id XOR tables, the
// colouring buffers, the per-slot clocks, the walk counter and the check flag)
// lives in
// the file-scope array below, kNoAllocScratchBytes bytes on every GPU that loads
// the library, held until the process exits.
//
// Set-up: the array's device address is obtained once per device with
// cudaGetSymbolAddress, with that device current, during the first call made on
// that device; that first call should come before any stream capture.  Every
// call shares the one array and leaves its contents behind, so each call clears
// the part it uses before its kernel runs; calls whose work overlaps on the GPU
// (e.g. on two streams) race on the array and give unspecified results.
// A failed device-side check is recorded in the array's flag word; plse_sync on
// the calling handle reads it (and clears it) like the flag of
// plse_local_search, until the next call of this entry point clears it.
#include <algorithm>
#include <mutex>

#include "plse_handle.cuh"

namespace plse {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr size_t kCounterBytes = 256;                       // walk counter + check flag
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device
int scratch_address(plse_instance *h, int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices)
        return fail(h, PLSE_ENOTSUP, "plse_local_search_noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(h, e, "plse_local_search_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_ptr[device]);
    return PLSE_OK;
}

}  // namespace
}  // namespace plse

using namespace plse;

extern "C" int plse_local_search_noalloc(plse_handle h, const uint8_t *S_in, uint8_t *S_out, int count,
                                         int ind0, int gen, int64_t iters, uint64_t seed, int flags,
                                         int32_t *f_out, int64_t *F_out, plse_walk_stats *stats, void *stream)
{
    if (!h || count < 0 || ind0 < 0 || gen < 0 || gen >= (1 << 24) || iters < 0 || iters > (1ll << 30) ||
        (flags & ~15) || !flags || ((flags & PLSE_LS_PARTIALCOL) && (flags & (PLSE_LS_PHASE1 | PLSE_LS_PHASE2))))
        return fail(h, PLSE_EINVAL, "plse_local_search_noalloc: invalid argument");
    if (count == 0) return PLSE_OK;
    if (!S_in || !S_out) return fail(h, PLSE_EINVAL, "plse_local_search_noalloc: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    if (h->nv == 0) {
        if (f_out && cudaMemsetAsync(f_out, 0, sizeof(int32_t) * count, st) != cudaSuccess) return PLSE_ECUDA;
        if (F_out && cudaMemsetAsync(F_out, 0, sizeof(int64_t) * count, st) != cudaSuccess) return PLSE_ECUDA;
        if (stats && cudaMemsetAsync(stats, 0, sizeof(plse_walk_stats) * count, st) != cudaSuccess) return PLSE_ECUDA;
        return PLSE_OK;
    }
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(h, e, "plse_local_search_noalloc: cudaGetDevice");
    unsigned char *scratch = nullptr;
    int rc = scratch_address(h, device, &scratch);
    if (rc) return rc;

    // walk slots that fit: each needs an evicted-tabu table (4 * |V| * n1p bytes),
    // a tabu cache (8 * |V| bytes), a candidate list (2 * |V| bytes), a member-id
    // XOR table (4 * n * n1p bytes), the high colour-count planes, a colouring
    // buffer (|V| rounded up to 16 bytes) and a clock word
    const size_t xr_bytes = 4 * (size_t)h->di.n * h->di.n1p;
    const size_t hp_bytes = 4 * hp_words(h->di);
    const size_t sw = sw_bytes(h->di);
    const size_t table_bytes =
        4 * (size_t)h->di.nv * h->di.n1p + 10 * (size_t)h->di.nv + xr_bytes + hp_bytes + sw;
    const size_t max_slots = (kNoAllocScratchBytes - kCounterBytes - 1536) / (table_bytes + 4);   // 1536: alignment
    if (max_slots < 1)
        return fail(h, PLSE_ENOTSUP,
                    "plse_local_search_noalloc: one walk slot needs %zu bytes of scratch, more than the %zu "
                    "available", table_bytes + 4, kNoAllocScratchBytes - kCounterBytes);
    LSLaunch L = plan_local_search(h->di, device, count, h->ls_lanes, h->ls_walks, h->ls_splace);
    if (L.blocks <= 0) return fail(h, PLSE_ENOTSUP, "plse_local_search_noalloc: local search does not fit");
    if ((size_t)L.slots() > max_slots) {
        if ((size_t)L.walks > max_slots) {
            const int cap = h->ls_walks > 0 ? std::min(h->ls_walks, (int)max_slots) : (int)max_slots;
            L = plan_local_search(h->di, device, count, h->ls_lanes, cap, h->ls_splace);
        }
        L.blocks = (int)std::min<size_t>((size_t)L.blocks, max_slots / (size_t)L.walks);
        if (L.blocks <= 0) return fail(h, PLSE_ENOTSUP, "plse_local_search_noalloc: no walk slot fits");
    }
    const size_t slots = (size_t)L.slots();
    // layout: [counters][slot clocks][evicted-tabu tables][tabu caches][lists][XOR
    // tables][high planes][colourings]; the first three must start at zero, the
    // rest is rebuilt by every walk
    int *counters = reinterpret_cast<int *>(scratch);
    uint32_t *clocks = reinterpret_cast<uint32_t *>(scratch + kCounterBytes);
    const size_t tables_off = (kCounterBytes + 4 * slots + 255) & ~size_t(255);
    uint32_t *tables = reinterpret_cast<uint32_t *>(scratch + tables_off);
    const size_t tc_off = (tables_off + slots * 4 * (size_t)h->di.nv * h->di.n1p + 255) & ~size_t(255);
    uint2 *tcache = reinterpret_cast<uint2 *>(scratch + tc_off);
    const size_t list_off = (tc_off + slots * 8 * (size_t)h->di.nv + 255) & ~size_t(255);
    uint16_t *lists = reinterpret_cast<uint16_t *>(scratch + list_off);
    const size_t xr_off = (list_off + slots * 2 * (size_t)h->di.nv + 255) & ~size_t(255);
    uint16_t *xrs = reinterpret_cast<uint16_t *>(scratch + xr_off);
    const size_t hp_off = (xr_off + slots * xr_bytes + 255) & ~size_t(255);
    uint32_t *hps = reinterpret_cast<uint32_t *>(scratch + hp_off);
    const size_t sw_off = (hp_off + slots * hp_bytes + 255) & ~size_t(255);
    uint8_t *sws = scratch + sw_off;
    const size_t used = sw_off + slots * sw;
    if (used > kNoAllocScratchBytes) return fail(h, PLSE_ENOTSUP, "plse_local_search_noalloc: scratch overflow");
    e = cudaMemsetAsync(scratch, 0, tc_off, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "plse_local_search_noalloc: clear scratch");

    const plse_params &p = h->params;
    LSArgs a;
    a.S_in = S_in;
    a.S_out = S_out;
    a.count = count;
    a.ind0 = ind0;
    a.gen = gen;
    a.flags = flags;
    a.iters1 = iters;
    a.iters2 = (int64_t)p.phase2_iter_per_v * h->nv;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.phi2_1 = p.phase1_phi2;
    a.phi2_2 = p.phase2_phi2_per_v * h->nv;
    a.alpha_num = p.alpha_num;
    a.alpha_den = p.alpha_den;
    a.tenure_rand = p.tenure_rand;
    a.alpha_recip = h->alpha_recip;
    const int tmax = max_tenure(h);
    a.span1 = (int)(a.iters1 + tmax + 2);
    a.span2 = (int)(a.iters2 + tmax + 2);
    a.f_out = f_out;
    a.F_out = F_out;
    a.stats = stats;
    a.G = tables;
    a.TC = tcache;
    a.LIST = lists;
    a.XR = xrs;
    a.HP = hps;
    a.SW = sws;
    a.slot_clock = clocks;
    set_ls_strides(h->di, a);
    a.work_counter = counters;
    a.error_flag = counters + 1;
    a.skip = nullptr;
    e = launch_local_search(h->di, a, L, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "plse_local_search_noalloc: launch");
    h->noalloc_flag = counters + 1;    // plse_sync reads (and clears) it
    return PLSE_OK;
}
