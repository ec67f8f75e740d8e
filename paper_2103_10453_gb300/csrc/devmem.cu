// devmem.cu -- device and pinned host memory of the library's handles.
//
// Device buffers come from a library-owned, stream-ordered memory pool per
// device (cudaMallocFromPoolAsync / cudaFreeAsync).  Unlike cudaFree, a
// stream-ordered free never synchronizes the device, so handles can be created
// and destroyed while other runs keep the GPU busy (the request server does so
// for every request); freed blocks stay cached in the pool for the next handle.
//
// The per-run flag buffers the host polls (two generations x (f*, done)) are
// 16-byte slots cut from pinned chunks that are allocated once and reused,
// because cudaHostAlloc / cudaFreeHost are slow and may synchronize.
//
// Every call that enqueues work for a handle runs inside a StreamScope: the
// stream first waits for the handle's previous work (on whatever stream it was
// enqueued), and the handle's event is recorded after the new work.  Work on
// one handle (which shares its scratch) is thereby ordered across streams, and
// plse_destroy can free in stream order after the last of it.
#include <mutex>
#include <vector>

#include "plse_handle.cuh"

namespace plse {
namespace {

constexpr int kMaxDev = 64;
constexpr uint64_t kPoolKeepBytes = 16ull << 30;   // cached in the pool across frees

std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kMaxDev] = {};

cudaError_t pool_of(cudaStream_t st, cudaMemPool_t *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    (void)st;
    *out = g_pool[dev];
    return cudaSuccess;
}

std::mutex g_pinned_mutex;
std::vector<int *> g_pinned_free;
constexpr int kSlotInts = 4;          // one slot: 16 bytes
constexpr int kSlotsPerChunk = 1024;

}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = pool_of(st, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
}

void dev_free(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

cudaError_t h_malloc(plse_instance *h, void **p, size_t bytes, cudaStream_t st)
{
    if (!h->arena) return dev_malloc(p, bytes, st);
    const size_t off = ws_align(h->arena_used), need = bytes ? bytes : 16;
    if (off > h->arena_size || need > h->arena_size - off) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    *p = h->arena + off;
    h->arena_used = off + need;
    return cudaSuccess;
}

void h_free(plse_instance *h, void *p, cudaStream_t st)
{
    if (!p) return;
    const char *q = static_cast<const char *>(p);
    if (h->arena && q >= h->arena && q < h->arena + h->arena_size) return;   // part of the bound range
    dev_free(p, st);
}

int *pinned_slot_get()
{
    std::lock_guard<std::mutex> lk(g_pinned_mutex);
    if (g_pinned_free.empty()) {
        int *chunk = nullptr;
        if (cudaHostAlloc(reinterpret_cast<void **>(&chunk), sizeof(int) * kSlotInts * kSlotsPerChunk,
                          cudaHostAllocPortable) != cudaSuccess)
            return nullptr;
        for (int k = kSlotsPerChunk - 1; k >= 0; --k) g_pinned_free.push_back(chunk + k * kSlotInts);
    }
    int *s = g_pinned_free.back();
    g_pinned_free.pop_back();
    for (int k = 0; k < kSlotInts; ++k) s[k] = 0;
    return s;
}

void pinned_slot_put(int *s)
{
    if (!s) return;
    std::lock_guard<std::mutex> lk(g_pinned_mutex);
    g_pinned_free.push_back(s);
}

StreamScope::StreamScope(plse_instance *h_, cudaStream_t st_) : h(h_), st(st_)
{
    if (h->done_recorded) cudaStreamWaitEvent(st, h->done_ev, 0);
}

StreamScope::~StreamScope()
{
    if (cudaEventRecord(h->done_ev, st) == cudaSuccess) h->done_recorded = true;
}

}  // namespace plse
