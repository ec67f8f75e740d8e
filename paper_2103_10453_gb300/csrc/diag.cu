// diag.cu -- a shared-memory bandwidth probe: the measured peak against which
// the local search's byte rate is reported.  Every thread of a block streams
// 16-byte loads from its own bank-aligned slots of a 32 KB shared buffer
// (conflict-free: a warp's 32 loads cover all 32 banks four times, the
// 128-byte-per-clock width of one SM), folding the data into a register so that
// nothing is optimised away.  Two blocks of 1024 threads per SM, timed by CUDA
// events on a private stream.
#include <cuda_runtime.h>

#include "plse.h"

namespace {

constexpr int kThreads = 1024;
constexpr int kWords = 32 * 1024 / 16;     // uint4 slots of the buffer

__global__ void __launch_bounds__(kThreads) smem_stream_kernel(int iters, uint32_t seed, uint32_t *sink)
{
    __shared__ uint4 buf[kWords];
    for (int q = threadIdx.x; q < kWords; q += kThreads)
        buf[q] = make_uint4(seed ^ q, seed + q, seed * 3u + q, seed ^ (q << 7));
    __syncthreads();
    uint32_t acc = 0;
    for (int it = 0; it < iters; ++it) {
        const int base = (it * 160 + threadIdx.x) & (kWords - 1);   // moves every round
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint4 x = buf[(base + u * 512) & (kWords - 1)];
            acc ^= x.x + x.y + x.z + x.w;
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;        // keeps the loads live; practically never true
}

}  // namespace

extern "C" int plse_smem_bandwidth(int iters, double *bytes_per_s, double *ms)
{
    if (iters < 1 || !bytes_per_s) return PLSE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PLSE_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t *sink = nullptr;
    int rc = PLSE_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMallocAsync(reinterpret_cast<void **>(&sink), sizeof(uint32_t), st) != cudaSuccess) {
        rc = PLSE_ECUDA;
    } else {
        smem_stream_kernel<<<2 * sms, kThreads, 0, st>>>(iters / 4 + 1, 7u, sink);   // warm-up
        cudaEventRecord(e0, st);
        smem_stream_kernel<<<2 * sms, kThreads, 0, st>>>(iters, 11u, sink);
        cudaEventRecord(e1, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = PLSE_ECUDA;
        } else {
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            const double bytes = 2.0 * sms * kThreads * (double)iters * 4.0 * 16.0;
            *bytes_per_s = t > 0 ? bytes / (t * 1e-3) : 0.0;
            if (ms) *ms = t;
        }
        cudaFreeAsync(sink, st);
        cudaStreamSynchronize(st);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return rc;
}
