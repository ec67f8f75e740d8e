// k_local_search.cu -- population initialisation (Sec. 3.2) and the launch
// planning and colour-word dispatch of the tabu local search (Alg. 3, Sec. 3.3;
// Sec. 3.7).  The walk itself and its kernels are in ls_walk.cuh; each
// colour-word class (1..4 words of 32 colours) is compiled in its own
// translation unit, k_ls_w1.cu .. k_ls_w4.cu.
#include <algorithm>

#include "ls_walk.cuh"

namespace plse {
namespace {

// one thread per (individual, block of four vertices): one Philox block each
__global__ void init_population_kernel(const DevInst I, int pop, uint32_t k0, uint32_t k1, uint8_t *P)
{
    const int nblk = (I.nv + 3) >> 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)pop * nblk) return;
    const int i = (int)(idx / nblk), b = (int)(idx % nblk);
    const uint4 u = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)i, kPurposeInit << 4, 0u), k0, k1);
    const uint32_t us[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = 4 * b + q;
        if (v >= I.nv) break;
        uint32_t k = bounded(us[q], (uint32_t)__ldg(&I.ndom[v]) - 1u);   // k-th colour of D(v)\{0}
        const uint4 d = __ldg(&I.dom[v]);
        uint32_t m[4] = {d.x & ~1u, d.y, d.z, d.w};
        int colour = 0;
        for (int wq = 0; wq < 4 && !colour; ++wq) {
            const uint32_t cnt = __popc(m[wq]);
            if (k < cnt) {
                uint32_t x = m[wq];
                for (uint32_t s = 0; s < k; ++s) x &= x - 1;
                colour = wq * 32 + __ffs(x) - 1;
            } else {
                k -= cnt;
            }
        }
        P[(size_t)i * I.nv + v] = (uint8_t)colour;
    }
}

}  // namespace

LSLaunch plan_local_search(const DevInst &I, int device, int count, int group, int max_walks, int s_place)
{
    LSLaunch L;
    L.blocks = 0;
    L.walks = 0;
    L.smem = 0;
    if (group <= 0) group = 32;                    // automatic: one warp per walk
    L.group = group <= 16 ? 16 : group <= 32 ? 32 : group <= 64 ? 64 : group <= 128 ? 128 : 256;
    L.colour_words = colour_words(I.n);
    const int warps = L.group < 32 ? 1 : L.group / 32;
    int max_smem = 0, sms = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    // one block per SM holding as many walk slots as fit (at most the kernel's
    // thread limit: 640 for 64 <= n < 96, 384 from 96, 256 below 64 with two
    // blocks); the colouring stays in the slot unless that would cut the walks
    long long by_threads = std::max(1, max_threads_for(L.colour_words) / L.group);
    if (max_walks > 0) by_threads = std::min<long long>(by_threads, max_walks);
    const SmemPlan ps = make_plan(I, warps, true), pg = make_plan(I, warps, false);
    const long long walks_s = ((long long)max_smem - (long long)ps.inst) / (long long)ps.slot;
    const long long walks_g = ((long long)max_smem - (long long)pg.inst) / (long long)pg.slot;
    bool s_smem = s_place == 1 ? true : s_place == 2 ? false : walks_s >= by_threads;
    long long walks = std::min<long long>(s_smem ? walks_s : walks_g, by_threads);
    if (L.group == 16) walks &= ~1ll;              // 16-lane groups run in pairs, one pair per warp
    if (walks < 1) return L;
    const SmemPlan &p = s_smem ? ps : pg;
    L.s_smem = s_smem ? 1 : 0;
    L.walks = (int)walks;
    L.smem = p.total(L.walks);
    const int threads = L.group * L.walks;
    int per_sm = 0;
    switch (L.colour_words) {
        case 1: per_sm = LSKernels<1>::set_smem(L.group, L.smem, threads); break;
        case 2: per_sm = LSKernels<2>::set_smem(L.group, L.smem, threads); break;
        case 3: per_sm = LSKernels<3>::set_smem(L.group, L.smem, threads); break;
        default: per_sm = LSKernels<4>::set_smem(L.group, L.smem, threads); break;
    }
    long long blocks = ((long long)count + walks - 1) / walks;
    blocks = std::min<long long>(blocks, (long long)sms * std::max(per_sm, 1));
    L.blocks = per_sm > 0 ? (int)blocks : 0;
    return L;
}

LSLaunch plan_local_search_multi(const DevInst *insts, int count, int device, int group, int max_walks, int s_place)
{
    LSLaunch L;
    if (count <= 0) return L;
    if (group <= 0) group = 32;
    L.group = group <= 16 ? 16 : group <= 32 ? 32 : group <= 64 ? 64 : group <= 128 ? 128 : 256;
    L.colour_words = colour_words(insts[0].n);
    for (int k = 1; k < count; ++k)
        if (colour_words(insts[k].n) != L.colour_words) return L;   // one colour-word class per launch
    const int warps = L.group < 32 ? 1 : L.group / 32;
    int max_smem = 0, sms = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    long long by_threads = std::max(1, max_threads_for(L.colour_words) / L.group);
    if (max_walks > 0) by_threads = std::min<long long>(by_threads, max_walks);
    // one group's part of shared memory: its job descriptor and a slot of the
    // largest job's layout
    size_t slot_s = 0, slot_g = 0;
    for (int k = 0; k < count; ++k) {
        slot_s = std::max(slot_s, make_plan(insts[k], warps, true).slot);
        slot_g = std::max(slot_g, make_plan(insts[k], warps, false).slot);
    }
    const size_t desc = align16(sizeof(JobDesc));
    const long long walks_s = (long long)max_smem / (long long)(desc + slot_s);
    const long long walks_g = (long long)max_smem / (long long)(desc + slot_g);
    const bool s_smem = s_place == 1 ? true : s_place == 2 ? false : walks_s >= by_threads;
    const long long walks = std::min<long long>(s_smem ? walks_s : walks_g, by_threads);
    if (walks < 1) return L;
    L.s_smem = s_smem ? 1 : 0;
    L.walks = (int)walks;
    L.stride = desc + (s_smem ? slot_s : slot_g);
    L.smem = L.stride * (size_t)L.walks;
    const int threads = L.group * L.walks;
    int per_sm = 0;
    switch (L.colour_words) {
        case 1: per_sm = LSKernels<1>::set_smem_multi(L.group, L.smem, threads); break;
        case 2: per_sm = LSKernels<2>::set_smem_multi(L.group, L.smem, threads); break;
        case 3: per_sm = LSKernels<3>::set_smem_multi(L.group, L.smem, threads); break;
        default: per_sm = LSKernels<4>::set_smem_multi(L.group, L.smem, threads); break;
    }
    L.blocks = per_sm > 0 ? sms * per_sm : 0;
    return L;
}

cudaError_t launch_local_search_multi(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st)
{
    if (L.blocks <= 0 || njobs <= 0) return cudaErrorInvalidConfiguration;
    switch (L.colour_words) {
        case 1: return LSKernels<1>::launch_multi(jobs, njobs, L, st);
        case 2: return LSKernels<2>::launch_multi(jobs, njobs, L, st);
        case 3: return LSKernels<3>::launch_multi(jobs, njobs, L, st);
        default: return LSKernels<4>::launch_multi(jobs, njobs, L, st);
    }
}

cudaError_t launch_local_search(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    if (L.blocks <= 0) return cudaErrorInvalidConfiguration;
    LSArgs b = a;
    b.s_smem = L.s_smem;
    switch (L.colour_words) {
        case 1: return LSKernels<1>::launch(I, b, L, st);
        case 2: return LSKernels<2>::launch(I, b, L, st);
        case 3: return LSKernels<3>::launch(I, b, L, st);
        default: return LSKernels<4>::launch(I, b, L, st);
    }
}

cudaError_t launch_init_population(const DevInst &I, int pop, uint64_t seed, uint8_t *P, cudaStream_t st)
{
    const long long total = (long long)pop * ((I.nv + 3) / 4);
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const long long blocks = (total + threads - 1) / threads;
    init_population_kernel<<<(unsigned)blocks, threads, 0, st>>>(I, pop, (uint32_t)seed, (uint32_t)(seed >> 32), P);
    return cudaGetLastError();
}

}  // namespace plse