// plse_pop.cuh -- population-level kernels (k_population.cu), library-internal.
#pragma once

#include "plse_internal.cuh"

namespace plse {

constexpr int kChunk = 128;   // Alg. 4 candidates resolved per sequential step

// device-side progress of one Alg. 4 pass
struct SelState {
    int nacc;             // members accepted so far
    int nrej;             // candidates rejected so far (in rank order)
    int done;             // nacc reached p
    int pad;
};

// dataflow words of one Alg. 4 pass (zeroed before it), followed by
// int32 upd[chunks] (finished tile updates covering chunk k) and
// int32 accn[chunks] (members accepted once chunk k is resolved)
struct SelFlow {
    unsigned next;        // next work item to claim
    int resolved;         // chunks resolved so far
    int err;              // nonzero: a block gave up waiting
    int pad;
};
constexpr int kSelFlowHeader = 4;   // int32 words of SelFlow
inline size_t sel_flow_ints(int nchunks) { return kSelFlowHeader + 2 * (size_t)nchunks; }

// device scratch of Alg. 4 for populations of up to `cap_p`
struct PopScratch {
    int cap_p = 0;
    int32_t *order = nullptr;  // [2p] candidates in (e, index) order
    int32_t *mind = nullptr;   // [2p] min distance to the accepted set, by rank
    int32_t *acc = nullptr;    // [p] accepted candidates in acceptance order
    int32_t *rej = nullptr;    // [2p] rejected candidates in rank order
    uint16_t *Dloc = nullptr;  // [chunks][kChunk][kChunk] chunk-local distances
    SelState *sel_state = nullptr;
    int32_t *flow = nullptr;   // SelFlow + upd[chunks] + accn[chunks]
    const uint32_t *planes_ref = nullptr;  // set by launch_pop_update for its kernels
    int *error_flag = nullptr;             // set by the caller: a failed pass is reported here
};

cudaError_t launch_planes(const DevInst &I, const uint8_t *P, int count, uint32_t *planes, cudaStream_t st);
cudaError_t launch_distance_matrix(const DevInst &I, const uint32_t *planesA, int na,
                                   const uint32_t *planesB, int nb, int32_t *D, cudaStream_t st);
cudaError_t launch_pop_update(const DevInst &I, int p, const uint32_t *planes, const int64_t *e,
                              int gamma, const PopScratch &ps, int32_t *sel, int32_t *filled,
                              const int *skip, cudaStream_t st,
                              long long *kernels = nullptr);
cudaError_t launch_matching(const DevInst &I, int p, const uint32_t *planes, const uint32_t *uid,
                            uint32_t *tested, int32_t *tcount, int cap, int random, int gen,
                            uint64_t seed, int32_t *partner, int32_t *dist, const int *skip,
                            cudaStream_t st);
cudaError_t launch_crossover(const DevInst &I, int p, const uint8_t *P, const int32_t *partner,
                             const int32_t *dist, int gen, uint64_t seed, int beta, int ux, uint8_t *O,
                             const int *skip, cudaStream_t st);

}  // namespace plse
