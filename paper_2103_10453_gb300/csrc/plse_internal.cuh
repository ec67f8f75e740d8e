// plse_internal.cuh -- shared declarations of the sm_103a kernels and the C ABI
// layer of libplse.so.  Nothing here is visible outside the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "plse.h"

namespace plse {

constexpr int kMaxN = 127;            // colours 0..127 fit one 128-bit mask
constexpr int kMaxTenure = 16383;     // relative u16 tabu clocks need T < 2^14
constexpr int kKeyScale = 256;        // move key = 2dF * 256 + colour
constexpr int kMaxD2 = (1 << 23) - 1; // |2dF| bound so that the key fits int32

// Philox counter purposes (third counter word = gen << 8 | purpose << 4 | phase)
enum : uint32_t { kPurposeInit = 1, kPurposeTabu = 2, kPurposeXover = 3, kPurposeMatch = 4 };

// Read-only device image of one reduced instance (Sec. 2.1-2.2, Alg. 1).
struct DevInst {
    int n;        // order
    int n1p;      // row stride of the per-row / per-column colour count tables
    int nv;       // |V|, reduced vertices in row-major cell order
    int nw;       // ceil(nv / 32): words of a vertex bitmask or of a bit plane
    int nb;       // bit planes needed for colours 0..n
    const uint16_t *rc;      // [nv] row << 8 | column
    const uint4 *dom;        // [nv] D(v) as a 128-bit mask, bit k = colour k
    const uint8_t *ndom;     // [nv] |D(v)| (colour 0 included)
    const int32_t *row_ptr;  // [n + 1] vertices of row r: row_v[row_ptr[r] .. row_ptr[r+1])
    const uint16_t *row_v;   // [nv]
    const int32_t *col_ptr;  // [n + 1]
    const uint16_t *col_v;   // [nv]
    const uint4 *allow_row;  // [n] colours 1..n not prefilled in row r (bit k = colour k)
    const uint4 *allow_col;  // [n] colours 1..n not prefilled in column c (= allow_row + n)
    const uint8_t *linelen;  // [2n] reduced vertices per row, then per column
    // D(v) \ {0} = allow_row[row(v)] & allow_col[col(v)] for every reduced vertex
};

// Scalar parameters of one local-search launch.
struct LSArgs {
    const uint8_t *S_in;
    uint8_t *S_out;
    int count, ind0, gen, flags;
    int64_t iters1, iters2;       // phase-1 / PartialCol iterations, phase-2 iterations
    uint32_t key0, key1;          // Philox key = seed
    int phi2_1, phi2_2;           // 2*phi of phase 1 and phase 2
    int alpha_num, alpha_den, tenure_rand;
    uint32_t alpha_recip;         // ceil(2^32 / alpha_den) if exact for every x <= alpha_num*|V|, else 0
    int span1, span2;             // clock span reserved per phase (iterations + max tenure + 2)
    int32_t *f_out;
    int64_t *F_out;
    plse_walk_stats *stats;
    // scratch (global memory owned by the handle's workspace)
    uint32_t *G;                  // [slots][nv * n1p] evicted tabu expiries (absolute clock)
    uint2 *TC;                    // [slots][nv] two-entry tabu caches (relative clock)
    uint16_t *LIST;               // [slots][nv] candidate lists
    uint16_t *XR;                 // [slots][2n][n1p] member-id XOR per line and colour
    uint32_t *HP;                 // [slots][2n][cw][8] colour-count planes 2..6
    uint8_t *SW;                  // [slots][nv rounded up to 16] current colourings (when not
                                  // kept in shared memory)
    uint32_t *slot_clock;         // [slots] next free clock value of each slot
    // elements per walk slot of G, TC, LIST, XR, HP and SW (a launch over several
    // instances shares one scratch set sized for the largest of them)
    size_t g_stride, tc_stride, list_stride, xr_stride, hp_stride, sw_stride;
    int *work_counter;            // dynamic walk scheduler, zeroed before launch
    int *error_flag;              // nonzero after a failed device bound check
    const int *skip;              // if non-null and nonzero at launch: return at once
    int s_smem;                   // set by the launcher: colourings in shared memory
};

struct LSLaunch {
    int blocks = 0;      // persistent blocks (one per SM at most, two below n = 64)
    int group = 32;      // threads per walk (16: two walks per warp; 32, 64, 128, 256)
    int walks = 0;       // concurrent walks per block, each with its own shared-memory slot
    size_t smem = 0;     // dynamic shared memory per block
    int colour_words = 1;// 32-bit words of a colour mask actually used (1..4)
    int s_smem = 1;      // current colourings in the shared-memory slots (else global)
    size_t stride = 0;   // multi-instance launch: shared memory per walk group
    int slots() const { return blocks * walks; }
};

// Shared-memory plan of one block (bytes): instance part, then `walks` slots.
struct SmemPlan {
    size_t inst;       // vertex coordinates, allowed-colour masks and line lengths
    size_t slot;       // one walk: [colouring], count planes 0-1, high OR, candidate masks, scalars
    size_t off_S, off_P01, off_PH, off_cmask, off_lmask, off_red;   // within a slot
    size_t total(int walks) const { return inst + slot * (size_t)walks; }
};

// One job of a multi-instance local-search launch.
struct LSJob {
    DevInst I;
    LSArgs a;
};

// Launchers (return cudaError_t of the launch; asynchronous).
cudaError_t launch_init_population(const DevInst &I, int pop, uint64_t seed, uint8_t *P,
                                   cudaStream_t st);
cudaError_t launch_local_search(const DevInst &I, const LSArgs &a, const LSLaunch &L,
                                cudaStream_t st);
// group = threads per walk (0: automatic); max_walks caps the walks per block
// (0 = no cap); s_place: 0 = colourings in shared memory unless that cuts the
// walks per block, 1 = shared memory, 2 = global memory.
LSLaunch plan_local_search(const DevInst &I, int device, int count, int group, int max_walks = 0,
                           int s_place = 0);
// One persistent launch over `count` instances of one colour-word class: as many
// blocks as are resident, walks per block and shared memory fitting the largest
// instance.  blocks = 0 if the instances differ in class or nothing fits.
LSLaunch plan_local_search_multi(const DevInst *insts, int count, int device, int group, int max_walks = 0,
                                 int s_place = 0);
// jobs: device array [njobs]; each job's work counter must be zero at launch and
// each job's scratch must hold L.slots() walk slots.
cudaError_t launch_local_search_multi(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st);

// Launch entry points of the local-search kernels of one colour-word class
// (NWC = 32-colour words, 1..4); each class is instantiated in its own
// translation unit (k_ls_w1.cu .. k_ls_w4.cu).
template <int NWC>
struct LSKernels {
    static cudaError_t launch(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st);
    // sets the block's shared-memory size; returns resident blocks per SM
    static int set_smem(int group, size_t smem, int threads);
    static cudaError_t launch_multi(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st);
    static int set_smem_multi(int group, size_t smem, int threads);
};
extern template struct LSKernels<1>;
extern template struct LSKernels<2>;
extern template struct LSKernels<3>;
extern template struct LSKernels<4>;

// 32-colour words of a colour mask over colours 0..n
__host__ __device__ inline int colour_words(int n) { return n < 32 ? 1 : n < 64 ? 2 : n < 96 ? 3 : 4; }

// bytes per walk slot of the global colouring buffer
inline size_t sw_bytes(const DevInst &I) { return ((size_t)I.nv + 15) & ~size_t(15); }

// u32 words per walk slot of the colour-count planes 2..6 kept in global memory
// ([2n lines][colour words][8])
inline size_t hp_words(const DevInst &I) { return 2 * (size_t)I.n * colour_words(I.n) * 8; }

}  // namespace plse
