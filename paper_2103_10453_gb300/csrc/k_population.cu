// k_population.cu -- population-level steps of MPMA for sm_103a: Hamming
// distances (Sec. 3.4), the population update (Alg. 4), nearest-untested parent
// matching (Sec. 3.5.1), AUX / UX crossover (Sec. 3.5.2, Eq. 10, Alg. 5), the
// best-solution update of Alg. 2 and the bookkeeping around them.
//
// Distances are never stored as p x p matrices.  Every colouring is kept as nb
// bit planes (bit b of the colour of 32 consecutive vertices per word), and
// D(x, y) = sum over words of popc(OR_b (X_b ^ Y_b)) is recomputed wherever a
// step needs it, 64 x 64 pairs per block with both operand tiles staged in
// shared memory.  For the planes of a 2p population at n = 70 this is about
// 3 KB per individual (L2-resident), against 2p^2 bytes of u16 matrices per
// generation in HBM for the paper's stored-matrix design.
#include <algorithm>
#include <climits>

#include "plse_pop.cuh"

namespace plse {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = x.x * 0xD2511F53u, hi0 = __umulhi(x.x, 0xD2511F53u);
        const uint32_t lo1 = x.z * 0xCD9E8D57u, hi1 = __umulhi(x.z, 0xCD9E8D57u);
        x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return x;
}

// ---- bit planes -------------------------------------------------------------
// one warp per (individual, 32-vertex word): a ballot per plane
__global__ void planes_kernel(const DevInst I, const uint8_t *__restrict__ P, int count,
                              uint32_t *__restrict__ planes)
{
    const int lane = threadIdx.x & 31;
    const long long total = (long long)count * I.nw;
    const long long step = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < total; gw += step) {
        const int x = (int)(gw / I.nw), wd = (int)(gw % I.nw);
        const int v = wd * 32 + lane;
        const uint32_t c = v < I.nv ? P[(size_t)x * I.nv + v] : 0u;
        uint32_t *dst = planes + (size_t)x * I.nw * I.nb + (size_t)wd * I.nb;
        for (int b = 0; b < I.nb; ++b) {
            const uint32_t word = __ballot_sync(FULL, (c >> b) & 1u);
            if (lane == b) dst[b] = word;
        }
    }
}

// ---- 64 x 64 distance tiles ---------------------------------------------------
// 256 threads as 16 x 16; thread (tx, ty) owns rows 4ty..4ty+3 and columns
// 4tx..4tx+3 of the tile.  Operand words are staged as [w][b][64] so that each
// thread reads its four rows (columns) with one 16-byte shared load.
constexpr int kTile = 64;
constexpr int kWC = 8;   // words per staged chunk

template <int NB>
struct TileSmem {
    uint32_t A[kWC][NB][kTile];
    uint32_t B[kWC][NB][kTile];
};

// Row swizzle of a staged (word, plane) slot: consecutive staging threads write
// one row of 56 consecutive slots, 64 words apart, which would all fall in one
// bank; XOR-ing the row with a multiple of 4 that depends on the slot spreads
// them over 16 banks and keeps every aligned group of 4 rows contiguous (the
// 16-byte row reads stay aligned).
__device__ __forceinline__ int tile_swz(int slot) { return (slot & 15) << 2; }

struct KeepAll {
    __device__ __forceinline__ bool operator()(const int (&)[4][4]) const { return true; }
};

// Distances between rows ra[0..63] and columns cb[0..63] (indices into the
// plane array; -1 = padding) accumulated into acc[4][4].  With PRUNE, after
// every staged chunk of kWC words each thread asks keep(acc) whether one of its
// pairs still needs the rest of the words; when no thread does, the tile stops
// there and acc holds partial sums (a lower bound of each distance).
template <int NB, bool PRUNE = false, class Keep = KeepAll>
__device__ __forceinline__ void tile_distances(const uint32_t *__restrict__ planesA,
                                               const uint32_t *__restrict__ planesB, int nw,
                                               const int *ra, const int *cb, TileSmem<NB> &sm,
                                               int (&acc)[4][4], const Keep &keep = Keep())
{
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const size_t stride = (size_t)nw * NB;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0;
    bool need = true;
    for (int w0 = 0; w0 < nw; w0 += kWC) {
        const int wc = min(kWC, nw - w0);
        if constexpr (PRUNE) {
            if (!__syncthreads_or(need)) break;      // no pair of the tile can still matter
        } else {
            __syncthreads();
        }
        // stage: 64 rows x wc*NB words for A and for B
        for (int q = tid; q < kTile * kWC * NB; q += 256) {
            const int r = q / (kWC * NB), rest = q % (kWC * NB);
            const int wq = rest / NB, b = rest % NB;
            uint32_t va = 0u, vb = 0u;
            if (wq < wc) {
                const int xa = ra[r], xb = cb[r];
                if (xa >= 0) va = __ldg(planesA + (size_t)xa * stride + (size_t)(w0 + wq) * NB + b);
                if (xb >= 0) vb = __ldg(planesB + (size_t)xb * stride + (size_t)(w0 + wq) * NB + b);
            }
            const int rs = r ^ tile_swz(wq * NB + b);
            sm.A[wq][b][rs] = va;
            sm.B[wq][b][rs] = vb;
        }
        __syncthreads();
        for (int wq = 0; wq < wc; ++wq) {
            uint32_t x[4], y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) x[a] = y[a] = 0u;
            uint32_t o[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) o[a][b] = 0u;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int sw = tile_swz(wq * NB + b);
                const uint4 xa = *reinterpret_cast<const uint4 *>(&sm.A[wq][b][(4 * ty) ^ sw]);
                const uint4 yb = *reinterpret_cast<const uint4 *>(&sm.B[wq][b][(4 * tx) ^ sw]);
                x[0] = xa.x; x[1] = xa.y; x[2] = xa.z; x[3] = xa.w;
                y[0] = yb.x; y[1] = yb.y; y[2] = yb.z; y[3] = yb.w;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) o[a][c] |= x[a] ^ y[c];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] += __popc(o[a][c]);
        }
        if constexpr (PRUNE) need = keep(acc);
    }
}

// D[a][b] for an arbitrary A x B (plse_distances)
template <int NB>
__global__ void __launch_bounds__(256) distance_matrix_kernel(const DevInst I, const uint32_t *planesA,
                                                              int na, const uint32_t *planesB, int nb,
                                                              int32_t *D)
{
    __shared__ TileSmem<NB> sm;
    __shared__ int ra[kTile], cb[kTile];
    const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    if (threadIdx.x < kTile) {
        const int r = r0 + threadIdx.x, c = c0 + threadIdx.x;
        ra[threadIdx.x] = r < na ? r : -1;
        cb[threadIdx.x] = c < nb ? c : -1;
    }
    __syncthreads();
    int acc[4][4];
    tile_distances<NB>(planesA, planesB, I.nw, ra, cb, sm, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int r = r0 + 4 * ty + a, q = c0 + 4 * tx + c;
            if (r < na && q < nb) D[(size_t)r * nb + q] = acc[a][c];
        }
}

// ---- Alg. 4 -------------------------------------------------------------------
// rank of each candidate in the (e, index) order
__global__ void rank_kernel(const int64_t *__restrict__ e, int m, int32_t *__restrict__ order,
                            const int *skip)
{
    if (skip && *skip) return;
    __shared__ int64_t ks[1024];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ex = x < m ? e[x] : 0;
    int rank = 0;
    for (int base = 0; base < m; base += 1024) {
        __syncthreads();
        for (int q = threadIdx.x; q < 1024 && base + q < m; q += blockDim.x) ks[q] = e[base + q];
        __syncthreads();
        const int lim = min(1024, m - base);
        if (x < m)
            for (int q = 0; q < lim; ++q) {
                const int64_t ey = ks[q];
                rank += (ey < ex) || (ey == ex && base + q < x);
            }
    }
    if (x < m) order[rank] = x;
}

// chunk-local distance tiles: D between sorted positions of one chunk
template <int NB>
__global__ void __launch_bounds__(256) chunk_local_kernel(const DevInst I, const uint32_t *planes,
                                                          const int32_t *order, int m,
                                                          uint16_t *Dloc, const int *skip)
{
    if (skip && *skip) return;
    __shared__ TileSmem<NB> sm;
    __shared__ int ra[kTile], cb[kTile];
    const int chunk = blockIdx.x, ti = blockIdx.y >> 1, tj = blockIdx.y & 1;
    const int base = chunk * kChunk;
    if (threadIdx.x < kTile) {
        const int pr = base + ti * kTile + threadIdx.x, pc = base + tj * kTile + threadIdx.x;
        ra[threadIdx.x] = pr < m ? order[pr] : -1;
        cb[threadIdx.x] = pc < m ? order[pc] : -1;
    }
    __syncthreads();
    int acc[4][4];
    tile_distances<NB>(planes, planes, I.nw, ra, cb, sm, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    uint16_t *out = Dloc + (size_t)chunk * kChunk * kChunk;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
            out[(ti * kTile + 4 * ty + a) * kChunk + tj * kTile + 4 * tx + c] = (uint16_t)acc[a][c];
}

// Sequential greedy over one chunk of sorted candidates (one warp).  Lane l
// holds positions l, l+32, l+64, l+96 of the chunk with their current minimum
// distance to the accepted set; the chunk's own distances are staged in shared
// memory (Dc) so each sequential step costs only shared loads and one shuffle.
// Values other blocks write during the pass (mind, the state) are read through
// L2 (ld.global.cg), never from a possibly stale L1 line.
__device__ __forceinline__ void resolve_chunk(int chunk, int m, int p, int nv, int gamma, const int32_t *order,
                                              const int32_t *mind, const uint16_t *Dloc, int32_t *acc,
                                              int32_t *rej, SelState *s, uint16_t *Dc)
{
    const int lane = threadIdx.x & 31;
    const int base = chunk * kChunk;
    const uint4 *src = reinterpret_cast<const uint4 *>(Dloc + (size_t)chunk * kChunk * kChunk);
    uint4 *dst = reinterpret_cast<uint4 *>(Dc);
    for (int q = lane; q < kChunk * kChunk / 8; q += 32) dst[q] = src[q];
    int md[kChunk / 32], cd[kChunk / 32];
#pragma unroll
    for (int q = 0; q < kChunk / 32; ++q) {
        const int pos = base + lane + 32 * q;
        md[q] = pos < m ? __ldcg(&mind[pos]) : INT_MAX;
        cd[q] = pos < m ? order[pos] : -1;
    }
    __syncwarp();
    int nacc = __ldcg(&s->nacc), nrej = __ldcg(&s->nrej);
    const int lim = min(kChunk, m - base);
    for (int qpos = 0; qpos < lim && nacc < p; ++qpos) {
        int mine = INT_MAX, cmine = -1;
#pragma unroll
        for (int q = 0; q < kChunk / 32; ++q)
            if (q == (qpos >> 5)) { mine = md[q]; cmine = cd[q]; }
        const int dmin = __shfl_sync(FULL, mine, qpos & 31);
        const int cand = __shfl_sync(FULL, cmine, qpos & 31);
        const bool accept = (nacc == 0) || ((long long)gamma * dmin > nv);   // D > |V| / gamma
        if (accept) {
            if (lane == 0) acc[nacc] = cand;
            ++nacc;
#pragma unroll
            for (int q = 0; q < kChunk / 32; ++q) {
                const int qq = lane + 32 * q;
                if (qq > qpos) md[q] = min(md[q], (int)Dc[qpos * kChunk + qq]);
            }
        } else {
            if (lane == 0) rej[nrej] = cand;
            ++nrej;
        }
    }
    if (lane == 0) {
        s->nacc = nacc;
        s->nrej = nrej;
        if (nacc >= p) s->done = 1;
    }
}

// Alg. 4 uses a minimum distance only in the test gamma * D > |V|, i.e.
// D >= cut with cut = floor(|V| / gamma) + 1.  A tile of the minimum-distance
// update therefore stops counting once every valid pair has reached cut: the
// minimum it stores is then a partial sum >= cut, which passes the test exactly
// when the true minimum does, and a minimum below cut is always exact (the tile
// runs to the end while one of its pairs is below cut).
struct KeepBelowCut {
    int cut;
    bool rv[4], cv[4];
    __device__ __forceinline__ bool operator()(const int (&acc)[4][4]) const
    {
        bool k = false;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) k |= rv[a] && cv[c] && acc[a][c] < cut;
        return k;
    }
};

// min distance of the 64 candidates of tile `tb` after chunk `chunk` to the
// members accepted in that chunk (acc[a0 .. a1)), exact below `cut`; every
// thread of the block
template <int NB>
__device__ __forceinline__ void update_mind_tile(const DevInst &I, const uint32_t *planes, int chunk, int tb, int m,
                                                 const int32_t *order, int32_t *mind, const int32_t *accl, int a0,
                                                 int a1, int cut, TileSmem<NB> &sm, int *ra, int *cb,
                                                 int (*rowmin)[17])
{
    const int first = (chunk + 1) * kChunk + tb * kTile;
    if (first >= m) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int best[4] = {INT_MAX, INT_MAX, INT_MAX, INT_MAX};
    for (int c0 = a0; c0 < a1; c0 += kTile) {
        __syncthreads();
        if (threadIdx.x < kTile) {
            const int pr = first + threadIdx.x, ac = c0 + threadIdx.x;
            ra[threadIdx.x] = pr < m ? order[pr] : -1;
            cb[threadIdx.x] = ac < a1 ? __ldcg(&accl[ac]) : -1;
        }
        __syncthreads();
        KeepBelowCut keep;
        keep.cut = cut;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            keep.rv[q] = ra[4 * ty + q] >= 0;
            keep.cv[q] = cb[4 * tx + q] >= 0;
        }
        int acc[4][4];
        tile_distances<NB, true>(planes, planes, I.nw, ra, cb, sm, acc, keep);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (cb[4 * tx + c] >= 0) best[a] = min(best[a], acc[a][c]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) rowmin[4 * ty + a][tx] = best[a];
    __syncthreads();
    if (threadIdx.x < kTile) {
        int v = INT_MAX;
        for (int q = 0; q < 16; ++q) v = min(v, rowmin[threadIdx.x][q]);
        const int pos = first + threadIdx.x;
        if (pos < m && v != INT_MAX) atomicMin(&mind[pos], v);   // tiles of several chunks may overlap in time
    }
    __syncthreads();
}

// Alg. 4 after the ranking, as one dataflow launch.  The pass is a fixed list
// of work items in dependency order: for each chunk k of 128 ranked candidates
// the item R_k (the sequential greedy of resolve_chunk on chunk k), then one
// item U_{k,t} per 64-candidate tile t after chunk k (the minimum distances of
// those candidates to the members accepted in chunk k).  Blocks claim items
// from one counter in list order.  R_k waits until R_{k-1} and every U_{k',t}
// covering chunk k (k' < k) have finished; U_{k,t} waits for R_k.  Each wait is
// on an item claimed earlier, i.e. held by a block that is already running, so
// the pass completes with any number of resident blocks (no cooperative launch:
// it can share the GPU with other kernels), and the updates of chunk k overlap
// the resolution of chunk k+1, which needs only the two tiles covering it.
// Tiles of different chunks may lower one candidate's minimum at the same time:
// atomicMin, whose result does not depend on their order.  Every wait is
// bounded (kFlowSpins polls); a block that gives up sets the error word and
// leaves, and the blocks waiting behind it leave as soon as they see it.
constexpr unsigned long long kFlowSpins = 1ull << 24;

// first item of chunk k: chunk k' < C-1 holds 1 + tiles(k') items with
// tiles(k') = 2 (C-2-k') + e, e = tiles covering the last (partial) chunk
__device__ __forceinline__ long long flow_start(int k, int C, int e)
{
    return (long long)k * (1 + e) + 2LL * k * (C - 2) - (long long)k * (k - 1);
}

// thread 0: wait until *w >= target; false (error word set) if the bound runs
// out or another block has already given up
__device__ __forceinline__ bool flow_wait(const int *w, int target, int *err)
{
    const volatile int *vw = w;
    const volatile int *ve = err;
    unsigned long long spins = 0;
    while (*vw < target) {
        if (++spins > kFlowSpins || *ve) {
            atomicOr(err, 1);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

template <int NB>
__global__ void __launch_bounds__(256) select_flow_kernel(const DevInst I, const uint32_t *planes, int m, int p,
                                                          int gamma, const int32_t *order, int32_t *mind,
                                                          const uint16_t *Dloc, int32_t *acc, int32_t *rej,
                                                          SelState *s, int32_t *flow, const int *skip)
{
    if (skip && *skip) return;
    extern __shared__ __align__(16) uint8_t dsm[];
    TileSmem<NB> &sm = *reinterpret_cast<TileSmem<NB> *>(dsm);
    uint16_t *Dc = reinterpret_cast<uint16_t *>(dsm + sizeof(TileSmem<NB>));
    __shared__ int ra[kTile], cb[kTile];
    __shared__ int rowmin[kTile][17];
    __shared__ int it_k, it_t, it_ok, it_done, it_a0, it_a1;
    SelFlow *f = reinterpret_cast<SelFlow *>(flow);
    const int C = (m + kChunk - 1) / kChunk;
    int *upd = flow + kSelFlowHeader, *accn = flow + kSelFlowHeader + C;
    const int e = (m - (C - 1) * kChunk + kTile - 1) / kTile;
    const long long total = flow_start(C - 1, C, e) + 1;
    const int cut = (int)((long long)I.nv / gamma + 1);     // gamma * D > |V|  <=>  D >= cut
    for (;;) {
        if (threadIdx.x == 0) {
            const long long x = (long long)atomicAdd(&f->next, 1u);
            int k = -1, t = 0, ok = 1, done = 0, a0 = 0, a1 = 0;
            if (x < total) {
                int lo = 0, hi = C - 1;                  // the last chunk k with flow_start(k) <= x
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (flow_start(mid, C, e) <= x) lo = mid; else hi = mid - 1;
                }
                k = lo;
                t = (int)(x - flow_start(k, C, e)) - 1;  // -1: R_k, else tile t of U_k
                if (t < 0) {
                    ok = flow_wait(&f->resolved, k, &f->err) &&
                         flow_wait(&upd[k], k * (k == C - 1 ? e : 2), &f->err);
                } else {
                    ok = flow_wait(&f->resolved, k + 1, &f->err);
                    if (ok) {
                        a0 = k ? __ldcg(&accn[k - 1]) : 0;
                        a1 = __ldcg(&accn[k]);
                    }
                }
                if (ok) done = __ldcg(&s->done);
            }
            it_k = k; it_t = t; it_ok = ok; it_done = done; it_a0 = a0; it_a1 = a1;
        }
        __syncthreads();
        const int k = it_k, t = it_t;
        if (k < 0 || !it_ok) return;
        if (t < 0) {
            // R_k; thread 0 (lane 0 of the resolving warp) wrote the state, acc and rej
            if (!it_done && threadIdx.x < 32) resolve_chunk(k, m, p, I.nv, gamma, order, mind, Dloc, acc, rej, s, Dc);
            __syncthreads();
            if (threadIdx.x == 0) {
                accn[k] = __ldcg(&s->nacc);
                __threadfence();
                atomicAdd(&f->resolved, 1);
            }
        } else {
            if (!it_done && it_a1 > it_a0)
                update_mind_tile<NB>(I, planes, k, t, m, order, mind, acc, it_a0, it_a1, cut, sm, ra, cb, rowmin);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0) atomicAdd(&upd[k + 1 + t / 2], 1);
        }
        __syncthreads();
    }
}

// fill rule and the final selection list
__global__ void finish_selection_kernel(int p, const SelState *s, const int32_t *acc, const int32_t *rej,
                                        int32_t *sel, int32_t *filled, const SelFlow *flow, int *error_flag,
                                        const int *skip)
{
    if (skip && *skip) return;
    if (flow && flow->err) {               // a wait of the dataflow pass gave up: the selection
        for (int q = threadIdx.x; q < p; q += blockDim.x) sel[q] = q;   // stays valid, the error is reported
        if (threadIdx.x == 0 && error_flag) atomicOr(error_flag, 2);
        return;
    }
    const int nacc = s->nacc;
    const int need = p - nacc;
    for (int q = threadIdx.x; q < p; q += blockDim.x)
        sel[q] = q < nacc ? acc[q] : rej[q - nacc];
    if (threadIdx.x == 0 && filled) *filled = need > 0 ? need : 0;
}

// ---- parent matching (Sec. 3.5.1, Alg. 5) ---------------------------------------
template <int NB>
__global__ void __launch_bounds__(256) matching_kernel(const DevInst I, const uint32_t *planes, int p,
                                                       const uint32_t *uid, uint32_t *tested,
                                                       int32_t *tcount, int cap, int32_t *partner,
                                                       int32_t *dist, const int *skip)
{
    if (skip && *skip) return;
    __shared__ TileSmem<NB> sm;
    __shared__ int ra[kTile], cb[kTile];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.x * kTile;
    if (threadIdx.x < kTile) ra[threadIdx.x] = (r0 + threadIdx.x) < p ? r0 + (int)threadIdx.x : -1;
    // per owned row: best allowed key and best plain key, key = d << 16 | j
    uint32_t ballow[4], bplain[4];
    int tc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ballow[a] = bplain[a] = 0xffffffffu;
        const int i = r0 + 4 * ty + a;
        tc[a] = i < p ? tcount[i] : 0;
    }
    for (int c0 = 0; c0 < p; c0 += kTile) {
        __syncthreads();
        if (threadIdx.x < kTile) cb[threadIdx.x] = (c0 + threadIdx.x) < p ? c0 + (int)threadIdx.x : -1;
        __syncthreads();
        int acc[4][4];
        tile_distances<NB>(planes, planes, I.nw, ra, cb, sm, acc);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = r0 + 4 * ty + a;
            if (i >= p) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = c0 + 4 * tx + c;
                if (j >= p || j == i) continue;
                const uint32_t key = ((uint32_t)acc[a][c] << 16) | (uint32_t)j;
                bplain[a] = min(bplain[a], key);
                if (key < ballow[a]) {
                    const uint32_t uj = __ldg(&uid[j]);
                    const uint32_t *L = tested + (size_t)i * cap;
                    bool seen = false;
                    for (int q = 0; q < tc[a]; ++q) seen |= (L[q] == uj);
                    if (!seen) ballow[a] = key;
                }
            }
        }
    }
    // reduce over the 16 threads of each row group (same warp half)
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            ballow[a] = min(ballow[a], __shfl_xor_sync(FULL, ballow[a], o));
            bplain[a] = min(bplain[a], __shfl_xor_sync(FULL, bplain[a], o));
        }
    }
    if (tx == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = r0 + 4 * ty + a;
            if (i >= p) continue;
            const uint32_t key = ballow[a] != 0xffffffffu ? ballow[a] : bplain[a];
            const int j = (int)(key & 0xffffu);
            partner[i] = j;
            dist[i] = (int)(key >> 16);
            uint32_t *L = tested + (size_t)i * cap;
            const int cnt = tcount[i];
            if (cnt == cap) {
                for (int q = 0; q + 1 < cap; ++q) L[q] = L[q + 1];
                L[cap - 1] = uid[j];
            } else {
                L[cnt] = uid[j];
                tcount[i] = cnt + 1;
            }
        }
    }
}

template <int NB>
__global__ void random_matching_kernel(const DevInst I, const uint32_t *planes, int p, int gen,
                                       uint32_t k0, uint32_t k1, int32_t *partner, int32_t *dist,
                                       const int *skip)
{
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p) return;
    const uint4 u = philox4x32_10(make_uint4(0u, (uint32_t)i, ((uint32_t)gen << 8) | (kPurposeMatch << 4), 0u), k0, k1);
    int j = (int)__umulhi(u.x, (uint32_t)(p - 1));
    if (j >= i) ++j;
    partner[i] = j;
    const size_t stride = (size_t)I.nw * NB;
    const uint32_t *X = planes + (size_t)i * stride, *Y = planes + (size_t)j * stride;
    int d = 0;
    for (int wd = 0; wd < I.nw; ++wd) {
        uint32_t o = 0;
#pragma unroll
        for (int b = 0; b < NB; ++b) o |= X[wd * NB + b] ^ Y[wd * NB + b];
        d += __popc(o);
    }
    dist[i] = d;
}

__global__ void fill_int_kernel(int32_t *x, int n, int value, const int *skip)
{
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = value;
}

// ---- AUX / UX crossover -----------------------------------------------------------
__global__ void crossover_kernel(const DevInst I, int p, const uint8_t *__restrict__ P,
                                 const int32_t *__restrict__ partner, const int32_t *__restrict__ dist,
                                 int gen, uint32_t k0, uint32_t k1, int beta, int ux,
                                 uint8_t *__restrict__ O, const int *skip)
{
    if (skip && *skip) return;
    const int nblk = (I.nv + 3) >> 2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)p * nblk) return;
    const int i = (int)(idx / nblk), b = (int)(idx % nblk);
    const int j = partner[i];
    const long long d = dist[i];
    long long a, bb;
    if (ux) { a = 1; bb = 2; }
    else {
        bb = (long long)beta * d;          // p_ij = 1 - |V| / (beta D), Eq. 10
        a = bb - I.nv;
        if (a < 0) a = 0;
    }
    const uint4 u = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)i, ((uint32_t)gen << 8) | (kPurposeXover << 4), 0u), k0, k1);
    const uint32_t us[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = 4 * b + q;
        if (v >= I.nv) break;
        const bool take_i = (d == 0) || ((unsigned long long)us[q] * (unsigned long long)bb <
                                         ((unsigned long long)a << 32));
        O[(size_t)i * I.nv + v] = take_i ? P[(size_t)i * I.nv + v] : P[(size_t)j * I.nv + v];
    }
}

}  // namespace

// ---- host launchers ------------------------------------------------------------
#define NB_DISPATCH(nb, CALL)                  \
    switch (nb) {                              \
        case 1: { constexpr int NBV = 1; CALL; } break; \
        case 2: { constexpr int NBV = 2; CALL; } break; \
        case 3: { constexpr int NBV = 3; CALL; } break; \
        case 4: { constexpr int NBV = 4; CALL; } break; \
        case 5: { constexpr int NBV = 5; CALL; } break; \
        case 6: { constexpr int NBV = 6; CALL; } break; \
        default: { constexpr int NBV = 7; CALL; } break; \
    }

static unsigned grid_for(long long threads, int block)
{
    long long g = (threads + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 0x7fffffffLL) g = 0x7fffffffLL;
    return (unsigned)g;
}

cudaError_t launch_planes(const DevInst &I, const uint8_t *P, int count, uint32_t *planes, cudaStream_t st)
{
    if (count <= 0 || I.nv == 0) return cudaSuccess;
    const long long warps = (long long)count * I.nw;
    unsigned blocks = grid_for(warps * 32, 256);
    if (blocks > 65535u * 16u) blocks = 65535u * 16u;
    planes_kernel<<<blocks, 256, 0, st>>>(I, P, count, planes);
    return cudaGetLastError();
}

cudaError_t launch_distance_matrix(const DevInst &I, const uint32_t *planesA, int na,
                                   const uint32_t *planesB, int nb, int32_t *D, cudaStream_t st)
{
    if (na <= 0 || nb <= 0) return cudaSuccess;
    dim3 grid((nb + kTile - 1) / kTile, (na + kTile - 1) / kTile);
    NB_DISPATCH(I.nb, (distance_matrix_kernel<NBV><<<grid, 256, 0, st>>>(I, planesA, na, planesB, nb, D)));
    return cudaGetLastError();
}

template <int NB>
static cudaError_t launch_select_flow(const DevInst &I, int m, int p, int gamma, const PopScratch &ps,
                                      const int *skip, cudaStream_t st)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorUnknown;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t dyn = sizeof(TileSmem<NB>) + sizeof(uint16_t) * kChunk * kChunk;
    cudaError_t e = cudaFuncSetAttribute(select_flow_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, select_flow_kernel<NB>, 256, dyn);
    if (e != cudaSuccess) return e;
    // one block per item at most, and no more than fit on the device at once
    // (the pass needs only one to be resident; more overlap the tile updates)
    const int C = (m + kChunk - 1) / kChunk;
    const long long items = (long long)C + (long long)(C - 1) * C;      // an upper bound
    const int blocks = (int)std::max(1LL, std::min(items, (long long)sms * std::max(per_sm, 1)));
    select_flow_kernel<NB><<<blocks, 256, dyn, st>>>(I, ps.planes_ref, m, p, gamma, ps.order, ps.mind, ps.Dloc,
                                                     ps.acc, ps.rej, ps.sel_state, ps.flow, skip);
    return cudaGetLastError();
}

cudaError_t launch_pop_update(const DevInst &I, int p, const uint32_t *planes, const int64_t *e,
                              int gamma, const PopScratch &ps_in, int32_t *sel, int32_t *filled,
                              const int *skip, cudaStream_t st, long long *kernels)
{
    const int m = 2 * p;
    PopScratch ps = ps_in;
    ps.planes_ref = planes;
    const int nchunks = (m + kChunk - 1) / kChunk;
    cudaError_t err = cudaMemsetAsync(ps.sel_state, 0, sizeof(SelState), st);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(ps.flow, 0, sizeof(int32_t) * sel_flow_ints(nchunks), st);
    if (err != cudaSuccess) return err;
    rank_kernel<<<grid_for(m, 256), 256, 0, st>>>(e, m, ps.order, skip);
    fill_int_kernel<<<grid_for(m, 256), 256, 0, st>>>(ps.mind, m, INT_MAX, skip);
    NB_DISPATCH(I.nb, (chunk_local_kernel<NBV><<<dim3(nchunks, 4), 256, 0, st>>>(I, planes, ps.order, m, ps.Dloc, skip)));
    NB_DISPATCH(I.nb, (err = launch_select_flow<NBV>(I, m, p, gamma, ps, skip, st)));
    if (err != cudaSuccess) return err;
    finish_selection_kernel<<<1, 256, 0, st>>>(p, ps.sel_state, ps.acc, ps.rej, sel, filled,
                                               reinterpret_cast<const SelFlow *>(ps.flow), ps.error_flag, skip);
    if (kernels) *kernels = 5;
    return cudaGetLastError();
}

cudaError_t launch_matching(const DevInst &I, int p, const uint32_t *planes, const uint32_t *uid,
                            uint32_t *tested, int32_t *tcount, int cap, int random, int gen,
                            uint64_t seed, int32_t *partner, int32_t *dist, const int *skip,
                            cudaStream_t st)
{
    if (p <= 1) return cudaSuccess;
    if (random) {
        NB_DISPATCH(I.nb, (random_matching_kernel<NBV><<<grid_for(p, 256), 256, 0, st>>>(I, planes, p, gen, (uint32_t)seed, (uint32_t)(seed >> 32), partner, dist, skip)));
    } else {
        NB_DISPATCH(I.nb, (matching_kernel<NBV><<<(p + kTile - 1) / kTile, 256, 0, st>>>(I, planes, p, uid, tested, tcount, cap, partner, dist, skip)));
    }
    return cudaGetLastError();
}

cudaError_t launch_crossover(const DevInst &I, int p, const uint8_t *P, const int32_t *partner,
                             const int32_t *dist, int gen, uint64_t seed, int beta, int ux, uint8_t *O,
                             const int *skip, cudaStream_t st)
{
    const long long total = (long long)p * ((I.nv + 3) / 4);
    if (total == 0) return cudaSuccess;
    crossover_kernel<<<grid_for(total, 256), 256, 0, st>>>(I, p, P, partner, dist, gen, (uint32_t)seed,
                                                           (uint32_t)(seed >> 32), beta, ux, O, skip);
    return cudaGetLastError();
}

}  // namespace plse
