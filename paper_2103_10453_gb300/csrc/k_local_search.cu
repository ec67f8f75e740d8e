// k_local_search.cu -- population initialisation (Sec. 3.2) and the tabu local
// search of MPMA (Alg. 3: PLITS phases 1 and 2, Sec. 3.3; PartialCol and the
// greedy conflict removal, Sec. 3.7) for sm_103a.
//
// Design (GB300-first):
//  * One thread block per walk (1, 2, 4 or 8 warps), persistent over walks
//    handed out by an atomic counter.  Everything an iteration touches lives in
//    the block's shared memory: the colouring, the gamma table, the tabu cache,
//    the candidate set and the instance's vertex coordinates and colour masks.
//  * The gamma table of the incremental evaluation (Sec. 3.3) is held in
//    factored form.  On a Latin-square graph the neighbours of v = (r, c) are
//    exactly its row- and column-mates, so
//        gamma[v][k] = R[r][k] + K[c][k] - 2*[S(v) = k],
//    with R / K the per-row / per-column colour counts.  A move updates four
//    counters instead of deg(v) table entries.  The counts are kept twice:
//    as bytes (single lookups) and as 7 bit planes per 32 colours, so that the
//    best colour of a candidate vertex, min over its domain of R + K, comes out
//    of a bit-sliced add and a most-significant-plane-first elimination over
//    whole 32-colour words instead of a loop over colours.
//  * The tabu list (expiry per (v, colour)) is a 2-entry per-vertex cache with
//    16-bit clocks relative to the phase, backed by an exact global table G for
//    entries evicted while possibly live.  A vertex whose evicted entries have
//    all expired never touches G.
//  * The candidate set V0 u C(S) is a bitmask updated after each move from the
//    row and column of the moved vertex only.  Each warp compacts and scans its
//    own slice of the bitmask; the best move is the minimum of the key
//    (2dF, (v - r) mod |V|, j) over all threads -- a total order, so the result
//    does not depend on how the work is split.  Two block barriers per move.
#include <climits>

#include "plse_internal.cuh"

namespace plse {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t kRebaseAt = 49152;   // relative clock rebased before it reaches this
constexpr uint32_t kRebaseBy = 32768;
constexpr uint32_t kNoKey = 0xffffffffu;
constexpr int kPlanes = 8;              // plane slots per 32-colour word (7 used)

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 multiplies,
// a word permutation and a key xor; Weyl key schedule.
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

__device__ __forceinline__ uint32_t bounded(uint32_t u, uint32_t k) { return __umulhi(u, k); }

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline int colour_words(int n) { return n < 32 ? 1 : n < 64 ? 2 : n < 96 ? 3 : 4; }

__host__ __device__ inline SmemPlan make_plan(const DevInst &I, int warps)
{
    const int cw = colour_words(I.n);
    SmemPlan p;
    p.off_rc = 0;
    p.off_allow = align16(2 * (size_t)I.nv);
    p.off_S = p.off_allow + 2 * 16 * (size_t)I.n;
    p.off_B = align16(p.off_S + (size_t)I.nv);
    p.off_R = align16(p.off_B + (size_t)I.nv);
    p.off_K = p.off_R + (size_t)I.n * I.n1p;
    p.off_RP = align16(p.off_K + (size_t)I.n * I.n1p);
    p.off_KP = p.off_RP + 4 * (size_t)I.n * cw * kPlanes;
    p.off_cmask = p.off_KP + 4 * (size_t)I.n * cw * kPlanes;
    p.off_clist = align16(p.off_cmask + 4 * (size_t)I.nw);
    p.off_tc = align16(p.off_clist + 2 * 32 * (size_t)I.nw);
    p.off_red = align16(p.off_tc + 8 * (size_t)I.nv);
    p.total = align16(p.off_red + 2 * 16 * (size_t)warps + 64);
    return p;
}

// Per-block view of the shared memory of one walk slot.
struct Ctx {
    const uint16_t *rc;   // [nv] row << 8 | column
    const uint4 *allow;   // [2n]: allowed colours per row, then per column
    uint8_t *S, *B;       // current / best colouring
    uint8_t *R8, *K8;     // colour counts per row / column [n][n1p]
    uint32_t *RP, *KP;    // colour-count bit planes [n][cw][8]
    uint32_t *cmask;      // candidate bitmask [nw]
    uint16_t *clist;      // per-warp compacted candidates [nw * 32]
    uint2 *tc;            // tabu cache [nv]: x = e0 | e1 << 16, y = c0 | c1 << 8 | emax << 16
    uint2 *red;           // [2][warps] best key per warp (double-buffered by iteration parity)
    int *red_cnt;         // [2][warps] candidates per warp
    int *scal;            // [8] block scalars
    int cw;
};

template <int NW>
__device__ __forceinline__ Ctx carve(uint8_t *base, const DevInst &I)
{
    const SmemPlan p = make_plan(I, NW);
    Ctx c;
    c.rc = reinterpret_cast<const uint16_t *>(base + p.off_rc);
    c.allow = reinterpret_cast<const uint4 *>(base + p.off_allow);
    c.S = base + p.off_S;
    c.B = base + p.off_B;
    c.R8 = base + p.off_R;
    c.K8 = base + p.off_K;
    c.RP = reinterpret_cast<uint32_t *>(base + p.off_RP);
    c.KP = reinterpret_cast<uint32_t *>(base + p.off_KP);
    c.cmask = reinterpret_cast<uint32_t *>(base + p.off_cmask);
    c.clist = reinterpret_cast<uint16_t *>(base + p.off_clist);
    c.tc = reinterpret_cast<uint2 *>(base + p.off_tc);
    c.red = reinterpret_cast<uint2 *>(base + p.off_red);
    c.red_cnt = reinterpret_cast<int *>(base + p.off_red + 2 * 8 * NW);
    c.scal = c.red_cnt + 2 * NW;
    c.cw = colour_words(I.n);
    return c;
}

struct LaneStats {
    long long iterations, moves, cand, pairs, deg, improvements, uncolored;
};

template <int NW>
__device__ __forceinline__ long long block_sum64(long long x, long long *scratch)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = x;
    __syncthreads();
    long long t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += scratch[k];
    __syncthreads();
    return t;
}

template <int NW>
__device__ __forceinline__ int block_sum(int x, const Ctx &c)
{
    x = __reduce_add_sync(FULL, x);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) c.scal[threadIdx.x >> 5] = x;
    __syncthreads();
    int t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += c.scal[k];
    __syncthreads();
    return t;
}

template <int NW>
__device__ __forceinline__ uint32_t block_max(uint32_t x, const Ctx &c)
{
    x = __reduce_max_sync(FULL, x);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) c.scal[threadIdx.x >> 5] = (int)x;
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t = max(t, (uint32_t)c.scal[k]);
    __syncthreads();
    return t;
}

// ---- colour counts ---------------------------------------------------------------
__device__ __forceinline__ void plane_step(uint32_t *P, uint32_t bit, bool inc)
{
    uint32_t carry = bit;
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        const uint32_t x = P[p];
        const uint32_t t = inc ? (x & carry) : (~x & carry);
        P[p] = x ^ carry;
        carry = t;
    }
}

// +1 / -1 on count[line][k] in bytes and planes (one thread)
__device__ __forceinline__ void count_step(uint8_t *C8, uint32_t *CP, const DevInst &I, int cw, int line,
                                           int k, bool inc)
{
    C8[line * I.n1p + k] += inc ? 1 : (uint8_t)0xFF;
    plane_step(CP + ((size_t)line * cw + (k >> 5)) * kPlanes, 1u << (k & 31), inc);
}

template <int NW>
__device__ void build_counts(const DevInst &I, const Ctx &c)
{
    const int tid = threadIdx.x, T = 32 * NW;
    uint32_t *RK = reinterpret_cast<uint32_t *>(c.R8);
    for (int q = tid; q < (2 * I.n * I.n1p) / 4; q += T) RK[q] = 0u;
    __syncthreads();
    for (int r = tid; r < 2 * I.n; r += T) {
        const bool col = r >= I.n;
        const int line = col ? r - I.n : r;
        const int32_t *ptr = col ? I.col_ptr : I.row_ptr;
        const uint16_t *lst = col ? I.col_v : I.row_v;
        uint8_t *C8 = (col ? c.K8 : c.R8) + line * I.n1p;
        for (int q = __ldg(&ptr[line]); q < __ldg(&ptr[line + 1]); ++q) {
            const int k = c.S[__ldg(&lst[q])];
            if (k) C8[k] += 1;
        }
    }
    __syncthreads();
    // bit planes from the byte counts: one task per (table, line, colour word)
    const int tasks = 2 * I.n * c.cw;
    for (int q = tid; q < tasks; q += T) {
        const bool col = q >= I.n * c.cw;
        const int rem = col ? q - I.n * c.cw : q;
        const int line = rem / c.cw, wq = rem % c.cw;
        const uint8_t *C8 = (col ? c.K8 : c.R8) + line * I.n1p;
        uint32_t pl[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < 32; ++b) {
            const int k = wq * 32 + b;
            const uint32_t v = k <= I.n ? C8[k] : 0u;
#pragma unroll
            for (int p = 0; p < 7; ++p) pl[p] |= ((v >> p) & 1u) << b;
        }
        uint32_t *dst = (col ? c.KP : c.RP) + ((size_t)line * c.cw + wq) * kPlanes;
#pragma unroll
        for (int p = 0; p < 7; ++p) dst[p] = pl[p];
        dst[7] = 0u;
    }
    __syncthreads();
}

__device__ __forceinline__ int gamma_own(const DevInst &I, const Ctx &c, int v, int k)
{
    const uint16_t rc = c.rc[v];
    return c.R8[(rc >> 8) * I.n1p + k] + c.K8[(rc & 255) * I.n1p + k] - 2;
}

// candidate bitmask: PLITS -> V0 u C(S); PartialCol -> V0.  Returns f and |C|.
template <int NW>
__device__ void build_cands(const DevInst &I, const Ctx &c, bool only_v0, int &f, int &nconf)
{
    int lf = 0, lc = 0;
    for (int wd = threadIdx.x; wd < I.nw; wd += 32 * NW) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int v = wd * 32 + b;
            if (v >= I.nv) break;
            const int k = c.S[v];
            if (k == 0) {
                bits |= 1u << b;
                ++lf;
            } else if (gamma_own(I, c, v, k) > 0) {
                ++lc;
                if (!only_v0) bits |= 1u << b;
            }
        }
        c.cmask[wd] = bits;
    }
    f = block_sum<NW>(lf, c);
    nconf = block_sum<NW>(lc, c);
}

// conflicting edges c(S) = sum over rows and columns of C(count, 2)
template <int NW>
__device__ int conflict_edges(const DevInst &I, const Ctx &c)
{
    int s = 0;
    for (int q = threadIdx.x; q < 2 * I.n * I.n1p; q += 32 * NW) {
        const int x = c.R8[q];
        s += x * (x - 1) / 2;
    }
    return block_sum<NW>(s, c);
}

template <int NW>
__device__ __forceinline__ void block_copy(uint8_t *dst, const uint8_t *src, int n)
{
    for (int q = threadIdx.x; q < n; q += 32 * NW) dst[q] = src[q];
}

// compacts this warp's slice of the candidate bitmask; returns its count
template <int NW>
__device__ __forceinline__ int compact_warp(const DevInst &I, const Ctx &c, int &w0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    w0 = (warp * I.nw) / NW;
    const int w1 = ((warp + 1) * I.nw) / NW;
    int cnt = 0;
    for (int wd = w0 + lane; wd < w1; wd += 32) cnt += __popc(c.cmask[wd]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    int pos = w0 * 32 + incl - cnt;
    const int total = __shfl_sync(FULL, incl, 31);
    for (int wd = w0 + lane; wd < w1; wd += 32) {
        uint32_t bits = c.cmask[wd];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            c.clist[pos++] = (uint16_t)(wd * 32 + b);
        }
    }
    __syncwarp();
    return total;
}

// ---- tabu cache ---------------------------------------------------------------
struct Clock {
    uint32_t base;    // absolute clock of iteration 0 of the phase
    uint32_t shift;   // relative clock = t - shift
};

template <int NW>
__device__ __forceinline__ void tabu_reset(const DevInst &I, const Ctx &c)
{
    for (int v = threadIdx.x; v < I.nv; v += 32 * NW) c.tc[v] = make_uint2(0u, 0xFFFFu);
}

template <int NW>
__device__ void tabu_rebase(const DevInst &I, const Ctx &c)
{
    for (int v = threadIdx.x; v < I.nv; v += 32 * NW) {
        const uint2 x = c.tc[v];
        uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16, em = x.y >> 16;
        e0 = e0 > kRebaseBy ? e0 - kRebaseBy : 0u;
        e1 = e1 > kRebaseBy ? e1 - kRebaseBy : 0u;
        em = em > kRebaseBy ? em - kRebaseBy : 0u;
        c.tc[v] = make_uint2(e0 | (e1 << 16), (x.y & 0xFFFFu) | (em << 16));
    }
}

// (v, k) tabu until relative clock e (inclusive); evicts to G when needed
__device__ __forceinline__ void tabu_insert(const DevInst &I, const Ctx &c, uint32_t *G, const Clock &ck,
                                            int v, int k, uint32_t e)
{
    const uint2 x = c.tc[v];
    uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16;
    uint32_t c0 = x.y & 0xFFu, c1 = (x.y >> 8) & 0xFFu, em = x.y >> 16;
    if (c0 == (uint32_t)k) {
        e0 = e;
    } else if (c1 == (uint32_t)k) {
        e1 = e;
    } else {
        const bool second = e1 < e0;                     // evict the earlier expiry
        const uint32_t ev = second ? e1 : e0, cv = second ? c1 : c0;
        if (cv != 0xFFu) {
            G[(size_t)v * I.n1p + cv] = ck.base + ck.shift + ev;
            em = max(em, ev);
        }
        if (second) { c1 = (uint32_t)k; e1 = e; } else { c0 = (uint32_t)k; e0 = e; }
    }
    c.tc[v] = make_uint2(e0 | (e1 << 16), c0 | (c1 << 8) | (em << 16));
}

template <int NWC>
__device__ __forceinline__ void clear_bit(uint32_t (&m)[NWC], uint32_t k)
{
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (q == (int)(k >> 5)) m[q] &= ~(1u << (k & 31));
}

template <int NWC>
__device__ __forceinline__ bool test_bit(const uint32_t (&m)[NWC], uint32_t k)
{
    bool r = false;
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (q == (int)(k >> 5)) r = (m[q] >> (k & 31)) & 1u;
    return r;
}

// min over colours j in m of s_j = R[r][j] + K[c][j], lowest j on ties, from
// the bit planes: bit-sliced add, then most-significant-plane-first
// elimination.  Returns -1 if m is empty.
template <int NWC>
__device__ __forceinline__ int bits_min(const uint32_t *RPr, const uint32_t *KPc, const uint32_t (&m)[NWC],
                                        int &smin)
{
    uint32_t s[NWC][8];
    uint32_t anym = 0;
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        const uint4 r0 = *reinterpret_cast<const uint4 *>(RPr + q * kPlanes);
        const uint4 r1 = *reinterpret_cast<const uint4 *>(RPr + q * kPlanes + 4);
        const uint4 k0 = *reinterpret_cast<const uint4 *>(KPc + q * kPlanes);
        const uint4 k1 = *reinterpret_cast<const uint4 *>(KPc + q * kPlanes + 4);
        const uint32_t a[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
        const uint32_t b[7] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z};
        uint32_t carry = 0u;
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            const uint32_t x = a[p] ^ b[p];
            s[q][p] = x ^ carry;
            carry = (a[p] & b[p]) | (carry & x);
        }
        s[q][7] = carry;
        anym |= m[q];
    }
    if (!anym) return -1;
    uint32_t set[NWC];
    uint32_t any0 = 0, any1 = 0, hi = 0;
    uint32_t h1[NWC];
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        h1[q] = s[q][1] | s[q][2] | s[q][3] | s[q][4] | s[q][5] | s[q][6] | s[q][7];
        hi |= s[q][3] | s[q][4] | s[q][5] | s[q][6] | s[q][7];
        set[q] = m[q] & ~(s[q][0] | h1[q]);      // s_j = 0
        any0 |= set[q];
    }
    if (any0) {
        smin = 0;
    } else {
#pragma unroll
        for (int q = 0; q < NWC; ++q) {
            set[q] = m[q] & s[q][0] & ~h1[q];    // s_j = 1
            any1 |= set[q];
        }
        if (any1) {
            smin = 1;
        } else {
            uint32_t val = 0;
#pragma unroll
            for (int q = 0; q < NWC; ++q) set[q] = m[q];
#pragma unroll
            for (int p = 7; p >= 0; --p) {
                if (p > 2 && !hi) continue;
                uint32_t t[NWC], anyt = 0;
#pragma unroll
                for (int q = 0; q < NWC; ++q) {
                    t[q] = set[q] & ~s[q][p];
                    anyt |= t[q];
                }
                if (anyt) {
#pragma unroll
                    for (int q = 0; q < NWC; ++q) set[q] = t[q];
                } else {
                    val |= 1u << p;
                }
            }
            smin = (int)val;
        }
    }
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (set[q]) return q * 32 + __ffs(set[q]) - 1;
    return -1;
}

// Best admissible move of candidate v as key 2dF*256 + j (INT_MAX: none).
//   v uncoloured:  2dF(j) = base_unc + mult*s_j        (j != 0)
//   v coloured i:  2dF(j) = mult*(s_j - g_i)            (j != 0, j != i)
//                  2dF(0) = 2 - mult*g_i
// with s_j = R[r][j] + K[c][j] and g_i = gamma[v][i] (Sec. 3.3).  A move is
// admissible if not tabu, or if 2dF < A (aspiration by the phase's best).
template <int NWC>
__device__ __forceinline__ int eval_vertex(const DevInst &I, const Ctx &c, const uint32_t *G, const Clock &ck,
                                           uint32_t trel, int v, int mult, int base_unc, int A, int &pairs)
{
    const int i = c.S[v];
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255;
    const uint8_t *R8r = c.R8 + r * I.n1p;
    const uint8_t *K8c = c.K8 + cc * I.n1p;
    const int gi = i ? (int)R8r[i] + (int)K8c[i] - 2 : 0;
    const int base2 = i ? -mult * gi : base_unc;
    const int d2zero = 2 - mult * gi;
    const uint4 ar = c.allow[r], ac = c.allow[I.n + cc];
    const uint32_t ar4[4] = {ar.x, ar.y, ar.z, ar.w}, ac4[4] = {ac.x, ac.y, ac.z, ac.w};
    uint32_t m[NWC];
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        m[q] = ar4[q] & ac4[q];
        cnt += __popc(m[q]);
    }
    pairs = cnt;                                   // |D(v)| - 1 scanned moves
    if (i) clear_bit<NWC>(m, (uint32_t)i);
    bool has0 = (i != 0);

    const uint2 te = c.tc[v];
    const uint32_t e0 = te.x & 0xFFFFu, e1 = te.x >> 16;
    const uint32_t c0 = te.y & 0xFFu, c1 = (te.y >> 8) & 0xFFu, em = te.y >> 16;
    int best = INT_MAX;
    if (em < trel) {
        // fast path: only the cached colours c0, c1 can be tabu
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
            const uint32_t cs = sx ? c1 : c0, es = sx ? e1 : e0;
            if (cs == 0u) {
                if (has0) {
                    has0 = false;
                    if (es < trel || d2zero < A) best = min(best, d2zero * kKeyScale);
                }
            } else if (cs < 128u && test_bit<NWC>(m, cs)) {
                clear_bit<NWC>(m, cs);
                const int d2 = base2 + mult * ((int)R8r[cs] + (int)K8c[cs]);
                if (es < trel || d2 < A) best = min(best, d2 * kKeyScale + (int)cs);
            }
        }
        if (has0) best = min(best, d2zero * kKeyScale);
        int smin = 0;
        const int jb = bits_min<NWC>(c.RP + (size_t)r * NWC * kPlanes, c.KP + (size_t)cc * NWC * kPlanes, m, smin);
        if (jb >= 0) best = min(best, (base2 + mult * smin) * kKeyScale + jb);
    } else {
        // slow path: evicted entries of v may still be live, consult G
        const uint32_t tabs = ck.base + ck.shift + trel;
        const uint32_t *Gv = G + (size_t)v * I.n1p;
        if (has0) {
            const bool tabu = (c0 == 0u) ? (e0 >= trel) : (c1 == 0u) ? (e1 >= trel) : (Gv[0] >= tabs);
            if (!tabu || d2zero < A) best = min(best, d2zero * kKeyScale);
        }
#pragma unroll
        for (int q = 0; q < NWC; ++q) {
            uint32_t bits = m[q];
            while (bits) {
                const uint32_t j = q * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                const int d2 = base2 + mult * ((int)R8r[j] + (int)K8c[j]);
                const bool tabu = (j == c0) ? (e0 >= trel) : (j == c1) ? (e1 >= trel) : (Gv[j] >= tabs);
                if (!tabu || d2 < A) best = min(best, d2 * kKeyScale + (int)j);
            }
        }
    }
    return best;
}

__device__ __forceinline__ int vertex_degree(const DevInst &I, const Ctx &c, int v)
{
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255;
    return (__ldg(&I.row_ptr[r + 1]) - __ldg(&I.row_ptr[r]) - 1) +
           (__ldg(&I.col_ptr[cc + 1]) - __ldg(&I.col_ptr[cc]) - 1);
}

// reserve a clock range for one phase of this slot
template <int NW>
__device__ Clock claim_clock(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, int slot, int span)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t base = a.slot_clock[slot] + 1u;
        if (base > 0x7FFFFFFFu - (uint32_t)span) base = 0u;   // wrap: clear the slot
        c.scal[0] = (int)base;
    }
    __syncthreads();
    uint32_t base = (uint32_t)c.scal[0];
    if (base == 0u) {
        const size_t words = (size_t)I.nv * I.n1p;
        for (size_t q = threadIdx.x; q < words; q += 32 * NW) G[q] = 0u;
        base = 1u;
    }
    __syncthreads();
    if (threadIdx.x == 0) a.slot_clock[slot] = base + (uint32_t)span;
    Clock ck;
    ck.base = base;
    ck.shift = 0u;
    return ck;
}

// the move key of a candidate: hi = 2dF + 2^30; lo = rot << 16 | j << 8 | i
__device__ __forceinline__ void key_update(int kv, int v, int rsh, int nv, int i, uint32_t &khi, uint32_t &klo)
{
    int rot = v - rsh;
    if (rot < 0) rot += nv;
    const uint32_t hi = (uint32_t)((kv >> 8) + (1 << 30));
    const uint32_t lo = ((uint32_t)rot << 16) | ((uint32_t)(kv & 255) << 8) | (uint32_t)i;
    if (hi < khi || (hi == khi && lo < klo)) { khi = hi; klo = lo; }
}

// block-wide best key; returns the number of candidates counted by all warps
template <int NW>
__device__ __forceinline__ int block_best(const Ctx &c, int parity, uint32_t khi, uint32_t klo, int nloc,
                                          uint32_t &mhi, uint32_t &mlo)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t whi = __reduce_min_sync(FULL, khi);
    uint32_t wlo = __reduce_min_sync(FULL, khi == whi ? klo : kNoKey);
    if (lane == 0) {
        c.red[parity * NW + warp] = make_uint2(whi, wlo);
        c.red_cnt[parity * NW + warp] = nloc;
    }
    __syncthreads();
    mhi = kNoKey;
    mlo = kNoKey;
    int total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const uint2 x = c.red[parity * NW + k];
        if (x.x < mhi || (x.x == mhi && x.y < mlo)) { mhi = x.x; mlo = x.y; }
        total += c.red_cnt[parity * NW + k];
    }
    return total;
}

// ---- PLITS phase (Alg. 3 with phi2 = 2*phi) --------------------------------
template <int NWC, int NW>
__device__ bool plits_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, int slot, int ind,
                            int phase, int64_t N, int phi2, int span, LaneStats &st, long long &F2best_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    build_counts<NW>(I, c);
    int f, nconf;
    build_cands<NW>(I, c, false, f, nconf);
    const int cedges = conflict_edges<NW>(I, c);
    long long F2 = 2LL * f + (long long)phi2 * cedges;
    long long F2best = F2;
    block_copy<NW>(c.B, c.S, I.nv);
    tabu_reset<NW>(I, c);
    Clock ck = claim_clock<NW>(I, a, c, G, slot, span);

    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | (uint32_t)phase;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    for (long long t = 1; t <= N; ++t) {
        if (f + nconf == 0) break;                       // nothing left to improve
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            __syncthreads();
            tabu_rebase<NW>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            __syncthreads();
        }
        const int q = (int)((t - 1) & 31);
        if (q == 0) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + lane), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(FULL, Lr, q);
        const int rsh = (int)__shfl_sync(FULL, rotr, q);
        const long long A64 = F2best - F2;
        const int A = A64 < -(1LL << 30) ? -(1 << 30) : (int)A64;

        int w0;
        const int nloc = compact_warp<NW>(I, c, w0);
        uint32_t khi = kNoKey, klo = kNoKey;
        for (int qq = lane; qq < nloc; qq += 32) {
            const int v = c.clist[w0 * 32 + qq];
            int pairs;
            const int kv = eval_vertex<NWC>(I, c, G, ck, trel, v, phi2, -2, A, pairs);
            st.pairs += pairs;
            if (kv != INT_MAX) key_update(kv, v, rsh, I.nv, c.S[v], khi, klo);
        }
        uint32_t mhi, mlo;
        const int ncand = block_best<NW>(c, (int)(t & 1), khi, klo, nloc, mhi, mlo);   // barrier
        if (ncand != f + nconf) { ok = false; break; }
        st.iterations += 1;
        st.cand += ncand;
        if (mhi == kNoKey) continue;                     // every move tabu

        const int d2 = (int)mhi - (1 << 30);
        const int j = (int)((mlo >> 8) & 255u), i = (int)(mlo & 255u);
        int v = (int)(mlo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        f += (j == 0) - (i == 0);
        F2 += d2;
        if (warp == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            if (lane == 0) {
                c.S[v] = (uint8_t)j;
                if (i) { count_step(c.R8, c.RP, I, c.cw, r, i, false); count_step(c.K8, c.KP, I, c.cw, cc, i, false); }
                if (j) { count_step(c.R8, c.RP, I, c.cw, r, j, true); count_step(c.K8, c.KP, I, c.cw, cc, j, true); }
            }
            __syncwarp();
            // conflict status of the row- and column-mates coloured i or j
            int dconf = 0;
            for (int side = 0; side < 2; ++side) {
                const int32_t *ptr = side ? I.col_ptr : I.row_ptr;
                const uint16_t *lst = side ? I.col_v : I.row_v;
                const int line = side ? cc : r;
                const int qb = __ldg(&ptr[line]), qe = __ldg(&ptr[line + 1]);
                for (int qq = qb + lane; qq < qe; qq += 32) {
                    const int u = __ldg(&lst[qq]);
                    if (u == v) continue;
                    const int su = c.S[u];
                    if (su == 0 || (su != i && su != j)) continue;
                    const int nc = gamma_own(I, c, u, su) > 0;
                    const int oc = (c.cmask[u >> 5] >> (u & 31)) & 1;
                    if (nc != oc) {
                        atomicXor(&c.cmask[u >> 5], 1u << (u & 31));
                        dconf += nc - oc;
                    }
                }
            }
            if (lane == 0) {
                const int newc = j ? (int)(gamma_own(I, c, v, j) > 0) : 0;
                if (j != 0 && !newc) atomicAnd(&c.cmask[v >> 5], ~(1u << (v & 31)));
                dconf += newc - (i != 0 ? 1 : 0);
            }
            dconf = __reduce_add_sync(FULL, dconf);
            if (lane == 0) {
                const int k = f + nconf + dconf;
                const int T = L + (a.alpha_num * k) / a.alpha_den;
                tabu_insert(I, c, G, ck, v, i, trel + (uint32_t)T);
                c.scal[4] = nconf + dconf;
            }
        }
        __syncthreads();
        nconf = c.scal[4];
        st.moves += 1;
        if (threadIdx.x == 0) st.deg += vertex_degree(I, c, v);
        if (F2 < F2best) {
            F2best = F2;
            st.improvements += 1;
            block_copy<NW>(c.B, c.S, I.nv);
        }
    }
    __syncthreads();
    block_copy<NW>(c.S, c.B, I.nv);
    __syncthreads();
    F2best_out = F2best;
    return ok;
}

// ---- greedy conflict removal (Sec. 3.7) ------------------------------------
template <int NW>
__device__ void repair(const DevInst &I, const Ctx &c)
{
    build_counts<NW>(I, c);
    for (int step = 0; step < I.nv; ++step) {
        uint32_t key = 0;
        for (int v = threadIdx.x; v < I.nv; v += 32 * NW) {
            const int k = c.S[v];
            if (!k) continue;
            const int g = gamma_own(I, c, v, k);
            if (g > 0) key = max(key, ((uint32_t)g << 16) | (0xFFFFu - (uint32_t)v));
        }
        const uint32_t m = block_max<NW>(key, c);
        if (m == 0u) break;
        const int v = (int)(0xFFFFu - (m & 0xFFFFu));
        if (threadIdx.x == 0) {
            const int k = c.S[v];
            const uint16_t rc = c.rc[v];
            c.S[v] = 0;
            count_step(c.R8, c.RP, I, c.cw, rc >> 8, k, false);
            count_step(c.K8, c.KP, I, c.cw, rc & 255, k, false);
        }
        __syncthreads();
    }
}

// ---- PartialCol (Sec. 3.7): legal partial colourings only ------------------
template <int NWC, int NW>
__device__ bool partialcol_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, int slot, int ind,
                                 int64_t N, int span, LaneStats &st, long long &fbest_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    build_counts<NW>(I, c);
    int f, nconf;
    build_cands<NW>(I, c, true, f, nconf);
    if (conflict_edges<NW>(I, c) != 0) return false;    // needs a legal start
    int fbest = f;
    block_copy<NW>(c.B, c.S, I.nv);
    tabu_reset<NW>(I, c);
    Clock ck = claim_clock<NW>(I, a, c, G, slot, span);
    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | 3u;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    int *ulist = c.scal + 8;   // never more than 2 entries in a legal colouring; bounded below
    for (long long t = 1; t <= N; ++t) {
        if (f == 0) break;
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            __syncthreads();
            tabu_rebase<NW>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            __syncthreads();
        }
        const int q = (int)((t - 1) & 31);
        if (q == 0) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + lane), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(FULL, Lr, q);
        const int rsh = (int)__shfl_sync(FULL, rotr, q);
        const int A = fbest - f;
        int w0;
        const int nloc = compact_warp<NW>(I, c, w0);
        uint32_t khi = kNoKey, klo = kNoKey;
        for (int qq = lane; qq < nloc; qq += 32) {
            const int v = c.clist[w0 * 32 + qq];
            int pairs;
            const int kv = eval_vertex<NWC>(I, c, G, ck, trel, v, 1, -1, A, pairs);
            st.pairs += pairs;
            if (kv != INT_MAX) key_update(kv, v, rsh, I.nv, 0, khi, klo);
        }
        uint32_t mhi, mlo;
        const int ncand = block_best<NW>(c, (int)(t & 1), khi, klo, nloc, mhi, mlo);
        if (ncand != f) { ok = false; break; }
        st.iterations += 1;
        st.cand += ncand;
        if (mhi == kNoKey) continue;

        const int d = (int)mhi - (1 << 30);
        const int j = (int)((mlo >> 8) & 255u);
        int v = (int)(mlo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        if (warp == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            const int T = L + (a.alpha_num * (f + d)) / a.alpha_den;
            if (lane == 0) c.scal[5] = 0;
            __syncwarp();
            // row- and column-mates coloured j lose their colour
            for (int side = 0; side < 2; ++side) {
                const int32_t *ptr = side ? I.col_ptr : I.row_ptr;
                const uint16_t *lst = side ? I.col_v : I.row_v;
                const int line = side ? cc : r;
                const int qb = __ldg(&ptr[line]), qe = __ldg(&ptr[line + 1]);
                for (int qq = qb + lane; qq < qe; qq += 32) {
                    const int u = __ldg(&lst[qq]);
                    if (u == v || c.S[u] != j) continue;
                    const int slot_u = atomicAdd(&c.scal[5], 1);
                    if (slot_u < 8) ulist[slot_u] = u;
                }
            }
            __syncwarp();
            if (lane == 0) {
                const int nunc = c.scal[5];
                if (nunc > 8 || nunc - 1 != d) {
                    c.scal[6] = 1;                       // inconsistent: abandon the walk
                } else {
                    c.scal[6] = 0;
                    for (int k = 0; k < nunc; ++k) {
                        const int u = ulist[k];
                        const uint16_t rcu = c.rc[u];
                        c.S[u] = 0;
                        count_step(c.R8, c.RP, I, c.cw, rcu >> 8, j, false);
                        count_step(c.K8, c.KP, I, c.cw, rcu & 255, j, false);
                        atomicOr(&c.cmask[u >> 5], 1u << (u & 31));
                        tabu_insert(I, c, G, ck, u, j, trel + (uint32_t)T);
                    }
                    c.S[v] = (uint8_t)j;
                    count_step(c.R8, c.RP, I, c.cw, r, j, true);
                    count_step(c.K8, c.KP, I, c.cw, cc, j, true);
                    atomicAnd(&c.cmask[v >> 5], ~(1u << (v & 31)));
                }
            }
        }
        __syncthreads();
        if (c.scal[6]) { ok = false; break; }
        if (threadIdx.x == 0) st.uncolored += c.scal[5];
        f += d;
        st.moves += 1;
        if (threadIdx.x == 0) st.deg += vertex_degree(I, c, v);
        if (f < fbest) {
            fbest = f;
            st.improvements += 1;
            block_copy<NW>(c.B, c.S, I.nv);
        }
    }
    __syncthreads();
    block_copy<NW>(c.S, c.B, I.nv);
    __syncthreads();
    fbest_out = fbest;
    return ok;
}

template <int NWC, int NW>
__global__ void __launch_bounds__(32 * NW, 16 / NW) local_search_kernel(const DevInst I, const LSArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    if (a.skip && *a.skip) return;
    const int slot = blockIdx.x;
    const Ctx c = carve<NW>(smem, I);
    uint32_t *G = a.G + (size_t)slot * I.nv * I.n1p;
    __shared__ long long red64[NW];

    // instance data shared by every walk of this block
    for (int v = threadIdx.x; v < I.nv; v += 32 * NW) const_cast<uint16_t *>(c.rc)[v] = __ldg(&I.rc[v]);
    for (int r = threadIdx.x; r < 2 * I.n; r += 32 * NW)
        const_cast<uint4 *>(c.allow)[r] = r < I.n ? I.allow_row[r] : I.allow_col[r - I.n];
    __syncthreads();

    for (;;) {
        if (threadIdx.x == 0) c.scal[7] = atomicAdd(a.work_counter, 1);
        __syncthreads();
        const int wk = c.scal[7];
        __syncthreads();
        if (wk >= a.count) break;
        const int ind = a.ind0 + wk;
        const uint8_t *gin = a.S_in + (size_t)wk * I.nv;
        uint8_t *gout = a.S_out + (size_t)wk * I.nv;
        block_copy<NW>(c.S, gin, I.nv);
        __syncthreads();

        LaneStats st = {0, 0, 0, 0, 0, 0, 0};
        long long Flast = 0;
        bool ok = true;
        if (a.flags & PLSE_LS_PARTIALCOL) {
            if (a.flags & PLSE_LS_REPAIR) repair<NW>(I, c);
            ok = partialcol_phase<NWC, NW>(I, a, c, G, slot, ind, a.iters1, a.span1, st, Flast);
        } else {
            if (a.flags & PLSE_LS_PHASE1)
                ok = plits_phase<NWC, NW>(I, a, c, G, slot, ind, 1, a.iters1, a.phi2_1, a.span1, st, Flast);
            if (ok && (a.flags & PLSE_LS_PHASE2))
                ok = plits_phase<NWC, NW>(I, a, c, G, slot, ind, 2, a.iters2, a.phi2_2, a.span2, st, Flast);
            if (ok && (a.flags & PLSE_LS_REPAIR)) repair<NW>(I, c);
        }
        __syncthreads();
        if (!ok && threadIdx.x == 0) atomicOr(a.error_flag, 1);
        block_copy<NW>(gout, c.S, I.nv);
        int z = 0;
        for (int q = threadIdx.x; q < I.nv; q += 32 * NW) z += (c.S[q] == 0);
        const int fz = block_sum<NW>(z, c);
        const long long pairs = block_sum64<NW>(st.pairs, red64);
        if (threadIdx.x == 0) {
            if (a.f_out) a.f_out[wk] = fz;
            if (a.F_out) a.F_out[wk] = Flast;
            if (a.stats) {
                plse_walk_stats s;
                s.iterations = st.iterations;
                s.moves = st.moves;
                s.cand = st.cand;
                s.pairs = pairs;
                s.deg = st.deg;
                s.improvements = st.improvements;
                s.uncolored = st.uncolored;
                a.stats[wk] = s;
            }
        }
        __syncthreads();
    }
}

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

template <int NWC, int NW>
cudaError_t launch_t(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    local_search_kernel<NWC, NW><<<L.blocks, 32 * NW, L.smem, st>>>(I, a);
    return cudaGetLastError();
}

template <int NWC, int NW>
int occupancy_t(size_t smem)
{
    cudaFuncSetAttribute(local_search_kernel<NWC, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_search_kernel<NWC, NW>, 32 * NW, smem) !=
        cudaSuccess)
        per_sm = 0;
    return per_sm;
}

template <int NWC>
int occupancy_w(int warps, size_t smem)
{
    switch (warps) {
        case 1: return occupancy_t<NWC, 1>(smem);
        case 2: return occupancy_t<NWC, 2>(smem);
        case 4: return occupancy_t<NWC, 4>(smem);
        default: return occupancy_t<NWC, 8>(smem);
    }
}

template <int NWC>
cudaError_t launch_w(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    switch (L.warps) {
        case 1: return launch_t<NWC, 1>(I, a, L, st);
        case 2: return launch_t<NWC, 2>(I, a, L, st);
        case 4: return launch_t<NWC, 4>(I, a, L, st);
        default: return launch_t<NWC, 8>(I, a, L, st);
    }
}

}  // namespace

SmemPlan smem_plan(const DevInst &I) { return make_plan(I, 1); }

int default_ls_warps(const DevInst &I)
{
    if (I.nv <= 256) return 1;
    if (I.nv <= 1024) return 2;
    return 4;
}

LSLaunch plan_local_search(const DevInst &I, int device, int count, int warps)
{
    LSLaunch L;
    L.warps = warps == 1 || warps == 2 || warps == 4 ? warps : 8;
    L.smem = make_plan(I, L.warps).total;
    L.colour_words = colour_words(I.n);
    int per_sm = 0;
    switch (L.colour_words) {
        case 1: per_sm = occupancy_w<1>(L.warps, L.smem); break;
        case 2: per_sm = occupancy_w<2>(L.warps, L.smem); break;
        case 3: per_sm = occupancy_w<3>(L.warps, L.smem); break;
        default: per_sm = occupancy_w<4>(L.warps, L.smem); break;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    long long blocks = (long long)per_sm * sms;
    if (blocks > count) blocks = count;
    L.blocks = (int)(blocks > 0 ? blocks : 0);
    return L;
}

cudaError_t launch_local_search(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    if (L.blocks <= 0) return cudaErrorInvalidConfiguration;
    switch (L.colour_words) {
        case 1: return launch_w<1>(I, a, L, st);
        case 2: return launch_w<2>(I, a, L, st);
        case 3: return launch_w<3>(I, a, L, st);
        default: return launch_w<4>(I, a, L, st);
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
