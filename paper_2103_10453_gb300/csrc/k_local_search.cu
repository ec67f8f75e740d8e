// k_local_search.cu -- population initialisation (Sec. 3.2) and the tabu local
// search of MPMA (Alg. 3: PLITS phases 1 and 2, Sec. 3.3; PartialCol and the
// greedy conflict removal, Sec. 3.7) for sm_103a.
//
// Design (GB300-first):
//  * A walk is owned by a group of NW warps (NW = 1, 2, 4, 8).  A block holds
//    W independent groups, each with its own shared-memory slot, plus one copy
//    of the instance's vertex coordinates and colour masks shared by all of
//    them.  Groups take walks from an atomic counter and never wait for each
//    other; a group of one warp needs no block barrier at all.
//  * The gamma table of the incremental evaluation (Sec. 3.3) is held in
//    factored form.  On a Latin-square graph the neighbours of v = (r, c) are
//    exactly its row- and column-mates, so
//        gamma[v][k] = R[r][k] + K[c][k] - 2*[S(v) = k],
//    with R / K the per-row / per-column colour counts.  A move updates four
//    counters instead of deg(v) table entries.  The counts are stored as 7 bit
//    planes per 32 colours: the best colour of a candidate, min over its domain
//    of R + K, comes out of a bit-sliced add and a most-significant-plane-first
//    elimination on whole 32-colour words, and a single count is 7 bit reads.
//  * The tabu list (expiry per (v, colour)) is a 2-entry per-vertex cache with
//    16-bit clocks relative to the phase, backed by an exact global table G for
//    entries evicted while possibly live.  A vertex whose evicted entries have
//    all expired never touches G.
//  * The candidate set V0 u C(S) is a bitmask plus a persistent list of its
//    members (stale entries are skipped and the list is rebuilt when half of it
//    is stale).  A move changes the status of its own vertex and of row- and
//    column-mates only, so no per-iteration compaction is needed.  The chosen
//    move is the minimum of the key (2dF, (v - r) mod |V|, j): a total order, so
//    the result does not depend on how candidates are split among threads.
//  * The walk's best colouring S'* is kept in the output row in global memory.
#include <algorithm>
#include <climits>

#include "plse_internal.cuh"

namespace plse {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t kRebaseAt = 49152;   // relative clock rebased before it reaches this
constexpr uint32_t kRebaseBy = 32768;
constexpr unsigned long long kNoKey = ~0ull;

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

// floor(x / alpha_den) by the reciprocal the host checked exact over the range used
__device__ __forceinline__ int tenure_div(const LSArgs &a, int x)
{
    return a.alpha_recip ? (int)__umulhi((uint32_t)x, a.alpha_recip) : x / a.alpha_den;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// threads per block of the local search: one block per SM at n >= 64 with 16
// one-warp walks (n < 96) or 12 (n >= 96, whose kernel needs more registers),
// two blocks of 8 walks per SM below
template <int NWC>
constexpr int kMaxThreads = NWC == 3 ? 512 : NWC == 4 ? 384 : 256;

// colour counts per (line, 32-colour word) are bit planes: planes 0, 1 and the OR
// of planes 2..6 (a count >= 4) in shared memory, planes 2..6 in global memory,
// where they are touched only when a count crosses a multiple of 4
constexpr int kLo = 4;    // shared words: plane 0, plane 1, high OR, pad
constexpr int kHi = 8;    // global words: planes 2..6, pad

__host__ __device__ inline SmemPlan make_plan(const DevInst &I, int warps)
{
    const int cw = colour_words(I.n);
    SmemPlan p;
    p.inst = align16(align16(2 * (size_t)I.nv) + 32 * (size_t)I.n + 2 * (size_t)I.n);
    size_t o = 0;
    p.off_S = o;      o = align16(o + (size_t)I.nv);
    p.off_RP = o;     o += 4 * kLo * (size_t)I.n * cw;
    p.off_KP = o;     o += 4 * kLo * (size_t)I.n * cw;
    p.off_cmask = o;  o += 4 * (size_t)I.nw;
    p.off_lmask = o;  o += 4 * (size_t)I.nw;
    p.off_red = align16(o);
    o = p.off_red;
    o = p.off_red + 8 * 2 * (size_t)warps + 4 * 2 * (size_t)warps + 4 * 16;
    p.slot = align16(o);
    return p;
}

// One walk's shared-memory slot.
struct Slot {
    uint8_t *S;                 // current colouring [nv]
    uint32_t *RP, *KP;          // colour-count planes 0, 1 and high OR [n][cw][kLo] per row / column
    uint32_t *RH, *KH;          // colour-count planes 2..6 [n][cw][kHi] per row / column, global
    uint32_t *cmask;            // candidate bitmask [nw]
    uint32_t *lmask;            // vertices present in the candidate list [nw]
    uint16_t *list;             // candidate list (may hold stale entries) [nv], global memory
    uint16_t *xr;               // [2n][n1p] XOR of the ids of a line's vertices of each colour, global
    uint2 *tc;                  // tabu cache [nv] in global memory (L1-resident for the candidates):
                                // x = e0 | e1 << 16, y = c0 | c1 << 8 | emax << 16
    unsigned long long *red;    // [2][NW] best key per warp (double-buffered)
    int *red_cnt;               // [2][NW] live candidates seen per warp
    int *scal;                  // [16]: 0 list length, 4 |C(S)|, 5..6 PartialCol, 7 walk id, 8.. reductions
};

// Per-thread view: instance data, its slot and its place in the group.
struct Ctx {
    const uint16_t *rc;         // [nv] row << 8 | column (shared by the block)
    const uint4 *allow;         // [2n] allowed colours per row, then per column (shared)
    const uint8_t *linelen;     // [2n] reduced vertices per row, then per column (shared)
    Slot s;
    int cw;                     // colour words of the plane layout
    int g;                      // group (walk slot) within the block
    int gt;                     // thread index within the group
    int lane, wg;               // lane, warp within the group
};

template <int NW>
__device__ __forceinline__ void gsync(const Ctx &c)
{
    if (NW == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(c.g + 1), "r"(32 * NW) : "memory");
}

template <int NW>
__device__ __forceinline__ Ctx make_ctx(uint8_t *base, const DevInst &I)
{
    const SmemPlan p = make_plan(I, NW);
    Ctx c;
    c.rc = reinterpret_cast<const uint16_t *>(base);
    c.allow = reinterpret_cast<const uint4 *>(base + align16(2 * (size_t)I.nv));
    c.linelen = base + align16(2 * (size_t)I.nv) + 32 * (size_t)I.n;
    c.g = threadIdx.x / (32 * NW);
    c.gt = threadIdx.x % (32 * NW);
    c.lane = threadIdx.x & 31;
    c.wg = c.gt >> 5;
    uint8_t *sb = base + p.inst + p.slot * c.g;
    c.s.S = sb + p.off_S;
    c.s.RP = reinterpret_cast<uint32_t *>(sb + p.off_RP);
    c.s.KP = reinterpret_cast<uint32_t *>(sb + p.off_KP);
    c.s.cmask = reinterpret_cast<uint32_t *>(sb + p.off_cmask);
    c.s.lmask = reinterpret_cast<uint32_t *>(sb + p.off_lmask);
    c.s.list = nullptr;         // set once the walk slot is known
    c.s.RH = c.s.KH = nullptr;
    c.s.xr = nullptr;
    c.s.tc = nullptr;           // set once the walk slot is known
    c.s.red = reinterpret_cast<unsigned long long *>(sb + p.off_red);
    c.s.red_cnt = reinterpret_cast<int *>(sb + p.off_red + 16 * NW);
    c.s.scal = c.s.red_cnt + 2 * NW;
    c.cw = colour_words(I.n);
    return c;
}

struct LaneStats {
    long long iterations, moves, cand, pairs, deg, improvements, uncolored;
};

template <int NW>
__device__ __forceinline__ int gsum(int x, const Ctx &c)
{
    x = __reduce_add_sync(FULL, x);
    if (NW == 1) return x;
    gsync<NW>(c);
    if (c.lane == 0) c.s.scal[8 + c.wg] = x;
    gsync<NW>(c);
    int t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += c.s.scal[8 + k];
    gsync<NW>(c);
    return t;
}

template <int NW>
__device__ __forceinline__ uint32_t gmax(uint32_t x, const Ctx &c)
{
    x = __reduce_max_sync(FULL, x);
    if (NW == 1) return x;
    gsync<NW>(c);
    if (c.lane == 0) c.s.scal[8 + c.wg] = (int)x;
    gsync<NW>(c);
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t = max(t, (uint32_t)c.s.scal[8 + k]);
    gsync<NW>(c);
    return t;
}

template <int NW>
__device__ __forceinline__ long long gsum64(long long x, const Ctx &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    if (NW == 1) return x;
    gsync<NW>(c);
    if (c.lane == 0) c.s.red[c.wg] = (unsigned long long)x;
    gsync<NW>(c);
    long long t = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) t += (long long)c.s.red[k];
    gsync<NW>(c);
    return t;
}

template <int NW>
__device__ __forceinline__ void gcopy(uint8_t *dst, const uint8_t *src, int n, const Ctx &c)
{
    for (int q = c.gt; q < n; q += 32 * NW) dst[q] = src[q];
}

// ---- colour-count planes ----------------------------------------------------
__device__ __forceinline__ const uint32_t *line_planes(const uint32_t *P, int cw, int line)
{
    return P + (size_t)line * cw * kLo;
}

__device__ __forceinline__ uint4 *lo_word(const Ctx &c, int side, int line, int k)
{
    return reinterpret_cast<uint4 *>(side ? c.s.KP : c.s.RP) + (size_t)line * c.cw + (k >> 5);
}

__device__ __forceinline__ uint32_t *hi_words(const Ctx &c, int side, int line, int k)
{
    return (side ? c.s.KH : c.s.RH) + ((size_t)line * c.cw + (k >> 5)) * kHi;
}

// +1 / -1 on count[side][line][k] (one thread per line at a time).  Returns the
// change in the number of counts >= 4, which selects the evaluation path, and
// the updated shared word in *lo_out (may be null).
__device__ __forceinline__ int count_step(const Ctx &c, int side, int line, int k, bool inc, uint4 *lo_out = nullptr)
{
    uint4 *w = lo_word(c, side, line, k);
    uint4 a = *w;
    const uint32_t bit = 1u << (k & 31);
    const int old_hi = (a.z & bit) ? 1 : 0;
    uint32_t carry = bit, t;
    t = inc ? (a.x & carry) : (~a.x & carry);
    a.x ^= carry;
    carry = t;
    t = inc ? (a.y & carry) : (~a.y & carry);
    a.y ^= carry;
    carry = t;
    if (carry) {                                   // crosses a multiple of 4: planes 2..6
        uint32_t *g = hi_words(c, side, line, k);
        const uint4 g0 = *reinterpret_cast<const uint4 *>(g);
        uint32_t x[5] = {g0.x, g0.y, g0.z, g0.w, g[4]};
#pragma unroll
        for (int p = 0; p < 5; ++p) {
            t = inc ? (x[p] & carry) : (~x[p] & carry);
            x[p] ^= carry;
            carry = t;
        }
        *reinterpret_cast<uint4 *>(g) = make_uint4(x[0], x[1], x[2], x[3]);
        g[4] = x[4];
        a.z = ((x[0] | x[1] | x[2] | x[3] | x[4]) & bit) ? (a.z | bit) : (a.z & ~bit);
    }
    *w = a;
    if (lo_out) *lo_out = a;
    return ((a.z & bit) ? 1 : 0) - old_hi;
}

// count from a shared word: exact below 4, reported as 4 + (count mod 4) from 4 on,
// which decides every "count > t" test with t <= 3 like the exact count
__device__ __forceinline__ int count_low(const uint4 &a, int k)
{
    const uint32_t b = k & 31;
    return (int)(((a.x >> b) & 1u) | (((a.y >> b) & 1u) << 1) | (((a.z >> b) & 1u) << 2));
}

__device__ __forceinline__ int count_of_fast(const Ctx &c, int side, int line, int k)
{
    return count_low(*lo_word(c, side, line, k), k);
}

// exact count (planes 2..6 read from global memory only when the count is >= 4)
__device__ __forceinline__ int count_of(const Ctx &c, int side, int line, int k)
{
    const uint4 a = *lo_word(c, side, line, k);
    const uint32_t b = k & 31;
    int x = (int)(((a.x >> b) & 1u) | (((a.y >> b) & 1u) << 1));
    if ((a.z >> b) & 1u) {
        const uint32_t *g = hi_words(c, side, line, k);
#pragma unroll
        for (int p = 0; p < 5; ++p) x |= (int)((g[p] >> b) & 1u) << (p + 2);
    }
    return x;
}

__device__ __forceinline__ int gamma_of(const DevInst &I, const Ctx &c, int v, int k)
{
    const uint16_t rc = c.rc[v];
    return count_of(c, 0, rc >> 8, k) + count_of(c, 1, rc & 255, k) - 2;
}

template <int NW>
__device__ __forceinline__ void build_planes(const DevInst &I, const Ctx &c)
{
    const int lo_words = 2 * I.n * c.cw * kLo, hi_words_n = 2 * I.n * c.cw * kHi;
    for (int q = c.gt; q < lo_words; q += 32 * NW) c.s.RP[q] = 0u;   // RP and KP are contiguous
    for (int q = c.gt; q < hi_words_n; q += 32 * NW) c.s.RH[q] = 0u;  // RH and KH are contiguous
    gsync<NW>(c);
    for (int l = c.gt; l < 2 * I.n; l += 32 * NW) {
        const bool col = l >= I.n;
        const int line = col ? l - I.n : l;
        const int32_t *ptr = col ? I.col_ptr : I.row_ptr;
        const uint16_t *lst = col ? I.col_v : I.row_v;
        uint16_t *X = c.s.xr + (size_t)l * I.n1p;
        for (int k = 0; k < I.n1p; ++k) X[k] = 0;
        for (int q = __ldg(&ptr[line]); q < __ldg(&ptr[line + 1]); ++q) {
            const int u = __ldg(&lst[q]);
            const int k = c.s.S[u];
            if (k) {
                count_step(c, col ? 1 : 0, line, k, true);
                X[k] ^= (uint16_t)u;
            }
        }
    }
    gsync<NW>(c);
    int hi = 0;
    for (int t = c.gt; t < 2 * I.n * c.cw; t += 32 * NW) hi += __popc(c.s.RP[(size_t)t * kLo + 2]);
    hi = gsum<NW>(hi, c);
    if (c.gt == 0) c.s.scal[2] = hi;
    gsync<NW>(c);
}

// conflicting edges c(S) = sum over lines and colours of C(count, 2), from the
// planes: sum of count^2 = sum_{p,q} 2^(p+q) popc(P_p & P_q)
template <int NW>
__device__ __forceinline__ int conflict_edges(const DevInst &I, const Ctx &c)
{
    long long s = 0;
    for (int t = c.gt; t < 2 * I.n * c.cw; t += 32 * NW) {
        const uint32_t *lo = c.s.RP + (size_t)t * kLo, *g = c.s.RH + (size_t)t * kHi;
        const bool high = lo[2] != 0u;
        const uint32_t w[7] = {lo[0], lo[1], high ? g[0] : 0u, high ? g[1] : 0u, high ? g[2] : 0u,
                               high ? g[3] : 0u, high ? g[4] : 0u};
        long long sq = 0, lin = 0;
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            lin += (long long)__popc(w[p]) << p;
#pragma unroll
            for (int q = 0; q < 7; ++q) sq += (long long)__popc(w[p] & w[q]) << (p + q);
        }
        s += (sq - lin) / 2;
    }
    return gsum<NW>((int)s, c);
}

// candidate bits (PLITS: V0 u C(S); PartialCol: V0), f and |C|; list = members
template <int NW>
__device__ __forceinline__ void build_cands(const DevInst &I, const Ctx &c, bool only_v0, int &f, int &nconf)
{
    int lf = 0, lc = 0;
    for (int wd = c.gt; wd < I.nw; wd += 32 * NW) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int v = wd * 32 + b;
            if (v >= I.nv) break;
            const int k = c.s.S[v];
            if (k == 0) {
                bits |= 1u << b;
                ++lf;
            } else if (gamma_of(I, c, v, k) > 0) {
                ++lc;
                if (!only_v0) bits |= 1u << b;
            }
        }
        c.s.cmask[wd] = bits;
    }
    f = gsum<NW>(lf, c);
    nconf = gsum<NW>(lc, c);
}

// rebuilds the candidate list from the bitmask (order is irrelevant)
template <int NW>
__device__ __forceinline__ void rebuild_list(const DevInst &I, const Ctx &c)
{
    gsync<NW>(c);
    const int w0 = (c.wg * I.nw) / NW, w1 = ((c.wg + 1) * I.nw) / NW;
    int cnt = 0;
    for (int wd = w0 + c.lane; wd < w1; wd += 32) cnt += __popc(c.s.cmask[wd]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (c.lane >= o) incl += y;
    }
    const int wtotal = __shfl_sync(FULL, incl, 31);
    int base = 0, total = wtotal;
    if (NW > 1) {
        if (c.lane == 0) c.s.scal[8 + c.wg] = wtotal;
        gsync<NW>(c);
        total = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int x = c.s.scal[8 + k];
            if (k < c.wg) base += x;
            total += x;
        }
    }
    int pos = base + incl - cnt;
    for (int wd = w0 + c.lane; wd < w1; wd += 32) {
        uint32_t bits = c.s.cmask[wd];
        c.s.lmask[wd] = bits;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            c.s.list[pos++] = (uint16_t)(wd * 32 + b);
        }
    }
    gsync<NW>(c);
    if (c.gt == 0) c.s.scal[0] = total;
    gsync<NW>(c);
}

// ---- tabu cache -------------------------------------------------------------
struct Clock {
    uint32_t base;    // absolute clock of iteration 0 of the phase
    uint32_t shift;   // relative clock = t - shift
};

template <int NW>
__device__ __forceinline__ void tabu_reset(const DevInst &I, const Ctx &c)
{
    for (int v = c.gt; v < I.nv; v += 32 * NW) c.s.tc[v] = make_uint2(0u, 0xFFFFu);
}

template <int NW>
__device__ __forceinline__ void tabu_rebase(const DevInst &I, const Ctx &c)
{
    for (int v = c.gt; v < I.nv; v += 32 * NW) {
        const uint2 x = c.s.tc[v];
        uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16, em = x.y >> 16;
        e0 = e0 > kRebaseBy ? e0 - kRebaseBy : 0u;
        e1 = e1 > kRebaseBy ? e1 - kRebaseBy : 0u;
        em = em > kRebaseBy ? em - kRebaseBy : 0u;
        c.s.tc[v] = make_uint2(e0 | (e1 << 16), (x.y & 0xFFFFu) | (em << 16));
    }
}

// (v, k) tabu until relative clock e (inclusive); evicts to G when needed
__device__ __forceinline__ void tabu_insert(const DevInst &I, const Ctx &c, uint32_t *G, const Clock &ck,
                                            int v, int k, uint32_t e)
{
    const uint2 x = c.s.tc[v];
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
    c.s.tc[v] = make_uint2(e0 | (e1 << 16), c0 | (c1 << 8) | (em << 16));
}

// Word selection by mask arithmetic (a compare-and-select loop over a register
// array is turned into an indexed local-memory access by the compiler).
template <int NWC>
__device__ __forceinline__ void word_masks(uint32_t k, uint32_t (&sel)[NWC])
{
    const uint32_t wq = k >> 5;
#pragma unroll
    for (int q = 0; q < NWC; ++q) sel[q] = 0u - (uint32_t)(wq == (uint32_t)q);
}

template <int NWC>
__device__ __forceinline__ void clear_bit(uint32_t (&m)[NWC], uint32_t k)
{
    uint32_t sel[NWC];
    word_masks<NWC>(k, sel);
    const uint32_t bit = 1u << (k & 31);
#pragma unroll
    for (int q = 0; q < NWC; ++q) m[q] &= ~(bit & sel[q]);
}

template <int NWC>
__device__ __forceinline__ bool test_bit(const uint32_t (&m)[NWC], uint32_t k)
{
    uint32_t sel[NWC];
    word_masks<NWC>(k, sel);
    uint32_t w = 0;
#pragma unroll
    for (int q = 0; q < NWC; ++q) w |= m[q] & sel[q];
    return (w >> (k & 31)) & 1u;
}

// min over colours j in m of s_j (lowest j on ties) by most-significant-plane-
// first elimination; returns -1 if m is empty
template <int NWC>
__device__ __forceinline__ int bits_min(const uint32_t (&s)[NWC][8], const uint32_t (&m)[NWC], int &smin)
{
    uint32_t set[NWC], anym = 0, any0 = 0, any1 = 0, hi = 0, h1[NWC];
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        anym |= m[q];
        h1[q] = s[q][1] | s[q][2] | s[q][3] | s[q][4] | s[q][5] | s[q][6] | s[q][7];
        hi |= s[q][3] | s[q][4] | s[q][5] | s[q][6] | s[q][7];
        set[q] = m[q] & ~(s[q][0] | h1[q]);      // s_j = 0
        any0 |= set[q];
    }
    if (!anym) return -1;
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
// 3-plane variants, exact while every count is <= 3 (sums <= 6)
template <int NWC>
__device__ __forceinline__ int value3(const uint32_t (&s0)[NWC], const uint32_t (&s1)[NWC],
                                      const uint32_t (&s2)[NWC], uint32_t k)
{
    uint32_t sel[NWC];
    word_masks<NWC>(k, sel);
    uint32_t w0 = 0, w1 = 0, w2 = 0;
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        w0 |= s0[q] & sel[q];
        w1 |= s1[q] & sel[q];
        w2 |= s2[q] & sel[q];
    }
    const uint32_t b = k & 31;
    return (int)(((w0 >> b) & 1u) | (((w1 >> b) & 1u) << 1) | (((w2 >> b) & 1u) << 2));
}

template <int NWC>
__device__ __forceinline__ int bits_min3(const uint32_t (&s0)[NWC], const uint32_t (&s1)[NWC],
                                         const uint32_t (&s2)[NWC], const uint32_t (&m)[NWC], int &smin)
{
    uint32_t set[NWC], anym = 0, any0 = 0;
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        anym |= m[q];
        set[q] = m[q] & ~(s0[q] | s1[q] | s2[q]);
        any0 |= set[q];
    }
    if (!anym) return -1;
    if (any0) {
        smin = 0;
    } else {
        uint32_t val = 0;
#pragma unroll
        for (int q = 0; q < NWC; ++q) set[q] = m[q];
#pragma unroll
        for (int p = 2; p >= 0; --p) {
            uint32_t t[NWC], anyt = 0;
#pragma unroll
            for (int q = 0; q < NWC; ++q) {
                const uint32_t sp = p == 2 ? s2[q] : p == 1 ? s1[q] : s0[q];
                t[q] = set[q] & ~sp;
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
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (set[q]) return q * 32 + __ffs(set[q]) - 1;
    return -1;
}

// eval_vertex while all counts are <= 3: planes 0-1 of R and K only
template <int NWC>
__device__ __forceinline__ int eval_vertex_low(const DevInst &I, const Ctx &c, const uint32_t *G, const Clock &ck,
                                               uint32_t trel, int v, int mult, int base_unc, int A, int &pairs,
                                               bool &slow)
{
    // the tabu-cache entry (global memory) is loaded first and used last, so its
    // latency overlaps the shared-memory loads and the bit-sliced arithmetic
    const uint2 te = c.s.tc[v];
    const int i = c.s.S[v];
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255;
    const uint32_t *RPr = line_planes(c.s.RP, NWC, r), *KPc = line_planes(c.s.KP, NWC, cc);
    uint32_t s0[NWC], s1[NWC], s2[NWC];
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        const uint2 ra = *reinterpret_cast<const uint2 *>(RPr + q * kLo);
        const uint2 ka = *reinterpret_cast<const uint2 *>(KPc + q * kLo);
        const uint32_t x0 = ra.x ^ ka.x, cy = ra.x & ka.x, x1 = ra.y ^ ka.y;
        s0[q] = x0;
        s1[q] = x1 ^ cy;
        s2[q] = (ra.y & ka.y) | (cy & x1);
    }
    const int gi = i ? value3<NWC>(s0, s1, s2, (uint32_t)i) - 2 : 0;
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
    pairs = cnt;
    if (i) clear_bit<NWC>(m, (uint32_t)i);
    bool has0 = (i != 0);
    int best = INT_MAX;
    const uint32_t e0 = te.x & 0xFFFFu, e1 = te.x >> 16;
    const uint32_t c0 = te.y & 0xFFu, c1 = (te.y >> 8) & 0xFFu, em = te.y >> 16;
    slow = em >= trel;                        // evicted entries may apply: full evaluation
    if (slow) return INT_MAX;
#pragma unroll
    // a cached colour whose tabu has expired is an ordinary admissible colour
    // and stays in m; a still-tabu one is taken out and admitted by aspiration only
    for (int sx = 0; sx < 2; ++sx) {
        const uint32_t cs = sx ? c1 : c0, es = sx ? e1 : e0;
        if (es < trel) continue;
        if (cs == 0u) {
            if (has0) {
                has0 = false;
                if (d2zero < A) best = min(best, d2zero * kKeyScale);
            }
        } else if (cs < 128u && test_bit<NWC>(m, cs)) {
            clear_bit<NWC>(m, cs);
            const int d2 = base2 + mult * value3<NWC>(s0, s1, s2, cs);
            if (d2 < A) best = min(best, d2 * kKeyScale + (int)cs);
        }
    }
    if (has0) best = min(best, d2zero * kKeyScale);
    int smin = 0;
    const int jb = bits_min3<NWC>(s0, s1, s2, m, smin);
    if (jb >= 0) best = min(best, (base2 + mult * smin) * kKeyScale + jb);
    return best;
}

template <int NWC>
__device__ __forceinline__ int eval_vertex(const DevInst &I, const Ctx &c, const uint32_t *G, const Clock &ck,
                                           uint32_t trel, int v, int mult, int base_unc, int A, int &pairs)
{
    const int i = c.s.S[v];
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255;
    const uint32_t *RPr = line_planes(c.s.RP, NWC, r), *KPc = line_planes(c.s.KP, NWC, cc);
    // s = R[r] + K[c] for every colour, bit-sliced
    uint32_t s[NWC][8];
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        const uint4 r0 = *reinterpret_cast<const uint4 *>(RPr + q * kLo);
        const uint4 k0 = *reinterpret_cast<const uint4 *>(KPc + q * kLo);
        uint32_t a[7] = {r0.x, r0.y, 0u, 0u, 0u, 0u, 0u};
        uint32_t b[7] = {k0.x, k0.y, 0u, 0u, 0u, 0u, 0u};
        if (r0.z) {
            const uint32_t *g = c.s.RH + ((size_t)r * NWC + q) * kHi;
#pragma unroll
            for (int p = 0; p < 5; ++p) a[p + 2] = g[p];
        }
        if (k0.z) {
            const uint32_t *g = c.s.KH + ((size_t)cc * NWC + q) * kHi;
#pragma unroll
            for (int p = 0; p < 5; ++p) b[p + 2] = g[p];
        }
        uint32_t carry = 0u;
#pragma unroll
        for (int p = 0; p < 7; ++p) {
            const uint32_t x = a[p] ^ b[p];
            s[q][p] = x ^ carry;
            carry = (a[p] & b[p]) | (carry & x);
        }
        s[q][7] = carry;
    }
    const int gi = i ? count_of(c, 0, r, i) + count_of(c, 1, cc, i) - 2 : 0;
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

    const uint2 te = c.s.tc[v];
    const uint32_t e0 = te.x & 0xFFFFu, e1 = te.x >> 16;
    const uint32_t c0 = te.y & 0xFFu, c1 = (te.y >> 8) & 0xFFu, em = te.y >> 16;
    int best = INT_MAX;
    if (em < trel) {
        // fast path: only the cached colours c0, c1 can be tabu
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
            const uint32_t cs = sx ? c1 : c0, es = sx ? e1 : e0;
            if (es < trel) continue;                  // expired: stays in m
            if (cs == 0u) {
                if (has0) {
                    has0 = false;
                    if (d2zero < A) best = min(best, d2zero * kKeyScale);
                }
            } else if (cs < 128u && test_bit<NWC>(m, cs)) {
                clear_bit<NWC>(m, cs);
                const int d2 = base2 + mult * (count_of(c, 0, r, (int)cs) + count_of(c, 1, cc, (int)cs));
                if (d2 < A) best = min(best, d2 * kKeyScale + (int)cs);
            }
        }
        if (has0) best = min(best, d2zero * kKeyScale);
        int smin = 0;
        const int jb = bits_min<NWC>(s, m, smin);
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
                const int d2 = base2 + mult * (count_of(c, 0, r, (int)j) + count_of(c, 1, cc, (int)j));
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
    return (int)c.linelen[rc >> 8] + (int)c.linelen[I.n + (rc & 255)] - 2;
}

// reserve a clock range for one phase of this slot
template <int NW>
__device__ __forceinline__ Clock claim_clock(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, int slot, int span)
{
    gsync<NW>(c);
    if (c.gt == 0) {
        uint32_t base = a.slot_clock[slot] + 1u;
        if (base > 0x7FFFFFFFu - (uint32_t)span) base = 0u;   // wrap: clear the slot
        c.s.scal[1] = (int)base;
    }
    gsync<NW>(c);
    uint32_t base = (uint32_t)c.s.scal[1];
    if (base == 0u) {
        const size_t words = (size_t)I.nv * I.n1p;
        for (size_t q = c.gt; q < words; q += 32 * NW) G[q] = 0u;
        base = 1u;
    }
    gsync<NW>(c);
    if (c.gt == 0) a.slot_clock[slot] = base + (uint32_t)span;
    Clock ck;
    ck.base = base;
    ck.shift = 0u;
    return ck;
}

// key = (2dF + 2^30) << 32 | rot << 16 | j << 8 | i: unsigned order = (2dF, rot, j)
__device__ __forceinline__ unsigned long long make_key(int kv, int v, int rsh, int nv, int i)
{
    int rot = v - rsh;
    if (rot < 0) rot += nv;
    const uint32_t hi = (uint32_t)((kv >> 8) + (1 << 30));
    const uint32_t lo = ((uint32_t)rot << 16) | ((uint32_t)(kv & 255) << 8) | (uint32_t)i;
    return ((unsigned long long)hi << 32) | lo;
}

// group-wide minimum key and number of live candidates scanned
template <int NW>
__device__ __forceinline__ unsigned long long group_best(const Ctx &c, int parity, unsigned long long key,
                                                         int live, int &total)
{
    const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
    const uint32_t whi = __reduce_min_sync(FULL, hi);
    const uint32_t wlo = __reduce_min_sync(FULL, hi == whi ? lo : 0xffffffffu);
    const unsigned long long wk = ((unsigned long long)whi << 32) | wlo;
    const int wl = __reduce_add_sync(FULL, live);
    if (NW == 1) {
        total = wl;
        return wk;
    }
    if (c.lane == 0) {
        c.s.red[parity * NW + c.wg] = wk;
        c.s.red_cnt[parity * NW + c.wg] = wl;
    }
    gsync<NW>(c);
    unsigned long long best = kNoKey;
    total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        best = min(best, c.s.red[parity * NW + k]);
        total += c.s.red_cnt[parity * NW + k];
    }
    return best;
}

// warp 0 of the group: appends the lanes' flagged vertices to the candidate list
__device__ __forceinline__ void list_append(const Ctx &c, bool want, int u, int &len)
{
    const uint32_t b = __ballot_sync(FULL, want);
    if (want) {
        const int pos = len + __popc(b & ((1u << c.lane) - 1u));
        c.s.list[pos] = (uint16_t)u;
        atomicOr(&c.s.lmask[u >> 5], 1u << (u & 31));
    }
    len += __popc(b);
}

// One scan pass of a one-warp walk over list entries base .. base+31: stale
// entries (no longer candidates) are dropped and lose their membership bit, live
// ones are written back contiguously at wpos, so the list stays about as long as
// the candidate set and a scan needs no pass over stale entries.  Returns the
// lane's live vertex or -1.
__device__ __forceinline__ int list_pass(const Ctx &c, int base, int len, int &wpos)
{
    const int qq = base + c.lane;
    int v = -1;
    bool lv = false;
    if (qq < len) {
        v = c.s.list[qq];
        lv = (c.s.cmask[v >> 5] >> (v & 31)) & 1u;
        if (!lv) atomicAnd(&c.s.lmask[v >> 5], ~(1u << (v & 31)));
    }
    const uint32_t b = __ballot_sync(FULL, lv);
    __syncwarp();                                     // every entry of the pass read before any write
    const int to = wpos + __popc(b & ((1u << c.lane) - 1u));
    if (lv && to != qq) c.s.list[to] = (uint16_t)v;  // entries that do not move stay cached
    wpos += __popc(b);
    return lv ? v : -1;
}

// ---- PLITS phase (Alg. 3 with phi2 = 2*phi) --------------------------------
template <int NWC, int NW>
__device__ __forceinline__ bool plits_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, uint8_t *gbest,
                            int slot, int ind, int phase, int64_t N, int phi2, int span, LaneStats &st,
                            long long &F2best_out)
{
    build_planes<NW>(I, c);
    int f, nconf;
    build_cands<NW>(I, c, false, f, nconf);
    const int cedges = conflict_edges<NW>(I, c);
    long long F2 = 2LL * f + (long long)phi2 * cedges;
    long long F2best = F2;
    gcopy<NW>(gbest, c.s.S, I.nv, c);
    tabu_reset<NW>(I, c);
    rebuild_list<NW>(I, c);
    Clock ck = claim_clock<NW>(I, a, c, G, slot, span);

    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | (uint32_t)phase;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    for (long long t = 1; t <= N; ++t) {
        if (f + nconf == 0) break;                       // nothing left to improve
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            gsync<NW>(c);
            tabu_rebase<NW>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            gsync<NW>(c);
        }
        int len = c.s.scal[0];
        if (len > 2 * (f + nconf) + 64) {
            rebuild_list<NW>(I, c);
            len = c.s.scal[0];
        }
        const int q = (int)((t - 1) & 31);
        if (q == 0) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + c.lane), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(FULL, Lr, q);
        const int rsh = (int)__shfl_sync(FULL, rotr, q);
        const long long A64 = F2best - F2;
        const int A = A64 < -(1LL << 30) ? -(1 << 30) : (int)A64;

        const bool low = c.s.scal[2] == 0;            // every count <= 3
        unsigned long long key = kNoKey;
        int live = 0;
        auto consider = [&](int v) {
            ++live;
            int pairs;
            bool slow = true;
            int kv = INT_MAX;
            if (low) kv = eval_vertex_low<NWC>(I, c, G, ck, trel, v, phi2, -2, A, pairs, slow);
            if (slow) kv = eval_vertex<NWC>(I, c, G, ck, trel, v, phi2, -2, A, pairs);
            st.pairs += pairs;
            if (kv != INT_MAX) key = min(key, make_key(kv, v, rsh, I.nv, c.s.S[v]));
        };
        if constexpr (NW == 1) {
            int wpos = 0;
            for (int base = 0; base < len; base += 32) {
                const int v = list_pass(c, base, len, wpos);
                if (v >= 0) consider(v);
            }
            if (c.lane == 0) c.s.scal[0] = wpos;
            __syncwarp();
            len = wpos;
        } else {
            for (int qq = c.gt; qq < len; qq += 32 * NW) {
                const int v = c.s.list[qq];
                if ((c.s.cmask[v >> 5] >> (v & 31)) & 1u) consider(v);   // else a stale entry
            }
        }
        int ncand;
        const unsigned long long best = group_best<NW>(c, (int)(t & 1), key, live, ncand);
        if (ncand != f + nconf) { ok = false; break; }
        st.iterations += 1;
        st.cand += ncand;
        if (best == kNoKey) continue;                    // every move tabu

        const uint32_t bhi = (uint32_t)(best >> 32), blo = (uint32_t)best;
        const int d2 = (int)bhi - (1 << 30);
        const int j = (int)((blo >> 8) & 255u), i = (int)(blo & 255u);
        int v = (int)(blo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        f += (j == 0) - (i == 0);
        F2 += d2;
        if (c.wg == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            // count updates: lane 0 row r / colour i, lane 1 column cc / colour i,
            // lanes 2-3 the same for colour j (folded into lanes 0-1 when i and j
            // share a 32-colour word, so that no two lanes touch one plane word)
            const bool same = i && j && ((i >> 5) == (j >> 5));
            // member-id XOR of (row r | column cc, colour i | j), read first so that
            // its latency overlaps the count updates: lane 0 row/i, 1 column/i,
            // 2 row/j, 3 column/j
            const int xk = c.lane < 2 ? i : j;
            const size_t xidx = (size_t)((c.lane & 1) ? I.n + cc : r) * I.n1p + xk;
            const int xold = (c.lane < 4 && xk) ? (int)c.s.xr[xidx] : 0;
            int cnt_i = 0, cnt_j = 0;
            if (c.lane < 4) {
                const int side = c.lane & 1;
                const int line = side ? cc : r;
                int dh = 0;
                uint4 w;
                if (c.lane < 2) {
                    if (i) dh += count_step(c, side, line, i, false, &w);
                    if (same) dh += count_step(c, side, line, j, true, &w);
                    if (i) cnt_i = count_low(w, i);       // counts after the move (4 = four or more)
                    if (same) cnt_j = count_low(w, j);
                } else if (j && !same) {
                    dh += count_step(c, side, line, j, true, &w);
                    cnt_j = count_low(w, j);
                }
                if (dh) atomicAdd(&c.s.scal[2], dh);
                if (c.lane == 0) c.s.S[v] = (uint8_t)j;
                if (xk) c.s.xr[xidx] = (uint16_t)(xold ^ v);   // v leaves i, joins j
            }
            // counts of colours i and j on the moved row and column, after the move
            const int Ri = __shfl_sync(FULL, cnt_i, 0), Ki = __shfl_sync(FULL, cnt_i, 1);
            const int Rj = __shfl_sync(FULL, cnt_j, same ? 0 : 2), Kj = __shfl_sync(FULL, cnt_j, same ? 1 : 3);
            __syncwarp();
            // The mates whose conflict status can change, one per (line, colour) at
            // most: the only other holder of colour i (count after the move 1) and
            // the other holder of colour j (count after 2).  Each is read from the
            // member-id XOR of its line: lane 0 row/i, 1 column/i, 2 row/j, 3 column/j.
            int dconf = 0;
            int u = -1, su = 0, cl = 0;
            const bool row_mate = (c.lane & 1) == 0;
            if (c.lane == 0 && i && Ri == 1) { u = xold ^ v; su = i; cl = Ri; }   // the last holder of i
            if (c.lane == 1 && i && Ki == 1) { u = xold ^ v; su = i; cl = Ki; }
            if (c.lane == 2 && j && Rj == 2) { u = xold; su = j; cl = Rj; }       // the other holder of j
            if (c.lane == 3 && j && Kj == 2) { u = xold; su = j; cl = Kj; }
            bool want = false, bad_mate = false;
            if (u >= 0) {
                if (u >= I.nv || u == v || c.s.S[u] != su) {
                    bad_mate = true;                     // inconsistent table: report, touch nothing
                } else {
                    const uint16_t urc = c.rc[u];
                    const int g = cl + (row_mate ? count_of_fast(c, 1, urc & 255, su)
                                                 : count_of_fast(c, 0, urc >> 8, su)) - 2;
                    const int nc = g > 0, oc = (c.s.cmask[u >> 5] >> (u & 31)) & 1;
                    if (nc != oc) {
                        atomicXor(&c.s.cmask[u >> 5], 1u << (u & 31));
                        dconf += nc - oc;
                        want = nc && !((c.s.lmask[u >> 5] >> (u & 31)) & 1u);
                    }
                }
            }
            list_append(c, want, u, len);
            const bool any_bad = __any_sync(FULL, bad_mate);
            if (c.lane == 0) {
                const int newc = j ? (int)(Rj + Kj - 2 > 0) : 0;
                if (j != 0 && !newc) atomicAnd(&c.s.cmask[v >> 5], ~(1u << (v & 31)));
                dconf += newc - (i != 0 ? 1 : 0);
            }
            dconf = __reduce_add_sync(FULL, dconf);
            if (c.lane == 0) {
                const int k = f + nconf + dconf;
                const int T = L + tenure_div(a, a.alpha_num * k);
                tabu_insert(I, c, G, ck, v, i, trel + (uint32_t)T);
                c.s.scal[4] = nconf + dconf;
                c.s.scal[0] = len;
                c.s.scal[6] = any_bad ? 1 : 0;
            }
        }
        gsync<NW>(c);
        if (c.s.scal[6]) { ok = false; break; }
        nconf = c.s.scal[4];
        st.moves += 1;
        if (c.gt == 0) st.deg += vertex_degree(I, c, v);
        if (F2 < F2best) {
            F2best = F2;
            st.improvements += 1;
            gcopy<NW>(gbest, c.s.S, I.nv, c);
        }
    }
    gsync<NW>(c);
    gcopy<NW>(c.s.S, gbest, I.nv, c);
    gsync<NW>(c);
    F2best_out = F2best;
    return ok;
}

// ---- greedy conflict removal (Sec. 3.7) ------------------------------------
template <int NW>
__device__ __forceinline__ void repair(const DevInst &I, const Ctx &c)
{
    build_planes<NW>(I, c);
    for (int step = 0; step < I.nv; ++step) {
        uint32_t key = 0;
        for (int v = c.gt; v < I.nv; v += 32 * NW) {
            const int k = c.s.S[v];
            if (!k) continue;
            const int g = gamma_of(I, c, v, k);
            if (g > 0) key = max(key, ((uint32_t)g << 16) | (0xFFFFu - (uint32_t)v));
        }
        const uint32_t m = gmax<NW>(key, c);
        if (m == 0u) break;
        const int v = (int)(0xFFFFu - (m & 0xFFFFu));
        gsync<NW>(c);
        if (c.gt == 0) {
            const int k = c.s.S[v];
            const uint16_t rc = c.rc[v];
            c.s.S[v] = 0;
            c.s.scal[2] += count_step(c, 0, rc >> 8, k, false) + count_step(c, 1, rc & 255, k, false);
        }
        gsync<NW>(c);
    }
}

// ---- PartialCol (Sec. 3.7): legal partial colourings only ------------------
template <int NWC, int NW>
__device__ __forceinline__ bool partialcol_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, uint8_t *gbest,
                                 int slot, int ind, int64_t N, int span, LaneStats &st, long long &fbest_out)
{
    build_planes<NW>(I, c);
    int f, nconf;
    build_cands<NW>(I, c, true, f, nconf);
    if (conflict_edges<NW>(I, c) != 0) return false;    // needs a legal start
    int fbest = f;
    gcopy<NW>(gbest, c.s.S, I.nv, c);
    tabu_reset<NW>(I, c);
    rebuild_list<NW>(I, c);
    Clock ck = claim_clock<NW>(I, a, c, G, slot, span);
    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | 3u;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    int *ulist = c.s.scal + 8;   // a legal colouring has at most 2 mates of one colour
    for (long long t = 1; t <= N; ++t) {
        if (f == 0) break;
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            gsync<NW>(c);
            tabu_rebase<NW>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            gsync<NW>(c);
        }
        int len = c.s.scal[0];
        if (len > 2 * f + 64) {
            rebuild_list<NW>(I, c);
            len = c.s.scal[0];
        }
        const int q = (int)((t - 1) & 31);
        if (q == 0) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + c.lane), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(FULL, Lr, q);
        const int rsh = (int)__shfl_sync(FULL, rotr, q);
        const int A = fbest - f;
        const bool low = c.s.scal[2] == 0;            // every count <= 3
        unsigned long long key = kNoKey;
        int live = 0;
        auto consider = [&](int v) {
            ++live;
            int pairs;
            bool slow = true;
            int kv = INT_MAX;
            if (low) kv = eval_vertex_low<NWC>(I, c, G, ck, trel, v, 1, -1, A, pairs, slow);
            if (slow) kv = eval_vertex<NWC>(I, c, G, ck, trel, v, 1, -1, A, pairs);
            st.pairs += pairs;
            if (kv != INT_MAX) key = min(key, make_key(kv, v, rsh, I.nv, 0));
        };
        if constexpr (NW == 1) {
            int wpos = 0;
            for (int base = 0; base < len; base += 32) {
                const int v = list_pass(c, base, len, wpos);
                if (v >= 0) consider(v);
            }
            if (c.lane == 0) c.s.scal[0] = wpos;
            __syncwarp();
            len = wpos;
        } else {
            for (int qq = c.gt; qq < len; qq += 32 * NW) {
                const int v = c.s.list[qq];
                if ((c.s.cmask[v >> 5] >> (v & 31)) & 1u) consider(v);
            }
        }
        int ncand;
        const unsigned long long best = group_best<NW>(c, (int)(t & 1), key, live, ncand);
        if (ncand != f) { ok = false; break; }
        st.iterations += 1;
        st.cand += ncand;
        if (best == kNoKey) continue;

        const int d = (int)(uint32_t)(best >> 32) - (1 << 30);
        const uint32_t blo = (uint32_t)best;
        const int j = (int)((blo >> 8) & 255u);
        int v = (int)(blo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        if (c.wg == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            const int T = L + tenure_div(a, a.alpha_num * (f + d));
            if (c.lane == 0) c.s.scal[5] = 0;
            __syncwarp();
            // row- and column-mates coloured j lose their colour
            for (int side = 0; side < 2; ++side) {
                const int32_t *ptr = side ? I.col_ptr : I.row_ptr;
                const uint16_t *lst = side ? I.col_v : I.row_v;
                const int line = side ? cc : r;
                const int qb = __ldg(&ptr[line]), qe = __ldg(&ptr[line + 1]);
                for (int qq = qb + c.lane; qq < qe; qq += 32) {
                    const int u = __ldg(&lst[qq]);
                    if (u == v || c.s.S[u] != j) continue;
                    const int k = atomicAdd(&c.s.scal[5], 1);
                    if (k < 8) ulist[k] = u;
                }
            }
            __syncwarp();
            const int nunc = c.s.scal[5];
            const bool bad = nunc > 8 || nunc - 1 != d;
            int wantu = 0;
            bool want = false;
            if (!bad && c.lane < nunc) {
                wantu = ulist[c.lane];
                want = !((c.s.lmask[wantu >> 5] >> (wantu & 31)) & 1u);
            }
            __syncwarp();
            if (!bad) {
                if (c.lane == 0) {
                    for (int k = 0; k < nunc; ++k) {
                        const int u = ulist[k];
                        const uint16_t rcu = c.rc[u];
                        c.s.S[u] = 0;
                        c.s.scal[2] += count_step(c, 0, rcu >> 8, j, false) +
                                       count_step(c, 1, rcu & 255, j, false);
                        atomicOr(&c.s.cmask[u >> 5], 1u << (u & 31));
                        tabu_insert(I, c, G, ck, u, j, trel + (uint32_t)T);
                    }
                    c.s.S[v] = (uint8_t)j;
                    c.s.scal[2] += count_step(c, 0, r, j, true) + count_step(c, 1, cc, j, true);
                    atomicAnd(&c.s.cmask[v >> 5], ~(1u << (v & 31)));
                }
                __syncwarp();
                list_append(c, want, wantu, len);
            }
            if (c.lane == 0) {
                c.s.scal[6] = bad ? 1 : 0;
                c.s.scal[0] = len;
            }
        }
        gsync<NW>(c);
        if (c.s.scal[6]) { ok = false; break; }
        if (c.gt == 0) st.uncolored += c.s.scal[5];
        f += d;
        st.moves += 1;
        if (c.gt == 0) st.deg += vertex_degree(I, c, v);
        if (f < fbest) {
            fbest = f;
            st.improvements += 1;
            gcopy<NW>(gbest, c.s.S, I.nv, c);
        }
    }
    gsync<NW>(c);
    gcopy<NW>(c.s.S, gbest, I.nv, c);
    gsync<NW>(c);
    fbest_out = fbest;
    return ok;
}

template <int NWC, int NW>
__global__ void __launch_bounds__(kMaxThreads<NWC>, NWC >= 3 ? 1 : 2) local_search_kernel(const DevInst I, const LSArgs a, int walks)
{
    extern __shared__ __align__(16) uint8_t smem[];
    if (a.skip && *a.skip) return;
    // instance data shared by every walk slot of the block
    uint16_t *rc_s = reinterpret_cast<uint16_t *>(smem);
    uint4 *allow_s = reinterpret_cast<uint4 *>(smem + align16(2 * (size_t)I.nv));
    for (int v = threadIdx.x; v < I.nv; v += blockDim.x) rc_s[v] = __ldg(&I.rc[v]);
    uint8_t *len_s = smem + align16(2 * (size_t)I.nv) + 32 * (size_t)I.n;
    for (int r = threadIdx.x; r < 2 * I.n; r += blockDim.x) {
        allow_s[r] = r < I.n ? I.allow_row[r] : I.allow_col[r - I.n];
        len_s[r] = (uint8_t)(r < I.n ? I.row_ptr[r + 1] - I.row_ptr[r] : I.col_ptr[r - I.n + 1] - I.col_ptr[r - I.n]);
    }
    __syncthreads();

    Ctx c = make_ctx<NW>(smem, I);
    if (c.g >= walks) return;
    const int slot = blockIdx.x * walks + c.g;
    uint32_t *G = a.G + (size_t)slot * I.nv * I.n1p;
    c.s.tc = a.TC + (size_t)slot * I.nv;
    c.s.list = a.LIST + (size_t)slot * I.nv;
    c.s.xr = a.XR + (size_t)slot * 2 * I.n * I.n1p;
    c.s.RH = a.HP + (size_t)slot * 2 * I.n * c.cw * kHi;
    c.s.KH = c.s.RH + (size_t)I.n * c.cw * kHi;

    for (;;) {
        if (c.gt == 0) c.s.scal[7] = atomicAdd(a.work_counter, 1);
        gsync<NW>(c);
        const int wk = c.s.scal[7];
        gsync<NW>(c);
        if (wk >= a.count) break;
        const int ind = a.ind0 + wk;
        const uint8_t *gin = a.S_in + (size_t)wk * I.nv;
        uint8_t *gout = a.S_out + (size_t)wk * I.nv;
        gcopy<NW>(c.s.S, gin, I.nv, c);
        gsync<NW>(c);

        LaneStats st = {0, 0, 0, 0, 0, 0, 0};
        long long Flast = 0;
        bool ok = true;
        if (a.flags & PLSE_LS_PARTIALCOL) {
            if (a.flags & PLSE_LS_REPAIR) repair<NW>(I, c);
            ok = partialcol_phase<NWC, NW>(I, a, c, G, gout, slot, ind, a.iters1, a.span1, st, Flast);
        } else {
            if (a.flags & PLSE_LS_PHASE1)
                ok = plits_phase<NWC, NW>(I, a, c, G, gout, slot, ind, 1, a.iters1, a.phi2_1, a.span1, st, Flast);
            if (ok && (a.flags & PLSE_LS_PHASE2))
                ok = plits_phase<NWC, NW>(I, a, c, G, gout, slot, ind, 2, a.iters2, a.phi2_2, a.span2, st, Flast);
            if (ok && (a.flags & PLSE_LS_REPAIR)) repair<NW>(I, c);
        }
        gsync<NW>(c);
        if (!ok && c.gt == 0) atomicOr(a.error_flag, 1);
        gcopy<NW>(gout, c.s.S, I.nv, c);
        int z = 0;
        for (int q = c.gt; q < I.nv; q += 32 * NW) z += (c.s.S[q] == 0);
        const int fz = gsum<NW>(z, c);
        const long long pairs = gsum64<NW>(st.pairs, c);
        if (c.gt == 0) {
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
        gsync<NW>(c);
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
    local_search_kernel<NWC, NW><<<L.blocks, 32 * NW * L.walks, L.smem, st>>>(I, a, L.walks);
    return cudaGetLastError();
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

// sets the block's shared-memory size; returns resident blocks per SM
template <int NWC, int NW>
int set_smem_t(size_t smem, int threads)
{
    cudaFuncSetAttribute(local_search_kernel<NWC, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_search_kernel<NWC, NW>, threads, smem) !=
        cudaSuccess)
        per_sm = 0;
    return per_sm;
}

template <int NWC>
int set_smem_w(int warps, size_t smem, int threads)
{
    switch (warps) {
        case 1: return set_smem_t<NWC, 1>(smem, threads);
        case 2: return set_smem_t<NWC, 2>(smem, threads);
        case 4: return set_smem_t<NWC, 4>(smem, threads);
        default: return set_smem_t<NWC, 8>(smem, threads);
    }
}

}  // namespace

SmemPlan smem_plan(const DevInst &I, int warps) { return make_plan(I, warps); }

LSLaunch plan_local_search(const DevInst &I, int device, int count, int warps, int max_walks)
{
    LSLaunch L;
    if (warps <= 0) warps = 1;                     // automatic: one warp per walk
    L.warps = warps == 1 || warps == 2 || warps == 4 ? warps : 8;
    L.colour_words = colour_words(I.n);
    const SmemPlan p = make_plan(I, L.warps);
    int max_smem = 0, sms = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    // one block per SM holding as many walk slots as fit (at most kMaxThreads
    // threads: 512 for 64 <= n < 96, 384 from 96, 256 below 64 with two blocks)
    long long walks = ((long long)max_smem - (long long)p.inst) / (long long)p.slot;
    const int max_threads = L.colour_words == 1 ? kMaxThreads<1> : L.colour_words == 2 ? kMaxThreads<2>
                          : L.colour_words == 3 ? kMaxThreads<3> : kMaxThreads<4>;
    walks = std::min<long long>(walks, std::max(1, max_threads / (32 * L.warps)));
    if (max_walks > 0) walks = std::min<long long>(walks, max_walks);
    if (walks < 1) {
        L.blocks = 0;
        L.walks = 0;
        L.smem = 0;
        return L;
    }
    L.walks = (int)walks;
    L.smem = p.total(L.walks);
    const int threads = 32 * L.warps * L.walks;
    int per_sm = 0;
    switch (L.colour_words) {
        case 1: per_sm = set_smem_w<1>(L.warps, L.smem, threads); break;
        case 2: per_sm = set_smem_w<2>(L.warps, L.smem, threads); break;
        case 3: per_sm = set_smem_w<3>(L.warps, L.smem, threads); break;
        default: per_sm = set_smem_w<4>(L.warps, L.smem, threads); break;
    }
    long long blocks = ((long long)count + walks - 1) / walks;
    blocks = std::min<long long>(blocks, (long long)sms * std::max(per_sm, 1));
    L.blocks = per_sm > 0 ? (int)blocks : 0;
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
