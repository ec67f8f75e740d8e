// ls_walk.cuh -- the tabu local search of MPMA (Alg. 3: PLITS phases 1 and 2,
// Sec. 3.3; PartialCol and the greedy conflict removal, Sec. 3.7) for sm_103a.
//
// Design (GB300-first):
//  * A walk is owned by a group of GT threads: half a warp (GT = 16, two walks
//    per warp), one warp (32) or 2, 4, 8 warps.  A block holds W independent
//    groups, each with its own shared-memory slot, plus one copy of the
//    instance's vertex coordinates and colour masks shared by all of them.
//    Groups take walks from an atomic counter and never wait for each other; a
//    group within one warp needs no block barrier at all (its collectives use
//    the group's lane mask).
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
//    members, compacted during the scan.  A move changes the status of its own
//    vertex and of row- and column-mates only.  The chosen move is the minimum of
//    the key (2dF, (v - r) mod |V|, j): a total order, so the result does not
//    depend on how candidates are split among threads.
//  * The current colouring lives in the slot (shared memory) when the slots
//    still fit, else in a per-slot global buffer (L1-cached), which lets twice
//    as many walks share an SM.  The walk's best colouring S'* is kept in the
//    output row in global memory.
#pragma once

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

// threads per block of the local search: one block per SM at n >= 64 (640
// threads, 20 one-warp walks, for n < 96 at 95 registers without spills; 384
// from 96, whose kernel needs more registers), two blocks of 256 per SM below.
// The register budget per thread follows from it.
#ifndef PLSE_LS_THREADS_N64
#define PLSE_LS_THREADS_N64 640
#endif
template <int NWC>
constexpr int kMaxThreads = NWC == 3 ? PLSE_LS_THREADS_N64 : NWC == 4 ? 384 : 256;

// a walk group of GT threads: W lanes in each of its NW warps
template <int GT>
struct Grp {
    static constexpr int W = GT < 32 ? GT : 32;
    static constexpr int NW = GT < 32 ? 1 : GT / 32;
};

// colour counts per (line, 32-colour word) are bit planes: planes 0 and 1 (a
// uint2) and the OR of planes 2..6 (a count >= 4) in shared memory, planes 2..6
// in global memory, where they are touched only when a count crosses a
// multiple of 4
constexpr int kHi = 8;    // global words per (line, colour word): planes 2..6, pad

__host__ __device__ inline SmemPlan make_plan(const DevInst &I, int warps, bool s_smem)
{
    const int cw = colour_words(I.n);
    SmemPlan p;
    p.inst = align16(align16(2 * (size_t)I.nv) + 32 * (size_t)I.n + 2 * (size_t)I.n);
    size_t o = 0;
    p.off_S = o;
    if (s_smem) o = align16(o + (size_t)I.nv);
    p.off_P01 = o;    o += 8 * 2 * (size_t)I.n * cw;
    p.off_PH = o;     o += 4 * 2 * (size_t)I.n * cw;
    p.off_cmask = o;  o += 4 * (size_t)I.nw;
    p.off_lmask = o;  o += 4 * (size_t)I.nw;
    p.off_red = align16(o);
    o = p.off_red + 8 * 2 * (size_t)warps + 4 * 2 * (size_t)warps + 4 * 32;
    p.slot = align16(o);
    return p;
}

// One walk's slot.
struct Slot {
    uint8_t *S;                 // current colouring [nv] (shared or global memory)
    uint2 *P01;                 // colour-count planes 0, 1 [2n][cw] (rows, then columns)
    uint32_t *PH;               // OR of planes 2..6 [2n][cw]
    uint32_t *HP;               // planes 2..6 [2n][cw][kHi], global
    uint32_t *cmask;            // candidate bitmask [nw]
    uint32_t *lmask;            // vertices present in the candidate list [nw]
    uint16_t *list;             // candidate list (may hold stale entries) [nv], global memory
    uint16_t *xr;               // [2n][n1p] XOR of the ids of a line's vertices of each colour, global
    uint2 *tc;                  // tabu cache [nv] in global memory (L1-resident for the candidates):
                                // x = e0 | e1 << 16, y = c0 | c1 << 8 | emax << 16
    unsigned long long *red;    // [2][NW] best key per warp (double-buffered)
    int *red_cnt;               // [2][NW] live candidates seen per warp
    int *scal;                  // [32]: 0 list length, 2 counts >= 4, 4 |C(S)|, 5..6 move
                                // scratch, 7 walk id, 8..15 reductions, 16..29 the walk's
                                // 64-bit work totals (WalkTotals)
};

// Per-thread view: instance data, its slot and its place in the group.
struct Ctx {
    const uint16_t *rc;         // [nv] row << 8 | column (shared by the block)
    const uint4 *allow;         // [2n] allowed colours per row, then per column (shared)
    const uint8_t *linelen;     // [2n] reduced vertices per row, then per column (shared)
    Slot s;
    int n;                      // order: line index of column c is n + c
    int cw;                     // colour words of the plane layout
    int g;                      // group (walk slot) within the block
    int gt;                     // thread index within the group
    int lane;                   // lane within the warp
    int gl;                     // lane within the group's part of the warp
    int wg;                     // warp within the group
    unsigned gm;                // the group's lanes within the warp
};

template <int GT>
__device__ __forceinline__ void gsync(const Ctx &c)
{
    if (Grp<GT>::NW == 1) __syncwarp(c.gm);
    else asm volatile("bar.sync %0, %1;" ::"r"(c.g + 1), "r"(GT) : "memory");
}

// context of thread threadIdx.x in group g: instance data at rc / allow /
// linelen (shared or global memory), the walk's slot at sb; NWC = colour words
// of the instance (a compile-time constant of the kernel)
template <int NWC, int GT>
__device__ __forceinline__ Ctx make_ctx_at(const DevInst &I, bool s_smem, const uint16_t *rc, const uint4 *allow,
                                           const uint8_t *linelen, uint8_t *sb)
{
    const SmemPlan p = make_plan(I, Grp<GT>::NW, s_smem);
    Ctx c;
    c.rc = rc;
    c.allow = allow;
    c.linelen = linelen;
    c.g = threadIdx.x / GT;
    c.gt = threadIdx.x % GT;
    c.lane = threadIdx.x & 31;
    c.gl = c.lane & (Grp<GT>::W - 1);
    c.wg = c.gt >> 5;
    c.gm = Grp<GT>::W == 32 ? FULL : (((1u << Grp<GT>::W) - 1u) << (c.lane & ~(Grp<GT>::W - 1)));
    c.s.S = s_smem ? sb + p.off_S : nullptr;      // global buffer set once the slot is known
    c.s.P01 = reinterpret_cast<uint2 *>(sb + p.off_P01);
    c.s.PH = reinterpret_cast<uint32_t *>(sb + p.off_PH);
    c.s.cmask = reinterpret_cast<uint32_t *>(sb + p.off_cmask);
    c.s.lmask = reinterpret_cast<uint32_t *>(sb + p.off_lmask);
    c.s.list = nullptr;         // set once the walk slot is known
    c.s.HP = nullptr;
    c.s.xr = nullptr;
    c.s.tc = nullptr;
    c.s.red = reinterpret_cast<unsigned long long *>(sb + p.off_red);
    c.s.red_cnt = reinterpret_cast<int *>(sb + p.off_red + 16 * Grp<GT>::NW);
    c.s.scal = c.s.red_cnt + 2 * Grp<GT>::NW;
    c.n = I.n;
    c.cw = NWC;
    return c;
}

// block layout of the single-instance kernel: instance part, then the slots
template <int NWC, int GT>
__device__ __forceinline__ Ctx make_ctx(uint8_t *base, const DevInst &I, bool s_smem)
{
    const SmemPlan p = make_plan(I, Grp<GT>::NW, s_smem);
    const int g = threadIdx.x / GT;
    return make_ctx_at<NWC, GT>(I, s_smem, reinterpret_cast<const uint16_t *>(base),
                           reinterpret_cast<const uint4 *>(base + align16(2 * (size_t)I.nv)),
                           base + align16(2 * (size_t)I.nv) + 32 * (size_t)I.n, base + p.inst + p.slot * g);
}

// Work counters of a walk (plse_walk_stats), kept as 64-bit totals in the
// slot's shared memory.  Iterations and moves are added per phase from the
// iteration count (a move is counted unless the iteration had none).  The sums
// that grow every iteration are 32-bit registers (the scanned pairs per lane),
// folded into the totals every 2^14 iterations and at the end of each phase,
// which keeps them below 2^32 at any instance size (fewer than 2^14 candidates
// of at most 127 colours per iteration).  After a failed device check the
// counters are unspecified.
struct WalkTotals {
    long long iterations, moves, cand, pairs, deg, improvements, uncolored;
};

struct IterCounters {
    uint32_t cand, pairs, deg;
};

constexpr int kFoldMask = (1 << 14) - 1;

__device__ __forceinline__ WalkTotals *walk_totals(const Ctx &c)
{
    return reinterpret_cast<WalkTotals *>(c.s.scal + 16);
}

template <int GT>
__device__ __forceinline__ int gsum(int x, const Ctx &c)
{
    x = __reduce_add_sync(c.gm, x);
    if (Grp<GT>::NW == 1) return x;
    gsync<GT>(c);
    if (c.lane == 0) c.s.scal[8 + c.wg] = x;
    gsync<GT>(c);
    int t = 0;
#pragma unroll
    for (int k = 0; k < Grp<GT>::NW; ++k) t += c.s.scal[8 + k];
    gsync<GT>(c);
    return t;
}

template <int GT>
__device__ __forceinline__ uint32_t gmax(uint32_t x, const Ctx &c)
{
    x = __reduce_max_sync(c.gm, x);
    if (Grp<GT>::NW == 1) return x;
    gsync<GT>(c);
    if (c.lane == 0) c.s.scal[8 + c.wg] = (int)x;
    gsync<GT>(c);
    uint32_t t = 0;
#pragma unroll
    for (int k = 0; k < Grp<GT>::NW; ++k) t = max(t, (uint32_t)c.s.scal[8 + k]);
    gsync<GT>(c);
    return t;
}

template <int GT>
__device__ __forceinline__ long long gsum64(long long x, const Ctx &c)
{
#pragma unroll
    for (int o = Grp<GT>::W / 2; o > 0; o >>= 1) x += __shfl_xor_sync(c.gm, x, o, Grp<GT>::W);
    if (Grp<GT>::NW == 1) return x;
    gsync<GT>(c);
    if (c.lane == 0) c.s.red[c.wg] = (unsigned long long)x;
    gsync<GT>(c);
    long long t = 0;
#pragma unroll
    for (int k = 0; k < Grp<GT>::NW; ++k) t += (long long)c.s.red[k];
    gsync<GT>(c);
    return t;
}

// adds the iteration counters to the walk's totals and clears them (the whole
// group calls it)
template <int GT>
__device__ __forceinline__ void fold_counters(const Ctx &c, IterCounters &k)
{
    const long long pairs = gsum64<GT>((long long)k.pairs, c);
    if (c.gt == 0) {
        WalkTotals *w = walk_totals(c);
        w->cand += k.cand;
        w->pairs += pairs;
        w->deg += k.deg;
    }
    k = IterCounters{0u, 0u, 0u};
}

// iterations 1 .. t-1 of a phase were executed; every one of them made a move
// unless it was counted off when it had none
__device__ __forceinline__ void count_iterations(const Ctx &c, int t)
{
    if (c.gt == 0) {
        WalkTotals *w = walk_totals(c);
        w->iterations += t - 1;
        w->moves += t - 1;
    }
}

template <int GT>
__device__ __forceinline__ void gcopy(uint8_t *dst, const uint8_t *src, int n, const Ctx &c)
{
    for (int q = c.gt; q < n; q += GT) dst[q] = src[q];
}

// ---- colour-count planes ----------------------------------------------------
// Lines are numbered 0..n-1 for rows and n..2n-1 for columns.
__device__ __forceinline__ size_t plane_word(const Ctx &c, int line, int k)
{
    return (size_t)line * c.cw + (k >> 5);
}

// +1 / -1 on count[line][k] (one thread per line at a time).  Returns the change
// in the number of counts >= 4, which selects the evaluation path, and the
// updated shared words (plane 0, plane 1, high OR) in *lo_out (may be null).
__device__ __forceinline__ int count_step(const Ctx &c, int line, int k, bool inc, uint4 *lo_out = nullptr)
{
    const size_t w = plane_word(c, line, k);
    uint2 a = c.s.P01[w];
    uint32_t z = c.s.PH[w];
    const uint32_t bit = 1u << (k & 31);
    const int old_hi = (z & bit) ? 1 : 0;
    uint32_t carry = bit, t;
    t = inc ? (a.x & carry) : (~a.x & carry);
    a.x ^= carry;
    carry = t;
    t = inc ? (a.y & carry) : (~a.y & carry);
    a.y ^= carry;
    carry = t;
    if (carry) {                                   // crosses a multiple of 4: planes 2..6
        uint32_t *g = c.s.HP + w * kHi;
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
        z = ((x[0] | x[1] | x[2] | x[3] | x[4]) & bit) ? (z | bit) : (z & ~bit);
        c.s.PH[w] = z;
    }
    c.s.P01[w] = a;
    if (lo_out) *lo_out = make_uint4(a.x, a.y, z, 0u);
    return ((z & bit) ? 1 : 0) - old_hi;
}

// count from the shared words: exact below 4, reported as 4 + (count mod 4) from
// 4 on, which decides every "count > t" test with t <= 3 like the exact count
__device__ __forceinline__ int count_low(const uint4 &a, int k)
{
    const uint32_t b = k & 31;
    return (int)(((a.x >> b) & 1u) | (((a.y >> b) & 1u) << 1) | (((a.z >> b) & 1u) << 2));
}

__device__ __forceinline__ int count_of_fast(const Ctx &c, int line, int k)
{
    const size_t w = plane_word(c, line, k);
    const uint2 a = c.s.P01[w];
    return count_low(make_uint4(a.x, a.y, c.s.PH[w], 0u), k);
}

// exact count (planes 2..6 read from global memory only when the count is >= 4)
__device__ __forceinline__ int count_of(const Ctx &c, int line, int k)
{
    const size_t w = plane_word(c, line, k);
    const uint2 a = c.s.P01[w];
    const uint32_t b = k & 31;
    int x = (int)(((a.x >> b) & 1u) | (((a.y >> b) & 1u) << 1));
    if ((c.s.PH[w] >> b) & 1u) {
        const uint32_t *g = c.s.HP + w * kHi;
#pragma unroll
        for (int p = 0; p < 5; ++p) x |= (int)((g[p] >> b) & 1u) << (p + 2);
    }
    return x;
}

__device__ __forceinline__ int gamma_of(const Ctx &c, int v, int k)
{
    const uint16_t rc = c.rc[v];
    return count_of(c, rc >> 8, k) + count_of(c, c.n + (rc & 255), k) - 2;
}

// planes and member-id XOR tables from the colouring; returns the number of
// counts >= 4 (also left in scal[2])
template <int GT>
__device__ __forceinline__ int build_planes(const DevInst &I, const Ctx &c)
{
    const int words = 2 * I.n * c.cw, hi_words_n = 2 * I.n * c.cw * kHi;
    for (int q = c.gt; q < words; q += GT) {
        c.s.P01[q] = make_uint2(0u, 0u);
        c.s.PH[q] = 0u;
    }
    for (int q = c.gt; q < hi_words_n; q += GT) c.s.HP[q] = 0u;
    gsync<GT>(c);
    for (int l = c.gt; l < 2 * I.n; l += GT) {
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
                count_step(c, l, k, true);
                X[k] ^= (uint16_t)u;
            }
        }
    }
    gsync<GT>(c);
    int hi = 0;
    for (int t = c.gt; t < words; t += GT) hi += __popc(c.s.PH[t]);
    hi = gsum<GT>(hi, c);
    if (c.gt == 0) c.s.scal[2] = hi;
    gsync<GT>(c);
    return hi;
}

// conflicting edges c(S) = sum over lines and colours of C(count, 2), from the
// planes: sum of count^2 = sum_{p,q} 2^(p+q) popc(P_p & P_q)
template <int GT>
__device__ __forceinline__ int conflict_edges(const DevInst &I, const Ctx &c)
{
    long long s = 0;
    for (int t = c.gt; t < 2 * I.n * c.cw; t += GT) {
        const uint2 lo = c.s.P01[t];
        const uint32_t *g = c.s.HP + (size_t)t * kHi;
        const bool high = c.s.PH[t] != 0u;
        const uint32_t w[7] = {lo.x, lo.y, high ? g[0] : 0u, high ? g[1] : 0u, high ? g[2] : 0u,
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
    return gsum<GT>((int)s, c);
}

// candidate bits (PLITS: V0 u C(S); PartialCol: V0), f and |C|; list = members
template <int GT>
__device__ __forceinline__ void build_cands(const DevInst &I, const Ctx &c, bool only_v0, int &f, int &nconf)
{
    int lf = 0, lc = 0;
    for (int wd = c.gt; wd < I.nw; wd += GT) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int v = wd * 32 + b;
            if (v >= I.nv) break;
            const int k = c.s.S[v];
            if (k == 0) {
                bits |= 1u << b;
                ++lf;
            } else if (gamma_of(c, v, k) > 0) {
                ++lc;
                if (!only_v0) bits |= 1u << b;
            }
        }
        c.s.cmask[wd] = bits;
    }
    f = gsum<GT>(lf, c);
    nconf = gsum<GT>(lc, c);
}

// rebuilds the candidate list from the bitmask (order is irrelevant); returns
// its length (also left in scal[0])
template <int GT>
__device__ __forceinline__ int rebuild_list(const DevInst &I, const Ctx &c)
{
    constexpr int W = Grp<GT>::W, NW = Grp<GT>::NW;
    gsync<GT>(c);
    const int w0 = (c.wg * I.nw) / NW, w1 = ((c.wg + 1) * I.nw) / NW;
    int cnt = 0;
    for (int wd = w0 + c.gl; wd < w1; wd += W) cnt += __popc(c.s.cmask[wd]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const int y = __shfl_up_sync(c.gm, incl, o, W);
        if (c.gl >= o) incl += y;
    }
    const int wtotal = __shfl_sync(c.gm, incl, W - 1, W);
    int base = 0, total = wtotal;
    if (NW > 1) {
        if (c.lane == 0) c.s.scal[8 + c.wg] = wtotal;
        gsync<GT>(c);
        total = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int x = c.s.scal[8 + k];
            if (k < c.wg) base += x;
            total += x;
        }
    }
    int pos = base + incl - cnt;
    for (int wd = w0 + c.gl; wd < w1; wd += W) {
        uint32_t bits = c.s.cmask[wd];
        c.s.lmask[wd] = bits;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            c.s.list[pos++] = (uint16_t)(wd * 32 + b);
        }
    }
    gsync<GT>(c);
    if (c.gt == 0) c.s.scal[0] = total;
    gsync<GT>(c);
    return total;
}

// ---- tabu cache -------------------------------------------------------------
struct Clock {
    uint32_t base;    // absolute clock of iteration 0 of the phase
    uint32_t shift;   // relative clock = t - shift
};

template <int GT>
__device__ __forceinline__ void tabu_reset(const DevInst &I, const Ctx &c)
{
    for (int v = c.gt; v < I.nv; v += GT) c.s.tc[v] = make_uint2(0u, 0xFFFFu);
}

template <int GT>
__device__ __forceinline__ void tabu_rebase(const DevInst &I, const Ctx &c)
{
    for (int v = c.gt; v < I.nv; v += GT) {
        const uint2 x = c.s.tc[v];
        uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16, em = x.y >> 16;
        e0 = e0 > kRebaseBy ? e0 - kRebaseBy : 0u;
        e1 = e1 > kRebaseBy ? e1 - kRebaseBy : 0u;
        em = em > kRebaseBy ? em - kRebaseBy : 0u;
        c.s.tc[v] = make_uint2(e0 | (e1 << 16), (x.y & 0xFFFFu) | (em << 16));
    }
}

// (v, k) tabu until relative clock e (inclusive); evicts to G when needed
// as tabu_insert, with v's cache entry x already loaded (by the same thread)
__device__ __forceinline__ void tabu_insert_entry(const DevInst &I, const Ctx &c, uint32_t *G, const Clock &ck,
                                                  int v, int k, uint32_t e, const uint2 x)
{
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

__device__ __forceinline__ void tabu_insert(const DevInst &I, const Ctx &c, uint32_t *G, const Clock &ck,
                                            int v, int k, uint32_t e)
{
    tabu_insert_entry(I, c, G, ck, v, k, e, c.s.tc[v]);
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
// lowest set bit over the words (colour index), or -1; no branch
template <int NWC>
__device__ __forceinline__ int first_bit(const uint32_t (&set)[NWC])
{
    int jb = -1;
#pragma unroll
    for (int q = NWC - 1; q >= 0; --q) jb = set[q] ? q * 32 + __ffs(set[q]) - 1 : jb;
    return jb;
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

// min over colours j in m of s_j = s0 + 2 s1 + 4 s2 (lowest j on ties) by a
// most-significant-plane-first elimination, in straight-line code (selects, no
// branches, so the lanes of a warp never split on the values); -1 if m is empty
template <int NWC>
__device__ __forceinline__ int bits_min3(const uint32_t (&s0)[NWC], const uint32_t (&s1)[NWC],
                                         const uint32_t (&s2)[NWC], const uint32_t (&m)[NWC], int &smin)
{
    uint32_t set[NWC];
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
        const bool keep = anyt != 0u;              // some colour has bit p clear
#pragma unroll
        for (int q = 0; q < NWC; ++q) set[q] = keep ? t[q] : set[q];
        val |= keep ? 0u : (1u << p);
    }
    smin = (int)val;
    return first_bit<NWC>(set);
}

// The tabu rule of one candidate (Sec. 3.3).  The two cache entries of v are
// authoritative for their colours; while an evicted entry of v may still be
// live (emax >= t) any other colour is looked up in the global table G.  The
// colours of m are taken in increasing (s_j, j) order, the order of their keys
// 2dF*256 + j, and the first admissible one (not tabu, or aspirating: 2dF < A)
// is the best move of m; a lookup in G is needed only for the colours that come
// before it, usually none or one.
struct TabuView {
    uint32_t e0, e1, c0, c1;
    bool gslow;                 // an evicted entry may be live: colours outside the cache go to G
    uint32_t tabs;              // absolute clock of this iteration
    const uint32_t *G;          // the slot's table
    uint32_t row;               // v * n1p: G row of v (addressed only on a lookup)
};

__device__ __forceinline__ TabuView tabu_view(const DevInst &I, const uint2 &te, const Clock &ck, uint32_t trel,
                                              const uint32_t *G, int v)
{
    TabuView t;
    t.e0 = te.x & 0xFFFFu;
    t.e1 = te.x >> 16;
    t.c0 = te.y & 0xFFu;
    t.c1 = (te.y >> 8) & 0xFFu;
    t.gslow = (te.y >> 16) >= trel;
    t.tabs = ck.base + ck.shift + trel;
    t.G = G;
    t.row = (uint32_t)v * (uint32_t)I.n1p;
    return t;
}

// colour 0 (uncolouring v) and the cache colours still tabu (taken out of m,
// admitted by aspiration only); returns the best key so far
template <int NWC, typename SVAL>
__device__ __forceinline__ int eval_special(const TabuView &tv, uint32_t trel, int i, int base2, int d2zero,
                                            int mult, int A, uint32_t (&m)[NWC], SVAL sval)
{
    int best = INT_MAX;
    if (i != 0) {
        const bool tabu0 = tv.c0 == 0u ? tv.e0 >= trel : tv.c1 == 0u ? tv.e1 >= trel : (tv.gslow && tv.G[tv.row] >= tv.tabs);
        if (!tabu0 || d2zero < A) best = d2zero * kKeyScale;
    }
    // the live cache colours of m (an expired one stays in m as an ordinary
    // colour); a live one is tabu and admissible by aspiration only, which needs
    // 2dF < A, while 2dF >= base2 for every colour (s_j >= 0): the values are
    // needed only when base2 < A
    // (the word of each cache colour is selected once, for the test and the clear;
    // an empty entry, colour 255, selects no word)
    uint32_t sel0[NWC], sel1[NWC];
    word_masks<NWC>(tv.c0, sel0);
    word_masks<NWC>(tv.c1, sel1);
    const uint32_t b0 = 1u << (tv.c0 & 31u), b1 = 1u << (tv.c1 & 31u);
    uint32_t w0 = 0u, w1 = 0u;
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        w0 |= m[q] & sel0[q];
        w1 |= m[q] & sel1[q];
    }
    const bool l0 = tv.c0 != 0u && tv.e0 >= trel && (w0 & b0) != 0u;
    const bool l1 = tv.c1 != 0u && tv.e1 >= trel && (w1 & b1) != 0u;
    if ((l0 || l1) && base2 < A) {
#pragma unroll
        for (int sx = 0; sx < 2; ++sx) {
            const uint32_t cs = sx ? tv.c1 : tv.c0;
            if (sx ? l1 : l0) {
                const int d2 = base2 + mult * sval(cs);
                if (d2 < A) best = min(best, d2 * kKeyScale + (int)cs);
            }
        }
    }
    // out of m
    const uint32_t k0 = l0 ? b0 : 0u, k1 = l1 ? b1 : 0u;
#pragma unroll
    for (int q = 0; q < NWC; ++q) m[q] &= ~((k0 & sel0[q]) | (k1 & sel1[q]));
    return best;
}

// eval while all counts are <= 3: planes 0-1 of R and K only (sums <= 6)
template <int NWC>
__device__ __forceinline__ int eval_vertex_low(const DevInst &I, const Ctx &c, const uint32_t *G, const Clock &ck,
                                               uint32_t trel, int v, int mult, int base_unc, int A, int &pairs,
                                               int &iv)
{
    // the tabu-cache entry (global memory) is loaded first and used last, so its
    // latency overlaps the shared-memory loads and the bit-sliced arithmetic
    const uint2 te = c.s.tc[v];
    const int i = c.s.S[v];
    iv = i;
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255;
    const uint2 *Pr = c.s.P01 + (size_t)r * NWC, *Pc = c.s.P01 + (size_t)(I.n + cc) * NWC;
    uint32_t s0[NWC], s1[NWC], s2[NWC];
#pragma unroll
    for (int q = 0; q < NWC; ++q) {
        const uint2 ra = Pr[q];
        const uint2 ka = Pc[q];
        const uint32_t x0 = ra.x ^ ka.x, cy = ra.x & ka.x, x1 = ra.y ^ ka.y;
        s0[q] = x0;
        s1[q] = x1 ^ cy;
        s2[q] = (ra.y & ka.y) | (cy & x1);
    }
    // gamma[v][i] from the row and column words of colour i (counts <= 3 here)
    const uint2 ri = Pr[i >> 5], ki = Pc[i >> 5];
    const uint32_t bi = (uint32_t)i & 31u;
    const int gi = i ? (int)(((ri.x >> bi) & 1u) + ((ri.y >> bi) & 1u) * 2u + ((ki.x >> bi) & 1u) +
                             ((ki.y >> bi) & 1u) * 2u) - 2
                     : 0;
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
    clear_bit<NWC>(m, (uint32_t)i);                // colour 0 is never in m: no-op when i = 0
    const TabuView tv = tabu_view(I, te, ck, trel, G, v);
    int best = eval_special<NWC>(tv, trel, i, base2, d2zero, mult, A, m,
                                 [&](uint32_t k) { return value3<NWC>(s0, s1, s2, k); });
    for (;;) {
        int smin = 0;
        const int jb = bits_min3<NWC>(s0, s1, s2, m, smin);
        if (jb < 0) break;
        const int d2 = base2 + mult * smin;
        const bool tabu = tv.gslow && (uint32_t)jb != tv.c0 && (uint32_t)jb != tv.c1 && tv.G[tv.row + (uint32_t)jb] >= tv.tabs;
        if (!tabu || d2 < A) {
            best = min(best, d2 * kKeyScale + jb);
            break;
        }
        clear_bit<NWC>(m, (uint32_t)jb);
    }
    return best;
}

// s_j = R[line_r][j] + K[line_c][j] for the 32 colours of word q, bit-sliced
// (8 planes; planes 2..6 of a line read from global memory only when one of its
// counts in the word is >= 4)
__device__ __forceinline__ void word_sum(const Ctx &c, int rl, int cl, int q, uint32_t (&s)[8])
{
    const size_t wr = plane_word(c, rl, q * 32), wc = plane_word(c, cl, q * 32);
    const uint2 r0 = c.s.P01[wr];
    const uint2 k0 = c.s.P01[wc];
    uint32_t a[7] = {r0.x, r0.y, 0u, 0u, 0u, 0u, 0u};
    uint32_t b[7] = {k0.x, k0.y, 0u, 0u, 0u, 0u, 0u};
    if (c.s.PH[wr]) {
        const uint32_t *g = c.s.HP + wr * kHi;
#pragma unroll
        for (int p = 0; p < 5; ++p) a[p + 2] = g[p];
    }
    if (c.s.PH[wc]) {
        const uint32_t *g = c.s.HP + wc * kHi;
#pragma unroll
        for (int p = 0; p < 5; ++p) b[p + 2] = g[p];
    }
    uint32_t carry = 0u;
#pragma unroll
    for (int p = 0; p < 7; ++p) {
        const uint32_t x = a[p] ^ b[p];
        s[p] = x ^ carry;
        carry = (a[p] & b[p]) | (carry & x);
    }
    s[7] = carry;
}

// min over the colours j of m of s_j (lowest j on ties) with exact counts, one
// colour word at a time: each word's minimum by most-significant-plane-first
// elimination over its 8 planes, then the smallest (value, word); -1 if m is
// empty.  Only one word's planes are held at once.
template <int NWC>
__device__ __forceinline__ int exact_min(const Ctx &c, int rl, int cl, const uint32_t (&m)[NWC], int &smin)
{
    uint32_t bestv = 0xFFFFFFFFu;
    int jb = -1;
#pragma unroll 1
    for (int q = 0; q < NWC; ++q) {                 // not unrolled: one word's planes live at a time
        uint32_t mq = m[0];
#pragma unroll
        for (int w = 1; w < NWC; ++w) mq = q == w ? m[w] : mq;
        uint32_t s[8];
        word_sum(c, rl, cl, q, s);
        uint32_t set = mq, val = 0u;
#pragma unroll
        for (int p = 7; p >= 0; --p) {
            const uint32_t t = set & ~s[p];
            const bool keep = t != 0u;                  // some colour of the word has bit p clear
            set = keep ? t : set;
            val |= keep ? 0u : (1u << p);
        }
        const bool better = mq != 0u && val < bestv;    // strict: a lower word wins ties
        bestv = better ? val : bestv;
        jb = better ? q * 32 + __ffs(set) - 1 : jb;
    }
    smin = (int)bestv;
    return jb;
}

// eval with exact counts (planes 2..6 read where a count reaches 4)
template <int NWC>
__device__ __forceinline__ int eval_vertex(const DevInst &I, const Ctx &c, const uint32_t *G, const Clock &ck,
                                           uint32_t trel, int v, int mult, int base_unc, int A, int &pairs, int &iv)
{
    const uint2 te = c.s.tc[v];
    const int i = c.s.S[v];
    iv = i;
    const uint16_t rc = c.rc[v];
    const int r = rc >> 8, cc = rc & 255, rl = r, cl = I.n + cc;
    const int gi = i ? count_of(c, rl, i) + count_of(c, cl, i) - 2 : 0;
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
    clear_bit<NWC>(m, (uint32_t)i);                // colour 0 is never in m: no-op when i = 0
    const TabuView tv = tabu_view(I, te, ck, trel, G, v);
    int best = eval_special<NWC>(tv, trel, i, base2, d2zero, mult, A, m,
                                 [&](uint32_t k) { return count_of(c, rl, (int)k) + count_of(c, cl, (int)k); });
    for (;;) {
        int smin = 0;
        const int jb = exact_min<NWC>(c, rl, cl, m, smin);
        if (jb < 0) break;
        const int d2 = base2 + mult * smin;
        const bool tabu = tv.gslow && (uint32_t)jb != tv.c0 && (uint32_t)jb != tv.c1 && tv.G[tv.row + (uint32_t)jb] >= tv.tabs;
        if (!tabu || d2 < A) {
            best = min(best, d2 * kKeyScale + jb);
            break;
        }
        clear_bit<NWC>(m, (uint32_t)jb);
    }
    return best;
}

__device__ __forceinline__ int vertex_degree(const DevInst &I, const Ctx &c, int v)
{
    const uint16_t rc = c.rc[v];
    return (int)c.linelen[rc >> 8] + (int)c.linelen[I.n + (rc & 255)] - 2;
}

// reserve a clock range for one phase of this slot
template <int GT>
__device__ __forceinline__ Clock claim_clock(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, int slot, int span)
{
    gsync<GT>(c);
    if (c.gt == 0) {
        uint32_t base = a.slot_clock[slot] + 1u;
        if (base > 0x7FFFFFFFu - (uint32_t)span) base = 0u;   // wrap: clear the slot
        c.s.scal[1] = (int)base;
    }
    gsync<GT>(c);
    uint32_t base = (uint32_t)c.s.scal[1];
    if (base == 0u) {
        const size_t words = a.g_stride;              // the slot's whole table
        for (size_t q = c.gt; q < words; q += GT) G[q] = 0u;
        base = 1u;
    }
    gsync<GT>(c);
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
template <int GT>
__device__ __forceinline__ unsigned long long group_best(const Ctx &c, int parity, unsigned long long key,
                                                         int live, int &total)
{
    constexpr int NW = Grp<GT>::NW;
    const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
    const uint32_t whi = __reduce_min_sync(c.gm, hi);
    const uint32_t wlo = __reduce_min_sync(c.gm, hi == whi ? lo : 0xffffffffu);
    const unsigned long long wk = ((unsigned long long)whi << 32) | wlo;
    const int wl = __reduce_add_sync(c.gm, live);
    if (NW == 1) {
        total = wl;
        return wk;
    }
    if (c.lane == 0) {
        c.s.red[parity * NW + c.wg] = wk;
        c.s.red_cnt[parity * NW + c.wg] = wl;
    }
    gsync<GT>(c);
    unsigned long long best = kNoKey;
    total = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        best = min(best, c.s.red[parity * NW + k]);
        total += c.s.red_cnt[parity * NW + k];
    }
    return best;
}

// first warp of the group: appends the lanes' flagged vertices to the candidate list
__device__ __forceinline__ void list_append(const Ctx &c, bool want, int u, int &len)
{
    const uint32_t b = __ballot_sync(c.gm, want);
    if (want) {
        const int pos = len + __popc(b & ((1u << c.lane) - 1u));
        c.s.list[pos] = (uint16_t)u;
        atomicOr(&c.s.lmask[u >> 5], 1u << (u & 31));
    }
    len += __popc(b);
}

// One scan pass of a single-warp group over list entries base .. base+W-1:
// stale entries (no longer candidates) are dropped and lose their membership
// bit, live ones are written back contiguously at wpos, so the list stays about
// as long as the candidate set and a scan needs no pass over stale entries.
// Returns the lane's live vertex or -1.
template <int W>
__device__ __forceinline__ int list_pass(const Ctx &c, int base, int len, int &wpos)
{
    const int qq = base + c.gl;
    int v = -1;
    bool lv = false;
    if (qq < len) {
        v = c.s.list[qq];
        lv = (c.s.cmask[v >> 5] >> (v & 31)) & 1u;
        if (!lv) atomicAnd(&c.s.lmask[v >> 5], ~(1u << (v & 31)));
    }
    const uint32_t b = __ballot_sync(c.gm, lv);
    __syncwarp(c.gm);                                 // every entry of the pass read before any write
    const int to = wpos + __popc(b & ((1u << c.lane) - 1u));
    if (lv && to != qq) c.s.list[to] = (uint16_t)v;  // entries that do not move stay cached
    wpos += __popc(b);
    return lv ? v : -1;
}

// ---- PLITS phase (Alg. 3 with phi2 = 2*phi) --------------------------------
// Within one warp (GT <= 32) the list length, |C(S)|, the number of counts >= 4
// and the check result are known to every lane after the move's collectives
// and stay in registers; wider groups pass them through the slot's scalars.
template <int NWC, int GT>
__device__ __forceinline__ bool plits_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, uint8_t *gbest,
                            int slot, int ind, int phase, int64_t N, int phi2, int span,
                            long long &F2best_out)
{
    constexpr int W = Grp<GT>::W, NW = Grp<GT>::NW;
    int hi = build_planes<GT>(I, c);
    int f, nconf;
    build_cands<GT>(I, c, false, f, nconf);
    const int cedges = conflict_edges<GT>(I, c);
    long long F2 = 2LL * f + (long long)phi2 * cedges;
    long long F2best = F2;
    gcopy<GT>(gbest, c.s.S, I.nv, c);
    tabu_reset<GT>(I, c);
    int len = rebuild_list<GT>(I, c);
    Clock ck = claim_clock<GT>(I, a, c, G, slot, span);

    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    IterCounters wc = {0u, 0u, 0u};
    const int Nt = (int)N;                               // at most 2^30 (checked by the host)
    int t = 1;
    for (; t <= Nt; ++t) {
        if (f + nconf == 0) break;                       // nothing left to improve
        if ((t & kFoldMask) == 0) fold_counters<GT>(c, wc);
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            gsync<GT>(c);
            tabu_rebase<GT>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            gsync<GT>(c);
        }
        if (NW > 1) {
            len = c.s.scal[0];
            hi = c.s.scal[2];
        }
        if (len > 2 * (f + nconf) + 64) len = rebuild_list<GT>(I, c);
        const int q = (int)((t - 1) & (W - 1));
        if (q == 0) {
            // counter (iteration, individual, gen << 8 | purpose << 4 | phase)
            const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | (uint32_t)phase;
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + c.gl), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(c.gm, Lr, q, W);
        const int rsh = (int)__shfl_sync(c.gm, rotr, q, W);
        const long long A64 = F2best - F2;
        const int A = A64 < -(1LL << 30) ? -(1 << 30) : (int)A64;

        const bool low = hi == 0;                     // every count <= 3
        unsigned long long key = kNoKey;
        int live = 0;
        auto consider = [&](int v) {
            ++live;
            int pairs, iv;
            const int kv = low ? eval_vertex_low<NWC>(I, c, G, ck, trel, v, phi2, -2, A, pairs, iv)
                               : eval_vertex<NWC>(I, c, G, ck, trel, v, phi2, -2, A, pairs, iv);
            wc.pairs += (uint32_t)pairs;
            if (kv != INT_MAX) key = min(key, make_key(kv, v, rsh, I.nv, iv));
        };
        if constexpr (NW == 1) {
            int wpos = 0;
            for (int base = 0; base < len; base += W) {
                const int v = list_pass<W>(c, base, len, wpos);
                if (v >= 0) consider(v);
            }
            len = wpos;
        } else {
            for (int qq = c.gt; qq < len; qq += GT) {
                const int v = c.s.list[qq];
                if ((c.s.cmask[v >> 5] >> (v & 31)) & 1u) consider(v);   // else a stale entry
            }
        }
        int ncand;
        const unsigned long long best = group_best<GT>(c, (int)(t & 1), key, live, ncand);
        if (ncand != f + nconf) { ok = false; break; }
        wc.cand += (uint32_t)ncand;
        if (best == kNoKey) {                            // every move tabu
            if (c.gt == 0) walk_totals(c)->moves -= 1;
            continue;
        }

        const uint32_t bhi = (uint32_t)(best >> 32), blo = (uint32_t)best;
        const int d2 = (int)bhi - (1 << 30);
        const int j = (int)((blo >> 8) & 255u), i = (int)(blo & 255u);
        int v = (int)(blo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        f += (j == 0) - (i == 0);
        F2 += d2;
        bool bad = false;
        int degv = 0;
        if (c.wg == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            // v's tabu-cache entry and degree, needed last, loaded first
            const uint2 tcv = c.gl == 0 ? c.s.tc[v] : make_uint2(0u, 0u);
            degv = (int)c.linelen[r] + (int)c.linelen[I.n + cc] - 2;
            // member-id XOR of (row r | column cc, colour i | j), read first so that
            // its latency overlaps the count updates: lane 0 row/i, 1 column/i,
            // 2 row/j, 3 column/j
            const int xk = c.gl < 2 ? i : j;
            const int xline = (c.gl & 1) ? I.n + cc : r;
            const size_t xidx = (size_t)xline * I.n1p + xk;
            const int xold = (c.gl < 4 && xk) ? (int)c.s.xr[xidx] : 0;
            // count updates: lane 0 on row r, lane 1 on column cc, colour i then j
            // (one lane per line, so no two lanes touch one plane word)
            int cnt_i = 0, cnt_j = 0, dh = 0;
            if (c.gl < 2) {
                uint4 w;
                if (i) {
                    dh += count_step(c, xline, i, false, &w);
                    cnt_i = count_low(w, i);              // counts after the move (4 = four or more)
                }
                if (j) {
                    dh += count_step(c, xline, j, true, &w);
                    cnt_j = count_low(w, j);
                }
            }
            if (c.gl == 0) c.s.S[v] = (uint8_t)j;
            // counts of colours i and j on the moved row (lane 0) and column (lane 1)
            // after the move, packed i | j << 8: lane l reads line l & 1's, and lane
            // 0 also the column's
            const int packed = cnt_i | (cnt_j << 8);
            const int line_cnt = __shfl_sync(c.gm, packed, c.gl & 1, W);
            const int col_cnt = __shfl_xor_sync(c.gm, packed, 1, W);
            __syncwarp(c.gm);
            // The mates whose conflict status can change, one per (line, colour) at
            // most: the only other holder of colour i (count after the move 1) and
            // the other holder of colour j (count after 2).  Each is read from the
            // member-id XOR of its line: lane 0 row/i, 1 column/i, 2 row/j, 3 column/j
            // (colour xk, line xline).
            int dconf = 0;
            const int su = xk;
            const int cl = c.gl < 2 ? 1 : 2;              // the mate's count on that line
            const int cnt_l = c.gl < 2 ? (line_cnt & 255) : (line_cnt >> 8);
            const int u = (c.gl < 4 && xk && cnt_l == cl) ? (c.gl < 2 ? xold ^ v : xold) : -1;
            const bool row_mate = (c.gl & 1) == 0;
            bool want = false, bad_mate = false;
            if (u >= 0) {
                if (u >= I.nv || u == v || c.s.S[u] != su) {
                    bad_mate = true;                     // inconsistent table: report, touch nothing
                } else {
                    const uint16_t urc = c.rc[u];
                    const int g = cl + (row_mate ? count_of_fast(c, I.n + (urc & 255), su)
                                                 : count_of_fast(c, urc >> 8, su)) - 2;
                    const int nc = g > 0, oc = (c.s.cmask[u >> 5] >> (u & 31)) & 1;
                    if (nc != oc) {
                        atomicXor(&c.s.cmask[u >> 5], 1u << (u & 31));
                        dconf += nc - oc;
                        want = nc && !((c.s.lmask[u >> 5] >> (u & 31)) & 1u);
                    }
                }
            }
            list_append(c, want, u, len);
            if (c.gl < 4 && xk) c.s.xr[xidx] = (uint16_t)(xold ^ v);   // v leaves i, joins j
            if (c.gl == 0) {
                const int newc = j ? (int)(cnt_j + (col_cnt >> 8) - 2 > 0) : 0;   // v's own status at j
                if (j != 0 && !newc) atomicAnd(&c.s.cmask[v >> 5], ~(1u << (v & 31)));
                dconf += newc - (i != 0 ? 1 : 0);
            }
            // one reduction for three sums: the change of |C(S)| (|.| <= 6), of the
            // number of counts >= 4 (|.| <= 4) and the inconsistent mates (<= 4)
            const int packed3 = __reduce_add_sync(c.gm, dconf + 32 * dh + 1024 * (int)bad_mate);
            dconf = ((packed3 + 16) & 31) - 16;
            const int rest = (packed3 - dconf) >> 5;
            const int dh_tot = ((rest + 16) & 31) - 16;
            bad = rest - dh_tot != 0;
            if (c.gl == 0) {
                const int k = f + nconf + dconf;
                const int T = L + tenure_div(a, a.alpha_num * k);
                tabu_insert_entry(I, c, G, ck, v, i, trel + (uint32_t)T, tcv);
            }
            if (NW == 1) {
                nconf += dconf;
                hi += dh_tot;
            } else if (c.lane == 0) {
                c.s.scal[4] = nconf + dconf;
                c.s.scal[0] = len;
                c.s.scal[2] = hi + dh_tot;
                c.s.scal[6] = bad ? 1 : 0;
            }
        }
        gsync<GT>(c);
        if (NW > 1) {
            bad = c.s.scal[6] != 0;
            nconf = c.s.scal[4];
        }
        if (bad) { ok = false; break; }
        if (c.gt == 0) wc.deg += (uint32_t)degv;
        if (F2 < F2best) {
            F2best = F2;
            if (c.gt == 0) walk_totals(c)->improvements += 1;
            gcopy<GT>(gbest, c.s.S, I.nv, c);
        }
    }
    fold_counters<GT>(c, wc);
    count_iterations(c, t);
    gsync<GT>(c);
    gcopy<GT>(c.s.S, gbest, I.nv, c);
    gsync<GT>(c);
    F2best_out = F2best;
    return ok;
}

// ---- greedy conflict removal (Sec. 3.7) ------------------------------------
template <int GT>
__device__ __forceinline__ void repair(const DevInst &I, const Ctx &c)
{
    build_planes<GT>(I, c);
    for (int step = 0; step < I.nv; ++step) {
        uint32_t key = 0;
        for (int v = c.gt; v < I.nv; v += GT) {
            const int k = c.s.S[v];
            if (!k) continue;
            const int g = gamma_of(c, v, k);
            if (g > 0) key = max(key, ((uint32_t)g << 16) | (0xFFFFu - (uint32_t)v));
        }
        const uint32_t m = gmax<GT>(key, c);
        if (m == 0u) break;
        const int v = (int)(0xFFFFu - (m & 0xFFFFu));
        gsync<GT>(c);
        if (c.gt == 0) {
            const int k = c.s.S[v];
            const uint16_t rc = c.rc[v];
            c.s.S[v] = 0;
            c.s.scal[2] += count_step(c, rc >> 8, k, false) + count_step(c, I.n + (rc & 255), k, false);
        }
        gsync<GT>(c);
    }
}

// ---- PartialCol (Sec. 3.7): legal partial colourings only ------------------
template <int NWC, int GT>
__device__ __forceinline__ bool partialcol_phase(const DevInst &I, const LSArgs &a, const Ctx &c, uint32_t *G, uint8_t *gbest,
                                 int slot, int ind, int64_t N, int span, long long &fbest_out)
{
    constexpr int W = Grp<GT>::W, NW = Grp<GT>::NW;
    build_planes<GT>(I, c);
    int f, nconf;
    build_cands<GT>(I, c, true, f, nconf);
    if (conflict_edges<GT>(I, c) != 0) return false;    // needs a legal start
    int fbest = f;
    gcopy<GT>(gbest, c.s.S, I.nv, c);
    tabu_reset<GT>(I, c);
    rebuild_list<GT>(I, c);
    Clock ck = claim_clock<GT>(I, a, c, G, slot, span);
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    int *ulist = c.s.scal + 8;   // a legal colouring has at most 2 mates of one colour
    IterCounters wc = {0u, 0u, 0u};
    const int Nt = (int)N;                               // at most 2^30 (checked by the host)
    int t = 1;
    for (; t <= Nt; ++t) {
        if (f == 0) break;
        if ((t & kFoldMask) == 0) fold_counters<GT>(c, wc);
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            gsync<GT>(c);
            tabu_rebase<GT>(I, c);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
            gsync<GT>(c);
        }
        int len = c.s.scal[0];
        if (len > 2 * f + 64) len = rebuild_list<GT>(I, c);
        const int q = (int)((t - 1) & (W - 1));
        if (q == 0) {
            const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | 3u;   // phase 3: PartialCol
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + c.gl), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(c.gm, Lr, q, W);
        const int rsh = (int)__shfl_sync(c.gm, rotr, q, W);
        const int A = fbest - f;
        const bool low = c.s.scal[2] == 0;            // every count <= 3
        unsigned long long key = kNoKey;
        int live = 0;
        auto consider = [&](int v) {
            ++live;
            int pairs, iv;
            const int kv = low ? eval_vertex_low<NWC>(I, c, G, ck, trel, v, 1, -1, A, pairs, iv)
                               : eval_vertex<NWC>(I, c, G, ck, trel, v, 1, -1, A, pairs, iv);
            wc.pairs += (uint32_t)pairs;
            if (kv != INT_MAX) key = min(key, make_key(kv, v, rsh, I.nv, 0));
        };
        if constexpr (NW == 1) {
            int wpos = 0;
            for (int base = 0; base < len; base += W) {
                const int v = list_pass<W>(c, base, len, wpos);
                if (v >= 0) consider(v);
            }
            if (c.gl == 0) c.s.scal[0] = wpos;
            __syncwarp(c.gm);
            len = wpos;
        } else {
            for (int qq = c.gt; qq < len; qq += GT) {
                const int v = c.s.list[qq];
                if ((c.s.cmask[v >> 5] >> (v & 31)) & 1u) consider(v);
            }
        }
        int ncand;
        const unsigned long long best = group_best<GT>(c, (int)(t & 1), key, live, ncand);
        if (ncand != f) { ok = false; break; }
        wc.cand += (uint32_t)ncand;
        if (best == kNoKey) {
            if (c.gt == 0) walk_totals(c)->moves -= 1;
            continue;
        }

        const int d = (int)(uint32_t)(best >> 32) - (1 << 30);
        const uint32_t blo = (uint32_t)best;
        const int j = (int)((blo >> 8) & 255u);
        int v = (int)(blo >> 16) + rsh;
        if (v >= I.nv) v -= I.nv;
        if (c.wg == 0) {
            const uint16_t rc = c.rc[v];
            const int r = rc >> 8, cc = rc & 255;
            const int T = L + tenure_div(a, a.alpha_num * (f + d));
            if (c.gl == 0) c.s.scal[5] = 0;
            __syncwarp(c.gm);
            // row- and column-mates coloured j lose their colour
            for (int side = 0; side < 2; ++side) {
                const int32_t *ptr = side ? I.col_ptr : I.row_ptr;
                const uint16_t *lst = side ? I.col_v : I.row_v;
                const int line = side ? cc : r;
                const int qb = __ldg(&ptr[line]), qe = __ldg(&ptr[line + 1]);
                for (int qq = qb + c.gl; qq < qe; qq += W) {
                    const int u = __ldg(&lst[qq]);
                    if (u == v || c.s.S[u] != j) continue;
                    const int k = atomicAdd(&c.s.scal[5], 1);
                    if (k < 8) ulist[k] = u;
                }
            }
            __syncwarp(c.gm);
            const int nunc = c.s.scal[5];
            const bool bad = nunc > 8 || nunc - 1 != d;
            int wantu = 0;
            bool want = false;
            if (!bad && c.gl < nunc) {
                wantu = ulist[c.gl];
                want = !((c.s.lmask[wantu >> 5] >> (wantu & 31)) & 1u);
            }
            __syncwarp(c.gm);
            if (!bad) {
                if (c.gl == 0) {
                    for (int k = 0; k < nunc; ++k) {
                        const int u = ulist[k];
                        const uint16_t rcu = c.rc[u];
                        c.s.S[u] = 0;
                        c.s.scal[2] += count_step(c, rcu >> 8, j, false) +
                                       count_step(c, I.n + (rcu & 255), j, false);
                        atomicOr(&c.s.cmask[u >> 5], 1u << (u & 31));
                        tabu_insert(I, c, G, ck, u, j, trel + (uint32_t)T);
                    }
                    c.s.S[v] = (uint8_t)j;
                    c.s.scal[2] += count_step(c, r, j, true) + count_step(c, I.n + cc, j, true);
                    atomicAnd(&c.s.cmask[v >> 5], ~(1u << (v & 31)));
                }
                __syncwarp(c.gm);
                list_append(c, want, wantu, len);
            }
            if (c.gl == 0) {
                c.s.scal[6] = bad ? 1 : 0;
                c.s.scal[0] = len;
            }
        }
        gsync<GT>(c);
        if (c.s.scal[6]) { ok = false; break; }
        if (c.gt == 0) walk_totals(c)->uncolored += c.s.scal[5];
        f += d;
        if (c.gt == 0) wc.deg += (uint32_t)vertex_degree(I, c, v);
        if (f < fbest) {
            fbest = f;
            if (c.gt == 0) walk_totals(c)->improvements += 1;
            gcopy<GT>(gbest, c.s.S, I.nv, c);
        }
    }
    fold_counters<GT>(c, wc);
    count_iterations(c, t);
    gsync<GT>(c);
    gcopy<GT>(c.s.S, gbest, I.nv, c);
    gsync<GT>(c);
    fbest_out = fbest;
    return ok;
}

// instance data shared by every walk slot of the block
__device__ __forceinline__ void load_instance(const DevInst &I, uint8_t *smem)
{
    uint16_t *rc_s = reinterpret_cast<uint16_t *>(smem);
    uint4 *allow_s = reinterpret_cast<uint4 *>(smem + align16(2 * (size_t)I.nv));
    for (int v = threadIdx.x; v < I.nv; v += blockDim.x) rc_s[v] = __ldg(&I.rc[v]);
    uint8_t *len_s = smem + align16(2 * (size_t)I.nv) + 32 * (size_t)I.n;
    for (int r = threadIdx.x; r < 2 * I.n; r += blockDim.x) {
        allow_s[r] = r < I.n ? I.allow_row[r] : I.allow_col[r - I.n];
        len_s[r] = (uint8_t)(r < I.n ? I.row_ptr[r + 1] - I.row_ptr[r] : I.col_ptr[r - I.n + 1] - I.col_ptr[r - I.n]);
    }
}

// The walk groups of one block take walks of one launch (instance I, arguments
// a) from its counter until none is left.
// PAIRED (single-instance launches with GT = 16): the two walks of a warp are
// pulled together and start together, so that their iterations run side by side
template <int NWC, int GT, bool PAIRED>
__device__ __forceinline__ void walk_loop(const DevInst &I, const LSArgs &a, int walks, Ctx c)
{
    if (c.g >= walks) return;
    const int slot = blockIdx.x * walks + c.g;
    uint32_t *G = a.G + (size_t)slot * a.g_stride;
    c.s.tc = a.TC + (size_t)slot * a.tc_stride;
    c.s.list = a.LIST + (size_t)slot * a.list_stride;
    c.s.xr = a.XR + (size_t)slot * a.xr_stride;
    c.s.HP = a.HP + (size_t)slot * a.hp_stride;
    if (!a.s_smem) c.s.S = a.SW + (size_t)slot * a.sw_stride;

    for (;;) {
        int wk;
        if constexpr (PAIRED) {
            // one pull of two walks per warp; a half without a walk waits for its
            // partner's (the launch holds an even number of 16-lane groups)
            __syncwarp(FULL);
            int base = 0;
            if (c.lane == 0) base = atomicAdd(a.work_counter, 2);
            base = __shfl_sync(FULL, base, 0);
            if (base >= a.count) break;
            wk = base + (c.lane >> 4);
            if (wk >= a.count) continue;
        } else {
            if (c.gt == 0) c.s.scal[7] = atomicAdd(a.work_counter, 1);
            gsync<GT>(c);
            wk = c.s.scal[7];
            gsync<GT>(c);
            if (wk >= a.count) break;
        }
        const int ind = a.ind0 + wk;
        const uint8_t *gin = a.S_in + (size_t)wk * I.nv;
        uint8_t *gout = a.S_out + (size_t)wk * I.nv;
        gcopy<GT>(c.s.S, gin, I.nv, c);
        if (c.gt == 0) *walk_totals(c) = WalkTotals{0, 0, 0, 0, 0, 0, 0};
        gsync<GT>(c);

        long long Flast = 0;
        bool ok = true;
        if (a.flags & PLSE_LS_PARTIALCOL) {
            if (a.flags & PLSE_LS_REPAIR) repair<GT>(I, c);
            ok = partialcol_phase<NWC, GT>(I, a, c, G, gout, slot, ind, a.iters1, a.span1, Flast);
        } else {
            if (a.flags & PLSE_LS_PHASE1)
                ok = plits_phase<NWC, GT>(I, a, c, G, gout, slot, ind, 1, a.iters1, a.phi2_1, a.span1, Flast);
            if (ok && (a.flags & PLSE_LS_PHASE2))
                ok = plits_phase<NWC, GT>(I, a, c, G, gout, slot, ind, 2, a.iters2, a.phi2_2, a.span2, Flast);
            if (ok && (a.flags & PLSE_LS_REPAIR)) repair<GT>(I, c);
        }
        gsync<GT>(c);
        if (!ok && c.gt == 0) atomicOr(a.error_flag, 1);
        gcopy<GT>(gout, c.s.S, I.nv, c);
        int z = 0;
        for (int q = c.gt; q < I.nv; q += GT) z += (c.s.S[q] == 0);
        const int fz = gsum<GT>(z, c);
        if (c.gt == 0) {
            if (a.f_out) a.f_out[wk] = fz;
            if (a.F_out) a.F_out[wk] = Flast;
            if (a.stats) {
                const WalkTotals w = *walk_totals(c);
                plse_walk_stats s;
                s.iterations = w.iterations;
                s.moves = w.moves;
                s.cand = w.cand;
                s.pairs = w.pairs;
                s.deg = w.deg;
                s.improvements = w.improvements;
                s.uncolored = w.uncolored;
                a.stats[wk] = s;
            }
        }
        gsync<GT>(c);
    }
}

template <int NWC, int GT>
__global__ void __launch_bounds__(kMaxThreads<NWC>, NWC >= 3 ? 1 : 2) local_search_kernel(const DevInst I, const LSArgs a, int walks)
{
    extern __shared__ __align__(16) uint8_t smem[];
    if (a.skip && *a.skip) return;
    load_instance(I, smem);
    __syncthreads();
    walk_loop<NWC, GT, GT == 16>(I, a, walks, make_ctx<NWC, GT>(smem, I, a.s_smem != 0));
}

// Several launches' worth of walks (one per job, e.g. the same generation of
// several runs) in one persistent launch.  Every walk group takes the jobs in
// order on its own: it copies a job's descriptor into its part of shared
// memory, takes the job's walks from the job's counter, and moves to the next
// job as soon as that counter runs out, so no group waits for another and the
// tail of one job is filled with walks of the next.  Instance data (vertex
// coordinates, allowed colours, line lengths) is read from global memory
// (L1-resident); each group's slot uses its job's own layout within a fixed
// stride.
struct JobDesc {
    DevInst I;
    LSArgs a;
};

template <int GT>
__device__ __forceinline__ void group_sync(int g, unsigned gm)
{
    if (Grp<GT>::NW == 1) __syncwarp(gm);
    else asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GT) : "memory");
}

template <int NWC, int GT>
__global__ void __launch_bounds__(kMaxThreads<NWC>, NWC >= 3 ? 1 : 2)
local_search_multi_kernel(const LSJob *jobs, int njobs, int walks, int s_smem, unsigned stride)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int g = threadIdx.x / GT, gt = threadIdx.x % GT, lane = threadIdx.x & 31;
    if (g >= walks) return;
    const unsigned gm = Grp<GT>::W == 32 ? FULL : (((1u << Grp<GT>::W) - 1u) << (lane & ~(Grp<GT>::W - 1)));
    uint8_t *gb = smem + (size_t)stride * g;
    JobDesc *jd = reinterpret_cast<JobDesc *>(gb);
    uint8_t *sb = gb + align16(sizeof(JobDesc));
    for (int j = 0; j < njobs; ++j) {
        group_sync<GT>(g, gm);                 // the previous job's descriptor is no longer read
        if (gt == 0) {
            jd->I = jobs[j].I;
            jd->a = jobs[j].a;
            jd->a.s_smem = s_smem;
        }
        group_sync<GT>(g, gm);
        if (jd->a.skip && *jd->a.skip) continue;
        const DevInst &I = jd->I;
        walk_loop<NWC, GT, false>(I, jd->a, walks, make_ctx_at<NWC, GT>(I, s_smem != 0, I.rc, I.allow_row, I.linelen, sb));
    }
}

template <int NWC, int GT>
cudaError_t launch_t(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    local_search_kernel<NWC, GT><<<L.blocks, GT * L.walks, L.smem, st>>>(I, a, L.walks);
    return cudaGetLastError();
}

template <int NWC>
cudaError_t launch_g(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    switch (L.group) {
        case 16: return launch_t<NWC, 16>(I, a, L, st);
        case 32: return launch_t<NWC, 32>(I, a, L, st);
        case 64: return launch_t<NWC, 64>(I, a, L, st);
        case 128: return launch_t<NWC, 128>(I, a, L, st);
        default: return launch_t<NWC, 256>(I, a, L, st);
    }
}

// sets the block's shared-memory size; returns resident blocks per SM
template <int NWC, int GT>
int set_smem_t(size_t smem, int threads)
{
    cudaFuncSetAttribute(local_search_kernel<NWC, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_search_kernel<NWC, GT>, threads, smem) !=
        cudaSuccess)
        per_sm = 0;
    return per_sm;
}

template <int NWC>
int set_smem_g(int group, size_t smem, int threads)
{
    switch (group) {
        case 16: return set_smem_t<NWC, 16>(smem, threads);
        case 32: return set_smem_t<NWC, 32>(smem, threads);
        case 64: return set_smem_t<NWC, 64>(smem, threads);
        case 128: return set_smem_t<NWC, 128>(smem, threads);
        default: return set_smem_t<NWC, 256>(smem, threads);
    }
}

inline int max_threads_for(int cw)
{
    return cw == 1 ? kMaxThreads<1> : cw == 2 ? kMaxThreads<2> : cw == 3 ? kMaxThreads<3> : kMaxThreads<4>;
}

template <int NWC, int GT>
cudaError_t launch_multi_t(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st)
{
    local_search_multi_kernel<NWC, GT><<<L.blocks, GT * L.walks, L.smem, st>>>(jobs, njobs, L.walks, L.s_smem,
                                                                                (unsigned)L.stride);
    return cudaGetLastError();
}

template <int NWC>
cudaError_t launch_multi_g(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st)
{
    switch (L.group) {
        case 16: return launch_multi_t<NWC, 16>(jobs, njobs, L, st);
        case 32: return launch_multi_t<NWC, 32>(jobs, njobs, L, st);
        case 64: return launch_multi_t<NWC, 64>(jobs, njobs, L, st);
        case 128: return launch_multi_t<NWC, 128>(jobs, njobs, L, st);
        default: return launch_multi_t<NWC, 256>(jobs, njobs, L, st);
    }
}

template <int NWC, int GT>
int set_smem_multi_t(size_t smem, int threads)
{
    cudaFuncSetAttribute(local_search_multi_kernel<NWC, GT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_search_multi_kernel<NWC, GT>, threads, smem) !=
        cudaSuccess)
        per_sm = 0;
    return per_sm;
}

template <int NWC>
int set_smem_multi_g(int group, size_t smem, int threads)
{
    switch (group) {
        case 16: return set_smem_multi_t<NWC, 16>(smem, threads);
        case 32: return set_smem_multi_t<NWC, 32>(smem, threads);
        case 64: return set_smem_multi_t<NWC, 64>(smem, threads);
        case 128: return set_smem_multi_t<NWC, 128>(smem, threads);
        default: return set_smem_multi_t<NWC, 256>(smem, threads);
    }
}

}  // namespace

// The launch entry points of one colour-word class (explicitly instantiated,
// one class per translation unit, so that the classes compile in parallel).
template <int NWC>
cudaError_t LSKernels<NWC>::launch(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    return launch_g<NWC>(I, a, L, st);
}

template <int NWC>
int LSKernels<NWC>::set_smem(int group, size_t smem, int threads)
{
    return set_smem_g<NWC>(group, smem, threads);
}

template <int NWC>
cudaError_t LSKernels<NWC>::launch_multi(const LSJob *jobs, int njobs, const LSLaunch &L, cudaStream_t st)
{
    return launch_multi_g<NWC>(jobs, njobs, L, st);
}

template <int NWC>
int LSKernels<NWC>::set_smem_multi(int group, size_t smem, int threads)
{
    return set_smem_multi_g<NWC>(group, smem, threads);
}

}  // namespace plse
