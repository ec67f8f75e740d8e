// k_local_search.cu -- population initialisation (Sec. 3.2) and the tabu local
// search of MPMA (Alg. 3: PLITS phases 1 and 2, Sec. 3.3; PartialCol and the
// greedy conflict removal, Sec. 3.7) for sm_103a.
//
// Design (GB300-first):
//  * One warp per walk, one walk slot per 32-thread block, walks handed out by
//    an atomic counter.  Every byte a walk touches per iteration lives in that
//    block's shared memory.
//  * The gamma table of the incremental evaluation (Sec. 3.3) is held in
//    factored form.  On a Latin-square graph the neighbours of v = (r, c) are
//    exactly its row- and column-mates, so
//        gamma[v][k] = R[r][k] + K[c][k] - 2*[S(v) = k],
//    with R / K the per-row / per-column colour counts (uint8, n x (n+1) each).
//    A move then updates four counters instead of deg(v) table entries, and
//    the table shrinks from |V| x (n+1) to 2 n (n+1) bytes.
//  * The tabu list (expiry per (v, colour)) is a 2-entry per-vertex cache in
//    shared memory (16-bit clocks relative to the phase) backed by an exact
//    global overflow table G for entries evicted while possibly live.  A vertex
//    whose evicted entries have all expired never touches G.
//  * A candidate list V0 u C(S) is kept as a shared bitmask, updated after each
//    move from the row and column of the moved vertex only, and compacted once
//    per iteration so lanes get equal numbers of candidates.  The best move is
//    the minimum of the key (2dF, (v - r) mod |V|, j) over lanes: a total order,
//    so the result does not depend on the scan order.
#include <climits>

#include "plse_internal.cuh"

namespace plse {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint32_t kRebaseAt = 49152;   // relative clock rebased before it reaches this
constexpr uint32_t kRebaseBy = 32768;
constexpr uint32_t kNoKey = 0xffffffffu;

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

struct WalkSmem {
    uint8_t *S;       // current colouring [nv]
    uint8_t *B;       // best colouring of the running phase [nv]
    uint8_t *R, *K;   // colour counts per row / per column, [n][n1p] each (contiguous)
    uint32_t *cmask;  // candidate bitmask [nw]
    uint16_t *clist;  // compacted candidates [nv]
    uint2 *tc;        // tabu cache [nv]: x = e0 | e1 << 16, y = c0 | c1 << 8 | emax << 16
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline SmemPlan make_plan(const DevInst &I)
{
    SmemPlan p;
    p.off_S = 0;
    const size_t nvp = align16((size_t)I.nv);
    p.off_R = 2 * nvp;                          // S and B
    p.off_K = p.off_R + (size_t)I.n * I.n1p;
    p.off_cmask = align16(p.off_K + (size_t)I.n * I.n1p);
    p.off_clist = align16(p.off_cmask + 4 * (size_t)I.nw);
    p.off_tc = align16(p.off_clist + 2 * (size_t)I.nv);
    p.total = align16(p.off_tc + 8 * (size_t)I.nv);
    return p;
}

__device__ __forceinline__ WalkSmem carve(uint8_t *base, const DevInst &I)
{
    const SmemPlan p = make_plan(I);
    WalkSmem w;
    w.S = base + p.off_S;
    w.B = base + align16((size_t)I.nv);
    w.R = base + p.off_R;
    w.K = base + p.off_K;
    w.cmask = reinterpret_cast<uint32_t *>(base + p.off_cmask);
    w.clist = reinterpret_cast<uint16_t *>(base + p.off_clist);
    w.tc = reinterpret_cast<uint2 *>(base + p.off_tc);
    return w;
}

// Per-lane work counters; uniform fields are counted on every lane and taken
// from lane 0, per-lane sums are reduced at the end of the walk.
struct LaneStats {
    long long iterations, moves, cand, pairs, deg, improvements, uncolored;
};

__device__ __forceinline__ long long warp_sum64(long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// ---- colour counts, candidate set, conflicts -------------------------------
__device__ void build_counts(const DevInst &I, const WalkSmem &w, int lane)
{
    const int words = (2 * I.n * I.n1p) >> 2;
    uint32_t *RK = reinterpret_cast<uint32_t *>(w.R);
    for (int q = lane; q < words; q += 32) RK[q] = 0u;
    __syncwarp();
    for (int r = lane; r < I.n; r += 32) {
        uint8_t *Rr = w.R + r * I.n1p;
        for (int q = __ldg(&I.row_ptr[r]); q < __ldg(&I.row_ptr[r + 1]); ++q) {
            const int k = w.S[__ldg(&I.row_v[q])];
            if (k) Rr[k] += 1;
        }
        uint8_t *Kc = w.K + r * I.n1p;
        for (int q = __ldg(&I.col_ptr[r]); q < __ldg(&I.col_ptr[r + 1]); ++q) {
            const int k = w.S[__ldg(&I.col_v[q])];
            if (k) Kc[k] += 1;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ int gamma_own(const DevInst &I, const WalkSmem &w, int v, int k)
{
    const uint16_t rc = __ldg(&I.rc[v]);
    return w.R[(rc >> 8) * I.n1p + k] + w.K[(rc & 255) * I.n1p + k] - 2;
}

// candidate bitmask: PLITS -> V0 u C(S); PartialCol -> V0.  Returns f and |C|.
__device__ void build_cands(const DevInst &I, const WalkSmem &w, int lane, bool only_v0,
                            int &f, int &nconf)
{
    int lf = 0, lc = 0;
    for (int wd = lane; wd < I.nw; wd += 32) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int v = wd * 32 + b;
            if (v >= I.nv) break;
            const int k = w.S[v];
            if (k == 0) {
                bits |= 1u << b;
                ++lf;
            } else if (gamma_own(I, w, v, k) > 0) {
                ++lc;
                if (!only_v0) bits |= 1u << b;
            }
        }
        w.cmask[wd] = bits;
    }
    f = __reduce_add_sync(FULL, lf);
    nconf = __reduce_add_sync(FULL, lc);
    __syncwarp();
}

// conflicting edges c(S) = sum over rows and columns of C(count, 2)
__device__ int conflict_edges(const DevInst &I, const WalkSmem &w, int lane)
{
    int s = 0;
    const int bytes = 2 * I.n * I.n1p;
    for (int q = lane; q < bytes; q += 32) {
        const int x = w.R[q];
        s += x * (x - 1) / 2;
    }
    return __reduce_add_sync(FULL, s);
}

__device__ __forceinline__ void copy_bytes(uint8_t *dst, const uint8_t *src, int n, int lane)
{
    for (int q = lane; q < n; q += 32) dst[q] = src[q];
    __syncwarp();
}

__device__ __forceinline__ int count_zero(const uint8_t *S, int nv, int lane)
{
    int z = 0;
    for (int q = lane; q < nv; q += 32) z += (S[q] == 0);
    return __reduce_add_sync(FULL, z);
}

// compacts the candidate bitmask into clist; returns the candidate count
__device__ int compact(const DevInst &I, const WalkSmem &w, int lane)
{
    int cnt = 0;
    for (int wd = lane; wd < I.nw; wd += 32) cnt += __popc(w.cmask[wd]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    int pos = incl - cnt;
    const int total = __shfl_sync(FULL, incl, 31);
    for (int wd = lane; wd < I.nw; wd += 32) {
        uint32_t bits = w.cmask[wd];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            w.clist[pos++] = (uint16_t)(wd * 32 + b);
        }
    }
    __syncwarp();
    return total;
}

// ---- tabu cache -------------------------------------------------------------
struct Clock {
    uint32_t base;    // absolute clock of iteration 0 of the phase
    uint32_t shift;   // relative clock = t - shift
};

__device__ __forceinline__ void tabu_reset(const DevInst &I, const WalkSmem &w, int lane)
{
    for (int v = lane; v < I.nv; v += 32) w.tc[v] = make_uint2(0u, 0xFFFFu);
    __syncwarp();
}

__device__ void tabu_rebase(const DevInst &I, const WalkSmem &w, int lane)
{
    for (int v = lane; v < I.nv; v += 32) {
        const uint2 x = w.tc[v];
        uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16, em = x.y >> 16;
        e0 = e0 > kRebaseBy ? e0 - kRebaseBy : 0u;
        e1 = e1 > kRebaseBy ? e1 - kRebaseBy : 0u;
        em = em > kRebaseBy ? em - kRebaseBy : 0u;
        w.tc[v] = make_uint2(e0 | (e1 << 16), (x.y & 0xFFFFu) | (em << 16));
    }
    __syncwarp();
}

// (v, c) tabu until relative clock e (inclusive); evicts to G when needed.
__device__ __forceinline__ void tabu_insert(const DevInst &I, const WalkSmem &w, uint32_t *G,
                                            const Clock &ck, int v, int c, uint32_t e)
{
    const uint2 x = w.tc[v];
    uint32_t e0 = x.x & 0xFFFFu, e1 = x.x >> 16;
    uint32_t c0 = x.y & 0xFFu, c1 = (x.y >> 8) & 0xFFu, em = x.y >> 16;
    if (c0 == (uint32_t)c) {
        e0 = e;
    } else if (c1 == (uint32_t)c) {
        e1 = e;
    } else {
        const bool second = e1 < e0;                     // evict the earlier expiry
        const uint32_t ev = second ? e1 : e0, cv = second ? c1 : c0;
        if (cv != 0xFFu) {
            G[(size_t)v * I.n1p + cv] = ck.base + ck.shift + ev;
            em = max(em, ev);
        }
        if (second) { c1 = (uint32_t)c; e1 = e; } else { c0 = (uint32_t)c; e0 = e; }
    }
    w.tc[v] = make_uint2(e0 | (e1 << 16), c0 | (c1 << 8) | (em << 16));
}

template <int NWC>
__device__ __forceinline__ void clear_bit(uint32_t (&m)[4], uint32_t c)
{
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (q == (int)(c >> 5)) m[q] &= ~(1u << (c & 31));
}

template <int NWC>
__device__ __forceinline__ bool test_bit(const uint32_t (&m)[4], uint32_t c)
{
    bool r = false;
#pragma unroll
    for (int q = 0; q < NWC; ++q)
        if (q == (int)(c >> 5)) r = (m[q] >> (c & 31)) & 1u;
    return r;
}

// Best admissible move of candidate v as key 2dF*256 + j (INT_MAX: none).
//   v uncoloured:  2dF(j) = base_unc + mult*s_j       (j != 0)
//   v coloured i:  2dF(j) = mult*(s_j - g_i)           (j != 0, j != i)
//                  2dF(0) = 2 - mult*g_i
// with s_j = R[r][j] + K[c][j] and g_i = gamma[v][i] (Sec. 3.3).  A move is
// admissible if not tabu, or if 2dF < A (aspiration by the phase's best).
template <int NWC>
__device__ __forceinline__ int eval_vertex(const DevInst &I, const WalkSmem &w, const uint32_t *G,
                                           const Clock &ck, uint32_t trel, int v, int mult,
                                           int base_unc, int A)
{
    const int i = w.S[v];
    const uint16_t rc = __ldg(&I.rc[v]);
    const uint8_t *Rr = w.R + (rc >> 8) * I.n1p;
    const uint8_t *Kc = w.K + (rc & 255) * I.n1p;
    const int gi = i ? (int)Rr[i] + (int)Kc[i] - 2 : 0;
    const int base2 = i ? -mult * gi : base_unc;
    const uint4 d = __ldg(&I.dom[v]);
    uint32_t m[4] = {d.x, d.y, d.z, d.w};
    clear_bit<NWC>(m, (uint32_t)i);
    bool has0 = (i != 0) && (m[0] & 1u);
    m[0] &= ~1u;
    const int d2zero = 2 - mult * gi;

    const uint2 te = w.tc[v];
    const uint32_t e0 = te.x & 0xFFFFu, e1 = te.x >> 16;
    const uint32_t c0 = te.y & 0xFFu, c1 = (te.y >> 8) & 0xFFu, em = te.y >> 16;
    int best = INT_MAX;
    if (em < trel) {
        // fast path: only the cached colours c0, c1 can be tabu
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const uint32_t cs = s ? c1 : c0, es = s ? e1 : e0;
            if (cs == 0u) {
                if (has0) {
                    has0 = false;
                    if (es < trel || d2zero < A) best = min(best, d2zero * kKeyScale);
                }
            } else if (cs < 128u && test_bit<NWC>(m, cs)) {
                clear_bit<NWC>(m, cs);
                const int d2 = base2 + mult * ((int)Rr[cs] + (int)Kc[cs]);
                if (es < trel || d2 < A) best = min(best, d2 * kKeyScale + (int)cs);
            }
        }
        if (has0) best = min(best, d2zero * kKeyScale);
        const int kb = base2 * kKeyScale, km = mult * kKeyScale;
#pragma unroll
        for (int q = 0; q < NWC; ++q) {
            uint32_t bits = m[q];
            while (bits) {
                const int j = q * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                best = min(best, kb + j + km * ((int)Rr[j] + (int)Kc[j]));
            }
        }
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
                const int d2 = base2 + mult * ((int)Rr[j] + (int)Kc[j]);
                const bool tabu = (j == c0) ? (e0 >= trel) : (j == c1) ? (e1 >= trel) : (Gv[j] >= tabs);
                if (!tabu || d2 < A) best = min(best, d2 * kKeyScale + (int)j);
            }
        }
    }
    return best;
}

__device__ __forceinline__ int vertex_degree(const DevInst &I, int v)
{
    const uint16_t rc = __ldg(&I.rc[v]);
    const int r = rc >> 8, c = rc & 255;
    return (__ldg(&I.row_ptr[r + 1]) - __ldg(&I.row_ptr[r]) - 1) +
           (__ldg(&I.col_ptr[c + 1]) - __ldg(&I.col_ptr[c]) - 1);
}

// reserve a clock range for one phase of this slot
__device__ Clock claim_clock(const DevInst &I, const LSArgs &a, uint32_t *G, int slot, int span, int lane)
{
    uint32_t base = 0;
    if (lane == 0) {
        base = a.slot_clock[slot] + 1u;
        if (base > 0x7FFFFFFFu - (uint32_t)span) base = 0u;   // wrap: clear the slot
    }
    base = __shfl_sync(FULL, base, 0);
    if (base == 0u) {
        const size_t words = (size_t)I.nv * I.n1p;
        for (size_t q = lane; q < words; q += 32) G[q] = 0u;
        base = 1u;
        __syncwarp();
    }
    if (lane == 0) a.slot_clock[slot] = base + (uint32_t)span;
    Clock ck;
    ck.base = base;
    ck.shift = 0u;
    return ck;
}

__device__ __forceinline__ void warp_best(uint32_t khi, uint32_t klo, uint32_t &mhi, uint32_t &mlo)
{
    mhi = __reduce_min_sync(FULL, khi);
    mlo = __reduce_min_sync(FULL, khi == mhi ? klo : kNoKey);
}

// ---- PLITS phase (Alg. 3 with phi2 = 2*phi) --------------------------------
template <int NWC>
__device__ bool plits_phase(const DevInst &I, const LSArgs &a, const WalkSmem &w, uint32_t *G,
                            int slot, int ind, int phase, int64_t N, int phi2, int span,
                            LaneStats &st, long long &F2best_out, int lane)
{
    build_counts(I, w, lane);
    int f, nconf;
    build_cands(I, w, lane, false, f, nconf);
    int cedges = conflict_edges(I, w, lane);
    long long F2 = 2LL * f + (long long)phi2 * cedges;
    long long F2best = F2;
    copy_bytes(w.B, w.S, I.nv, lane);
    tabu_reset(I, w, lane);
    Clock ck = claim_clock(I, a, G, slot, span, lane);

    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | (uint32_t)phase;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    for (long long t = 1; t <= N; ++t) {
        if (f + nconf == 0) break;                       // nothing left to improve
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            tabu_rebase(I, w, lane);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
        }
        const int q = (int)((t - 1) & 31);
        if (q == 0) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)(t + lane), (uint32_t)ind, ctr2, 0u), a.key0, a.key1);
            Lr = bounded(u.x, (uint32_t)a.tenure_rand);
            rotr = bounded(u.y, (uint32_t)I.nv);
        }
        const int L = (int)__shfl_sync(FULL, Lr, q);
        const int rsh = (int)__shfl_sync(FULL, rotr, q);
        long long A64 = F2best - F2;
        const int A = A64 < -(1LL << 30) ? -(1 << 30) : (int)A64;

        const int ncand = compact(I, w, lane);
        if (ncand != f + nconf) { ok = false; break; }
        uint32_t khi = kNoKey, klo = kNoKey;
        for (int qq = lane; qq < ncand; qq += 32) {
            const int v = w.clist[qq];
            st.pairs += __ldg(&I.ndom[v]) - 1;
            const int kv = eval_vertex<NWC>(I, w, G, ck, trel, v, phi2, -2, A);
            if (kv != INT_MAX) {
                int rot = v - rsh;
                if (rot < 0) rot += I.nv;
                const uint32_t hi = (uint32_t)((kv >> 8) + (1 << 30));
                const uint32_t lo = ((uint32_t)rot << 8) | (uint32_t)(kv & 255);
                if (hi < khi || (hi == khi && lo < klo)) { khi = hi; klo = lo; }
            }
        }
        st.iterations += 1;
        if (lane == 0) st.cand += ncand;
        uint32_t mhi, mlo;
        warp_best(khi, klo, mhi, mlo);
        if (mhi == kNoKey) continue;                     // every move tabu

        const int d2 = (int)mhi - (1 << 30);
        const int j = (int)(mlo & 255u);
        int v = (int)(mlo >> 8) + rsh;
        if (v >= I.nv) v -= I.nv;
        const int i = w.S[v];
        const uint16_t rc = __ldg(&I.rc[v]);
        const int r = rc >> 8, cc = rc & 255;
        uint8_t *Rr = w.R + r * I.n1p;
        uint8_t *Kc = w.K + cc * I.n1p;
        const int sj = j ? (int)Rr[j] + (int)Kc[j] : 0;
        const int gi = i ? (int)Rr[i] + (int)Kc[i] - 2 : 0;
        __syncwarp();
        if (lane == 0) {
            w.S[v] = (uint8_t)j;
            if (i) { Rr[i] -= 1; Kc[i] -= 1; }
            if (j) { Rr[j] += 1; Kc[j] += 1; }
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
                const int su = w.S[u];
                if (su == 0 || (su != i && su != j)) continue;
                const int nc = gamma_own(I, w, u, su) > 0;
                const int oc = (w.cmask[u >> 5] >> (u & 31)) & 1;
                if (nc != oc) {
                    atomicXor(&w.cmask[u >> 5], 1u << (u & 31));
                    dconf += nc - oc;
                }
            }
        }
        if (lane == 0) {
            const int newc = j ? (int)((int)Rr[j] + (int)Kc[j] - 2 > 0) : 0;
            if (j != 0 && !newc) atomicAnd(&w.cmask[v >> 5], ~(1u << (v & 31)));
            dconf += newc - (i != 0 ? 1 : 0);
        }
        dconf = __reduce_add_sync(FULL, dconf);
        f += (j == 0) - (i == 0);
        nconf += dconf;
        cedges += sj - gi;
        F2 += d2;
        const int k = f + nconf;
        const int T = L + (a.alpha_num * k) / a.alpha_den;
        if (lane == 0) tabu_insert(I, w, G, ck, v, i, trel + (uint32_t)T);
        st.moves += 1;
        st.deg += vertex_degree(I, v);
        if (F2 < F2best) {
            F2best = F2;
            st.improvements += 1;
            __syncwarp();
            for (int qq = lane; qq < I.nv; qq += 32) w.B[qq] = w.S[qq];
        }
        __syncwarp();
    }
    copy_bytes(w.S, w.B, I.nv, lane);
    F2best_out = F2best;
    return ok;
}

// ---- greedy conflict removal (Sec. 3.7) ------------------------------------
__device__ void repair(const DevInst &I, const WalkSmem &w, int lane)
{
    build_counts(I, w, lane);
    for (int step = 0; step < I.nv; ++step) {
        uint32_t key = 0;
        for (int v = lane; v < I.nv; v += 32) {
            const int k = w.S[v];
            if (!k) continue;
            const int g = gamma_own(I, w, v, k);
            if (g > 0) key = max(key, ((uint32_t)g << 16) | (0xFFFFu - (uint32_t)v));
        }
        const uint32_t m = __reduce_max_sync(FULL, key);
        if (m == 0u) break;
        const int v = (int)(0xFFFFu - (m & 0xFFFFu));
        if (lane == 0) {
            const int k = w.S[v];
            const uint16_t rc = __ldg(&I.rc[v]);
            w.S[v] = 0;
            w.R[(rc >> 8) * I.n1p + k] -= 1;
            w.K[(rc & 255) * I.n1p + k] -= 1;
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void byte_dec(uint8_t *p)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    atomicSub(reinterpret_cast<unsigned int *>(a & ~uintptr_t(3)), 1u << (8 * (a & 3)));
}

// ---- PartialCol (Sec. 3.7): legal partial colourings only ------------------
template <int NWC>
__device__ bool partialcol_phase(const DevInst &I, const LSArgs &a, const WalkSmem &w, uint32_t *G,
                                 int slot, int ind, int64_t N, int span, LaneStats &st,
                                 long long &fbest_out, int lane)
{
    build_counts(I, w, lane);
    int f, nconf;
    build_cands(I, w, lane, true, f, nconf);
    if (conflict_edges(I, w, lane) != 0) return false;   // needs a legal start
    int fbest = f;
    copy_bytes(w.B, w.S, I.nv, lane);
    tabu_reset(I, w, lane);
    Clock ck = claim_clock(I, a, G, slot, span, lane);
    const uint32_t ctr2 = ((uint32_t)a.gen << 8) | (kPurposeTabu << 4) | 3u;
    uint32_t Lr = 0, rotr = 0;
    bool ok = true;
    for (long long t = 1; t <= N; ++t) {
        if (f == 0) break;
        uint32_t trel = (uint32_t)(t - ck.shift);
        if (trel >= kRebaseAt) {
            tabu_rebase(I, w, lane);
            ck.shift += kRebaseBy;
            trel -= kRebaseBy;
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
        const int ncand = compact(I, w, lane);
        if (ncand != f) { ok = false; break; }
        uint32_t khi = kNoKey, klo = kNoKey;
        for (int qq = lane; qq < ncand; qq += 32) {
            const int v = w.clist[qq];
            st.pairs += __ldg(&I.ndom[v]) - 1;
            const int kv = eval_vertex<NWC>(I, w, G, ck, trel, v, 1, -1, A);
            if (kv != INT_MAX) {
                int rot = v - rsh;
                if (rot < 0) rot += I.nv;
                const uint32_t hi = (uint32_t)((kv >> 8) + (1 << 30));
                const uint32_t lo = ((uint32_t)rot << 8) | (uint32_t)(kv & 255);
                if (hi < khi || (hi == khi && lo < klo)) { khi = hi; klo = lo; }
            }
        }
        st.iterations += 1;
        if (lane == 0) st.cand += ncand;
        uint32_t mhi, mlo;
        warp_best(khi, klo, mhi, mlo);
        if (mhi == kNoKey) continue;

        const int d = (int)mhi - (1 << 30);
        const int j = (int)(mlo & 255u);
        int v = (int)(mlo >> 8) + rsh;
        if (v >= I.nv) v -= I.nv;
        const uint16_t rc = __ldg(&I.rc[v]);
        const int r = rc >> 8, cc = rc & 255;
        const int T = L + (a.alpha_num * (f + d)) / a.alpha_den;
        __syncwarp();
        // uncolour the row- and column-mates of colour j
        int nunc = 0;
        for (int side = 0; side < 2; ++side) {
            const int32_t *ptr = side ? I.col_ptr : I.row_ptr;
            const uint16_t *lst = side ? I.col_v : I.row_v;
            const int line = side ? cc : r;
            const int qb = __ldg(&ptr[line]), qe = __ldg(&ptr[line + 1]);
            for (int qq = qb + lane; qq < qe; qq += 32) {
                const int u = __ldg(&lst[qq]);
                if (u == v || w.S[u] != j) continue;
                const uint16_t rcu = __ldg(&I.rc[u]);
                w.S[u] = 0;
                byte_dec(w.R + (rcu >> 8) * I.n1p + j);
                byte_dec(w.K + (rcu & 255) * I.n1p + j);
                atomicOr(&w.cmask[u >> 5], 1u << (u & 31));
                tabu_insert(I, w, G, ck, u, j, trel + (uint32_t)T);
                ++nunc;
            }
        }
        __syncwarp();
        nunc = __reduce_add_sync(FULL, nunc);
        if (lane == 0) {
            w.S[v] = (uint8_t)j;
            w.R[r * I.n1p + j] += 1;
            w.K[cc * I.n1p + j] += 1;
            atomicAnd(&w.cmask[v >> 5], ~(1u << (v & 31)));
        }
        if (nunc - 1 != d) { ok = false; break; }
        f += d;
        st.moves += 1;
        st.deg += vertex_degree(I, v);
        if (lane == 0) st.uncolored += nunc;
        __syncwarp();
        if (f < fbest) {
            fbest = f;
            st.improvements += 1;
            for (int qq = lane; qq < I.nv; qq += 32) w.B[qq] = w.S[qq];
        }
        __syncwarp();
    }
    copy_bytes(w.S, w.B, I.nv, lane);
    fbest_out = fbest;
    return ok;
}

template <int NWC>
__global__ void __launch_bounds__(32) local_search_kernel(const DevInst I, const LSArgs a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x;
    const int slot = blockIdx.x;
    const WalkSmem w = carve(smem, I);
    uint32_t *G = a.G + (size_t)slot * I.nv * I.n1p;

    for (;;) {
        int wk = 0;
        if (lane == 0) wk = atomicAdd(a.work_counter, 1);
        wk = __shfl_sync(FULL, wk, 0);
        if (wk >= a.count) break;
        const int ind = a.ind0 + wk;
        const uint8_t *gin = a.S_in + (size_t)wk * I.nv;
        uint8_t *gout = a.S_out + (size_t)wk * I.nv;
        copy_bytes(w.S, gin, I.nv, lane);

        LaneStats st = {0, 0, 0, 0, 0, 0, 0};
        long long Flast = 0;
        bool ok = true;
        if (a.flags & PLSE_LS_PARTIALCOL) {
            if (a.flags & PLSE_LS_REPAIR) repair(I, w, lane);
            ok = partialcol_phase<NWC>(I, a, w, G, slot, ind, a.iters1, a.span1, st, Flast, lane);
        } else {
            if (a.flags & PLSE_LS_PHASE1)
                ok = plits_phase<NWC>(I, a, w, G, slot, ind, 1, a.iters1, a.phi2_1, a.span1, st, Flast, lane);
            if (ok && (a.flags & PLSE_LS_PHASE2))
                ok = plits_phase<NWC>(I, a, w, G, slot, ind, 2, a.iters2, a.phi2_2, a.span2, st, Flast, lane);
            if (ok && (a.flags & PLSE_LS_REPAIR)) repair(I, w, lane);
        }
        if (!ok && lane == 0) atomicOr(a.error_flag, 1);
        __syncwarp();
        for (int q = lane; q < I.nv; q += 32) gout[q] = w.S[q];
        const int fz = count_zero(w.S, I.nv, lane);
        const long long pairs = warp_sum64(st.pairs);
        if (lane == 0) {
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
        __syncwarp();
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
            const uint32_t c = __popc(m[wq]);
            if (k < c) {
                uint32_t x = m[wq];
                for (uint32_t s = 0; s < k; ++s) x &= x - 1;
                colour = wq * 32 + __ffs(x) - 1;
            } else {
                k -= c;
            }
        }
        P[(size_t)i * I.nv + v] = (uint8_t)colour;
    }
}

template <int NWC>
cudaError_t launch_ls_t(const DevInst &I, const LSArgs &a, const LSLaunch &L, cudaStream_t st)
{
    local_search_kernel<NWC><<<L.blocks, 32, L.smem, st>>>(I, a);
    return cudaGetLastError();
}

template <int NWC>
int occupancy_t(size_t smem)
{
    cudaFuncSetAttribute(local_search_kernel<NWC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, local_search_kernel<NWC>, 32, smem) != cudaSuccess)
        per_sm = 0;
    return per_sm;
}

}  // namespace

SmemPlan smem_plan(const DevInst &I) { return make_plan(I); }

LSLaunch plan_local_search(const DevInst &I, int device, int count)
{
    LSLaunch L;
    L.smem = make_plan(I).total;
    L.colour_words = I.n < 32 ? 1 : I.n < 64 ? 2 : I.n < 96 ? 3 : 4;
    int per_sm = 0;
    switch (L.colour_words) {
        case 1: per_sm = occupancy_t<1>(L.smem); break;
        case 2: per_sm = occupancy_t<2>(L.smem); break;
        case 3: per_sm = occupancy_t<3>(L.smem); break;
        default: per_sm = occupancy_t<4>(L.smem); break;
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
        case 1: return launch_ls_t<1>(I, a, L, st);
        case 2: return launch_ls_t<2>(I, a, L, st);
        case 3: return launch_ls_t<3>(I, a, L, st);
        default: return launch_ls_t<4>(I, a, L, st);
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
