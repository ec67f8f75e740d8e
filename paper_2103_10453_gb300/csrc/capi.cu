// capi.cu -- the extern "C" boundary of libplse.so (declared in include/plse.h):
// instance construction (Sec. 2.1-2.2, Alg. 1), parameters, device workspace
// and the step entry points.  The whole-solve driver lives in solve.cu.
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>

#include "plse_handle.cuh"

using namespace plse;

namespace plse {

int fail(plse_instance *h, int code, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

int cuda_fail(plse_instance *h, cudaError_t e, const char *where)
{
    return fail(h, PLSE_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// 128-bit colour set helpers (bit k = colour k)
struct Mask128 {
    uint64_t lo = 0, hi = 0;
    void set(int k) { if (k < 64) lo |= 1ull << k; else hi |= 1ull << (k - 64); }
    bool has(int k) const { return k < 64 ? (lo >> k) & 1 : (hi >> (k - 64)) & 1; }
};

int build_instance(plse_instance *h, int n, const int8_t *grid)
{
    h->n = n;
    h->grid.assign(grid, grid + (size_t)n * n);
    std::vector<Mask128> rowm(n), colm(n);
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            const int k = grid[r * n + c];
            if (k < 0 || k > n) return fail(h, PLSE_EINVAL, "cell (%d,%d) holds %d, outside 0..%d", r, c, k, n);
            if (!k) continue;
            if (rowm[r].has(k)) return fail(h, PLSE_EINVAL, "symbol %d twice in row %d", k, r);
            if (colm[c].has(k)) return fail(h, PLSE_EINVAL, "symbol %d twice in column %d", k, c);
            rowm[r].set(k);
            colm[c].set(k);
        }
    // colours still allowed by each row and each column
    h->allow_row.assign(n, make_uint4(0, 0, 0, 0));
    h->allow_col.assign(n, make_uint4(0, 0, 0, 0));
    for (int r = 0; r < n; ++r)
        for (int k = 1; k <= n; ++k) {
            uint32_t *ar = &h->allow_row[r].x, *ac = &h->allow_col[r].x;
            if (!rowm[r].has(k)) ar[k >> 5] |= 1u << (k & 31);
            if (!colm[r].has(k)) ac[k >> 5] |= 1u << (k & 31);
        }
    // D(v) = {0} u ({1..n} minus the row's and column's symbols); empty cells
    // with D(v) = {0} are removed and counted in l (Alg. 1).
    h->cell.clear();
    h->rc.clear();
    h->dom.clear();
    h->ndom.clear();
    h->l = 0;
    h->nfixed = 0;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            if (grid[r * n + c]) { ++h->nfixed; continue; }
            uint32_t m[4] = {1u, 0u, 0u, 0u};
            int cnt = 0;
            for (int k = 1; k <= n; ++k)
                if (!rowm[r].has(k) && !colm[c].has(k)) {
                    m[k >> 5] |= 1u << (k & 31);
                    ++cnt;
                }
            if (cnt == 0) { ++h->l; continue; }
            h->cell.push_back(r * n + c);
            h->rc.push_back((uint16_t)((r << 8) | c));
            h->dom.push_back(make_uint4(m[0], m[1], m[2], m[3]));
            h->ndom.push_back((uint8_t)(cnt + 1));
        }
    h->nv = (int)h->cell.size();
    h->ub = (h->l == 1) ? n * n - 2 : n * n - h->l;
    // row and column member lists
    h->row_ptr.assign(n + 1, 0);
    h->col_ptr.assign(n + 1, 0);
    for (int v = 0; v < h->nv; ++v) {
        h->row_ptr[(h->rc[v] >> 8) + 1]++;
        h->col_ptr[(h->rc[v] & 255) + 1]++;
    }
    for (int r = 0; r < n; ++r) {
        h->row_ptr[r + 1] += h->row_ptr[r];
        h->col_ptr[r + 1] += h->col_ptr[r];
    }
    h->row_v.assign(h->nv, 0);
    h->col_v.assign(h->nv, 0);
    std::vector<int32_t> rfill(h->row_ptr.begin(), h->row_ptr.end() - 1), cfill(h->col_ptr.begin(), h->col_ptr.end() - 1);
    for (int v = 0; v < h->nv; ++v) {
        h->row_v[rfill[h->rc[v] >> 8]++] = (uint16_t)v;
        h->col_v[cfill[h->rc[v] & 255]++] = (uint16_t)v;
    }
    return PLSE_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

int upload_instance(plse_instance *h)
{
    const int nv = h->nv, n = h->n;
    size_t off = 0;
    const size_t o_rc = off; off = up256(off + 2 * (size_t)nv + 2);
    const size_t o_dom = off; off = up256(off + 16 * (size_t)nv + 16);
    const size_t o_nd = off; off = up256(off + (size_t)nv + 1);
    const size_t o_rp = off; off = up256(off + 4 * (size_t)(n + 1));
    const size_t o_rv = off; off = up256(off + 2 * (size_t)nv + 2);
    const size_t o_cp = off; off = up256(off + 4 * (size_t)(n + 1));
    const size_t o_cv = off; off = up256(off + 2 * (size_t)nv + 2);
    const size_t o_ar = off; off = off + 16 * (size_t)n;          // columns right after rows
    const size_t o_ac = off; off = up256(off + 16 * (size_t)n);
    const size_t o_ll = off; off = up256(off + 2 * (size_t)n);
    cudaError_t e = dev_malloc(&h->inst_mem, off, cudaStreamLegacy);
    if (e != cudaSuccess) return fail(h, PLSE_ENOMEM, "instance upload: %s", cudaGetErrorString(e));
    h->inst_bytes = off;
    std::vector<uint8_t> img(off, 0);
    if (nv) {
        memcpy(img.data() + o_rc, h->rc.data(), 2 * (size_t)nv);
        memcpy(img.data() + o_dom, h->dom.data(), 16 * (size_t)nv);
        memcpy(img.data() + o_nd, h->ndom.data(), (size_t)nv);
        memcpy(img.data() + o_rv, h->row_v.data(), 2 * (size_t)nv);
        memcpy(img.data() + o_cv, h->col_v.data(), 2 * (size_t)nv);
    }
    memcpy(img.data() + o_ar, h->allow_row.data(), 16 * (size_t)n);
    memcpy(img.data() + o_ac, h->allow_col.data(), 16 * (size_t)n);
    memcpy(img.data() + o_rp, h->row_ptr.data(), 4 * (size_t)(n + 1));
    memcpy(img.data() + o_cp, h->col_ptr.data(), 4 * (size_t)(n + 1));
    for (int l = 0; l < 2 * n; ++l)      // reduced vertices per row, then per column
        img[o_ll + l] = (uint8_t)(l < n ? h->row_ptr[l + 1] - h->row_ptr[l] : h->col_ptr[l - n + 1] - h->col_ptr[l - n]);
    // A pageable host-to-device copy may return before its DMA has landed, and
    // the legacy stream orders it (and the allocation) for blocking streams only:
    // wait for both, so that kernels on any stream see the whole image.
    e = cudaMemcpyAsync(h->inst_mem, img.data(), off, cudaMemcpyHostToDevice, cudaStreamLegacy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
    if (e != cudaSuccess) return cuda_fail(h, e, "instance upload");
    uint8_t *b = static_cast<uint8_t *>(h->inst_mem);
    DevInst &I = h->di;
    I.n = n;
    I.n1p = (n + 1 + 3) & ~3;
    I.nv = nv;
    I.nw = (nv + 31) / 32;
    int nb = 1;
    while ((1 << nb) <= n) ++nb;
    I.nb = nb;
    I.rc = reinterpret_cast<const uint16_t *>(b + o_rc);
    I.dom = reinterpret_cast<const uint4 *>(b + o_dom);
    I.ndom = b + o_nd;
    I.row_ptr = reinterpret_cast<const int32_t *>(b + o_rp);
    I.row_v = reinterpret_cast<const uint16_t *>(b + o_rv);
    I.col_ptr = reinterpret_cast<const int32_t *>(b + o_cp);
    I.col_v = reinterpret_cast<const uint16_t *>(b + o_cv);
    I.allow_row = reinterpret_cast<const uint4 *>(b + o_ar);
    I.allow_col = reinterpret_cast<const uint4 *>(b + o_ac);
    I.linelen = b + o_ll;
    return PLSE_OK;
}

int check_params(plse_instance *h, const plse_params &p)
{
    if (p.alpha_num < 0 || p.alpha_den < 1 || p.tenure_rand < 1 || p.phase1_phi2 < 1 ||
        p.phase2_phi2_per_v < 1 || p.phase2_iter_per_v < 0 || p.spacing_gamma < 1 || p.beta < 1 ||
        (p.mode != PLSE_MODE_PLITS && p.mode != PLSE_MODE_PARTIALCOL && p.mode != PLSE_MODE_AUTO) ||
        (p.matching != PLSE_MATCH_NEAREST && p.matching != PLSE_MATCH_RANDOM) ||
        (p.crossover != PLSE_XOVER_AUX && p.crossover != PLSE_XOVER_UX) ||
        p.tested_cap < 1 || p.tested_cap > 256 || (p.stop_at_bound != 0 && p.stop_at_bound != 1))
        return fail(h, PLSE_EINVAL, "parameter out of range");
    return PLSE_OK;
}

// bounds that keep the kernels' fixed-width arithmetic exact
int check_exactness(plse_instance *h, const plse_params &p)
{
    const long long nv = h->nv, n = h->n;
    const long long tmax = (long long)p.tenure_rand - 1 + (long long)p.alpha_num * nv / p.alpha_den;
    if (tmax > kMaxTenure)
        return fail(h, PLSE_ENOTSUP, "maximum tabu tenure %lld exceeds %d", tmax, kMaxTenure);
    const long long phi2 = std::max<long long>(p.phase1_phi2, (long long)p.phase2_phi2_per_v * nv);
    if (phi2 * 2 * (n > 0 ? n - 1 : 0) + 2 > kMaxD2)
        return fail(h, PLSE_ENOTSUP, "penalty too large for exact 2dF keys");
    if ((long long)p.phase2_iter_per_v * nv > (1ll << 30))   // the walks count iterations in 32 bits
        return fail(h, PLSE_ENOTSUP, "phase-2 iterations %lld exceed 2^30", (long long)p.phase2_iter_per_v * nv);
    return PLSE_OK;
}

// ceil(2^32 / d) if floor(x / d) == high word of x * that for every x the
// tenure formula can produce (x <= alpha_num * |V|), else 0 (the kernel divides)
uint32_t tenure_reciprocal(int alpha_num, int alpha_den, int nv)
{
    if (alpha_den <= 1) return 0;
    const uint64_t m = ((1ull << 32) + (uint64_t)alpha_den - 1) / (uint64_t)alpha_den;
    if (m > 0xFFFFFFFFull) return 0;
    const uint64_t xmax = (uint64_t)alpha_num * (uint64_t)nv;
    for (uint64_t x = 0; x <= xmax; ++x)
        if (((x * m) >> 32) != x / (uint64_t)alpha_den) return 0;
    return (uint32_t)m;
}

int max_tenure(const plse_instance *h)
{
    const plse_params &p = h->params;
    return p.tenure_rand - 1 + (int)((long long)p.alpha_num * h->nv / p.alpha_den);
}

template <typename T>
static int grow(plse_instance *h, T *&ptr, size_t &cap, size_t need, bool zero, cudaStream_t st)
{
    if (need <= cap) return PLSE_OK;
    if (ptr) { h_free(h, ptr, st); ptr = nullptr; cap = 0; }
    void *q = nullptr;
    cudaError_t e = h_malloc(h, &q, need * sizeof(T), st);
    if (e != cudaSuccess) return fail(h, PLSE_ENOMEM, "workspace: %s", cudaGetErrorString(e));
    ptr = static_cast<T *>(q);
    if (zero) {
        e = cudaMemsetAsync(ptr, 0, need * sizeof(T), st);   // in order with the launch that needs it
        if (e != cudaSuccess) return cuda_fail(h, e, "workspace clear");
    }
    cap = need;
    return PLSE_OK;
}

void release_ls_workspace(plse_instance *h, cudaStream_t st)
{
    Workspace &ws = h->ws;
    h_free(h, ws.G, st);
    h_free(h, ws.TC, st);
    h_free(h, ws.LIST, st);
    h_free(h, ws.XR, st);
    h_free(h, ws.HP, st);
    h_free(h, ws.SW, st);
    h_free(h, ws.slot_clock, st);
    h_free(h, ws.counters, st);
    ws = Workspace();
}

// Device bytes ensure_ls_workspace takes for `slots` walk slots, each buffer
// rounded up as the bound-workspace allocator does.
size_t ls_workspace_bytes(const plse_instance *h, int slots)
{
    const DevInst &I = h->di;
    const size_t s = (size_t)slots;
    return ws_align(4 * s * I.nv * I.n1p) + ws_align(8 * s * I.nv) + ws_align(2 * s * I.nv) +
           ws_align(2 * s * 2 * I.n * I.n1p) + ws_align(4 * s * hp_words(I)) + ws_align(s * sw_bytes(I)) +
           ws_align(4 * s) + ws_align(4 * 8);
}

int ensure_counters(plse_instance *h, cudaStream_t st)
{
    return grow(h, h->ws.counters, h->ws.counters_cap, 8, true, st);
}

int ensure_ls_workspace(plse_instance *h, int slots, cudaStream_t st)
{
    Workspace &ws = h->ws;
    int rc = grow(h, ws.G, ws.G_cap, (size_t)slots * h->di.nv * h->di.n1p, true, st);
    if (rc) return rc;
    if ((size_t)slots > ws.clock_cap) {
        // the slot clocks index the same slots as G: reset both together
        if (ws.G && cudaMemsetAsync(ws.G, 0, ws.G_cap * sizeof(uint32_t), st) != cudaSuccess)
            return fail(h, PLSE_ECUDA, "workspace clear");
    }
    rc = grow(h, ws.TC, ws.TC_cap, (size_t)slots * h->di.nv, false, st);   // reset by every phase
    if (rc) return rc;
    rc = grow(h, ws.LIST, ws.LIST_cap, (size_t)slots * h->di.nv, false, st); // rebuilt by every phase
    if (rc) return rc;
    rc = grow(h, ws.XR, ws.XR_cap, (size_t)slots * 2 * h->di.n * h->di.n1p, false, st);   // idem
    if (rc) return rc;
    rc = grow(h, ws.HP, ws.HP_cap, (size_t)slots * hp_words(h->di), false, st);          // idem
    if (rc) return rc;
    rc = grow(h, ws.SW, ws.SW_cap, (size_t)slots * sw_bytes(h->di), false, st);          // idem
    if (rc) return rc;
    rc = grow(h, ws.slot_clock, ws.clock_cap, (size_t)slots, true, st);
    if (rc) return rc;
    return grow(h, ws.counters, ws.counters_cap, 8, true, st);
}

void set_ls_strides(const DevInst &I, LSArgs &a)
{
    a.g_stride = (size_t)I.nv * I.n1p;
    a.tc_stride = (size_t)I.nv;
    a.list_stride = (size_t)I.nv;
    a.xr_stride = 2 * (size_t)I.n * I.n1p;
    a.hp_stride = hp_words(I);
    a.sw_stride = sw_bytes(I);
}

LSArgs ls_args(plse_instance *h, const uint8_t *S_in, uint8_t *S_out, int count, int ind0, int gen, int64_t iters,
               uint64_t seed, int flags, int32_t *f_out, int64_t *F_out, plse_walk_stats *stats, const int *skip)
{
    const plse_params &p = h->params;
    LSArgs a{};
    a.S_in = S_in;
    a.S_out = S_out;
    a.count = count;
    a.ind0 = ind0;
    a.gen = gen;
    a.flags = flags;
    a.iters1 = iters;
    a.iters2 = (int64_t)p.phase2_iter_per_v * h->nv;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.phi2_1 = p.phase1_phi2;
    a.phi2_2 = p.phase2_phi2_per_v * h->nv;
    a.alpha_num = p.alpha_num;
    a.alpha_den = p.alpha_den;
    a.tenure_rand = p.tenure_rand;
    a.alpha_recip = h->alpha_recip;
    const int tmax = max_tenure(h);
    a.span1 = (int)(a.iters1 + tmax + 2);
    a.span2 = (int)(a.iters2 + tmax + 2);
    a.f_out = f_out;
    a.F_out = F_out;
    a.stats = stats;
    a.skip = skip;
    const Workspace &ws = h->ws;
    a.G = ws.G;
    a.TC = ws.TC;
    a.LIST = ws.LIST;
    a.XR = ws.XR;
    a.HP = ws.HP;
    a.SW = ws.SW;
    a.slot_clock = ws.slot_clock;
    set_ls_strides(h->di, a);
    a.work_counter = ws.counters;
    a.error_flag = ws.counters ? ws.counters + 1 : nullptr;
    return a;
}

int enqueue_local_search(plse_instance *h, const uint8_t *S_in, uint8_t *S_out, int count, int ind0,
                         int gen, int64_t iters, uint64_t seed, int flags, int32_t *f_out,
                         int64_t *F_out, plse_walk_stats *stats, cudaStream_t st, const int *skip)
{
    LSLaunch L = plan_local_search(h->di, h->device, count, h->ls_lanes, h->ls_walks, h->ls_splace);
    if (L.blocks <= 0) return fail(h, PLSE_ENOTSUP, "local search does not fit on this device");
    int rc = ensure_ls_workspace(h, L.slots(), st);
    if (rc) return rc;
    const LSArgs a = ls_args(h, S_in, S_out, count, ind0, gen, iters, seed, flags, f_out, F_out, stats, skip);
    cudaError_t e = cudaMemsetAsync(a.work_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "local search");
    e = launch_local_search(h->di, a, L, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "local search launch");
    return PLSE_OK;
}

}  // namespace plse

// ============================================================================
extern "C" {

const char *plse_strerror(int code)
{
    switch (code) {
        case PLSE_OK: return "success";
        case PLSE_EINVAL: return "invalid argument";
        case PLSE_ENOMEM: return "out of memory";
        case PLSE_ECUDA: return "CUDA error";
        case PLSE_EBUSY: return "busy: admission refused";
        case PLSE_ECANCELLED: return "cancelled";
        case PLSE_ENOTSUP: return "not supported";
        case PLSE_ECHECK: return "device-side check failed";
        default: return "unknown error";
    }
}

void plse_default_params(plse_params *p)
{
    if (!p) return;
    p->alpha_num = 6;
    p->alpha_den = 10;
    p->tenure_rand = 10;
    p->phase1_phi2 = 1;
    p->phase2_phi2_per_v = 2;
    p->phase2_iter_per_v = 2;
    p->spacing_gamma = 10;
    p->beta = 20;
    p->mode = PLSE_MODE_PLITS;
    p->matching = PLSE_MATCH_NEAREST;
    p->crossover = PLSE_XOVER_AUX;
    p->tested_cap = 64;
    p->stop_at_bound = 1;
}

int plse_create(int n, const int8_t *grid, plse_handle *out)
{
    if (!out || !grid || n < 1 || n > kMaxN) return PLSE_EINVAL;
    plse_instance *h = new (std::nothrow) plse_instance();
    if (!h) return PLSE_ENOMEM;
    plse_default_params(&h->params);
    int rc = build_instance(h, n, grid);
    if (rc == PLSE_OK) {
        cudaError_t e = cudaGetDevice(&h->device);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->done_ev, cudaEventDisableTiming);
        rc = (e != cudaSuccess) ? cuda_fail(h, e, "cudaGetDevice") : upload_instance(h);
    }
    if (rc == PLSE_OK) rc = check_exactness(h, h->params);
    if (rc == PLSE_OK) h->alpha_recip = tenure_reciprocal(h->params.alpha_num, h->params.alpha_den, h->nv);
    if (rc != PLSE_OK) {
        plse_destroy(h);
        return rc;
    }
    *out = h;
    return PLSE_OK;
}

void plse_destroy(plse_handle h)
{
    if (!h) return;
    run_drain(h);
    // free in stream order after the handle's last work, without waiting for it
    const cudaStream_t st = cudaStreamLegacy;
    if (h->done_recorded) cudaStreamWaitEvent(st, h->done_ev, 0);
    release_solver(h, st);
    dev_free(h->inst_mem, st);
    release_ls_workspace(h, st);
    if (h->done_ev) cudaEventDestroy(h->done_ev);
    delete h;
}

int plse_last_error_detail(plse_handle h, char *buf, size_t len)
{
    if (!h || !buf || len == 0) return PLSE_EINVAL;
    snprintf(buf, len, "%s", h->err.c_str());
    return PLSE_OK;
}

int plse_info(plse_handle h, int *nv, int *l, int *ub)
{
    if (!h) return PLSE_EINVAL;
    if (nv) *nv = h->nv;
    if (l) *l = h->l;
    if (ub) *ub = h->ub;
    return PLSE_OK;
}

int plse_set_params(plse_handle h, const plse_params *p)
{
    if (!h || !p) return PLSE_EINVAL;
    int rc = check_params(h, *p);
    if (rc) return rc;
    rc = check_exactness(h, *p);
    if (rc) return rc;
    h->params = *p;
    h->alpha_recip = tenure_reciprocal(p->alpha_num, p->alpha_den, h->nv);
    return PLSE_OK;
}

int plse_get_params(plse_handle h, plse_params *p)
{
    if (!h || !p) return PLSE_EINVAL;
    *p = h->params;
    return PLSE_OK;
}

int plse_set_launch(plse_handle h, int ls_lanes, int ls_walks, int ls_colourings)
{
    if (!h || !(ls_lanes == 0 || ls_lanes == 16 || ls_lanes == 32 || ls_lanes == 64 || ls_lanes == 128 ||
                ls_lanes == 256) ||
        ls_walks < 0 || ls_walks > 256 || ls_colourings < 0 || ls_colourings > 2)
        return PLSE_EINVAL;
    h->ls_lanes = ls_lanes;
    h->ls_walks = ls_walks;
    h->ls_splace = ls_colourings;
    return PLSE_OK;
}

int plse_workspace_size(plse_handle h, int pop, int max_generations, size_t *bytes)
{
    if (!h || !bytes || pop < 2 || pop > 65535 || max_generations < 0 || max_generations > 65534)
        return PLSE_EINVAL;
    *bytes = 0;
    if (h->nv == 0) return PLSE_OK;
    const LSLaunch L = plan_local_search(h->di, h->device, pop, h->ls_lanes, h->ls_walks, h->ls_splace);
    if (L.blocks <= 0) return fail(h, PLSE_ENOTSUP, "local search does not fit on this device");
    *bytes = solver_bytes(h, pop, max_generations) + ls_workspace_bytes(h, L.slots());
    return PLSE_OK;
}

int plse_bind_workspace(plse_handle h, void *dev_ptr, size_t bytes)
{
    if (!h) return PLSE_EINVAL;
    if (dev_ptr) {
        if (reinterpret_cast<uintptr_t>(dev_ptr) % kWsAlign != 0)
            return fail(h, PLSE_EINVAL, "plse_bind_workspace: range must start on a %zu-byte boundary", kWsAlign);
        cudaPointerAttributes at{};
        const cudaError_t e = cudaPointerGetAttributes(&at, dev_ptr);
        if (e != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != h->device) {
            cudaGetLastError();
            return fail(h, PLSE_EINVAL, "plse_bind_workspace: not device memory of device %d", h->device);
        }
    }
    int rc = run_drain(h);
    if (rc) return rc;
    if (h->done_recorded) {
        const cudaError_t e = cudaEventSynchronize(h->done_ev);
        if (e != cudaSuccess) return cuda_fail(h, e, "plse_bind_workspace");
    }
    // every run and scratch buffer leaves its old memory (the pool or the
    // previous range); the next call that needs one takes it from the new range
    release_solver(h, cudaStreamLegacy);
    release_ls_workspace(h, cudaStreamLegacy);
    h->session = Session();
    h->arena = dev_ptr ? static_cast<char *>(dev_ptr) : nullptr;
    h->arena_size = dev_ptr ? bytes : 0;
    h->arena_used = 0;
    return PLSE_OK;
}

int plse_sync(plse_handle h, void *stream)
{
    if (!h) return PLSE_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "plse_sync");
    // the flag of the handle's own workspace, then that of its last call of
    // plse_local_search_noalloc (a word of the library's fixed scratch array)
    int *flags[2] = {h->ws.counters ? h->ws.counters + 1 : nullptr, h->noalloc_flag};
    h->noalloc_flag = nullptr;
    int failed = 0;
    for (int *fp : flags) {
        if (!fp) continue;
        int flag = 0;
        e = cudaMemcpy(&flag, fp, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(h, e, "plse_sync");
        if (flag) {
            cudaMemsetAsync(fp, 0, sizeof(int), (cudaStream_t)stream);
            cudaStreamSynchronize((cudaStream_t)stream);
            failed = flag;
        }
    }
    if (failed) return fail(h, PLSE_ECHECK, "a device-side consistency check failed (flag %d)", failed);
    return PLSE_OK;
}

int plse_init_population(plse_handle h, int pop, uint64_t seed, uint8_t *P, void *stream)
{
    if (!h || pop < 0 || (pop > 0 && h->nv > 0 && !P)) return PLSE_EINVAL;
    StreamScope scope(h, (cudaStream_t)stream);
    cudaError_t e = launch_init_population(h->di, pop, seed, P, (cudaStream_t)stream);
    return e == cudaSuccess ? PLSE_OK : cuda_fail(h, e, "init_population");
}

int plse_local_search(plse_handle h, const uint8_t *S_in, uint8_t *S_out, int count, int ind0, int gen,
                      int64_t iters, uint64_t seed, int flags, int32_t *f_out, int64_t *F_out,
                      plse_walk_stats *stats, void *stream)
{
    if (!h || count < 0 || ind0 < 0 || gen < 0 || gen >= (1 << 24) || iters < 0 || iters > (1ll << 30) ||
        (flags & ~15) || !flags || ((flags & PLSE_LS_PARTIALCOL) && (flags & (PLSE_LS_PHASE1 | PLSE_LS_PHASE2))))
        return fail(h, PLSE_EINVAL, "plse_local_search: invalid argument");
    if (count == 0) return PLSE_OK;
    if (!S_in || !S_out) return fail(h, PLSE_EINVAL, "plse_local_search: null buffer");
    cudaStream_t st = (cudaStream_t)stream;
    StreamScope scope(h, st);
    if (h->nv == 0) {
        if (f_out) cudaMemsetAsync(f_out, 0, sizeof(int32_t) * count, st);
        if (F_out) cudaMemsetAsync(F_out, 0, sizeof(int64_t) * count, st);
        if (stats) cudaMemsetAsync(stats, 0, sizeof(plse_walk_stats) * count, st);
        return PLSE_OK;
    }
    return enqueue_local_search(h, S_in, S_out, count, ind0, gen, iters, seed, flags, f_out, F_out, stats, st);
}

}  // extern "C"
