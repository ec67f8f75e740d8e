/*
 * plse_oracle.c -- plain CPU oracle of the MPMA hot path (arXiv 2103.10453).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Shares no code with
 * the CUDA library.  Every routine restates one passage of the paper, in the
 * paper's order and notation, with the readings listed below where the paper is
 * silent or ambiguous.  No blocking, fusion or reordering: candidate sets are
 * rebuilt by a full vertex scan every iteration, |C(S)| is recounted from
 * scratch, and the gamma table is the explicit |V| x (n+1) table of the
 * incremental evaluation the paper uses (Sec. 3.3).
 *
 * Readings (the paper is silent or ambiguous):
 *  R1  F is carried as F2 = 2f + phi2*c, phi2 = 2*phi (exact integers).
 *  R2  Tenure T = L + floor(alpha_num*k/alpha_den), k = |V0|+|C(S)| after the
 *      move, L = floor(u*10/2^32) from the walk's Philox draw (Sec. 3.3).
 *  R3  Aspiration: a tabu move is admissible iff F2 + 2dF < best F2 of the
 *      current walk (Sec. 3.3 text; Alg. 3 says "better than S_i").
 *  R4  Move choice: minimum of the key (2dF, (v - r) mod |V|, j) over admissible
 *      moves, r = floor(u*|V|/2^32) drawn once per iteration.  No admissible
 *      move: the iteration passes with no move.  Empty candidate set (f = c = 0):
 *      the walk stops.
 *  R5  Iterations are numbered t = 1..N; (v, j) is tabu at t iff expiry >= t;
 *      a move of v from colour i at iteration t sets expiry[v][i] = t + T.
 *  R6  Phase 2 is a fresh walk (empty tabu list, best = start) started from
 *      phase-1's best S'*, with phi = |V| and 2|V| iterations (Sec. 3.3).
 *  R7  The phase-2 best is legalised by the greedy conflict removal of Sec. 3.7
 *      (most-conflicting vertex first, lowest index on ties).
 *  R8  Alg. 4 ranking score e(S) = f(S) + |V|*c(S); P_all is ordered by
 *      (e, index) with P_t before P'; every examined candidate leaves P_all;
 *      accepted iff gamma*min D > |V|; if P_all runs out, the rejected
 *      candidates fill the remaining places in the same order.
 *  R9  Matching: nearest partner whose uid is not in the first parent's
 *      tested list (lowest index on ties); if all are tested, plain nearest.
 *      uid = (generation of insertion) << 16 | slot; the list keeps the last
 *      tested_cap partners.
 *  R10 AUX coin: take S_i(v) iff u*b < a*2^32 with a = beta*D - |V| (clamped at
 *      0) and b = beta*D, i.e. with probability p_ij of Eq. 10.
 *  R11 Initial colouring: S(v) uniform over D(v) \ {0}.
 *  R12 Philox4x32-10 counter = (block or iteration, individual,
 *      generation<<8 | purpose<<4 | phase, 0), key = (seed low, seed high).
 *  R13 PartialCol (Sec. 3.7, cited method): a move colours v in V0 with
 *      j in D(v)\{0} and uncolours every neighbour of colour j; df = gamma-1;
 *      each uncoloured neighbour u gets (u, j) tabu with T = L + alpha*|V0|.
 */
#include "plse_oracle.h"
#include <stdlib.h>
#include <string.h>

enum { PURPOSE_INIT = 1, PURPOSE_TABU = 2, PURPOSE_XOVER = 3, PURPOSE_MATCH = 4 };

typedef struct {
    int n, nv, l, ub, nfixed;
    int8_t *grid;       /* n*n copy of the instance                          */
    int *cell;          /* [nv] row-major cell index of each vertex          */
    int *row, *col;     /* [nv]                                              */
    uint8_t *dom;       /* [nv*(n+1)] 1 iff colour in D(v); colour 0 always  */
    int *ndom;          /* [nv] |D(v)| including 0                           */
    int *adj_ptr;       /* [nv+1]                                            */
    int *adj;           /* edges of the reduced graph, both directions       */
} Inst;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two  */
/* 32x32->64 multiplies, a word swap and a key xor; the key is bumped by */
/* the Weyl constants between rounds.                                   */
/* ------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw4(uint64_t seed, uint32_t c0, uint32_t ind, uint32_t gen,
                  uint32_t purpose, uint32_t phase, uint32_t out[4])
{
    uint32_t ctr[4] = { c0, ind, (gen << 8) | (purpose << 4) | phase, 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_philox4x32_10(ctr, key, out);
}

/* uniform integer in [0, k): the high word of u * k */
static uint32_t bounded(uint32_t u, uint32_t k) { return (uint32_t)(((uint64_t)u * k) >> 32); }

void or_default_params(or_params *p)
{
    p->alpha_num = 6; p->alpha_den = 10;    /* alpha = 0.6 (Table 1)          */
    p->tenure_rand = 10;                    /* L in [0;9] (Sec. 3.3)          */
    p->phase1_phi2 = 1;                     /* phi = 0.5 (Sec. 3.3)           */
    p->phase2_phi2_per_v = 2;               /* phi = |V| (Sec. 3.3)           */
    p->phase2_iter_per_v = 2;               /* 2*|V| iterations (Sec. 3.3)    */
    p->spacing_gamma = 10;                  /* gamma = 10 (Table 1)           */
    p->beta = 20;                           /* beta = 20 (Table 1)            */
    p->mode = 0; p->matching = 0; p->crossover = 0;
    p->tested_cap = 64;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1-2.2 and Alg. 1: Latin square graph, domains, reduction.     */
/* ------------------------------------------------------------------ */
void *or_create(int32_t n, const int8_t *grid, int32_t *err)
{
    *err = 0;
    if (n < 1 || n > 127) { *err = -1; return NULL; }
    for (int i = 0; i < n * n; ++i)
        if (grid[i] < 0 || grid[i] > n) { *err = -2; return NULL; }
    /* partial Latin square: no symbol twice in a row or a column (Sec. 1) */
    for (int r = 0; r < n; ++r)
        for (int a = 0; a < n; ++a)
            for (int b = a + 1; b < n; ++b) {
                if (grid[r * n + a] && grid[r * n + a] == grid[r * n + b]) { *err = -3; return NULL; }
                if (grid[a * n + r] && grid[a * n + r] == grid[b * n + r]) { *err = -3; return NULL; }
            }

    Inst *I = (Inst *)calloc(1, sizeof(Inst));
    I->n = n;
    I->grid = (int8_t *)malloc((size_t)n * n);
    memcpy(I->grid, grid, (size_t)n * n);
    I->cell = (int *)malloc(sizeof(int) * n * n);
    I->row = (int *)malloc(sizeof(int) * n * n);
    I->col = (int *)malloc(sizeof(int) * n * n);
    I->dom = (uint8_t *)malloc((size_t)n * n * (n + 1));
    I->ndom = (int *)malloc(sizeof(int) * n * n);

    /* Full Latin square graph: D(v) = {k} for a prefilled cell, {0..n} for an
     * empty one.  Alg. 1, first loop: every prefilled vertex is removed and its
     * colour k is struck from the domains of its row- and column-mates. */
    uint8_t *D = (uint8_t *)malloc((size_t)n * n * (n + 1));
    for (int v = 0; v < n * n; ++v)
        for (int k = 0; k <= n; ++k)
            D[v * (n + 1) + k] = grid[v] ? (uint8_t)(k == grid[v]) : 1;
    for (int v = 0; v < n * n; ++v) {
        if (!grid[v]) continue;
        int k = grid[v], r = v / n, c = v % n;
        for (int u = 0; u < n * n; ++u) {
            if (u == v || grid[u]) continue;
            if (u / n == r || u % n == c) D[u * (n + 1) + k] = 0;
        }
    }
    /* Alg. 1, second loop: empty cells whose domain is {0} are removed and
     * counted in l.  The survivors, in row-major order, are the vertices V. */
    int nv = 0, l = 0, nfixed = 0;
    for (int v = 0; v < n * n; ++v) {
        if (grid[v]) { ++nfixed; continue; }
        int cnt = 0;
        for (int k = 1; k <= n; ++k) cnt += D[v * (n + 1) + k];
        if (cnt == 0) { ++l; continue; }
        I->cell[nv] = v; I->row[nv] = v / n; I->col[nv] = v % n;
        memcpy(I->dom + (size_t)nv * (n + 1), D + (size_t)v * (n + 1), (size_t)n + 1);
        I->ndom[nv] = cnt + 1;
        ++nv;
    }
    free(D);
    I->nv = nv; I->l = l; I->nfixed = nfixed;
    /* Upper bound n^2 - l, or n^2 - 2 when l = 1 (Sec. 2.2). */
    I->ub = n * n - l;
    if (l == 1) I->ub = n * n - 2;

    /* Edges of the reduced graph: same row or same column (Sec. 2.1). */
    I->adj_ptr = (int *)malloc(sizeof(int) * (nv + 1));
    int64_t m = 0;
    for (int v = 0; v < nv; ++v)
        for (int u = 0; u < nv; ++u)
            if (u != v && (I->row[u] == I->row[v] || I->col[u] == I->col[v])) ++m;
    I->adj = (int *)malloc(sizeof(int) * (m > 0 ? m : 1));
    m = 0;
    for (int v = 0; v < nv; ++v) {
        I->adj_ptr[v] = (int)m;
        for (int u = 0; u < nv; ++u)
            if (u != v && (I->row[u] == I->row[v] || I->col[u] == I->col[v])) I->adj[m++] = u;
    }
    I->adj_ptr[nv] = (int)m;
    return I;
}

void or_destroy(void *h)
{
    Inst *I = (Inst *)h;
    if (!I) return;
    free(I->grid); free(I->cell); free(I->row); free(I->col); free(I->dom);
    free(I->ndom); free(I->adj_ptr); free(I->adj); free(I);
}

void or_info(const void *h, int32_t *n, int32_t *nv, int32_t *l, int32_t *ub, int32_t *nfixed)
{
    const Inst *I = (const Inst *)h;
    *n = I->n; *nv = I->nv; *l = I->l; *ub = I->ub; *nfixed = I->nfixed;
}

void or_vertices(const void *h, int32_t *cell)
{
    const Inst *I = (const Inst *)h;
    for (int v = 0; v < I->nv; ++v) cell[v] = I->cell[v];
}

void or_domains(const void *h, uint8_t *dom)
{
    const Inst *I = (const Inst *)h;
    memcpy(dom, I->dom, (size_t)I->nv * (I->n + 1));
}

int64_t or_num_edges(const void *h)
{
    const Inst *I = (const Inst *)h;
    return I->adj_ptr[I->nv] / 2;
}

/* ------------------------------------------------------------------ */
/* Evaluation: f (Eq. 1), c (Eq. 3-4), F = f + phi*c (Eq. 5).           */
/* ------------------------------------------------------------------ */
int64_t or_eval(const void *h, const uint8_t *S, int32_t phi2, int64_t *f_out, int64_t *c_out)
{
    const Inst *I = (const Inst *)h;
    int64_t f = 0, c = 0;
    for (int v = 0; v < I->nv; ++v) {
        if (S[v] == 0) ++f;
        for (int e = I->adj_ptr[v]; e < I->adj_ptr[v + 1]; ++e) {
            int u = I->adj[e];
            if (u > v && S[u] == S[v] && S[v] != 0) ++c;   /* each edge once */
        }
    }
    if (f_out) *f_out = f;
    if (c_out) *c_out = c;
    return 2 * f + (int64_t)phi2 * c;
}

void or_gamma(const void *h, const uint8_t *S, int32_t *gamma)
{
    const Inst *I = (const Inst *)h;
    int n1 = I->n + 1;
    memset(gamma, 0, sizeof(int32_t) * (size_t)I->nv * n1);
    for (int v = 0; v < I->nv; ++v)
        for (int e = I->adj_ptr[v]; e < I->adj_ptr[v + 1]; ++e) {
            int k = S[I->adj[e]];
            if (k) gamma[v * n1 + k] += 1;
        }
}

/* C(S): coloured vertices with at least one neighbour of the same colour. */
static int64_t count_conflicting(const Inst *I, const uint8_t *S, const int32_t *gamma)
{
    int n1 = I->n + 1;
    int64_t cnt = 0;
    for (int v = 0; v < I->nv; ++v)
        if (S[v] != 0 && gamma[v * n1 + S[v]] > 0) ++cnt;
    return cnt;
}

int64_t or_num_conflicting(const void *h, const uint8_t *S)
{
    const Inst *I = (const Inst *)h;
    int32_t *g = (int32_t *)malloc(sizeof(int32_t) * (size_t)I->nv * (I->n + 1) + 4);
    or_gamma(h, S, g);
    int64_t r = count_conflicting(I, S, g);
    free(g);
    return r;
}

/* ------------------------------------------------------------------ */
/* Population initialisation (Sec. 3.2), reading R11.                   */
/* ------------------------------------------------------------------ */
void or_init_population(const void *h, int32_t p, uint64_t seed, uint8_t *P)
{
    const Inst *I = (const Inst *)h;
    int n1 = I->n + 1;
    for (int i = 0; i < p; ++i)
        for (int v = 0; v < I->nv; ++v) {
            uint32_t u[4];
            draw4(seed, (uint32_t)(v >> 2), (uint32_t)i, 0u, PURPOSE_INIT, 0u, u);
            uint32_t k = bounded(u[v & 3], (uint32_t)(I->ndom[v] - 1));
            /* the k-th colour (ascending) of D(v) \ {0} */
            int col = 0;
            for (int c = 1; c <= I->n; ++c)
                if (I->dom[v * n1 + c]) {
                    if (k == 0) { col = c; break; }
                    --k;
                }
            P[(size_t)i * I->nv + v] = (uint8_t)col;
        }
}

/* ------------------------------------------------------------------ */
/* Tabu walk, Alg. 3 (PLITS phase 1 / 2) and PartialCol (Sec. 3.7).     */
/* ------------------------------------------------------------------ */
typedef struct { int64_t d2; int rot; int j; int v; int valid; } MoveKey;

static int key_less(int64_t d2, int rot, int j, const MoveKey *b)
{
    if (!b->valid) return 1;
    if (d2 != b->d2) return d2 < b->d2;
    if (rot != b->rot) return rot < b->rot;
    return j < b->j;
}

static int64_t plits_walk(const Inst *I, const or_params *prm, uint8_t *S, int32_t ind,
                          int32_t gen, int32_t phase, int64_t iters, uint64_t seed,
                          int32_t debug, or_stats *st, int32_t *trace)
{
    const int n1 = I->n + 1, nv = I->nv;
    const int64_t phi2 = (phase == 1) ? prm->phase1_phi2
                                      : (int64_t)prm->phase2_phi2_per_v * nv;
    int32_t *gamma = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * n1 + 4);
    int64_t *expiry = (int64_t *)calloc((size_t)nv * n1 + 1, sizeof(int64_t));
    uint8_t *best = (uint8_t *)malloc((size_t)nv + 1);
    uint8_t *is_cand = (uint8_t *)malloc((size_t)nv + 1);
    int32_t *gchk = debug ? (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * n1 + 4) : NULL;
    int64_t ret;

    or_gamma(I, S, gamma);
    int64_t f, c;
    int64_t F2 = or_eval(I, S, (int32_t)phi2, &f, &c);
    memcpy(best, S, (size_t)nv);
    int64_t F2best = F2;

    for (int64_t t = 1; t <= iters; ++t) {
        /* candidate vertices V0 u C(S) (Sec. 3.3) */
        int64_t ncand = 0;
        for (int v = 0; v < nv; ++v) {
            int i = S[v];
            is_cand[v] = (uint8_t)(i == 0 || gamma[v * n1 + i] > 0);
            ncand += is_cand[v];
        }
        if (ncand == 0) break;            /* f = c = 0: nothing left to improve */
        if (st) { st->iterations++; st->cand += ncand; }
        if (trace) trace[3 * (t - 1)] = trace[3 * (t - 1) + 1] = trace[3 * (t - 1) + 2] = -1;

        uint32_t u[4];
        draw4(seed, (uint32_t)t, (uint32_t)ind, (uint32_t)gen, PURPOSE_TABU, (uint32_t)phase, u);
        const int64_t L = bounded(u[0], (uint32_t)prm->tenure_rand);
        const int r = (int)bounded(u[1], (uint32_t)nv);
        const int64_t A = F2best - F2;   /* aspiration: 2dF < A  <=>  F2' < F2best */

        MoveKey bestm = { 0, 0, 0, 0, 0 };
        for (int v = 0; v < nv; ++v) {
            if (!is_cand[v]) continue;
            const int i = S[v];
            const int rot = (v - r + nv) % nv;
            for (int j = 0; j <= I->n; ++j) {
                if (!I->dom[v * n1 + j] || j == i) continue;
                /* N0: i = 0 -> j != 0;  Nc: i != 0 -> any j != i, 0 allowed */
                const int64_t d2 = 2 * ((j == 0) - (i == 0))
                                 + phi2 * ((j ? gamma[v * n1 + j] : 0) - (i ? gamma[v * n1 + i] : 0));
                if (st) st->pairs++;
                if (debug >= 2) {
                    uint8_t save = S[v];
                    S[v] = (uint8_t)j;
                    int64_t F2j = or_eval(I, S, (int32_t)phi2, NULL, NULL);
                    S[v] = save;
                    if (F2j - F2 != d2) { ret = -1; goto out; }
                }
                const int tabu = expiry[v * n1 + j] >= t;
                if (tabu && !(d2 < A)) continue;
                if (key_less(d2, rot, j, &bestm)) {
                    bestm.d2 = d2; bestm.rot = rot; bestm.j = j; bestm.v = v; bestm.valid = 1;
                }
            }
        }
        if (!bestm.valid) continue;       /* every move tabu: no move this iteration */

        /* apply S <- S (+) <v, V_i, V_j> and update gamma incrementally */
        const int v = bestm.v, j = bestm.j, i = S[v];
        if (trace) { trace[3 * (t - 1)] = v; trace[3 * (t - 1) + 1] = i; trace[3 * (t - 1) + 2] = j; }
        if (st) { st->moves++; st->deg += I->adj_ptr[v + 1] - I->adj_ptr[v]; }
        f += (j == 0) - (i == 0);
        c += (j ? gamma[v * n1 + j] : 0) - (i ? gamma[v * n1 + i] : 0);
        F2 += bestm.d2;
        S[v] = (uint8_t)j;
        for (int e = I->adj_ptr[v]; e < I->adj_ptr[v + 1]; ++e) {
            const int w = I->adj[e];
            if (i) gamma[w * n1 + i] -= 1;
            if (j) gamma[w * n1 + j] += 1;
        }
        /* tenure from the eligible-vertex count after the move (R2) */
        const int64_t k = f + count_conflicting(I, S, gamma);
        const int64_t T = L + (prm->alpha_num * k) / prm->alpha_den;
        expiry[v * n1 + i] = t + T;

        if (debug) {
            or_gamma(I, S, gchk);
            if (memcmp(gchk, gamma, sizeof(int32_t) * (size_t)nv * n1) != 0) { ret = -1; goto out; }
            int64_t fc, cc;
            if (or_eval(I, S, (int32_t)phi2, &fc, &cc) != F2 || fc != f || cc != c) { ret = -1; goto out; }
        }
        if (F2 < F2best) {                /* Alg. 3: strict improvement only */
            F2best = F2;
            memcpy(best, S, (size_t)nv);
            if (st) st->improvements++;
        }
    }
    memcpy(S, best, (size_t)nv);
    ret = F2best;
out:
    free(gamma); free(expiry); free(best); free(is_cand); free(gchk);
    return ret;
}

static int64_t partialcol_walk(const Inst *I, const or_params *prm, uint8_t *S, int32_t ind,
                               int32_t gen, int64_t iters, uint64_t seed, int32_t debug,
                               or_stats *st, int32_t *trace)
{
    const int n1 = I->n + 1, nv = I->nv;
    int32_t *gamma = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * n1 + 4);
    int64_t *expiry = (int64_t *)calloc((size_t)nv * n1 + 1, sizeof(int64_t));
    uint8_t *best = (uint8_t *)malloc((size_t)nv + 1);
    int32_t *gchk = debug ? (int32_t *)malloc(sizeof(int32_t) * (size_t)nv * n1 + 4) : NULL;
    int64_t ret;

    or_gamma(I, S, gamma);
    int64_t f, c;
    or_eval(I, S, 0, &f, &c);
    if (c != 0) { ret = -1; goto out; }   /* PartialCol works on legal colourings */
    memcpy(best, S, (size_t)nv);
    int64_t fbest = f;

    for (int64_t t = 1; t <= iters; ++t) {
        if (f == 0) break;
        if (st) { st->iterations++; st->cand += f; }
        if (trace) trace[3 * (t - 1)] = trace[3 * (t - 1) + 1] = trace[3 * (t - 1) + 2] = -1;
        uint32_t u[4];
        draw4(seed, (uint32_t)t, (uint32_t)ind, (uint32_t)gen, PURPOSE_TABU, 3u, u);
        const int64_t L = bounded(u[0], (uint32_t)prm->tenure_rand);
        const int r = (int)bounded(u[1], (uint32_t)nv);
        const int64_t A = fbest - f;

        MoveKey bestm = { 0, 0, 0, 0, 0 };
        for (int v = 0; v < nv; ++v) {
            if (S[v] != 0) continue;      /* only uncoloured vertices move */
            const int rot = (v - r + nv) % nv;
            for (int j = 1; j <= I->n; ++j) {
                if (!I->dom[v * n1 + j]) continue;
                const int64_t d = (int64_t)gamma[v * n1 + j] - 1;
                if (st) st->pairs++;
                const int tabu = expiry[v * n1 + j] >= t;
                if (tabu && !(d < A)) continue;
                if (key_less(d, rot, j, &bestm)) {
                    bestm.d2 = d; bestm.rot = rot; bestm.j = j; bestm.v = v; bestm.valid = 1;
                }
            }
        }
        if (!bestm.valid) continue;

        const int v = bestm.v, j = bestm.j;
        if (trace) { trace[3 * (t - 1)] = v; trace[3 * (t - 1) + 1] = 0; trace[3 * (t - 1) + 2] = j; }
        if (st) { st->moves++; st->deg += I->adj_ptr[v + 1] - I->adj_ptr[v]; }
        /* neighbours currently coloured j lose their colour */
        int unc[2 * 128], nunc = 0;
        for (int e = I->adj_ptr[v]; e < I->adj_ptr[v + 1]; ++e)
            if (S[I->adj[e]] == j) unc[nunc++] = I->adj[e];
        for (int q = 0; q < nunc; ++q) {
            const int w = unc[q];
            S[w] = 0;
            for (int e = I->adj_ptr[w]; e < I->adj_ptr[w + 1]; ++e) gamma[I->adj[e] * n1 + j] -= 1;
        }
        S[v] = (uint8_t)j;
        for (int e = I->adj_ptr[v]; e < I->adj_ptr[v + 1]; ++e) gamma[I->adj[e] * n1 + j] += 1;
        f += bestm.d2;
        if (st) st->uncolored += nunc;
        const int64_t T = L + (prm->alpha_num * f) / prm->alpha_den;
        for (int q = 0; q < nunc; ++q) expiry[unc[q] * n1 + j] = t + T;

        if (debug) {
            or_gamma(I, S, gchk);
            if (memcmp(gchk, gamma, sizeof(int32_t) * (size_t)nv * n1) != 0) { ret = -1; goto out; }
            int64_t fc, cc;
            or_eval(I, S, 0, &fc, &cc);
            if (fc != f || cc != 0) { ret = -1; goto out; }
        }
        if (f < fbest) {
            fbest = f;
            memcpy(best, S, (size_t)nv);
            if (st) st->improvements++;
        }
    }
    memcpy(S, best, (size_t)nv);
    ret = fbest;
out:
    free(gamma); free(expiry); free(best); free(gchk);
    return ret;
}

int64_t or_tabu_walk_traced(const void *h, const or_params *prm, uint8_t *S, int32_t ind,
                            int32_t gen, int32_t phase, int64_t iters, uint64_t seed,
                            int32_t debug, or_stats *st, int32_t *trace)
{
    const Inst *I = (const Inst *)h;
    if (I->nv == 0) return 0;
    if (phase == 3) return partialcol_walk(I, prm, S, ind, gen, iters, seed, debug, st, trace);
    return plits_walk(I, prm, S, ind, gen, phase, iters, seed, debug, st, trace);
}

int64_t or_tabu_walk(const void *h, const or_params *prm, uint8_t *S, int32_t ind, int32_t gen,
                     int32_t phase, int64_t iters, uint64_t seed, int32_t debug, or_stats *st)
{
    return or_tabu_walk_traced(h, prm, S, ind, gen, phase, iters, seed, debug, st, NULL);
}

/* ------------------------------------------------------------------ */
/* Greedy conflict removal (Sec. 3.7), reading R7.                      */
/* ------------------------------------------------------------------ */
int32_t or_repair(const void *h, uint8_t *S)
{
    const Inst *I = (const Inst *)h;
    const int n1 = I->n + 1;
    int32_t *gamma = (int32_t *)malloc(sizeof(int32_t) * (size_t)I->nv * n1 + 4);
    or_gamma(h, S, gamma);
    int32_t steps = 0;
    for (;;) {
        int bv = -1, bg = 0;
        for (int v = 0; v < I->nv; ++v) {
            if (S[v] == 0) continue;
            int g = gamma[v * n1 + S[v]];
            if (g > bg) { bg = g; bv = v; }   /* strict: lowest index on ties */
        }
        if (bv < 0) break;                     /* c(S) = 0 */
        const int k = S[bv];
        S[bv] = 0;
        for (int e = I->adj_ptr[bv]; e < I->adj_ptr[bv + 1]; ++e) gamma[I->adj[e] * n1 + k] -= 1;
        ++steps;
    }
    free(gamma);
    return steps;
}

/* ------------------------------------------------------------------ */
/* Hamming distance (Sec. 3.4, Eq. 9).                                  */
/* ------------------------------------------------------------------ */
void or_distances(const void *h, const uint8_t *A, int32_t na, const uint8_t *B, int32_t nb, int32_t *D)
{
    const Inst *I = (const Inst *)h;
    const int nv = I->nv;
    for (int a = 0; a < na; ++a)
        for (int b = 0; b < nb; ++b) {
            int32_t d = 0;
            for (int v = 0; v < nv; ++v) d += A[(size_t)a * nv + v] != B[(size_t)b * nv + v];
            D[(size_t)a * nb + b] = d;
        }
}

/* ------------------------------------------------------------------ */
/* Population update, Alg. 4, reading R8.                               */
/* ------------------------------------------------------------------ */
static const int64_t *g_sort_e;
static int cmp_rank(const void *x, const void *y)
{
    int a = *(const int *)x, b = *(const int *)y;
    if (g_sort_e[a] != g_sort_e[b]) return g_sort_e[a] < g_sort_e[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

int32_t or_pop_update(const void *h, const or_params *prm, int32_t p, const int64_t *e,
                      const int32_t *Dall, int32_t *sel)
{
    const Inst *I = (const Inst *)h;
    const int m = 2 * p;
    int *order = (int *)malloc(sizeof(int) * m);
    int *rejected = (int *)malloc(sizeof(int) * m);
    for (int k = 0; k < m; ++k) order[k] = k;
    g_sort_e = e;
    qsort(order, (size_t)m, sizeof(int), cmp_rank);   /* argmin e, repeatedly */
    int nacc = 0, nrej = 0;
    for (int q = 0; q < m && nacc < p; ++q) {
        const int s = order[q];
        int accept = 1;
        if (nacc > 0) {
            int32_t dmin = INT32_MAX;
            for (int a = 0; a < nacc; ++a) {
                int32_t d = Dall[(size_t)s * m + sel[a]];
                if (d < dmin) dmin = d;
            }
            accept = (int64_t)prm->spacing_gamma * dmin > I->nv;   /* D > |V|/gamma */
        }
        if (accept) sel[nacc++] = s;
        else rejected[nrej++] = s;
    }
    int32_t filled = 0;
    for (int q = 0; nacc < p && q < nrej; ++q) { sel[nacc++] = rejected[q]; ++filled; }
    free(order); free(rejected);
    return filled;
}

/* ------------------------------------------------------------------ */
/* Parent matching (Sec. 3.5.1, Alg. 5), reading R9.                    */
/* ------------------------------------------------------------------ */
static int in_list(const uint32_t *list, int cnt, uint32_t x)
{
    for (int k = 0; k < cnt; ++k) if (list[k] == x) return 1;
    return 0;
}

void or_matching(const void *h, const or_params *prm, int32_t p, const int32_t *D,
                 const uint32_t *uid, uint32_t *tested, int32_t *tcount,
                 int32_t gen, uint64_t seed, int32_t *partner)
{
    (void)h;
    const int cap = prm->tested_cap;
    for (int i = 0; i < p; ++i) {
        int j = -1;
        if (prm->matching == 1) {               /* random matching (Sec. 5.3) */
            uint32_t u[4];
            draw4(seed, 0u, (uint32_t)i, (uint32_t)gen, PURPOSE_MATCH, 0u, u);
            j = (int)bounded(u[0], (uint32_t)(p - 1));
            if (j >= i) ++j;
            partner[i] = j;
            continue;
        }
        for (int q = 0; q < p; ++q) {
            if (q == i || in_list(tested + (size_t)i * cap, tcount[i], uid[q])) continue;
            if (j < 0 || D[(size_t)i * p + q] < D[(size_t)i * p + j]) j = q;
        }
        if (j < 0)                              /* every partner tested already */
            for (int q = 0; q < p; ++q) {
                if (q == i) continue;
                if (j < 0 || D[(size_t)i * p + q] < D[(size_t)i * p + j]) j = q;
            }
        partner[i] = j;
        uint32_t *L = tested + (size_t)i * cap;
        if (tcount[i] == cap) {                 /* keep the last cap partners */
            memmove(L, L + 1, sizeof(uint32_t) * (size_t)(cap - 1));
            L[cap - 1] = uid[j];
        } else {
            L[tcount[i]++] = uid[j];
        }
    }
}

/* ------------------------------------------------------------------ */
/* AUX crossover (Sec. 3.5.2, Eq. 10, Alg. 5), reading R10; UX variant. */
/* ------------------------------------------------------------------ */
void or_crossover(const void *h, const or_params *prm, int32_t p, const uint8_t *P,
                  const int32_t *partner, const int32_t *D, int32_t gen, uint64_t seed,
                  uint8_t *O)
{
    const Inst *I = (const Inst *)h;
    const int nv = I->nv;
    for (int i = 0; i < p; ++i) {
        const int j = partner[i];
        const int64_t d = D[(size_t)i * p + j];
        int64_t a, b;
        if (prm->crossover == 1) { a = 1; b = 2; }            /* UX: p_ij = 1/2 */
        else {
            b = (int64_t)prm->beta * d;                         /* p_ij = 1 - |V|/(beta D) */
            a = b - nv;
            if (a < 0) a = 0;
        }
        for (int v = 0; v < nv; ++v) {
            uint32_t u[4];
            draw4(seed, (uint32_t)(v >> 2), (uint32_t)i, (uint32_t)gen, PURPOSE_XOVER, 0u, u);
            const int take_i = (d == 0) || ((uint64_t)u[v & 3] * (uint64_t)b < ((uint64_t)a << 32));
            O[(size_t)i * nv + v] = take_i ? P[(size_t)i * nv + v] : P[(size_t)j * nv + v];
        }
    }
}

/* ------------------------------------------------------------------ */
/* The memetic loop, Alg. 2.                                            */
/* ------------------------------------------------------------------ */
static void add_stats(or_stats *a, const or_stats *b)
{
    a->iterations += b->iterations; a->moves += b->moves; a->cand += b->cand;
    a->pairs += b->pairs; a->deg += b->deg; a->improvements += b->improvements;
    a->uncolored += b->uncolored;
}

int32_t or_solve(const void *h, const or_params *prm, int32_t p, int32_t generations,
                 int64_t iters, uint64_t seed, int8_t *best_grid, int32_t *best_score,
                 int32_t *trace, or_stats *st_total, uint8_t *final_pop)
{
    const Inst *I = (const Inst *)h;
    const int nv = I->nv, cap = prm->tested_cap;
    const size_t PV = (size_t)p * nv;
    uint8_t *P = (uint8_t *)calloc(PV + 1, 1), *Pp = (uint8_t *)calloc(PV + 1, 1);
    uint8_t *SO = (uint8_t *)malloc(PV + 1), *Pn = (uint8_t *)malloc(PV + 1);
    uint8_t *Sstar = (uint8_t *)calloc((size_t)nv + 1, 1);
    int64_t *eall = (int64_t *)malloc(sizeof(int64_t) * 2 * p);
    int64_t *eP = (int64_t *)malloc(sizeof(int64_t) * p);
    int32_t *Dm = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * p);
    int32_t *Dall = (int32_t *)malloc(sizeof(int32_t) * (size_t)4 * p * p);
    int32_t *Dx = (int32_t *)malloc(sizeof(int32_t) * (size_t)p * p);
    int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * p);
    int32_t *partner = (int32_t *)malloc(sizeof(int32_t) * p);
    uint32_t *uid = (uint32_t *)malloc(sizeof(uint32_t) * p), *uidn = (uint32_t *)malloc(sizeof(uint32_t) * p);
    uint32_t *tested = (uint32_t *)calloc((size_t)p * cap + 1, sizeof(uint32_t));
    uint32_t *testedn = (uint32_t *)calloc((size_t)p * cap + 1, sizeof(uint32_t));
    int32_t *tcount = (int32_t *)calloc((size_t)p, sizeof(int32_t)), *tcountn = (int32_t *)calloc((size_t)p, sizeof(int32_t));
    if (st_total) memset(st_total, 0, sizeof(*st_total));

    /* S* = empty colouring, f(S*) = |V| (Alg. 2) */
    int64_t fstar = nv;
    const int64_t ftarget = (I->l == 1) ? 1 : 0;     /* optimality test (Sec. 3.2) */
    int32_t g_done = 0;

    if (nv > 0 && fstar > ftarget) {
        or_init_population(h, p, seed, P);
        for (int i = 0; i < p; ++i) {
            int64_t f, c;
            or_eval(h, P + (size_t)i * nv, 0, &f, &c);
            eP[i] = f + (int64_t)nv * c;
            uid[i] = (uint32_t)i;
        }
        or_distances(h, P, p, P, p, Dm);
        memcpy(SO, P, PV);

        for (int g = 0; g < generations; ++g) {
            /* two-phase local search of every offspring (Alg. 3 twice) */
            for (int i = 0; i < p; ++i) {
                uint8_t *S = Pp + (size_t)i * nv;
                memcpy(S, SO + (size_t)i * nv, (size_t)nv);
                or_stats st;
                memset(&st, 0, sizeof(st));
                if (prm->mode == 1) {
                    or_repair(h, S);
                    or_tabu_walk(h, prm, S, i, g, 3, iters, seed, 0, &st);
                } else {
                    or_tabu_walk(h, prm, S, i, g, 1, iters, seed, 0, &st);
                    or_tabu_walk(h, prm, S, i, g, 2, (int64_t)prm->phase2_iter_per_v * nv, seed, 0, &st);
                    or_repair(h, S);
                }
                if (st_total) add_stats(st_total, &st);
            }
            /* best-solution update, strict (Alg. 2) */
            int istar = -1;
            int64_t fbest = 0;
            for (int i = 0; i < p; ++i) {
                int64_t f, c;
                or_eval(h, Pp + (size_t)i * nv, 0, &f, &c);
                eall[p + i] = f + (int64_t)nv * c;
                if (c == 0 && (istar < 0 || f < fbest)) { istar = i; fbest = f; }
            }
            if (istar >= 0 && fbest < fstar) {
                fstar = fbest;
                memcpy(Sstar, Pp + (size_t)istar * nv, (size_t)nv);
            }
            if (trace) trace[g] = (int32_t)fstar;
            g_done = g + 1;
            if (fstar <= ftarget) break;

            /* distances P x P' and P' x P' (Sec. 3.4), assembled with the
             * population's own matrix into the 2p x 2p matrix of P_all */
            const int m = 2 * p;
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) Dall[(size_t)a * m + b] = Dm[(size_t)a * p + b];
            or_distances(h, P, p, Pp, p, Dx);
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) {
                    Dall[(size_t)a * m + p + b] = Dx[(size_t)a * p + b];
                    Dall[(size_t)(p + b) * m + a] = Dx[(size_t)a * p + b];
                }
            or_distances(h, Pp, p, Pp, p, Dx);
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) Dall[(size_t)(p + a) * m + p + b] = Dx[(size_t)a * p + b];
            for (int i = 0; i < p; ++i) eall[i] = eP[i];

            or_pop_update(h, prm, p, eall, Dall, sel);

            /* P_{t+1}: colourings, scores, uids, tested lists and distances */
            for (int q = 0; q < p; ++q) {
                const int s = sel[q];
                if (s < p) {
                    memcpy(Pn + (size_t)q * nv, P + (size_t)s * nv, (size_t)nv);
                    uidn[q] = uid[s];
                    tcountn[q] = tcount[s];
                    memcpy(testedn + (size_t)q * cap, tested + (size_t)s * cap, sizeof(uint32_t) * cap);
                } else {
                    memcpy(Pn + (size_t)q * nv, Pp + (size_t)(s - p) * nv, (size_t)nv);
                    uidn[q] = ((uint32_t)(g + 1) << 16) | (uint32_t)(s - p);
                    tcountn[q] = 0;
                }
                eP[q] = eall[s];
            }
            for (int a = 0; a < p; ++a)
                for (int b = 0; b < p; ++b) Dm[(size_t)a * p + b] = Dall[(size_t)sel[a] * m + sel[b]];
            { uint8_t *t8 = P; P = Pn; Pn = t8; }
            { uint32_t *tu = uid; uid = uidn; uidn = tu; }
            { uint32_t *tt = tested; tested = testedn; testedn = tt; }
            { int32_t *tc = tcount; tcount = tcountn; tcountn = tc; }

            /* offspring for the next generation (Alg. 5) */
            or_matching(h, prm, p, Dm, uid, tested, tcount, g, seed, partner);
            or_crossover(h, prm, p, P, partner, Dm, g, seed, SO);
        }
    }

    /* best grid: prefilled symbols + S* on the reduced vertices */
    for (int q = 0; q < I->n * I->n; ++q) best_grid[q] = I->grid[q];
    for (int v = 0; v < nv; ++v) best_grid[I->cell[v]] = (int8_t)Sstar[v];
    *best_score = I->n * I->n - I->l - (int32_t)fstar;
    if (final_pop && nv > 0) memcpy(final_pop, P, PV);

    free(P); free(Pp); free(SO); free(Pn); free(Sstar); free(eall); free(eP); free(Dm);
    free(Dall); free(Dx); free(sel); free(partner); free(uid); free(uidn); free(tested);
    free(testedn); free(tcount); free(tcountn);
    return g_done;
}
