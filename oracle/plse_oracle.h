/*
 * plse_oracle.h -- plain, slow CPU oracle for the MPMA hot path
 * (Goudet & Hao, "A massively parallel evolutionary algorithm for the partial
 * Latin square extension problem", arXiv 2103.10453).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it, and the two share no code:
 * this header is included by the oracle alone.
 *
 * Every routine is a direct, unoptimised restatement of one passage of the
 * paper (cited at each declaration).  All arithmetic is integer; the penalty
 * function F = f + phi*c (Sec. 3.1) is carried as F2 = 2F so that phi = 1/2 and
 * phi = |V| are both exact.
 *
 * Parity pins (tests/test_oracle_*.py): the n = 3 worked example of Sec. 2.2
 * (l = 1, bound 7), brute-force optima for n <= 5, closed forms of AUX
 * (Sec. 3.5.2), Alg. 4 spacing/elitism invariants, from-scratch recomputation of
 * the gamma table and of F after every move (debug mode), and the cuRAND host
 * Philox4x32-10 stream.  The whole-run heuristic trajectory has no external
 * value to compare with ("parity unpinned" for the paper's benchmark scores,
 * whose instances are not available).
 */
#ifndef PLSE_ORACLE_H
#define PLSE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Algorithm parameters (Table 1 and Sec. 3.3; integer forms of the reals). */
typedef struct {
    int32_t alpha_num, alpha_den;  /* tenure factor alpha = 6/10              */
    int32_t tenure_rand;           /* L uniform in [0, tenure_rand) = [0, 9]   */
    int32_t phase1_phi2;           /* 2*phi in phase 1 (phi = 0.5 -> 1)        */
    int32_t phase2_phi2_per_v;     /* 2*phi = this * |V| in phase 2 (phi=|V|)  */
    int32_t phase2_iter_per_v;     /* phase-2 iterations = this * |V| (2)      */
    int32_t spacing_gamma;         /* Alg. 4 spacing D > |V| / gamma (10)      */
    int32_t beta;                  /* AUX parameter beta (20)                  */
    int32_t mode;                  /* 0 = PLITS two-phase, 1 = PartialCol      */
    int32_t matching;              /* 0 = nearest untested, 1 = random         */
    int32_t crossover;             /* 0 = AUX, 1 = UX (p_ij = 1/2)             */
    int32_t tested_cap;            /* capacity of each tested-partner list     */
} or_params;

/* Per-walk work counters (the trajectory-dependent terms of the byte count). */
typedef struct {
    int64_t iterations;   /* iterations executed (early stop excluded)        */
    int64_t moves;        /* moves applied                                    */
    int64_t cand;         /* sum over iterations of |V0 u C(S)|               */
    int64_t pairs;        /* sum over iterations of scanned (v, j) pairs      */
    int64_t deg;          /* sum over applied moves of deg(v*)                */
    int64_t improvements; /* strict improvements of the walk's best           */
    int64_t uncolored;    /* PartialCol: neighbours uncoloured by moves       */
} or_stats;

void or_default_params(or_params *p);

/* Philox4x32-10 (Salmon et al., SC'11), written from its published definition. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Instance -> reduced graph (Sec. 2.1-2.2, Alg. 1).  Returns NULL and *err < 0
 * on an invalid grid (-1: bad n, -2: symbol out of range, -3: repeated symbol). */
void *or_create(int32_t n, const int8_t *grid, int32_t *err);
void  or_destroy(void *h);
void  or_info(const void *h, int32_t *n, int32_t *nv, int32_t *l, int32_t *ub, int32_t *nfixed);
void  or_vertices(const void *h, int32_t *cell);      /* [nv] row-major cell   */
void  or_domains(const void *h, uint8_t *dom);        /* [nv*(n+1)] 0/1        */
int64_t or_num_edges(const void *h);

/* f, c and F2 = 2f + phi2*c of a colouring (Eq. 1, 3, 5). */
int64_t or_eval(const void *h, const uint8_t *S, int32_t phi2, int64_t *f, int64_t *c);
/* gamma[v][k] = #neighbours of v with colour k (k >= 1), from scratch. */
void or_gamma(const void *h, const uint8_t *S, int32_t *gamma);
/* Number of conflicting vertices |C(S)| (Sec. 3.3). */
int64_t or_num_conflicting(const void *h, const uint8_t *S);

/* Random initial population (Sec. 3.2): S(v) uniform over D(v) \ {0}. */
void or_init_population(const void *h, int32_t p, uint64_t seed, uint8_t *P);

/* One tabu walk (Alg. 3).  phase 1 / 2 = PLITS with phi2 of that phase;
 * phase 3 = PartialCol (legal partial colourings, Sec. 3.7).  S: in = start,
 * out = best colouring found (S'*).  Returns F2 (PartialCol: f) of that best.
 * debug != 0 re-derives gamma, F and admissibility from scratch after every
 * move and returns -1 at the first disagreement. */
int64_t or_tabu_walk(const void *h, const or_params *prm, uint8_t *S,
                     int32_t ind, int32_t gen, int32_t phase, int64_t iters,
                     uint64_t seed, int32_t debug, or_stats *st);
/* As or_tabu_walk, also recording the move chosen at every iteration executed:
 * trace[3*(t-1) .. 3*(t-1)+2] = (v, colour before, colour after), or (-1, -1, -1)
 * for an iteration without an admissible move.  trace holds 3*iters int32
 * (entries past the last executed iteration are left untouched). */
int64_t or_tabu_walk_traced(const void *h, const or_params *prm, uint8_t *S,
                            int32_t ind, int32_t gen, int32_t phase, int64_t iters,
                            uint64_t seed, int32_t debug, or_stats *st, int32_t *trace);

/* Greedy conflict removal (Sec. 3.7): returns the number of vertices uncoloured. */
int32_t or_repair(const void *h, uint8_t *S);

/* Hamming distances (Sec. 3.4): D[a*nb+b] = #v with A_a(v) != B_b(v). */
void or_distances(const void *h, const uint8_t *A, int32_t na,
                  const uint8_t *B, int32_t nb, int32_t *D);

/* Alg. 4 over P_all = P (0..p-1) followed by P' (p..2p-1); Dall is the 2p x 2p
 * distance matrix of P_all and e[2p] the ranking scores.  Writes the p chosen
 * indices in acceptance order; returns how many were taken by the fill rule. */
int32_t or_pop_update(const void *h, const or_params *prm, int32_t p,
                      const int64_t *e, const int32_t *Dall, int32_t *sel);

/* Parent matching (Sec. 3.5.1, Alg. 5).  D: p x p of the new population;
 * uid[p]; tested[p*cap] with tcount[p] entries (oldest dropped when full).
 * Writes partner[p] and appends the partner uids to the lists. */
void or_matching(const void *h, const or_params *prm, int32_t p, const int32_t *D,
                 const uint32_t *uid, uint32_t *tested, int32_t *tcount,
                 int32_t gen, uint64_t seed, int32_t *partner);

/* AUX / UX crossover (Eq. 10, Alg. 5): offspring O[i] from (P[i], P[partner[i]]). */
void or_crossover(const void *h, const or_params *prm, int32_t p, const uint8_t *P,
                  const int32_t *partner, const int32_t *D, int32_t gen,
                  uint64_t seed, uint8_t *O);

/* Whole MPMA run (Alg. 2).  best_grid: n*n output; trace[generations] receives
 * f* after each generation (may be NULL).  Returns generations executed. */
int32_t or_solve(const void *h, const or_params *prm, int32_t p, int32_t generations,
                 int64_t iters, uint64_t seed, int8_t *best_grid, int32_t *best_score,
                 int32_t *trace, or_stats *st, uint8_t *final_pop);

#ifdef __cplusplus
}
#endif
#endif
