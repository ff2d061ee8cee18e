/*
 * perm_oracle.h -- plain, slow, single-threaded CPU reference for interacting
 * flatPERM on Z^d (d = 2, 3).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this library: only tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or constant generator with
 * the CUDA path.
 *
 * Paper: S. Campbell and E. J. Janse van Rensburg, "Parallel PERM".
 *   Sec. 1, eqs. (1)-(4): Rosenbluth growth, weight W = prod a_+, counting
 *                         theorem, sample average <W_n> = sum W_n / M.
 *   Sec. 2, eq. (6) and the text after it: flatPERM ratio r, enrichment,
 *                         pruning.
 *   Sec. 3, Algorithms 1 and 2 and Fig. 1: N sequences with private tables
 *                         (Alg. 1) or one shared table W (Alg. 2).
 *
 * Parity status of each function is stated in oracle/perm_oracle.c.
 */
#ifndef PERM_ORACLE_H
#define PERM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_EOVERFLOW = -3 };
enum { ORC_ALG2 = 2, ORC_ALG1 = 1 };
/* outcome of one node */
enum { ORC_LEAF_NMAX = 0, ORC_LEAF_TRAPPED = 1, ORC_LEAF_PRUNED = 2, ORC_CHILDREN = 3 };

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the paper. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Exact number c_k of self-avoiding walks of length k on Z^d, k = 0..n, by
 * depth-first enumeration.  Returns ORC_OK or ORC_EINVAL. */
int orc_enumerate(int d, int n, int64_t *c_out);
/* Same, and r2_out[k] = sum over those walks of the squared end-to-end distance. */
int orc_enumerate_r2(int d, int n, int64_t *c_out, int64_t *r2_out);

/* Power-of-two scale exponent E(n) of the stored weight (stored = W / 2^E(n)). */
int orc_scale_exp(int d, int n);

/* The ratio r = W / [W_n]^sample of Sec. 2 (eq. 6) in double precision, from
 * the node weight W, the sum Wsum of the weights recorded at length n before
 * this node and the number M of tours started: [W_n]^sample = (Wsum + W)/M
 * (own weight included).  n == 0 gives 1. */
double orc_ratio(int n, double W, double Wsum, int64_t M);

/* One node of the growth step on a snapshot state (walk coordinates given).
 * coords: (n+1)*d int32, site k at coords[k*d .. k*d+d-1], site 0 = origin.
 * W: the node's weight; Wsum: the sum of the weights recorded at length n
 * before it; M: tours started (both at the stored scale of length n).
 * Outputs: a_plus, free_mask (bit j = direction j free; order +x,-x,+y,-y,+z,-z),
 * r, c (children), dirs[0..c-1], child weight (stored scale of length n+1).
 * Returns the outcome code. */
int orc_step(int d, int n_max, int n, const int32_t *coords, double W, double Wsum,
             int64_t M, uint64_t ordinal, uint32_t seq, uint32_t tour,
             uint64_t seed, uint32_t run,
             int *a_plus, int *free_mask, double *r, int *c, int *dirs,
             double *child_w);

typedef struct orc_state orc_state;

/* A flatPERM simulation: d, n_max, N sequences, seed, run id, algorithm. */
int orc_create(orc_state **out, int d, int n_max, int n_seq, uint64_t seed,
               uint32_t run, int alg);
/* Original PERM with cut-offs (Sec. 2): from now on a node of length n >= 1 and
 * weight W > T_hi[n] is enriched into `copies` copies (distinct steps, at most
 * a_+, each W/c), one with W < t_lo[n] survives with probability 1/q (u0 < 1/q
 * in double precision) and then carries q W; the shared table no longer decides.
 * T_hi, t_lo: n_max+1 doubles at the stored scale, copied.  copies in
 * 1..2d, q >= 1.  Both NULL: back to flatPERM. */
int orc_set_cutoffs(orc_state *h, const double *T_hi, const double *t_lo, int copies, double q);
/* Continue the simulation by tours_per_seq tours of every sequence. */
int orc_run(orc_state *h, int64_t tours_per_seq);
/* The same on `threads` host threads sharing the table (Sec. 3, Algorithm 2 as
 * the paper ran it: threads take tour tickets, tables updated atomically and
 * read as they are at each node).  Algorithm 2 and flatPERM only (ORC_EINVAL
 * otherwise).  Not reproducible node by node: the interleaving decides. */
int orc_run_threads(orc_state *h, int64_t tours_per_seq, int threads);
/* Raw tables (stored scale): W_n, S_n, Q_n over n = 0..n_max (Alg. 2), or the
 * per-sequence rows concatenated (Alg. 1); M (tours started, per sequence for
 * Alg. 1 in M_out[0..N-1]); steps = nodes processed; max stack depth. */
int orc_tables(const orc_state *h, double *Wn, double *Sn, double *Qn,
               int64_t *M_out, int64_t *steps, int64_t *max_stack);
/* Estimates: log c_n (natural log), S_n, relative variance of c_n. */
int orc_estimates(const orc_state *h, double *log_cn, double *S_n, double *relvar_n);
/* Raw table of sum W |omega_n|^2 per length (eq. 5 numerator; stored scale),
 * rows as in orc_tables.  <R^2>_n = R_n / W_n (eq. 5). */
int orc_observable_r2(const orc_state *h, double *Rn);
void orc_destroy(orc_state *h);

#ifdef __cplusplus
}
#endif
#endif
