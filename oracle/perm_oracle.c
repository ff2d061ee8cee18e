/*
 * perm_oracle.c -- plain, slow, single-threaded CPU reference for interacting
 * flatPERM on the square (d = 2) and cubic (d = 3) lattices.
 *
 * TEST INFRASTRUCTURE ONLY: tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it; the product path never does.  It shares no code with
 * the CUDA path.  Build with -ffp-contract=off so that no multiply-add is fused
 * (every floating-point operation below is one IEEE round-to-nearest step).
 *
 * Paper: Campbell and Janse van Rensburg, "Parallel PERM".
 *
 * What each part follows, and how it is pinned (tests under tests/):
 *  - orc_philox4x32_10: Philox4x32 with 10 rounds, from Salmon et al.,
 *    "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  Pinned by the
 *    published known-answer vectors (tests/golden/philox4x32_10_kat.txt).
 *  - orc_enumerate: c_n by brute-force depth-first enumeration of all
 *    self-avoiding walks (the quantity of Sec. 1, eq. 3).  Pinned by closed
 *    forms for n <= 4, by an independent pure-Python brute force for small n,
 *    and by lattice symmetry.
 *  - node growth (orc_step / the run loop): Rosenbluth growth (Sec. 1, eqs.
 *    1-2), flatPERM ratio, enrichment and pruning (Sec. 2, eq. 6 and the
 *    paragraphs after it).  Pinned by exact c_0..c_3 in every run, by the
 *    counting theorem (Sec. 1, eq. 3: estimates within 4 sigma of the exact
 *    c_n from orc_enumerate), by weight conservation under enrichment and
 *    pruning, by the probabilities of the enrichment count and of survival,
 *    by the uniformity of the chosen directions, and by r = 1 wherever the
 *    own weight is the whole sum in the first tour.
 *  - original PERM with cut-offs (orc_set_cutoffs; Sec. 2, the paragraphs on
 *    T_k, t_k and q): pinned by its special cases -- no cut-off active is the
 *    Rosenbluth method (one sample per length per tour, exact c_2 and c_3 per
 *    tour); always enrich gives the deterministic tree of 2^(n-1) samples with
 *    exact c_2, c_3; always prune makes the survivors at n = 2 binomial with
 *    probability 1/q and each carry exactly q 12 -- and by the counting
 *    theorem with cut-offs active on both sides.
 *  - variance estimate: per-tour sums (the paper gives no error bars); pinned
 *    by the z-score calibration of the estimates against exact c_n over many
 *    seeds.
 *
 * Readings of the paper taken here:
 *  - The weight entering r is W(omega_k) before multiplication by
 *    a_+(omega_k); the children carry W'.a_+ (Sec. 2 with eq. 2).
 *  - M counts every tour started so far, the current one included; the own
 *    weight is included in the running average (Sec. 2; Sec. 3, Alg. 2).
 *  - r is 1 at the empty walk, so every tour has exactly one node of length 0
 *    and one of length 1.
 *  - r is the paper's definition evaluated in double precision:
 *    [W_n]^sample = (sum of the earlier weights at length n + W) / M and
 *    r = W / [W_n]^sample; u0 = w0 2^-32 is exact in double precision, and
 *    every comparison below is taken on these doubles.
 *  - Enriched copies take distinct steps, c is capped at a_+, each child has
 *    weight (W/c).a_+.  A survivor of pruning has its weight multiplied by
 *    1/r (Sec. 2).
 *  - Random numbers: one Philox4x32-10 block per node, counter = (DFS ordinal
 *    of the node within its tour, 64 bit; tour index; sequence index), key =
 *    (low seed word XOR run id, high seed word).  Word 0 decides c (or
 *    survival), word 1 picks the c distinct directions by a partial
 *    Fisher-Yates shuffle with batched multiply-high draws.
 *  - Directions are ordered +x, -x, +y, -y, +z, -z; the first chosen child is
 *    grown first and the others wait on the stack in order.
 *  - Weights are stored divided by 2^E(n), E(n) = floor(11n/8) (d = 2) or
 *    floor(9n/4) (d = 3), so that they stay inside the double range at long
 *    lengths; r is scale free and log c_n adds E(n) log 2 back.
 *  - Alg. 2 executed by one thread runs the tours of all sequences one after
 *    another; tour g (counted from 0) belongs to sequence g mod N, tour g div N.
 */
#include "perm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 3 and its Table 2 constants).    */
/* One round: two 32x32->64 multiplies of words 0 and 2; the high halves are  */
/* XORed with the other words and the round key, words are permuted.  The key */
/* is bumped by the Weyl constants between rounds.                            */
/* ------------------------------------------------------------------------- */
#define PHILOX_M4x32_0 0xD2511F53u
#define PHILOX_M4x32_1 0xCD9E8D57u
#define PHILOX_W32_0 0x9E3779B9u
#define PHILOX_W32_1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W32_0;
            k1 += PHILOX_W32_1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M4x32_0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M4x32_1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Exact enumeration (Sec. 1: c_n, the number of n-step self-avoiding walks). */
/* ------------------------------------------------------------------------- */
static void enum_rec(int d, int n, int depth, int *pos, unsigned char *occ,
                     const long *stride, int64_t *c, int64_t *r2) {
    c[depth] += 1;
    if (r2) {
        int64_t s = 0;
        for (int i = 0; i < d; ++i) s += (int64_t)pos[i] * pos[i];
        r2[depth] += s;
    }
    if (depth == n) return;
    for (int axis = 0; axis < d; ++axis) {
        for (int sgn = 1; sgn >= -1; sgn -= 2) {
            pos[axis] += sgn;
            long idx = 0;
            for (int i = 0; i < d; ++i) idx += (long)(pos[i] + n + 1) * stride[i];
            if (!occ[idx]) {
                occ[idx] = 1;
                enum_rec(d, n, depth + 1, pos, occ, stride, c, r2);
                occ[idx] = 0;
            }
            pos[axis] -= sgn;
        }
    }
}

int orc_enumerate(int d, int n, int64_t *c_out) { return orc_enumerate_r2(d, n, c_out, NULL); }

/* c_k and the sum over all walks of length k of the squared end-to-end distance
 * |omega_k - omega_0|^2 (the observable of Sec. 1, eq. 5), k = 0..n. */
int orc_enumerate_r2(int d, int n, int64_t *c_out, int64_t *r2_out) {
    if ((d != 2 && d != 3) || n < 0 || n > 24 || !c_out) return ORC_EINVAL;
    long side = 2L * n + 3;
    long total = 1, stride[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) { stride[i] = total; total *= side; }
    unsigned char *occ = (unsigned char *)calloc((size_t)total, 1);
    if (!occ) return ORC_ENOMEM;
    int pos[3] = {0, 0, 0};
    for (int k = 0; k <= n; ++k) { c_out[k] = 0; if (r2_out) r2_out[k] = 0; }
    long origin = 0;
    for (int i = 0; i < d; ++i) origin += (long)(n + 1) * stride[i];
    occ[origin] = 1;
    enum_rec(d, n, 0, pos, occ, stride, c_out, r2_out);
    free(occ);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Weight scale and the ratio r.                                              */
/* ------------------------------------------------------------------------- */
int orc_scale_exp(int d, int n) { return d == 2 ? (11 * n) / 8 : (9 * n) / 4; }

/* r = W / [W_n]^sample (Sec. 2, eq. 6), the running average of the weights
 * of length n including the node's own weight W: [W_n]^sample =
 * (Wsum + W) / M, where Wsum is the sum of the weights recorded at length n
 * before this node and M the number of tours started.  The empty walk has
 * r = 1 (every tour then visits lengths 0 and 1 exactly once). */
double orc_ratio(int n, double W, double Wsum, int64_t M) {
    if (n == 0) return 1.0;
    double avg = (Wsum + W) / (double)M;
    return W / avg;
}

/* ------------------------------------------------------------------------- */
/* Occupancy of the current walk: a dense byte box when it is small enough,   */
/* else a linear scan of the walk's sites.                                    */
/* ------------------------------------------------------------------------- */
typedef struct {
    int d, n_max;
    long side, stride[3];
    unsigned char *box;     /* NULL => linear scan */
    const int32_t *coords;  /* walk sites, (n+1)*d */
    int n;                  /* current endpoint index (for the scan) */
} occset;

static int occ_init(occset *o, int d, int n_max) {
    o->d = d; o->n_max = n_max; o->box = NULL; o->coords = NULL; o->n = -1;
    o->side = 2L * n_max + 3;
    long total = 1;
    for (int i = 0; i < d; ++i) { o->stride[i] = total; total *= o->side; }
    if (total <= (1L << 26)) {
        o->box = (unsigned char *)calloc((size_t)total, 1);
        if (!o->box) return ORC_ENOMEM;
    }
    return ORC_OK;
}

static long occ_index(const occset *o, const int32_t *p) {
    long idx = 0;
    for (int i = 0; i < o->d; ++i) idx += (long)(p[i] + o->n_max + 1) * o->stride[i];
    return idx;
}

static int occ_has(const occset *o, const int32_t *p) {
    if (o->box) return o->box[occ_index(o, p)];
    for (int k = 0; k <= o->n; ++k) {
        int same = 1;
        for (int i = 0; i < o->d; ++i) same &= (o->coords[k * o->d + i] == p[i]);
        if (same) return 1;
    }
    return 0;
}

static void occ_set(occset *o, const int32_t *p, unsigned char v) {
    if (o->box) o->box[occ_index(o, p)] = v;
}

/* unit step j: axis j/2, sign + for even j */
static void add_step(int d, const int32_t *from, int j, int32_t *to) {
    for (int i = 0; i < d; ++i) to[i] = from[i];
    to[j >> 1] += (j & 1) ? -1 : 1;
}

/* ------------------------------------------------------------------------- */
/* One node: a_+, r, the enrichment/pruning decision, the distinct steps and  */
/* the children's weight (Sec. 1 eqs. 1-2; Sec. 2).                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int a_plus, free_mask, c, dirs[6];
    double r;
    double child_w;
} node_out;

/* Original PERM (Sec. 2, the cut-offs T_k and t_k): a node of weight W above
 * T_n is enriched into `copies` copies, each with its weight divided by the
 * number made; one below t_n is pruned with probability 1 - 1/q and otherwise
 * has its weight multiplied by q.  Cut-offs are at the stored weight scale.
 * Readings: the copies take distinct steps, at most a_+ of them (as flatPERM's
 * copies); the survival test compares u0 with 1/q in double precision; the
 * empty walk is neither enriched nor pruned. */
typedef struct {
    const double *hi, *lo;   /* T_n and t_n, n = 0..n_max */
    int copies;
    double q;
} perm_cuts;

static int grow_node(int d, int n_max, int n, const int32_t *end, const occset *occ,
                     double W, double Wsum, int64_t M, uint64_t ordinal, uint32_t seq,
                     uint32_t tour, uint64_t seed, uint32_t run, const perm_cuts *cuts,
                     node_out *o) {
    o->a_plus = 0; o->free_mask = 0; o->c = 0; o->r = 0.0; o->child_w = 0.0;
    if (n == n_max) return ORC_LEAF_NMAX;                     /* walk complete */

    /* a_+: the free neighbours of the end-point (Sec. 1) */
    int free_list[6], a = 0;
    for (int j = 0; j < 2 * d; ++j) {
        int32_t nb[3];
        add_step(d, end, j, nb);
        if (!occ_has(occ, nb)) {
            free_list[a++] = j;
            o->free_mask |= 1 << j;
        }
    }
    o->a_plus = a;
    if (a == 0) return ORC_LEAF_TRAPPED;                       /* trapped: weight 0 beyond */

    /* the node's random block; u0 = w0 / 2^32 (exact in double precision) */
    uint32_t ctr[4] = {(uint32_t)ordinal, (uint32_t)(ordinal >> 32), tour, seq};
    uint32_t key[2] = {(uint32_t)seed ^ run, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double u0 = (double)w[0] * (1.0 / 4294967296.0);

    int c;
    double Wp;
    if (cuts && n > 0) {
        /* original PERM (Sec. 2): enrich above T_n, prune below t_n, else one copy */
        if (W > cuts->hi[n]) {
            o->r = (double)cuts->copies;
            c = cuts->copies < a ? cuts->copies : a;          /* distinct steps: at most a_+ */
            Wp = W / (double)c;
        } else if (W < cuts->lo[n]) {
            o->r = 1.0 / cuts->q;
            if (!(u0 < 1.0 / cuts->q)) return ORC_LEAF_PRUNED;   /* pruned w.p. 1 - 1/q */
            c = 1;
            Wp = W * cuts->q;                                     /* weight increased by q */
        } else {
            o->r = 1.0;
            c = 1;
            Wp = W;
        }
    } else {
        /* flatPERM (Sec. 2, eq. 6 and the two paragraphs after it) */
        double r = orc_ratio(n, W, Wsum, M);
        o->r = r;
        if (r >= 1.0) {
            /* enrichment: p = ceil(r) - r; c = floor(r) with probability p, else ceil(r) */
            double fl = floor(r), ce = ceil(r);
            double p = ce - r;
            double c_raw = (u0 < p) ? fl : ce;
            c = (c_raw >= (double)a) ? a : (int)c_raw;        /* distinct steps: at most a_+ */
            Wp = W / (double)c;                               /* each copy carries W/c */
        } else {
            /* pruning with probability 1 - r; a survivor's weight times 1/r */
            if (!(u0 < r)) return ORC_LEAF_PRUNED;
            c = 1;
            Wp = W * (1.0 / r);
        }
    }

    /* c distinct directions: partial Fisher-Yates over the free list, draws from word 1 */
    uint32_t x = w[1];
    for (int i = 0; i < c; ++i) {
        uint32_t m = (uint32_t)(a - i);
        uint64_t prod = (uint64_t)x * m;
        int j = i + (int)(prod >> 32);
        x = (uint32_t)prod;
        int tmp = free_list[i]; free_list[i] = free_list[j]; free_list[j] = tmp;
    }
    for (int i = 0; i < c; ++i) o->dirs[i] = free_list[i];
    o->c = c;
    /* each child: W' a_+ (eq. 2), stored at the scale of length n+1 */
    int dE = orc_scale_exp(d, n + 1) - orc_scale_exp(d, n);
    o->child_w = ldexp(Wp * (double)a, -dE);
    return ORC_CHILDREN;
}

int orc_step(int d, int n_max, int n, const int32_t *coords, double W, double Wsum,
             int64_t M, uint64_t ordinal, uint32_t seq, uint32_t tour,
             uint64_t seed, uint32_t run,
             int *a_plus, int *free_mask, double *r, int *c, int *dirs,
             double *child_w) {
    if ((d != 2 && d != 3) || n < 0 || n > n_max || n_max < 1 || !coords || M < 1)
        return ORC_EINVAL;
    /* the snapshot must be a self-avoiding walk from the origin */
    for (int i = 0; i < d; ++i) if (coords[i] != 0) return ORC_EINVAL;
    for (int k = 1; k <= n; ++k) {
        int dist = 0;
        for (int i = 0; i < d; ++i) dist += abs(coords[k * d + i] - coords[(k - 1) * d + i]);
        if (dist != 1) return ORC_EINVAL;
        for (int l = 0; l < k; ++l) {
            int same = 1;
            for (int i = 0; i < d; ++i) same &= (coords[k * d + i] == coords[l * d + i]);
            if (same) return ORC_EINVAL;
        }
    }
    occset occ;
    occ.d = d; occ.n_max = n_max; occ.box = NULL; occ.coords = coords; occ.n = n;
    node_out o;
    int rc = grow_node(d, n_max, n, coords + (long)n * d, &occ, W, Wsum, M, ordinal, seq,
                       tour, seed, run, NULL, &o);
    if (a_plus) *a_plus = o.a_plus;
    if (free_mask) *free_mask = o.free_mask;
    if (r) *r = o.r;
    if (c) *c = o.c;
    if (dirs) for (int i = 0; i < o.c; ++i) dirs[i] = o.dirs[i];
    if (child_w) *child_w = o.child_w;
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Simulation state: the shared table W (Alg. 2) or one table per sequence    */
/* (Alg. 1), the running walk, and the stack of waiting copies.               */
/* ------------------------------------------------------------------------- */
typedef struct { int depth, dir; double w; } stack_rec;

struct orc_state {
    int d, n_max, n_seq, alg;
    uint64_t seed;
    uint32_t run;
    int ntab;              /* 1 (Alg. 2) or n_seq (Alg. 1) */
    double *Wn, *Qn;       /* ntab * (n_max+1) */
    double *Rn;            /* ntab * (n_max+1): sum of W |omega_n|^2 (eq. 5 numerator) */
    int64_t *Sn;           /* ntab * (n_max+1) */
    int64_t *M;            /* ntab: tours started */
    int64_t *tours_done;   /* n_seq (Alg. 1); [0] counts tickets for Alg. 2 */
    double *X;             /* n_max+1: this tour's weight per length */
    int32_t *coords;       /* (n_max+1)*d */
    stack_rec *stack;
    long stack_cap;
    occset occ;
    int64_t steps, max_stack;
    double *cut_hi, *cut_lo;   /* original PERM's cut-offs (NULL: flatPERM) */
    perm_cuts cuts;
};

void orc_destroy(orc_state *h) {
    if (!h) return;
    free(h->Wn); free(h->Qn); free(h->Rn); free(h->Sn); free(h->M); free(h->tours_done);
    free(h->X); free(h->coords); free(h->stack); free(h->occ.box);
    free(h->cut_hi); free(h->cut_lo);
    free(h);
}

int orc_create(orc_state **out, int d, int n_max, int n_seq, uint64_t seed,
               uint32_t run, int alg) {
    if (!out) return ORC_EINVAL;
    *out = NULL;
    if ((d != 2 && d != 3) || n_max < 1 || n_max > 100000 || n_seq < 1 ||
        (alg != ORC_ALG1 && alg != ORC_ALG2))
        return ORC_EINVAL;
    orc_state *h = (orc_state *)calloc(1, sizeof(orc_state));
    if (!h) return ORC_ENOMEM;
    h->d = d; h->n_max = n_max; h->n_seq = n_seq; h->alg = alg; h->seed = seed; h->run = run;
    h->ntab = (alg == ORC_ALG1) ? n_seq : 1;
    size_t L = (size_t)n_max + 1;
    h->Wn = (double *)calloc(L * h->ntab, sizeof(double));
    h->Qn = (double *)calloc(L * h->ntab, sizeof(double));
    h->Rn = (double *)calloc(L * h->ntab, sizeof(double));
    h->Sn = (int64_t *)calloc(L * h->ntab, sizeof(int64_t));
    h->M = (int64_t *)calloc((size_t)h->ntab, sizeof(int64_t));
    h->tours_done = (int64_t *)calloc((size_t)n_seq, sizeof(int64_t));
    h->X = (double *)calloc(L, sizeof(double));
    h->coords = (int32_t *)calloc(L * d, sizeof(int32_t));
    h->stack_cap = (long)n_max * (2 * d - 2) + 2 * d;
    h->stack = (stack_rec *)calloc((size_t)h->stack_cap, sizeof(stack_rec));
    if (!h->Wn || !h->Qn || !h->Rn || !h->Sn || !h->M || !h->tours_done || !h->X || !h->coords ||
        !h->stack || occ_init(&h->occ, d, n_max) != ORC_OK) {
        orc_destroy(h);
        return ORC_ENOMEM;
    }
    h->occ.coords = h->coords;
    *out = h;
    return ORC_OK;
}

/* One tour: start at the empty walk and grow depth first until every copy has
 * ended (Sec. 2).  M is the number of tours started on this table, this one
 * included (Sec. 1, eq. 4; Sec. 3, Alg. 2). */
static int run_tour(orc_state *h, int tab, uint32_t seq, uint32_t tour, int64_t M) {
    const int d = h->d, n_max = h->n_max;
    double *Wn = h->Wn + (size_t)tab * (n_max + 1);
    double *Qn = h->Qn + (size_t)tab * (n_max + 1);
    double *Rn = h->Rn + (size_t)tab * (n_max + 1);
    int64_t *Sn = h->Sn + (size_t)tab * (n_max + 1);
    int32_t *co = h->coords;
    long sp = 0;
    int n = 0;
    double W = 1.0;
    uint64_t ordinal = 0;
    for (int i = 0; i < d; ++i) co[i] = 0;
    h->occ.n = 0;
    occ_set(&h->occ, co, 1);
    for (;;) {
        /* the sum of the earlier weights at this length, then accumulate the
         * node (eq. 4) */
        double Wsum = Wn[n];
        Wn[n] += W;
        Sn[n] += 1;
        h->X[n] += W;
        {   /* the observable |omega_n|^2 weighted by W (Sec. 1, eq. 5) */
            int64_t r2 = 0;
            for (int i = 0; i < d; ++i) {
                const int64_t x = co[(long)n * d + i];
                r2 += x * x;
            }
            Rn[n] += W * (double)r2;
        }
        h->steps += 1;
        node_out o;
        int rc = grow_node(d, n_max, n, co + (long)n * d, &h->occ, W, Wsum, M, ordinal,
                           seq, tour, h->seed, h->run, h->cut_hi ? &h->cuts : NULL, &o);
        ordinal += 1;
        if (rc == ORC_CHILDREN) {
            /* copies 1..c-1 wait on the stack (copy 1 on top); copy 0 grows now */
            for (int i = o.c - 1; i >= 1; --i) {
                if (sp >= h->stack_cap) return ORC_EOVERFLOW;
                h->stack[sp].depth = n;
                h->stack[sp].dir = o.dirs[i];
                h->stack[sp].w = o.child_w;
                ++sp;
            }
            if (sp > h->max_stack) h->max_stack = sp;
            add_step(d, co + (long)n * d, o.dirs[0], co + (long)(n + 1) * d);
            n += 1;
            h->occ.n = n;
            occ_set(&h->occ, co + (long)n * d, 1);
            W = o.child_w;
            continue;
        }
        /* leaf: resume the most recent waiting copy, or end the tour */
        if (sp == 0) break;
        --sp;
        int dp = h->stack[sp].depth;
        for (int k = n; k > dp; --k) occ_set(&h->occ, co + (long)k * d, 0);
        add_step(d, co + (long)dp * d, h->stack[sp].dir, co + (long)(dp + 1) * d);
        n = dp + 1;
        h->occ.n = n;
        occ_set(&h->occ, co + (long)n * d, 1);
        W = h->stack[sp].w;
    }
    for (int k = n; k >= 0; --k) occ_set(&h->occ, co + (long)k * d, 0);
    h->occ.n = -1;
    /* per-tour sums for the variance estimate */
    for (int k = 0; k <= n_max; ++k) {
        Qn[k] += h->X[k] * h->X[k];
        h->X[k] = 0.0;
    }
    return ORC_OK;
}

int orc_set_cutoffs(orc_state *h, const double *T_hi, const double *t_lo, int copies, double q) {
    if (!h) return ORC_EINVAL;
    free(h->cut_hi); free(h->cut_lo);
    h->cut_hi = h->cut_lo = NULL;
    if (!T_hi && !t_lo) return ORC_OK;                         /* back to flatPERM */
    if (!T_hi || !t_lo || copies < 1 || copies > 2 * h->d || !(q >= 1.0) || q > 4294967296.0)
        return ORC_EINVAL;
    size_t L = (size_t)h->n_max + 1;
    h->cut_hi = (double *)malloc(L * sizeof(double));
    h->cut_lo = (double *)malloc(L * sizeof(double));
    if (!h->cut_hi || !h->cut_lo) {
        free(h->cut_hi); free(h->cut_lo);
        h->cut_hi = h->cut_lo = NULL;
        return ORC_ENOMEM;
    }
    memcpy(h->cut_hi, T_hi, L * sizeof(double));
    memcpy(h->cut_lo, t_lo, L * sizeof(double));
    h->cuts.hi = h->cut_hi;
    h->cuts.lo = h->cut_lo;
    h->cuts.copies = copies;
    h->cuts.q = q;
    return ORC_OK;
}

int orc_run(orc_state *h, int64_t tours_per_seq) {
    if (!h || tours_per_seq < 0) return ORC_EINVAL;
    if (h->alg == ORC_ALG2) {
        /* Alg. 2 run by one thread: all sequences' tours in ticket order */
        int64_t first = h->M[0], last = h->M[0] + tours_per_seq * (int64_t)h->n_seq;
        for (int64_t g = first; g < last; ++g) {
            uint32_t seq = (uint32_t)(g % h->n_seq), tour = (uint32_t)(g / h->n_seq);
            h->M[0] = g + 1;
            int rc = run_tour(h, 0, seq, tour, h->M[0]);
            if (rc != ORC_OK) return rc;
        }
        h->tours_done[0] = h->M[0];
    } else {
        /* Alg. 1: every sequence against its own table */
        for (int s = 0; s < h->n_seq; ++s) {
            for (int64_t i = 0; i < tours_per_seq; ++i) {
                int64_t t = h->tours_done[s];
                h->M[s] = t + 1;
                int rc = run_tour(h, s, (uint32_t)s, (uint32_t)t, h->M[s]);
                if (rc != ORC_OK) return rc;
                h->tours_done[s] = t + 1;
            }
        }
    }
    return ORC_OK;
}

int orc_tables(const orc_state *h, double *Wn, double *Sn, double *Qn,
               int64_t *M_out, int64_t *steps, int64_t *max_stack) {
    if (!h) return ORC_EINVAL;
    size_t L = (size_t)(h->n_max + 1) * h->ntab;
    for (size_t i = 0; i < L; ++i) {
        if (Wn) Wn[i] = h->Wn[i];
        if (Sn) Sn[i] = (double)h->Sn[i];
        if (Qn) Qn[i] = h->Qn[i];
    }
    if (M_out) for (int t = 0; t < h->ntab; ++t) M_out[t] = h->M[t];
    if (steps) *steps = h->steps;
    if (max_stack) *max_stack = h->max_stack;
    return ORC_OK;
}

/* The raw table sum of W |omega_n|^2 (stored scale), rows as in orc_tables. */
int orc_observable_r2(const orc_state *h, double *Rn) {
    if (!h || !Rn) return ORC_EINVAL;
    size_t L = (size_t)(h->n_max + 1) * h->ntab;
    for (size_t i = 0; i < L; ++i) Rn[i] = h->Rn[i];
    return ORC_OK;
}

/* log c_n from <W_n> = W_n / M (eq. 4; Alg. 1 averages the sequences' own
 * estimates, eq. 7), S_n, and the relative variance of the estimate from the
 * per-tour sums: var = (Q/M - c^2)/(M - 1). */
int orc_estimates(const orc_state *h, double *log_cn, double *S_n, double *relvar_n) {
    if (!h) return ORC_EINVAL;
    const int L = h->n_max + 1;
    for (int n = 0; n < L; ++n) {
        double est = 0.0, var = 0.0, s = 0.0;
        int ok = 1;
        for (int t = 0; t < h->ntab; ++t) {
            int64_t M = h->M[t];
            double Wt = h->Wn[(size_t)t * L + n], Qt = h->Qn[(size_t)t * L + n];
            s += (double)h->Sn[(size_t)t * L + n];
            if (M < 1) { ok = 0; continue; }
            double c = Wt / (double)M;            /* the sample average (eq. 4), any M >= 1 */
            est += c;
            if (M < 2) { ok = 0; continue; }      /* the variance needs two tours */
            double v = (Qt / (double)M - c * c) / (double)(M - 1);
            if (v < 0.0) v = 0.0;
            var += v;
        }
        est /= (double)h->ntab;
        var /= (double)h->ntab * (double)h->ntab;
        if (log_cn) log_cn[n] = (est > 0.0) ? log(est) + orc_scale_exp(h->d, n) * log(2.0) : -INFINITY;
        if (S_n) S_n[n] = s;
        if (relvar_n) relvar_n[n] = (ok && est > 0.0) ? var / (est * est) : INFINITY;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2 on several host threads (Sec. 3: the paper ran one flatPERM    */
/* sequence per thread, every thread reading and updating the shared table W */
/* as it goes).  This is the CPU baseline of the benchmark; the parity tests */
/* use the sequential run above, which this section does not touch.  Each    */
/* thread takes tour tickets g (sequence g mod N, tour g div N) from a shared */
/* counter, so M counts every tour started by any thread; the tables are     */
/* updated with atomic adds, and a node reads W_n and M as they are at that  */
/* moment (the paper's "real time" sharing).  Results depend on the threads' */
/* interleaving, so only their statistics are reproducible.                  */
/* ------------------------------------------------------------------------- */
static void atomic_add_f64(double *p, double v) {
    uint64_t old_bits = __atomic_load_n((uint64_t *)p, __ATOMIC_RELAXED);
    for (;;) {
        double old, sum;
        memcpy(&old, &old_bits, 8);
        sum = old + v;
        uint64_t new_bits;
        memcpy(&new_bits, &sum, 8);
        if (__atomic_compare_exchange_n((uint64_t *)p, &old_bits, new_bits, 1, __ATOMIC_RELAXED,
                                        __ATOMIC_RELAXED))
            return;
    }
}

static double atomic_load_f64(const double *p) {
    uint64_t bits = __atomic_load_n((const uint64_t *)p, __ATOMIC_RELAXED);
    double v;
    memcpy(&v, &bits, 8);
    return v;
}

typedef struct {
    orc_state *h;
    int64_t last;            /* tickets below this are tours of this call */
    occset occ;
    int32_t *coords;
    stack_rec *stack;
    double *X;
    int64_t steps;
    int rc;
} mt_worker;

/* One tour on a worker's own walk state against the shared table. */
static int mt_tour(mt_worker *wk, uint32_t seq, uint32_t tour, int64_t g) {
    orc_state *h = wk->h;
    const int d = h->d, n_max = h->n_max;
    int32_t *co = wk->coords;
    long sp = 0;
    int n = 0;
    double W = 1.0;
    uint64_t ordinal = 0;
    for (int i = 0; i < d; ++i) co[i] = 0;
    wk->occ.n = 0;
    occ_set(&wk->occ, co, 1);
    for (;;) {
        /* the sum of the earlier weights at this length and the tours started so far
         * (this one included), read as they are now; then accumulate (eq. 4) */
        double Wsum = atomic_load_f64(&h->Wn[n]);
        int64_t M = __atomic_load_n(&h->M[0], __ATOMIC_RELAXED);
        if (M > wk->last) M = wk->last;
        if (M < g + 1) M = g + 1;
        atomic_add_f64(&h->Wn[n], W);
        __atomic_fetch_add(&h->Sn[n], 1, __ATOMIC_RELAXED);
        wk->X[n] += W;
        wk->steps += 1;
        node_out o;
        int rc = grow_node(d, n_max, n, co + (long)n * d, &wk->occ, W, Wsum, M, ordinal, seq, tour,
                           h->seed, h->run, NULL, &o);
        ordinal += 1;
        if (rc == ORC_CHILDREN) {
            for (int i = o.c - 1; i >= 1; --i) {
                if (sp >= h->stack_cap) return ORC_EOVERFLOW;
                wk->stack[sp].depth = n;
                wk->stack[sp].dir = o.dirs[i];
                wk->stack[sp].w = o.child_w;
                ++sp;
            }
            add_step(d, co + (long)n * d, o.dirs[0], co + (long)(n + 1) * d);
            n += 1;
            wk->occ.n = n;
            occ_set(&wk->occ, co + (long)n * d, 1);
            W = o.child_w;
            continue;
        }
        if (sp == 0) break;
        --sp;
        int dp = wk->stack[sp].depth;
        for (int k = n; k > dp; --k) occ_set(&wk->occ, co + (long)k * d, 0);
        add_step(d, co + (long)dp * d, wk->stack[sp].dir, co + (long)(dp + 1) * d);
        n = dp + 1;
        wk->occ.n = n;
        occ_set(&wk->occ, co + (long)n * d, 1);
        W = wk->stack[sp].w;
    }
    for (int k = n; k >= 0; --k) occ_set(&wk->occ, co + (long)k * d, 0);
    wk->occ.n = -1;
    for (int k = 0; k <= n_max; ++k) {
        if (wk->X[k] != 0.0) atomic_add_f64(&h->Qn[k], wk->X[k] * wk->X[k]);
        wk->X[k] = 0.0;
    }
    return ORC_OK;
}

static void *mt_main(void *arg) {
    mt_worker *wk = (mt_worker *)arg;
    orc_state *h = wk->h;
    for (;;) {
        int64_t g = __atomic_fetch_add(&h->M[0], 1, __ATOMIC_RELAXED);
        if (g >= wk->last) break;
        int rc = mt_tour(wk, (uint32_t)(g % h->n_seq), (uint32_t)(g / h->n_seq), g);
        if (rc != ORC_OK) { wk->rc = rc; break; }
    }
    return NULL;
}

int orc_run_threads(orc_state *h, int64_t tours_per_seq, int threads) {
    if (!h || tours_per_seq < 0 || threads < 1 || threads > 1024 || h->alg != ORC_ALG2 || h->cut_hi)
        return ORC_EINVAL;
    const int64_t first = h->M[0], last = first + tours_per_seq * (int64_t)h->n_seq;
    mt_worker *wk = (mt_worker *)calloc((size_t)threads, sizeof(mt_worker));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    int rc = (wk && tid) ? ORC_OK : ORC_ENOMEM;
    const size_t L = (size_t)h->n_max + 1;
    for (int t = 0; t < threads && rc == ORC_OK; ++t) {
        wk[t].h = h;
        wk[t].last = last;
        wk[t].coords = (int32_t *)calloc(L * h->d, sizeof(int32_t));
        wk[t].stack = (stack_rec *)calloc((size_t)h->stack_cap, sizeof(stack_rec));
        wk[t].X = (double *)calloc(L, sizeof(double));
        if (!wk[t].coords || !wk[t].stack || !wk[t].X || occ_init(&wk[t].occ, h->d, h->n_max) != ORC_OK)
            rc = ORC_ENOMEM;
        wk[t].occ.coords = wk[t].coords;
    }
    int started = 0;
    for (int t = 0; t < threads && rc == ORC_OK; ++t) {
        if (pthread_create(&tid[t], NULL, mt_main, &wk[t]) != 0) { rc = ORC_ENOMEM; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    if (started > 0) h->M[0] = last;            /* tickets handed out past the end are void */
    for (int t = 0; wk && t < threads; ++t) {
        h->steps += wk[t].steps;
        if (rc == ORC_OK && wk[t].rc != ORC_OK) rc = wk[t].rc;
        free(wk[t].coords); free(wk[t].stack); free(wk[t].X); free(wk[t].occ.box);
    }
    free(wk); free(tid);
    h->tours_done[0] = h->M[0];
    return rc;
}
