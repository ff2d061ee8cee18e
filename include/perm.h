/*
 * perm.h -- C ABI of the GB300 interacting-flatPERM library (libperm.so).
 *
 * The library runs the growth step of parallel flatPERM (Campbell and Janse
 * van Rensburg, "Parallel PERM") for self-avoiding walks on Z^d, d = 2, 3, on
 * one NVIDIA GB300 (sm_103a):
 *   - Sec. 1, eqs. (1)-(2): Rosenbluth growth -- a_+ free neighbours of the
 *     end-point, a step chosen uniformly among them, weight W = prod a_+;
 *   - Sec. 1, eq. (4): the sample average <W_n> = sum W_n / M estimates c_n,
 *     M being the number of tours started (passes through the empty walk);
 *   - Sec. 2, eq. (6) and the paragraphs after it: flatPERM ratio
 *     r = W / [W_n]^sample (own weight included), enrichment into c copies of
 *     weight W/c (c = floor r with probability ceil r - r, else ceil r),
 *     pruning with probability 1 - r and survival with weight W/r.  Every
 *     decision equals the one taken on r evaluated in double precision as
 *     defined (a single-precision estimate settles most nodes; the others
 *     evaluate r exactly);
 *   - Sec. 3, Algorithm 2 and Fig. 1: N sequences grow concurrently and share
 *     one table W; Algorithm 1: N sequences with private tables.
 *
 * Conventions (every entry point):
 *   - Return PERM_OK (0) on success or a negative PERM_E* code; perm_strerror
 *     names it.  No entry point aborts or traps; a failure inside a kernel is
 *     reported through the handle's status word as PERM_EOVERFLOW/PERM_EDEVICE.
 *   - The library owns all device memory it allocates; the caller owns every
 *     host array it passes, and every device pointer passed to
 *     perm_debug_step.  Host arrays of length n_max+1 are indexed by n.
 *   - A handle is not thread safe.  Work is queued on the handle's CUDA stream
 *     (perm_set_stream; default: a stream the library creates).
 */
#ifndef PERM_H
#define PERM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PERM_OK 0
#define PERM_EINVAL (-1)     /* bad argument (d, n_max, n_seq, pointer, mode) */
#define PERM_ENOMEM (-2)     /* device or host allocation failed */
#define PERM_EOVERFLOW (-3)  /* a kernel found a stack or hash bound exceeded; run invalid */
#define PERM_EDEVICE (-4)    /* CUDA error (launch, copy, no device) */
#define PERM_ETIMEOUT (-5)   /* a bounded device wait ran out; run invalid */
#define PERM_EUNSUPPORTED (-6) /* configuration this build does not handle */
#define PERM_ESCRATCH (-7)   /* perm_run_static: the requested walks need more scratch than
                                the static buffer (PERM_STATIC_SCRATCH_BYTES) holds */

typedef struct perm_run_s *perm_handle;

/* Algorithms (Sec. 3, Fig. 1). */
#define PERM_ALG2 2   /* N interacting sequences, one shared table W (default) */
#define PERM_ALG1 1   /* N independent sequences, one table each */

/* Where a node reads its threshold [W_n]^sample from (Algorithm 2). */
#define PERM_THRESH_SNAPSHOT 0  /* per-SM copy of W_n and M, refreshed every refresh_ns (default) */
#define PERM_THRESH_FRESH 1     /* global table read by the node's own atomic add (exact
                                   sequential flatPERM when N = 1) */

typedef struct {
    int d;             /* lattice dimension, 2 or 3 */
    int n_max;         /* longest walk length; 1..32766 (d=2), 1..1048574 (d=3) */
    int n_seq;         /* N, number of flatPERM sequences, >= 1 */
    uint64_t seed;     /* Philox key material */
    uint32_t run_id;   /* XORed into the low key word (distinct runs, one seed) */
    int alg;           /* PERM_ALG2 or PERM_ALG1 */
    int threshold;     /* PERM_THRESH_SNAPSHOT or PERM_THRESH_FRESH (Alg. 2 only) */
    int slots;         /* concurrent walks on the GPU; 0 = min(N, device capacity) */
    int lanes_per_warp;/* walks per warp, 1..32; 0 = automatic (about four warps per SM) */
    int refresh_ns;    /* snapshot refresh period in ns, paced on the SM cycle counter; 0 = default (8000) */
    double max_seconds;/* wall-clock bound of one launch; past it the kernel stops and the
                          run reports PERM_ETIMEOUT; 0 = default (600) */
    int ramp_c0;       /* Algorithm 2 admission: at most ramp_c0 + ramp_gamma * (finished
                          tours) tours are in flight.  0 = default (2); < 0 = no limit */
    double ramp_gamma; /* see ramp_c0; 0 = default (0.25) */
    int max_ctas;      /* at most this many CTAs (SMs) for the run's walks; 0 = all SMs;
                          -1 = as few CTAs as hold one walk per sequence (dense packing).
                          Lets concurrent runs share the device */
    int hash_scale;    /* per-walk occupancy hash has 2^hash_scale * 2 n_max slots
                          (rounded up to a power of 2); 0..2 */
    int share_copies;  /* Algorithm 2 with snapshot thresholds: a walk with no tour to
                          start (admission limit, or no tickets left) takes the oldest
                          waiting copy of another walk's tour and grows its subtree; the
                          copy's weights still count for that tour (Sec. 2: the copies
                          grow independently).  k >= 1: at most k parts of one tour grow
                          at once; 0 = on with the default cap (4); -1 = off.  Once no
                          tour of the run has finished for 5 ms (a start-up tree too
                          large for a few walks), the cap rises to 1024 */
    int stack_ring;    /* waiting-copy records per walk kept in shared memory (the rest
                          spill to global memory 8 at a time): 16, 32, 64 or 128;
                          0 = default (16) */
    int observables;   /* 1: also accumulate sum W |omega_n|^2 per length (the squared
                          end-to-end distance, for the ratio estimator of Sec. 1,
                          eq. 5; read with perm_observable_r2); 0 = off (default) */
    int walk_memory;   /* where each walk's occupancy hash, site list and stack ring
                          live: 0 = shared memory when at least one walk per CTA fits
                          beside the snapshot table, else a global-memory arena (long
                          walks: n_max of 10^4 and more); 1 = shared memory only
                          (PERM_EUNSUPPORTED when nothing fits); 2 = the global
                          arena (served through L1 and L2; the snapshot table stays
                          in shared memory while it fits) */
    int helper_walks;  /* walks beyond one per sequence that start no tour and grow
                          waiting copies of the sequences' tours only (shared copies,
                          Sec. 2: copies grow independently); at most N tours are in
                          flight whatever their number.  k > 0 needs Algorithm 2 with
                          snapshot thresholds and shared copies on; 0 (default) =
                          none; -1 = the walks the automatic layout has room for
                          beyond the tour walks (up to 4 warps of 8 per SM) when
                          shared copies are on, else none.  Fewer run when not all
                          fit.  They pay off for long walks from few sequences
                          (n_max 10^4 from 12); with many sequences or short walks
                          they gain nothing or cost time */
} perm_config;

/* Fill cfg with defaults for (d, n_max, n_seq, seed). */
void perm_config_init(perm_config *cfg, int d, int n_max, int n_seq, uint64_t seed);

/* Create a run with default settings (Algorithm 2, snapshot thresholds).
 * out: receives the handle (NULL on failure).  Allocates the shared tables
 * W_n, S_n, Q_n (FP64/u64, n_max+1 each), the tour counter M and per-walk
 * scratch (tour sums, stacks) in device memory. */
int perm_create(perm_handle *out, int d, int n_max, int n_seq, uint64_t seed);
/* Same with every setting explicit. */
int perm_create_ex(perm_handle *out, const perm_config *cfg);

/* Queue all later work of h on `stream` (a cudaStream_t; NULL = legacy default). */
int perm_set_stream(perm_handle h, void *stream);

/* Original PERM with cut-offs (Sec. 2, the paragraphs on T_k, t_k and q)
 * instead of flatPERM's ratio, for the runs that follow:
 *   - a node of length n >= 1 whose weight W exceeds T_hi[n] is enriched into
 *     `copies` copies, with distinct steps, at most a_+ of them, each carrying
 *     W/c for the c made;
 *   - one with W < t_lo[n] survives with probability 1/q (u0 < 1/q in double
 *     precision, u0 being the node's first random word over 2^32) and then
 *     carries q W;
 *   - otherwise it grows one copy, as in flatPERM with r = 1.
 * The empty walk is neither enriched nor pruned.  The shared table no longer
 * decides anything, so a run with sharing off (fresh thresholds, or
 * share_copies = -1) is deterministic for any number of sequences.
 * T_hi, t_lo: host arrays of n_max+1 doubles at the stored weight scale (the
 * scale of perm_tables' W_n; e.g. a multiple of W_n/M from an earlier run),
 * copied before return.  copies in 1..2d; 1 <= q <= 2^32.  Both arrays NULL:
 * back to flatPERM.  PERM_EINVAL on a bad argument. */
int perm_set_cutoffs(perm_handle h, const double *T_hi, const double *t_lo, int copies, double q);

/* Checkpoint and resume (no counterpart in the paper).  perm_save waits for the
 * handle's stream, then writes the run's state at that tour boundary to `path`:
 * the configuration, the tables W_n, S_n, Q_n (and the eq. 5 sums when
 * observables are on), the tour counters (M, tours per sequence), the cut-offs
 * if set, and the statistics.  The file is written beside `path` and renamed,
 * so a failure leaves no partial checkpoint.  A run whose status is an error is
 * not saved (that code is returned).  perm_load creates a new handle from such
 * a file (same library build; any GB300): runs on it continue where the saved
 * run stopped, with the same random streams, so a run with sharing off (fresh
 * thresholds, or share_copies = -1) continues exactly as if it had not been
 * interrupted.  PERM_EINVAL for a file that is not a complete checkpoint. */
int perm_save(perm_handle h, const char *path);
int perm_load(perm_handle *out, const char *path);
/* The configuration a handle runs with (defaults filled in), e.g. of a loaded one. */
int perm_get_config(perm_handle h, perm_config *out);

/* Grow tours_per_seq more tours of every sequence (cumulative: repeated calls
 * continue the same tables, tour counters and random streams).  Queues one
 * persistent kernel launch and returns without waiting unless `sync` is set
 * by perm_run_sync. */
int perm_run(perm_handle h, int64_t tours_per_seq);
/* perm_run, then wait for the stream and report any device-side status. */
int perm_run_sync(perm_handle h, int64_t tours_per_seq);

/* Start the run over: zero the tables, the tour counters and the statistics
 * (queued on the stream; the next perm_run begins at M = 0 with the same
 * random streams as a fresh handle). */
int perm_reset(perm_handle h);

/* Estimates after waiting for the stream (Sec. 1, eq. 4; Alg. 1: eq. 7):
 *   log_cn[n]   = log <W_n>, the natural log of the estimate of c_n
 *                 (-inf where no walk reached n);
 *   S_n[n]      = number of nodes of length n grown (histogram, as double);
 *   relvar_n[n] = estimated variance of <W_n> divided by <W_n>^2, from the
 *                 per-tour sums (variance = (Q_n/M - <W_n>^2)/(M-1)).
 * Any pointer may be NULL.  Arrays have n_max+1 entries. */
int perm_estimates(perm_handle h, double *log_cn, double *S_n, double *relvar_n);

/* Estimates from raw tables, without a handle (host arithmetic only; no device
 * call): e.g. tables pooled over several runs or replicas, or the per-sequence
 * rows of an Algorithm-1 run.  W_n, Q_n: `rows` rows of n_max+1 doubles at the
 * stored scale (as perm_tables returns them; Q_n may be NULL, then relvar_n is
 * +inf); M: `rows` tour counts (each >= 1).  Per row, c = W_n/M is the sample
 * average of Sec. 1, eq. 4, and (Q_n/M - c^2)/(M-1) its variance.
 *   PERM_COMBINE_MEAN:      log_cn = log of the mean over rows of c (Sec. 3's
 *                           average of the sequences' estimates; one row: eq. 4);
 *                           relvar_n = the variance of that mean over its square;
 *   PERM_COMBINE_GEOMETRIC: log_cn = the mean over rows of log c (the geometric
 *                           combination Sec. 4 uses for Algorithm 1); relvar_n =
 *                           the mean of the rows' relative variances / rows.
 * log_cn adds E(n) log 2 back (-inf where an estimate is 0); relvar_n is +inf
 * where a row has fewer than two tours.  Either output may be NULL.
 * PERM_EINVAL on a bad argument (d, n_max < 0, rows < 1, a NULL W_n or M, an
 * M below 1, an unknown combine). */
#define PERM_COMBINE_MEAN 0
#define PERM_COMBINE_GEOMETRIC 1
int perm_estimates_from_tables(int d, int n_max, int rows, const double *W_n, const double *Q_n,
                               const int64_t *M, int combine, double *log_cn, double *relvar_n);

/* Raw tables after waiting: W_n, S_n, Q_n at the stored scale (the weight of a
 * walk of length n is stored divided by 2^E(n), E(n) = floor(11n/8) for d=2,
 * floor(9n/4) for d=3), and M.  Alg. 1 returns n_seq rows of n_max+1 and one
 * M per sequence.  Any pointer may be NULL. */
int perm_tables(perm_handle h, double *W_n, double *S_n, double *Q_n, int64_t *M);

typedef struct {
    int64_t steps;        /* nodes processed (walk-growth steps), cumulative */
    int64_t tours;        /* tours started, cumulative */
    int64_t max_stack;    /* deepest per-walk stack of waiting copies seen */
    int64_t copies;       /* extra copies pushed by enrichment (c - 1 per node), cumulative */
    int64_t refreshes;    /* threshold refreshes summed over CTAs, cumulative */
    int64_t iterations;   /* main-loop iterations summed over worker warps, cumulative */
    int slots, ctas, lanes_per_warp, warps_per_cta;
    int hash_slots;       /* per-walk occupancy hash size */
    int status;           /* PERM_OK or the device-side error of the last run */
    int64_t device_bytes; /* device memory held by the handle */
    int64_t tours_finished; /* tours whose copies have all been grown, cumulative */
    int64_t shared;       /* waiting copies handed to other walks, cumulative */
    int64_t exact_steps;  /* nodes whose decision evaluated r in double precision because
                             the single-precision estimate lay too close to a decision
                             boundary to settle it, cumulative */
    int walk_memory;      /* where the walks' hashes, site lists and stack rings live:
                             1 shared memory, 2 the global arena */
    int pad;
} perm_stats_t;
int perm_stats(perm_handle h, perm_stats_t *out);

/* Mean squared end-to-end distance <|omega_n|^2>, n = 0..n_max, by the ratio
 * estimator of Sec. 1, eq. 5: sum W |omega_n|^2 / sum W (Algorithm 1: the average
 * over sequences of R/M divided by that of W/M).  mean_r2: caller-owned host
 * array of n_max+1 (NaN where no walk reached the length).  R_n: optional
 * (NULL allowed) host array receiving the raw sums at the stored weight scale,
 * n_max+1 values (Algorithm 1: one row per sequence).  Synchronises with the
 * run's stream.  PERM_EINVAL if the run was created with observables = 0. */
int perm_observable_r2(perm_handle h, double *mean_r2, double *R_n);

/* Sampled node trace (test support): every node whose DFS ordinal is a
 * multiple of `every`, in tours whose index within their sequence is a
 * multiple of `tour_every`, is recorded, up to `capacity` records, during later perm_run calls.
 * every = 0 switches tracing off.  perm_trace_read copies the records out.
 * Record: length n, a_plus, free_mask, c (copies; 0 when pruned), outcome (as
 * perm_debug_step), exact (1 if the decision evaluated r in double precision),
 * the chosen directions (-1 beyond c), the node's sequence, tour and DFS
 * ordinal, the M it used, its weight W, the sum Wsum of the weights at its
 * length that it saw (both at the stored scale), r as the decision used it
 * (the single-precision estimate widened, or the exact r) and the children's
 * weight (stored scale of length n+1). */
typedef struct {
    int32_t n, a_plus, free_mask, c, outcome, exact;
    int32_t dirs[6];
    uint32_t seq, tour;
    uint64_t ordinal, M;
    double W, Wsum, r, child_w;
} perm_trace_record;
int perm_trace_enable(perm_handle h, int64_t every, int64_t tour_every, int capacity);
/* count: records written (may exceed capacity; only capacity are kept).
 * recs: host array of `capacity` records; coords: host int32 array of
 * capacity*(n_max+1)*d, the walk of each record (site k at [k*d..k*d+d-1]). */
int perm_trace_read(perm_handle h, int64_t *count, perm_trace_record *recs, int32_t *coords);

void perm_destroy(perm_handle h);   /* NULL-safe; waits for the stream */
const char *perm_strerror(int code);

/* One growth step on B snapshot states (test support for step parity).
 * All arrays are DEVICE pointers owned by the caller:
 *   coords[B*(n_max+1)*d] int32  walk b: site k at (b*(n_max+1)+k)*d, origin first
 *   len[B]      int32   n, the length of walk b (0..n_max)
 *   W[B]        double  the node's weight (stored scale of length n)
 *   Wsum[B]     double  sum of the weights recorded at length n before the node
 *   M[B]        uint64  tours started (>= 1)
 *   ordinal[B]  uint64  DFS ordinal of the node; seq[B], tour[B] uint32
 *   out_i[B*11] int32   outcome, a_plus, free_mask, c, dirs[0..5], exact
 *   out_r[B]    double  r as the decision used it (estimate, or exact when exact = 1)
 *   out_w[B]    double  the children's weight (stored scale of length n+1)
 * force_exact = 1 takes every decision on r in double precision (0: the
 * kernel's own path).  Outcomes: 0 walk at n_max, 1 trapped, 2 pruned,
 * 3 children.  Requires d in {2,3} and n_max <= 512.  Queued on `stream`,
 * not waited for. */
int perm_debug_step(int d, int n_max, int B, const int32_t *coords, const int32_t *len,
                    const double *W, const double *Wsum, const uint64_t *M,
                    const uint64_t *ordinal, const uint32_t *seq, const uint32_t *tour,
                    uint64_t seed, uint32_t run_id, int force_exact, int32_t *out_i,
                    double *out_r, double *out_w, void *stream);

/* ---------------------------------------------------------------------------
 * Batched runs (many independent runs, one CUDA-graph launch).
 * perm_batch_create makes R runs (cfgs[r], grown tours_per_seq[r] tours per
 * sequence from empty tables) and captures all of their work -- table reset,
 * persistent growth kernel, tour-counter clamp -- into one CUDA graph with one
 * branch per stream (n_streams; 0 = min(R, 64)).  A run whose cfg.max_ctas is
 * 0 is packed into the fewest CTAs that hold one walk per sequence (as
 * max_ctas = -1), so that the runs' kernels share the SMs.
 * perm_batch_create_persistent makes the same batch grown by ONE persistent
 * kernel on every SM instead: each CTA joins the run with the most tours left
 * to start per CTA already on it (weighted by n_max + 1), grows at most one walk
 * per sequence of it, and moves to another run once the run has no tours left to
 * start; with no run left to start, CTAs help unfinished runs through their
 * waiting copies.  Every run must be Alg. 2 with snapshot thresholds
 * (PERM_EUNSUPPORTED otherwise); each is laid out for the whole grid (at most
 * 4 x 8 walks per CTA), so its per-walk scratch scales with the SM count; its
 * lanes_per_warp, slots and max_ctas are ignored.  The statistics and estimates
 * follow the same law as a single run's (the scheduling differs, so results are
 * not bit-identical to one).  The launch ends within the largest max_seconds
 * of its runs; a run not finished by then reports PERM_ETIMEOUT.
 * perm_batch_run replays the graph (every run starts again from empty tables)
 * and waits; estimates and statistics are then read per run as for a single
 * handle.  The batch owns its handles, streams and graph.
 * ------------------------------------------------------------------------- */
typedef struct perm_batch_s *perm_batch_handle;
int perm_batch_create(perm_batch_handle *out, const perm_config *cfgs, const int64_t *tours_per_seq,
                      int R, int n_streams);
int perm_batch_create_persistent(perm_batch_handle *out, const perm_config *cfgs,
                                 const int64_t *tours_per_seq, int R);
int perm_batch_run(perm_batch_handle b);
/* Grow extra_tours_per_seq[r] more tours per sequence of every run r on top of
 * its current tables (cumulative, as perm_run; 0 leaves a run as it is, e.g. one
 * that has met its target error), in one launch of the batch's form (the
 * persistent kernel over the runs with tours to grow, or each run's kernel on
 * its stream), and wait.  extra_tours_per_seq: host array of R values >= 0. */
int perm_batch_continue(perm_batch_handle b, const int64_t *extra_tours_per_seq);
int perm_batch_size(perm_batch_handle b);
int perm_batch_estimates(perm_batch_handle b, int r, double *log_cn, double *S_n, double *relvar_n);
int perm_batch_stats(perm_batch_handle b, int r, perm_stats_t *out);
void perm_batch_destroy(perm_batch_handle b);

/* Autotuner (no counterpart in the paper): for each walks-per-warp choice (auto,
 * 2, 4, 8, 16, 32), hash size (hash_scale 0, 1) and stack ring (16, 64 records),
 * times a complete run of probe_tours tours per sequence of cfg from empty
 * tables (twice; the faster counts).  The default layout (auto, 0, 16) is timed
 * first and kept unless another choice is at least 3% faster and then at least
 * 3% faster again on runs of 4 x probe_tours (the fastest of three runs of each,
 * alternated: complete runs vary by 10-30% in nodes), so the pick is never
 * slower than the default on that validation.  Writes the choice into cfg->lanes_per_warp,
 * cfg->hash_scale and cfg->stack_ring.  Equal tours in every trial, so the
 * comparison is at equal work, start-up included.  Results are cached per (d,
 * n_max, n_seq, max_ctas, alg, threshold) for the process.  Synchronous;
 * allocates and frees a handle per trial.  Returns PERM_EUNSUPPORTED if no
 * trial ran. */
int perm_autotune(perm_config *cfg, int64_t probe_tours);

/* perm_run_static -- one complete Algorithm-2 growth run that allocates
 * nothing (the paper has no counterpart: this serves callers that cannot
 * call cudaMalloc -- a process whose device memory is owned by another
 * allocator, a plugin inside one, or a loop that must not allocate because
 * cudaMalloc/cudaFree can synchronise the device).
 *
 * All scratch (tour counters, status, per-walk tour sums and stack spill
 * areas) lives in one file-scope device array of PERM_STATIC_SCRATCH_BYTES
 * that every GPU loading the library holds until exit.  The first call on a
 * device looks up the array's device address (make that first call before
 * any stream capture).  Every call shares the array and leaves its contents
 * behind; each call clears what must start at zero.  Calls whose work
 * overlaps on the GPU race on the array: do not overlap them.
 *
 * cfg: as for perm_create_ex; alg must be PERM_ALG2.  cfg->slots = 0 runs
 * as many walks at once as the buffer holds (sequences beyond that are
 * time-sliced at tour boundaries); an explicit cfg->slots (clamped to n_seq)
 * whose scratch exceeds the buffer is rejected with PERM_ESCRATCH.  The run
 * grows every waiting copy on the walk that made it (no shared copies:
 * share_copies 0 or -1 both mean that here) and uses the automatic layout;
 * observables, hash_scale, lanes_per_warp, stack_ring, max_ctas, walk_memory
 * other than 0, helper_walks > 0 or share_copies > 0 return PERM_EUNSUPPORTED (every walk's
 * state must then fit in shared memory).  Starts from empty tables and
 * grows tours_per_seq tours of each of cfg->n_seq sequences (M = n_seq *
 * tours_per_seq).
 * W_n, S_n, Q_n: caller-owned DEVICE arrays of n_max+1 entries, overwritten
 * with the raw tables at the stored scale (as perm_tables; S_n as uint64).
 * steps: host pointer (may be NULL) for the number of growth steps.
 * stream: a cudaStream_t (NULL = legacy default stream).  The call is
 * synchronous: it queues its work on `stream`, waits for that stream, and
 * returns after the run has finished.
 * Returns PERM_OK, PERM_EINVAL, PERM_EUNSUPPORTED, PERM_ESCRATCH (the requested
 * walks' scratch exceeds the buffer), PERM_EDEVICE, or a kernel status
 * (PERM_EOVERFLOW, PERM_ETIMEOUT).  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
#define PERM_STATIC_SCRATCH_BYTES (32u << 20)
int perm_run_static(const perm_config *cfg, int64_t tours_per_seq, double *W_n,
                    unsigned long long *S_n, double *Q_n, int64_t *steps, void *stream);

/* Philox4x32-10 on the device for B counters (test support).  ctr[B*4],
 * key[2] on the host, out[B*4]; ctr and out are DEVICE pointers.  Waits. */
int perm_debug_philox(int B, const uint32_t *ctr, const uint32_t *key, uint32_t *out);

#ifdef __cplusplus
}
#endif
#endif
