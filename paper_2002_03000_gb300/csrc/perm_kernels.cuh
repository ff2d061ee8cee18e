// perm_kernels.cuh -- parameters shared by the kernels and the C-ABI host code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "perm.h"

namespace perm {

enum ThreshMode { kSnapshot = 0, kFresh = 1 };
// Where a CTA's state lives: all in shared memory; the walk regions in a global
// arena (head in shared memory); or all of it in the arena.
enum ArenaMode { kArenaNone = 0, kArenaWalks = 1, kArenaAll = 2 };

// Everything one persistent launch needs (passed by value).
struct RunDev {
    int d, n_max, n_seq, alg;
    int run_index;       // position in a batch launch's run table (0 otherwise)
    int log2h;           // per-walk hash size 2^log2h
    int S;               // lanes per warp that hold walks
    int stride;          // interleave stride of per-walk shared arrays (power of 2, >= S)
    int worker_warps;    // per CTA
    int slots;           // walks on the device
    int tour_slots;      // walks that start tours (slots below it); the rest are helpers
    int stack_cache;     // stack records cached per walk in shared memory (power of 2)
    int arena_mode;      // ArenaMode
    long long arena_cta_bytes;     // bytes of one CTA's slice of the arena
    unsigned char *arena;          // global arena (nullptr unless arena_mode != kArenaNone)
    uint32_t key0, key1; // Philox key
    long long tour_limit;      // Alg. 2: tickets below this are tours of this launch or earlier
    long long seq_target;      // Alg. 1: tours per sequence after this launch
    int refresh_ns;
    long long max_ns;          // wall-clock bound of the launch (bounded waits)
    // global tables: Alg. 2 one row, Alg. 1 n_seq rows of n_max+1
    double *Wn;
    unsigned long long *Sn;
    double *Qn;
    double *Rn;                    // optional (nullptr: off): sum of W |omega_n|^2 per length
    // original PERM (nullptr: flatPERM): per length (T_n, t_n) at the stored scale; a node
    // above T_n makes cut_copies copies, one below t_n survives iff its first random
    // word is below cut_K = ceil(fl(1/q) 2^32) (u0 < 1/q) and then carries q W
    const double2 *cut;
    int cut_copies;
    double cut_q, cut_inv_q;
    unsigned long long cut_K;
    unsigned long long *tickets;   // Alg. 2: tours started (M); Alg. 1: next sequence
    unsigned long long *seq_M;     // Alg. 1: tours done per sequence
    // per-walk scratch
    double *X;                     // tour-sum rows x (n_max+1): a tour's weight per length
                                   // (rows: one per walk; two with shared copies)
    uint32_t *gstk_meta;           // slots x n_max
    double *gstk_w;                // slots x n_max
    // statistics and status
    unsigned long long *steps;
    unsigned long long *max_stack;
    unsigned long long *copies;
    unsigned long long *refreshes;
    unsigned long long *iterations;
    unsigned long long *exact_steps;   // nodes whose decision took r in double precision
    unsigned long long *finished;  // Alg. 2: tours finished (admission of new tours)
    long long ramp_c0;             // admission: in flight <= c0 + gamma * finished
    unsigned long long ramp_gamma_q16;
    // shared copies (snapshot form of Alg. 2): a walk with no tour to start
    // takes a waiting copy from the bottom of another walk's stack
    int share;                     // 0: off; else the most parts of one tour growing at once
    int share_boost;               // ... once no tour of the run has finished for stall_ns
    long long stall_ns;
    int dq_log2cap;                // ring of 2^dq_log2cap donation cells
    int dq_cell_bytes;             // header (32 bytes) + keys and hash slots of sites 0..n_max
    unsigned char *dq_cells;
    unsigned long long *dq_head;   // donations taken
    unsigned long long *dq_tail;   // donations reserved
    unsigned int *dq_ready;        // per cell: round + 1 once written for that round
    unsigned int *dq_free;         // per cell: first round that may write it
    unsigned int *outst;           // per tour-sum row: live parts of its tour (kRowFree: row unused)
    unsigned int *tmaxn;           // per tour-sum row: deepest length over the parts of its tour
    int *hungry;                   // walks waiting for work
    int *status;
    // optional sampled trace
    perm_trace_record *trace;
    int32_t *trace_coords;
    unsigned long long *trace_count;
    int trace_cap;
    long long trace_every, trace_tour_every;
};

// One launch growing several runs (snapshot form of Alg. 2): the runs' descriptors
// in device memory and the scheduling counters.
struct BatchDev {
    const RunDev *runs;   // R descriptors; run r's run_index is r
    int R;
    int *active;          // per run: CTAs on it now
    int *granted;         // per run: tour-growing walks handed to CTAs
    int *runs_open;       // runs with tours to start and walks to grant
    int *closed;          // per run: bit 0 tickets exhausted, bit 1 walks all granted
    long long max_ns;     // wall-clock bound of the launch
};

// Largest dynamic shared memory a batch CTA can have (and allow it).
cudaError_t batch_smem_budget(size_t *dynamic_max);
// CTAs of a batch launch: every SM, as many CTAs each as fit.
cudaError_t batch_grid(int threads, size_t smem, int *ctas);
// Counters reset, then the persistent batch kernel.
cudaError_t launch_batch(const BatchDev &B, int ctas, int threads, size_t smem, cudaStream_t stream);

// Host side of batch members (runs whose descriptors sit in a batch's table):
// a run laid out for `ctas` CTAs of at most 4 x 8 walks within smem_budget bytes
// of shared memory, and its descriptor for tours_per_seq tours per sequence from
// empty tables.
int member_create(perm_handle *out, const perm_config *cfg, int ctas, size_t smem_budget);
int member_params(perm_handle h, int64_t tours_per_seq, int run_index, RunDev *P, size_t *smem,
                  int *worker_warps);
// Empty tables and tour sums (every row, also after a failed run), on the run's stream.
int member_reset(perm_handle h);
// The descriptor after extra_tours_per_seq more tours per sequence on top of the
// run's current tables (cumulative, as perm_run).
int member_extend(perm_handle h, int64_t extra_tours_per_seq, int run_index, RunDev *P);

// Shared-memory bytes of one CTA (everything in shared memory), and its parts.
size_t cta_smem_bytes(int d, bool key64, int n_max, int log2h, int stack_cache, int worker_warps,
                      bool snapshot, int stride);
size_t cta_head_bytes(int n_max, bool snapshot);
size_t cta_warp_bytes(bool key64, int n_max, int log2h, int stack_cache, int stride);

cudaError_t launch_grow(const RunDev &P, int thresh_mode, bool key64, int ctas,
                        cudaStream_t stream);
cudaError_t launch_finalize(unsigned long long *tickets, long long limit, cudaStream_t stream);
cudaError_t set_smem_limits();

cudaError_t launch_debug_step(int d, int n_max, int B, const int32_t *coords, const int32_t *len,
                              const double *W, const double *Wsum, const uint64_t *M,
                              const uint64_t *ordinal, const uint32_t *seq, const uint32_t *tour,
                              uint32_t key0, uint32_t key1, int force_exact, int32_t *out_i,
                              double *out_r, double *out_w, cudaStream_t stream);
cudaError_t launch_debug_philox(int B, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                cudaStream_t stream);

}  // namespace perm
