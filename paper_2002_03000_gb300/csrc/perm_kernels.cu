// perm_kernels.cu -- persistent flatPERM growth kernel (Algorithms 1 and 2 of
// Campbell and Janse van Rensburg, "Parallel PERM", Sec. 3) for sm_103a.
//
// One thread grows one walk ("slot"); a warp holds up to 32 walks.  Per walk,
// shared memory holds the occupancy hash (triangular probing, deleted in LIFO
// order on backtrack), the hash slot of every site, and the top of the stack
// of waiting copies (the rest spills to global memory).  Each thread runs the
// tours handed to it one after another; a tour is a depth-first traversal of
// the tree of copies made by enrichment (Sec. 2).
//
// Threshold sources for Algorithm 2 (one shared table W, Fig. 1):
//  - snapshot: every node adds its weight to the global table with a
//    reduction that returns nothing; one extra warp per CTA reloads a
//    shared-memory copy of W_n and M every refresh period.  The nodes read
//    that copy (a stale but fixed threshold keeps the estimator unbiased:
//    enrichment and pruning conserve the expected weight for any r).  Walks
//    with no tour to start grow waiting copies of other walks' tours (shared
//    copies).
//  - fresh: every node adds its weight to the global table with an atomic that
//    returns the previous sum, and uses it at once (sequential flatPERM exactly
//    when one walk runs).
// Algorithm 1 (private tables) always uses the fresh form on its own rows.  The
// per-tour sums X_n go to a global row per walk and, squared, into Q_n when the
// tour ends.  With cut-offs set (original PERM, Sec. 2) r comes from the
// cut-offs instead of the table.  The batch kernel at the end grows many runs
// in one persistent launch with the same per-run body.
#include <cstdio>

#include "perm_device.cuh"
#include "perm_kernels.cuh"

namespace perm {

namespace {

constexpr int kStride = 32;        // interleave stride of the snapshot-state kernel
constexpr int kUnwind = 8;         // hash deletions per walk per iteration
constexpr int kNodePasses = 2;     // nodes a walk may grow per iteration
constexpr int kPoolExtra = 4;      // extra tour tickets fetched per warp (snapshot)
constexpr int kChunk = 8;          // stack records moved per spill or fill (ring >= 2 kChunk)
constexpr int kReloadBatch = 8;    // snapshot entries a refresher lane loads before storing them
constexpr unsigned kRowFree = 0xFFFFFFFFu;   // outst: the walk's tour-sum row is unused
constexpr int kMinShareGap = 8;    // share a waiting copy only if it may still grow this many steps
constexpr int kCellSpin = 1 << 20; // bounded wait for a donation cell being written
constexpr unsigned kFull = 0xFFFFFFFFu;

enum LaneState { kNeed = 0, kNode = 1, kUnwindState = 2, kFlush = 3, kDone = 4 };
enum Outcome { kLeafNmax = 0, kTrapped = 1, kPruned = 2, kChildren = 3 };

struct CtaHead {
    unsigned long long Ms;   // tours started, as of the last snapshot
    int done_warps;
    int want_don;            // copies this CTA may still hand to idle walks this period
    int queued;              // shared copies waiting in the ring, as of the last snapshot
    int status;              // run status, as of the last snapshot
    unsigned long long fin;  // tours finished, as of the last snapshot
    int cap;                 // parts of one tour that may grow at once (shared copies)
    int may_leave;           // batch launch: another run still has tours to start
    int stalled;             // no tour of the run has finished for stall_ns
    int pad[5];
};
static_assert(sizeof(CtaHead) == 64, "header size");

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A load of a table entry that other SMs update with atomics: an aligned 8-byte
// load is single-copy atomic; relaxed at GPU scope, so the loads of one batch
// stay in flight together.
__device__ __forceinline__ double ld_relaxed(const double *p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

__device__ __forceinline__ size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ __forceinline__ size_t warp_region_bytes(int n_max, int log2h, int K,
                                                             size_t key_bytes, int stride) {
    const size_t hash_b = ((((size_t)1 << log2h) * stride * key_bytes) + 15) & ~(size_t)15;
    const size_t sites_b = (((size_t)n_max * stride * 2) + 15) & ~(size_t)15;
    const size_t stk_b = (((size_t)K * stride * 4) + 15 & ~(size_t)15) + (size_t)K * stride * 8;
    return hash_b + sites_b + stk_b;
}

__host__ __device__ __forceinline__ size_t head_region_bytes(int n_max, bool snapshot) {
    const size_t L = (size_t)n_max + 1;
    size_t b = 64 + 2 * 64 * 8;   // header + two a/c tables
    if (snapshot) b += 8 * L;     // the snapshot of W_n
    return (b + 15) & ~(size_t)15;
}

// Weight factors for the two scale steps dE of the lattice (row t: dE = dE_lo + t):
// [a*8 + c] = (a/c) 2^-dE for c >= 1 (enrichment), [a*8 + 0] = a 2^-dE (exact).
__device__ void fill_aoc(double *aoc, int d, int tid, int nthreads) {
    const int dE_lo = (d == 2) ? 1 : 2;
    for (int i = tid; i < 128; i += nthreads) {
        const int t = i >> 6, a = (i >> 3) & 7, c = i & 7;
        double v = 0.0;
        const double s = __longlong_as_double((long long)((unsigned long long)(1023 - dE_lo - t) << 52));
        if (a >= 1 && c >= 1) v = __dmul_rn(__ddiv_rn((double)a, (double)c), s);
        else if (a >= 1) v = __dmul_rn((double)a, s);
        aoc[i] = v;
    }
}

// Original PERM's cut-offs (Sec. 2) as a node reads them: per length (T_n, t_n)
// at the stored scale, the copies made above T_n, and below t_n the survival
// threshold K (survive iff w0 < K, i.e. u0 < 1/q) and the factor q.
struct Cutoffs {
    const double2 *cut;        // nullptr: flatPERM
    int copies;
    double q, inv_q;
    unsigned long long K;
};

struct NodeOut {
    int outcome, a, mask, c;
    uint32_t dirs;
    double r;            // r as the decision used it (single-precision estimate or exact)
    double child_w;
    bool overflow;
    bool exact;          // the decision was taken on r in double precision
};

// The whole warp copies a donor's sites 0..bdp (key and hash slot) into a cell.
template <typename Key>
__device__ __noinline__ void copy_sites_to_cell(const Key *hash, const uint16_t *sites, int ST, int src,
                                                int bdp, Key *ck, uint16_t *cs, int lane) {
    for (int k = lane; k <= bdp; k += 32) {
        const uint16_t sl = sites[(uint32_t)k * ST + src];
        ck[k] = hash[(uint32_t)sl * ST + src];
        cs[k] = sl;
    }
}

// The whole warp places a taker's sites 0..dp from a cell at their hash slots.
template <typename Key>
__device__ __noinline__ void place_sites_from_cell(Key *hash, uint16_t *sites, int ST, int src, int dp,
                                                   const Key *ck, const uint16_t *cs, int lane) {
    for (int k = lane; k <= dp; k += 32) {
        const uint16_t sl = __ldcg(cs + k);
        hash[(uint32_t)sl * ST + src] = __ldcg(ck + k);
        sites[(uint32_t)k * ST + src] = sl;
    }
}

// One node's growth step (Sec. 1 and Sec. 2): a_+, r, decision, steps, child
// weight.  Wsum: sum of the weights recorded at length n before this node;
// M: tours started.  force_exact: take every decision on the double-precision r.
// Shared by the persistent kernel and the snapshot-state kernel.
template <int D, typename Key>
__device__ __forceinline__ NodeOut grow_node(const Key *hash, int stride, int lane, int log2h, int n,
                                             int n_max, int cx, int cy, int cz, double W, double Wsum,
                                             unsigned long long M, unsigned long long ordinal,
                                             uint32_t seq, uint32_t tour, uint32_t k0, uint32_t k1,
                                             const double *aoc, int (&eslot)[2 * D],
                                             const Cutoffs &cuts, double invM = 0.0, int back = -1,
                                             bool force_exact = false) {
    NodeOut o;
    o.a = 0; o.mask = 0; o.c = 0; o.dirs = 0u; o.child_w = 0.0; o.overflow = false; o.exact = false;
    // three independent chains: the node's random block, the estimate of r, and the probes
    const Philox4 w = philox4x32_10((uint32_t)ordinal, (uint32_t)(ordinal >> 32), tour, seq, k0, k1);
    bool odd = false;
    const float x = ratio_estimate(W, Wsum, M, odd);
    o.r = n == 0 ? 1.0 : widen(x);
    if (n == n_max) { o.outcome = kLeafNmax; return o; }
    bool ovf = false;
    const int fm = probe_neighbours<D, Key>(hash, stride, lane, log2h, cx, cy, cz, eslot, ovf, back);
    o.overflow = ovf;
    o.mask = fm;
    const int a = __popc(fm);
    o.a = a;
    if (a == 0) { o.outcome = kTrapped; return o; }
    uint32_t freelist = 0u;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) {
        if (fm >> j & 1) { freelist |= (uint32_t)j << (3 * cnt); ++cnt; }
    }
    const int dE = scale_exp(D, n + 1) - scale_exp(D, n);
    const int dE_lo = (D == 2) ? 1 : 2;
    const double *row = aoc + 64 * (dE - dE_lo);
    const double a_sc = row[a * 8];                      // a_+ 2^-dE, exact
    int c;
    bool surv = false;
    if (n == 0) {
        c = 1;                                           // r = 1 at the empty walk
        o.child_w = __dmul_rn(W, a_sc);
    } else if (cuts.cut != nullptr) {
        // original PERM (Sec. 2, cut-offs T_n, t_n): copies above T_n, survival with
        // probability 1/q (weight times q) below t_n, one copy between them
        const double2 tc = __ldg(cuts.cut + n);
        if (W > tc.x) {
            c = cuts.copies < a ? cuts.copies : a;
            o.r = (double)cuts.copies;
            o.child_w = __dmul_rn(W, row[a * 8 + c]);
        } else if (W < tc.y) {
            surv = (unsigned long long)w.x < cuts.K;
            c = surv ? 1 : 0;
            o.r = cuts.inv_q;
            o.child_w = __dmul_rn(__dmul_rn(W, cuts.q), a_sc);
        } else {
            c = 1;
            o.r = 1.0;
            o.child_w = __dmul_rn(W, a_sc);
        }
    } else {
        bool amb = false;
        c = decide_estimate(x, a, w.x, surv, amb);
        if (amb || odd || force_exact) {
            // the estimate cannot settle a comparison: r exactly as defined
            const double R = ratio_exact(W, Wsum, M);
            c = decide_exact(R, a, w.x, surv);
            o.r = R;
            o.exact = true;
            if (surv) o.child_w = __dmul_rn(__dmul_rn(W, __ddiv_rn(1.0, R)), a_sc);
            else if (c > 0) o.child_w = __dmul_rn(__ddiv_rn(W, (double)c), a_sc);
        } else {
            // a survivor carries W/r = [W_n]^sample = (Wsum + W)/M, a child of an
            // enrichment (W/c) a_+ 2^-dE: one double-precision product for both.
            // invM (when nonzero) is 1/M rounded to double; the survivor's factor
            // (1/M) a_+ 2^-dE is formed beside the sum Wsum + W, so that its weight
            // (within 2^-51 of the quotient, relative) takes two dependent double
            // operations.  The tests of invM and of the outcome are integer ones
            double base = W, fac = row[a * 8 + c];
            if (surv) {
                base = __dadd_rn(Wsum, W);
                if (__double_as_longlong(invM) != 0ll) fac = __dmul_rn(invM, a_sc);
                else { base = __ddiv_rn(base, __ull2double_rn(M)); fac = a_sc; }
            }
            o.child_w = __dmul_rn(base, fac);
        }
    }
    if (c == 0) { o.outcome = kPruned; o.child_w = 0.0; return o; }
    o.c = c;
    o.dirs = choose_steps(c, a, freelist, w.y);
    o.outcome = kChildren;
    return o;
}

template <int D>
__device__ __forceinline__ int select_slot(const int (&eslot)[2 * D], int dir) {
    int s = eslot[0];
#pragma unroll
    for (int j = 1; j < 2 * D; ++j) if (j == dir) s = eslot[j];
    return s;
}

// ---------------------------------------------------------------------------
// The persistent growth kernel.
// ---------------------------------------------------------------------------
// What lets a CTA leave a run before every tour of the run has finished: in a
// batch launch, another run still has walks to grant and tours to start
// (runs_open > 0).  The first walk to find a run's tickets exhausted marks it
// closed (bit 0 of its flag; bit 1: all its walks granted); the first of those two
// marks takes the run off runs_open.  Bit 2 of the flag says that no tour of the run has
// finished for a while (its CTAs' refreshers set and clear it): such a run
// draws helper CTAs before other unfinished runs do.
struct BatchLeave {
    int *runs_open;
    int *closed;
    const int *ctas_on_run;   // CTAs growing this run now
    bool helper;              // this CTA's walks take waiting copies only
};
constexpr int kStalledBit = 4;

// The growth of one run by one CTA (Secs. 1-3): the refresher warp and the walk
// warps.  A single-run launch calls it once (bl == nullptr: the CTA stays until
// the run is complete); a batch launch calls it for each run a CTA joins.
// SHARED: every region is in shared memory (no arena), known at compile time, so
// that the walks' hashes, site lists and stacks are reached by shared-memory
// instructions rather than generic ones (a generic load that lands in shared
// memory waits longer, and in the long-scoreboard queue).
template <int D, typename Key, int MODE, bool SHARED>
__device__ __forceinline__ void grow_run(const RunDev &P, unsigned char *smem, const BatchLeave *bl,
                                         int cta_walks) {
    const int L = P.n_max + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool snapshot = (MODE == kSnapshot);
    const int K = P.stack_cache;

    // The CTA's state: the head region (header, constant tables, snapshot of W_n)
    // and one region per walk warp (occupancy hashes, site lists, stack rings).
    // Both sit in shared memory, or, for walks too long for it, the walk regions
    // (and, if even the head does not fit, the head too) in this CTA's slice of a
    // global arena, served through L1 and L2.  Each walk's data is touched by its
    // own thread only, so the same code runs on either.
    const int ST = P.stride;
    const size_t hbytes = head_region_bytes(P.n_max, snapshot);
    const size_t wbytes = warp_region_bytes(P.n_max, P.log2h, K, sizeof(Key), ST);
    unsigned char *hbase = smem, *wbase = smem + hbytes;
    if (!SHARED && P.arena_mode != kArenaNone) {
        unsigned char *a = P.arena + (size_t)blockIdx.x * (size_t)P.arena_cta_bytes;
        if (P.arena_mode == kArenaAll) { hbase = a; wbase = a + hbytes; }
        else wbase = a;
    }
    CtaHead *head = reinterpret_cast<CtaHead *>(hbase);
    double *aoc = reinterpret_cast<double *>(hbase + 64);
    unsigned char *p = hbase + 64 + 1024;
    double *Wsnap = nullptr;
    if (snapshot) {
        Wsnap = reinterpret_cast<double *>(p); p += 8 * (size_t)L;
    }

    // zero everything (empty hashes, empty stacks), then the constant tables
    for (size_t i = threadIdx.x; i < hbytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(hbase)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (size_t i = threadIdx.x; i < wbytes * P.worker_warps / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(wbase)[i] = make_uint4(0u, 0u, 0u, 0u);
    if (P.arena_mode != kArenaNone) __threadfence_block();
    __syncthreads();
    fill_aoc(aoc, D, threadIdx.x, blockDim.x);
    const long long limit = P.tour_limit;
    if (snapshot) {
        unsigned long long Ms = *(volatile unsigned long long *)P.tickets;
        if ((long long)Ms > limit) Ms = (unsigned long long)limit;
        for (int k = threadIdx.x; k < L; k += blockDim.x) Wsnap[k] = *(volatile double *)(P.Wn + k);
        if (threadIdx.x == 0) head->Ms = Ms;
    }
    __syncthreads();

    // ----------------------------------------------------------------------
    // refresher warp (snapshot form): reload the snapshot of W_n and M
    // ----------------------------------------------------------------------
    if (snapshot && warp == P.worker_warps) {
        const long long t0 = global_ns();
        unsigned long long last_fin = *(volatile unsigned long long *)P.finished;
        long long t_change = t0;
        if (lane == 0) *(volatile int *)&head->cap = P.share;
        for (long long it = 0;; ++it) {
            const long long c_it = clock64();
            const int done = __shfl_sync(kFull, *(volatile int *)&head->done_warps, 0);
            __threadfence_block();
            if (done >= P.worker_warps) {
                if (lane == 0) atomicAdd(P.refreshes, (unsigned long long)it);
                break;
            }
            unsigned long long Ms = *(volatile unsigned long long *)P.tickets;
            if ((long long)Ms > limit) Ms = (unsigned long long)limit;
            for (int k0 = 0; k0 < L; k0 += 32 * kReloadBatch) {
                double v[kReloadBatch];
#pragma unroll
                for (int j = 0; j < kReloadBatch; ++j) {
                    const int k = k0 + j * 32 + lane;
                    v[j] = k < L ? ld_relaxed(P.Wn + k) : 0.0;
                }
#pragma unroll
                for (int j = 0; j < kReloadBatch; ++j) {
                    const int k = k0 + j * 32 + lane;
                    if (k < L) *(volatile double *)&Wsnap[k] = v[j];
                }
            }
            if (lane == 0) *(volatile unsigned long long *)&head->Ms = Ms;
            if (P.share && lane == 0) {
                // idle walks not yet served by a queued copy, split over the CTAs
                const long long hg = *(volatile int *)P.hungry;
                long long q = (long long)(*(volatile unsigned long long *)P.dq_tail -
                                          *(volatile unsigned long long *)P.dq_head);
                q = q < 0 ? 0 : (q > (1 << 30) ? (1 << 30) : q);
                const long long want = hg - q;
                const long long nct = bl != nullptr ? (long long)max(1, *(volatile const int *)bl->ctas_on_run)
                                                    : (long long)gridDim.x;
                const long long per = want > 0 ? (want + nct - 1) / nct : 0;
                *(volatile int *)&head->want_don = (int)(per < (1 << 20) ? per : (1 << 20));
                *(volatile int *)&head->queued = (int)q;
                *(volatile int *)&head->status = *(volatile int *)P.status;
                *(volatile int *)&head->may_leave = (bl != nullptr && *(volatile int *)bl->runs_open > 0) ? 1 : 0;
                const unsigned long long fin_now = *(volatile unsigned long long *)P.finished;
                *(volatile unsigned long long *)&head->fin = fin_now;
                // a run whose tours stop finishing is growing a start-up tree far
                // larger than its walks can grow a few parts at a time: let its
                // tours spread over every idle walk from then on
                const long long now = global_ns();
                if (fin_now != last_fin) { last_fin = fin_now; t_change = now; }
                else if (now - t_change > P.stall_ns) *(volatile int *)&head->cap = P.share_boost;
                const int st_now = (now - t_change > P.stall_ns) ? 1 : 0;
                if (st_now != *(volatile int *)&head->stalled) {
                    *(volatile int *)&head->stalled = st_now;
                    if (bl != nullptr) {
                        if (st_now) atomicOr(bl->closed + P.run_index, kStalledBit);
                        else atomicAnd(bl->closed + P.run_index, ~kStalledBit);
                    }
                }
            }
            __syncwarp();
            // one reload per refresh period, paced on the SM's cycle counter at two
            // cycles per ns (the 2 GHz SM clock): one __nanosleep may end well before
            // or after the time it is given
            for (int nap = 0; nap < 256; ++nap) {
                const long long left = __shfl_sync(kFull, (c_it + 2ll * P.refresh_ns - clock64()) >> 1, 0);
                if (left <= 0) break;
                __nanosleep((unsigned)(left < 1000 ? left : 1000));
            }
            const bool late = (it & 15) == 0 && global_ns() - t0 > P.max_ns;
            if (__any_sync(kFull, late)) {
                if (lane == 0) set_status(P.status, PERM_ETIMEOUT);
                break;
            }
        }
    } else if (warp < P.worker_warps) {

    // ----------------------------------------------------------------------
    // worker warps
    // ----------------------------------------------------------------------
    unsigned char *wb = wbase + wbytes * warp;
    Key *hash = reinterpret_cast<Key *>(wb);
    uint16_t *sites = reinterpret_cast<uint16_t *>(
        wb + (((((size_t)1 << P.log2h) * ST * sizeof(Key)) + 15) & ~(size_t)15));
    uint32_t *smeta = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(sites) +
                                                   ((((size_t)P.n_max * ST * 2) + 15) & ~(size_t)15));
    double *sw = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(smeta) +
                                            ((((size_t)K * ST * 4) + 15) & ~(size_t)15));

    const int gwarp = blockIdx.x * P.worker_warps + warp;
    const int slot = gwarp * P.S + lane;
    const bool active = lane < P.S && slot < P.slots && warp * P.S + lane < cta_walks;
    const int sidx = active ? slot : 0;
    uint32_t *gmeta = P.gstk_meta + (size_t)sidx * P.n_max;
    double *gwt = P.gstk_w + (size_t)sidx * P.n_max;
    const unsigned lt_mask = (1u << lane) - 1u;
    const Cutoffs cuts{P.cut, P.cut_copies, P.cut_q, P.cut_inv_q, P.cut_K};
    const int dE_lo = (D == 2) ? 1 : 2;
    (void)dE_lo;

    int state = active ? kNeed : kDone;
    int n = 0, cx = 0, cy = 0, cz = 0, maxn = 0;
    double W = 1.0;
    unsigned long long ordinal = 0ull, g = 0ull;
    uint32_t seq = 0u, tour = 0u;
    int top = 0, sbase = 0;
    int un_lo = 0, un_hi = -1, pend_dir = 0, pend_depth = 0;
    int back = -1;             // the direction from the end-point to the previous site (-1: empty walk)
    bool tour_end = false;
    double pend_w = 0.0;
    unsigned long long my_steps = 0ull, my_copies = 0ull, my_exact = 0ull;
    int my_max_stack = 0;
    int cur_seq = -1;
    long long seq_t = 0;
    unsigned long long pool_lo = 0ull, pool_hi = 0ull;
    bool waiting = false;
    // tour-sum rows: with shared copies a walk has two, so that it can start its
    // next tour while parts of its last one still grow on other walks
    const int rows_per_walk = P.share ? 2 : 1;
    int myrow = sidx * rows_per_walk;
    // shared copies: the walk grows either its own tour or a part of another
    // walk's tour (own = that tour's row, did = the part's donation id)
    int own = myrow, bot = 0;
    uint32_t did = 0u;
    bool donated = false;      // a part of this walk's own tour went to another walk
    bool xbusy = false;        // every tour-sum row of this walk is still used by such parts
    // no tour tickets left; a helper (of a batch, or a walk beyond the run's tour walks)
    // takes none and grows waiting copies only
    bool exhausted = (bl != nullptr && bl->helper) || sidx >= P.tour_slots;
    int my_hungry = 0;         // lane 0: this warp's share of P.hungry
    unsigned idle_ns = 500u;   // back-off of a warp with nothing to grow
    int frow = 0, fmaxn = 0;   // tour-sum row to flush at a part's end, and its depth
    bool do_flush = false, shared_flush = false;
    const uint32_t dq_mask = (1u << P.dq_log2cap) - 1u;
    // a hand-over made in this iteration's node passes, copied after them
    int don_cell = -1, don_bdp = 0;
    uint32_t don_round = 0u;
    // a donation cell: 32-byte header, the keys of sites 0..n_max, then their slots
    const size_t cell_key_bytes = align16(((size_t)P.n_max + 1) * sizeof(Key));
    unsigned long long my_iters = 0ull;
    unsigned long long inv_of = 0ull;   // the snapshot M whose reciprocal inv_ms holds
    double inv_ms = 0.0;
    double *Wrow = P.Wn;
    unsigned long long *Srow = P.Sn;
    double *Rrow = P.Rn;

    const long long t_start = global_ns();
    for (long long iter = 0;; ++iter) {
        const bool late = (iter & 255) == 0 && global_ns() - t_start > P.max_ns;
        if (__any_sync(kFull, late)) {
            if (lane == 0) set_status(P.status, PERM_ETIMEOUT);
            break;
        }
        // in a batch launch a failed run stops at once, so that its CTAs move on
        // (the whole warp leaves together: one lane's read decides)
        if (bl != nullptr && (iter & 255) == 0 && __shfl_sync(kFull, *(volatile int *)P.status, 0) != 0) break;
        // ---------------- tour tickets ----------------
        if (state == kNeed && xbusy) {
            if (*(volatile unsigned int *)(P.outst + myrow) == kRowFree) xbusy = false;
            else if (rows_per_walk == 2 && *(volatile unsigned int *)(P.outst + (myrow ^ 1)) == kRowFree) {
                myrow ^= 1;
                xbusy = false;
            }
        }
        const bool want_t = state == kNeed && !xbusy && !exhausted;
        const unsigned need = __ballot_sync(kFull, want_t);
        if (need) {
            if (P.alg == PERM_ALG2) {
                const unsigned cnt = __popc(need);
                const unsigned rank = __popc(need & lt_mask);
                const unsigned long long avail = pool_hi - pool_lo;
                unsigned long long base = 0ull, take = 0ull;
                if (avail < cnt) {
                    // fetch tickets; admission keeps tours in flight at most
                    // c0 + gamma * finished (a partial grant is allowed)
                    const int leader = __ffs(need) - 1;
                    const unsigned long long want = cnt - avail + (snapshot ? (unsigned long long)kPoolExtra : 0ull);
                    if (lane == leader) {
                        if (P.ramp_c0 < 0) {
                            base = atomicAdd(P.tickets, want);
                            take = want;
                        } else {
                            for (int attempt = 0; attempt < 64; ++attempt) {
                                const unsigned long long t_now = *(volatile unsigned long long *)P.tickets;
                                const unsigned long long f_now = *(volatile unsigned long long *)P.finished;
                                unsigned long long k = want;
                                if ((long long)t_now < limit) {
                                    const unsigned long long allow = (unsigned long long)P.ramp_c0 +
                                                                     ((f_now * P.ramp_gamma_q16) >> 16);
                                    const unsigned long long infl = t_now - (f_now < t_now ? f_now : t_now);
                                    k = allow > infl ? allow - infl : 0ull;
                                    k = k < want ? k : want;
                                }
                                if (k == 0ull) break;
                                if (atomicCAS(P.tickets, t_now, t_now + k) == t_now) {
                                    base = t_now;
                                    take = k;
                                    break;
                                }
                            }
                        }
                    }
                    base = __shfl_sync(kFull, base, leader);
                    take = __shfl_sync(kFull, take, leader);
                }
                const bool served = rank < avail + take;
                if (want_t && served) g = (rank < avail) ? pool_lo + rank : base + (rank - avail);
                if (avail >= cnt) {
                    pool_lo += cnt;
                } else if (avail + take > cnt) {
                    pool_lo = base + (cnt - avail);
                    pool_hi = base + take;
                } else {
                    pool_lo = pool_hi = 0ull;      // pool and grant all handed out
                }
                if (want_t && !served) {
                    waiting = true;                // not admitted yet: try again next round
                } else if (want_t) {
                    waiting = false;
                    if ((long long)g >= limit) {
                        if (P.share) exhausted = true;   // idle: may still take shared copies
                        else state = kDone;
                        if (bl != nullptr && (atomicOr(bl->closed + P.run_index, 1) & 3) == 0)
                            atomicSub(bl->runs_open, 1);
                    } else {
                        seq = (uint32_t)(g % (unsigned long long)P.n_seq);
                        tour = (uint32_t)(g / (unsigned long long)P.n_seq);
                    }
                }
            } else if (state == kNeed) {
                // Algorithm 1: a walk owns a sequence until its tours are done
                if (cur_seq < 0 || seq_t >= P.seq_target) {
                    const unsigned long long s = atomicAdd(P.tickets, 1ull);
                    if (s >= (unsigned long long)P.n_seq) {
                        state = kDone;
                    } else {
                        cur_seq = (int)s;
                        seq_t = (long long)P.seq_M[s];
                        Wrow = P.Wn + (size_t)s * L;
                        Srow = P.Sn + (size_t)s * L;
                        if (P.Rn != nullptr) Rrow = P.Rn + (size_t)s * L;
                    }
                }
                if (state == kNeed && cur_seq >= 0 && seq_t < P.seq_target) {
                    seq = (uint32_t)cur_seq;
                    tour = (uint32_t)seq_t;
                    g = (unsigned long long)seq_t;
                } else if (state == kNeed) {
                    cur_seq = -1;          // sequence finished: ask again next round
                }
            }
            if (state == kNeed && !waiting && !xbusy && !exhausted && (P.alg == PERM_ALG2 || cur_seq >= 0)) {
                // start a tour at the empty walk (Sec. 1: W(empty) = 1)
                n = 0; cx = cy = cz = 0; maxn = 0; W = 1.0; ordinal = 0ull; back = -1;
                top = 0; sbase = 0; bot = 0;
                own = myrow; did = 0u; donated = false;
                const int s0 = hash_insert<Key>(hash, ST, lane, P.log2h,
                                                KeyCodec<D, Key>::encode(0, 0, 0));
                if (s0 < 0) { set_status(P.status, PERM_EOVERFLOW); state = kDone; }
                else { sites[lane] = (uint16_t)s0; state = kNode; }
            }
        }
        if (P.share) {
            // ---------------- shared copies: idle walks take queued ones ----------------
            const bool idle = state == kNeed && (waiting || xbusy || exhausted);
            const unsigned hm = __ballot_sync(kFull, idle);
            // one lane's read of the queue length decides for the warp (the block
            // below exchanges values across all lanes)
            if (hm && __shfl_sync(kFull, *(volatile int *)&head->queued, 0) > 0) {
                const int leader = __ffs(hm) - 1;
                unsigned long long base = 0ull, take = 0ull;
                if (lane == leader) {
                    for (int attempt = 0; attempt < 8; ++attempt) {
                        const unsigned long long h0 = *(volatile unsigned long long *)P.dq_head;
                        const unsigned long long t0 = *(volatile unsigned long long *)P.dq_tail;
                        if (t0 <= h0) break;
                        unsigned long long k = t0 - h0;
                        k = k < (unsigned long long)__popc(hm) ? k : (unsigned long long)__popc(hm);
                        if (atomicCAS(P.dq_head, h0, h0 + k) == h0) { base = h0; take = k; break; }
                    }
                }
                base = __shfl_sync(kFull, base, leader);
                take = __shfl_sync(kFull, take, leader);
                const unsigned rk = __popc(hm & lt_mask);
                bool claiming = idle && rk < take;
                unsigned long long pos = 0ull;
                uint32_t cell = 0u, round = 0u;
                int cdp = -1;
                if (claiming) {
                    pos = base + rk;
                    cell = (uint32_t)pos & dq_mask;
                    round = (uint32_t)(pos >> P.dq_log2cap);
                    bool ok = false;
                    for (int spin = 0; spin < kCellSpin; ++spin) {
                        if (*(volatile unsigned int *)(P.dq_ready + cell) == round + 1u) { ok = true; break; }
                        __nanosleep(32);
                    }
                    if (!ok || pos + 1ull >= (1ull << 32)) {
                        set_status(P.status, ok ? PERM_EOVERFLOW : PERM_ETIMEOUT);
                        state = kDone;
                        claiming = false;
                    } else {
                        __threadfence();
                        cdp = (int)__ldcg(reinterpret_cast<const unsigned int *>(P.dq_cells + (size_t)cell *
                                                                                (size_t)P.dq_cell_bytes) + 3);
                    }
                }
                // the walk up to the branch point (Sec. 1), each site straight into the
                // slot it had in the donor's hash; the whole warp places one taker's
                // sites at a time (the taker's hash is empty: it had no walk)
                unsigned cm = __ballot_sync(kFull, claiming);
                while (cm) {
                    const int src = __ffs(cm) - 1;
                    cm &= cm - 1u;
                    const uint32_t scell = __shfl_sync(kFull, cell, src);
                    const int sdp = __shfl_sync(kFull, cdp, src);
                    const unsigned char *cb = P.dq_cells + (size_t)scell * (size_t)P.dq_cell_bytes;
                    const Key *ck = reinterpret_cast<const Key *>(cb + 32);
                    const uint16_t *cs = reinterpret_cast<const uint16_t *>(cb + 32 + cell_key_bytes);
                    place_sites_from_cell<Key>(hash, sites, ST, src, sdp, ck, cs, lane);
                }
                __syncwarp();
                if (claiming) {
                    const unsigned char *cb = P.dq_cells + (size_t)cell * (size_t)P.dq_cell_bytes;
                    const uint4 h0 = __ldcg(reinterpret_cast<const uint4 *>(cb));
                    const uint2 h1 = __ldcg(reinterpret_cast<const uint2 *>(cb + 16));
                    const double cw = __longlong_as_double(__ldcg(reinterpret_cast<const long long *>(cb + 24)));
                    const int dp = (int)h0.w;
                    const uint32_t meta = h1.x;
                    __threadfence();
                    *(volatile unsigned int *)(P.dq_free + cell) = round + 1u;
                    own = (int)h0.x; seq = h0.y; tour = h0.z;
                    g = (unsigned long long)tour * (unsigned long long)P.n_seq + seq;
                    did = (uint32_t)(pos + 1ull);
                    ordinal = (unsigned long long)did << 32;
                    donated = false; maxn = 0;
                    top = 0; sbase = 0; bot = 0;
                    const int cnt = (int)((meta >> 16) & 7u);
                    const uint32_t dirs = meta >> 19;
                    pend_dir = (int)(dirs & 7u);
                    pend_w = cw;
                    pend_depth = dp;
                    if (cnt > 1) {
                        smeta[lane] = (uint32_t)dp | ((uint32_t)(cnt - 1) << 16) | ((dirs >> 3) << 19);
                        sw[lane] = cw;
                        top = 1;
                    }
                    un_lo = dp + 1; un_hi = dp; tour_end = false;
                    waiting = false;
                    state = kUnwindState;      // resumes at the branch point below
                }
            }
            const int hcount = __popc(__ballot_sync(kFull, state == kNeed && (waiting || xbusy || exhausted)));
            if (lane == 0 && hcount != my_hungry) {
                atomicAdd(P.hungry, hcount - my_hungry);
                my_hungry = hcount;
            }
            // walks with no tickets left stop once every tour of the launch has
            // finished (or the run has failed)
            if (state == kNeed && exhausted &&
                ((long long)*(volatile unsigned long long *)&head->fin >= limit || *(volatile int *)&head->status != 0 ||
                 (!xbusy && *(volatile int *)&head->may_leave != 0)))
                state = kDone;
        }
        const unsigned live = __ballot_sync(kFull, state != kDone);
        if (!live) break;
        ++my_iters;
        if (__all_sync(kFull, state == kDone || (state == kNeed && (waiting || xbusy || exhausted)))) {
            __nanosleep(idle_ns);
            idle_ns = idle_ns < 4000u ? 2u * idle_ns : 4000u;
        } else {
            idle_ns = 500u;
        }

        // ---------------- nodes: up to kNodePasses per iteration ----------------
        // A walk whose node made children grows its next node in the same
        // iteration, so that the warp-wide parts of the loop are shared by more
        // nodes; a walk that reached a leaf waits for the backtrack below.
        for (int pass = 0; pass < kNodePasses; ++pass) {
        if (pass > 0 && !__any_sync(kFull, state == kNode)) break;
        // the snapshot's M for this pass, and its reciprocal (taken by the whole warp
        // once per new snapshot: double-precision arithmetic is slow on this part)
        unsigned long long Ms_p = 0ull;
        if (snapshot) {
            Ms_p = __shfl_sync(kFull, *(volatile unsigned long long *)&head->Ms, 0);
            if (Ms_p != inv_of) { inv_of = Ms_p; inv_ms = __drcp_rn(__ull2double_rn(Ms_p)); }
        }
        if (state == kNode) {
            // the sum of the weights recorded at this length before the node (a
            // snapshot, or the global table's value returned by the node's own add)
            // and the tours started, this one included
            double Wsum;
            unsigned long long Mb;
            if (snapshot) {
                // fire-and-forget reductions into the global table (no value comes back)
                atomicAdd(P.Wn + n, W);
                atomicAdd(P.Sn + n, 1ull);
                Wsum = *(volatile double *)&Wsnap[n];
                Mb = Ms_p > g + 1ull ? Ms_p : g + 1ull;
            } else {
                Wsum = atomicAdd(&Wrow[n], W);
                atomicAdd(&Srow[n], 1ull);
                if (P.alg == PERM_ALG2) {
                    unsigned long long Mt = *(volatile unsigned long long *)P.tickets;
                    if ((long long)Mt > limit) Mt = (unsigned long long)limit;
                    Mb = Mt > g + 1ull ? Mt : g + 1ull;
                } else {
                    Mb = (unsigned long long)seq_t + 1ull;
                }
            }
            atomicAdd(P.X + (size_t)own * L + n, W);
            if (P.Rn != nullptr) {
                // the observable of Sec. 1, eq. 5: W |omega_n|^2 (exact integer square)
                const long long r2 = (long long)cx * cx + (long long)cy * cy + (long long)cz * cz;
                atomicAdd(Rrow + n, __dmul_rn(W, (double)r2));
            }
            maxn = n > maxn ? n : maxn;
            ++my_steps;

            int eslot[2 * D];
#pragma unroll
            for (int j = 0; j < 2 * D; ++j) eslot[j] = 0;
            const NodeOut o = grow_node<D, Key>(hash, ST, lane, P.log2h, n, P.n_max, cx, cy, cz, W, Wsum,
                                                Mb, ordinal, seq, tour, P.key0, P.key1, aoc, eslot, cuts,
                                                (snapshot && Mb == Ms_p) ? inv_ms : 0.0, back);
            if (o.overflow) set_status(P.status, PERM_EOVERFLOW);
            my_exact += o.exact ? 1ull : 0ull;

            if (P.trace != nullptr && (ordinal % (unsigned long long)P.trace_every) == 0ull &&
                ((unsigned long long)tour % (unsigned long long)P.trace_tour_every) == 0ull) {
                const unsigned long long idx = atomicAdd(P.trace_count, 1ull);
                if (idx < (unsigned long long)P.trace_cap) {
                    perm_trace_record *rec = P.trace + idx;
                    rec->n = n; rec->a_plus = o.a; rec->free_mask = o.mask; rec->c = o.c;
                    rec->outcome = o.outcome; rec->exact = o.exact ? 1 : 0;
                    for (int i = 0; i < 6; ++i)
                        rec->dirs[i] = (i < o.c) ? (int)((o.dirs >> (3 * i)) & 7u) : -1;
                    rec->seq = seq; rec->tour = tour;
                    rec->ordinal = ordinal; rec->M = Mb;
                    rec->W = W; rec->Wsum = Wsum; rec->r = o.r; rec->child_w = o.child_w;
                    int32_t *cc = P.trace_coords + (size_t)idx * L * D;
                    for (int k = 0; k < n; ++k) {
                        int x, y, z;
                        KeyCodec<D, Key>::decode(hash[(uint32_t)sites[(uint32_t)k * ST + lane] * ST + lane], x, y, z);
                        cc[k * D] = x; cc[k * D + 1] = y;
                        if (D == 3) cc[k * D + 2] = z;
                    }
                    cc[n * D] = cx; cc[n * D + 1] = cy;
                    if (D == 3) cc[n * D + 2] = cz;
                }
            }

            if ((uint32_t)ordinal == 0xFFFFFFFFu) set_status(P.status, PERM_EOVERFLOW);
            ordinal += 1ull;
            if (o.outcome == kChildren) {
                const int c = o.c;
                my_copies += (unsigned long long)(c - 1);
                if (c > 1) {
                    // copies 1..c-1 wait in one record (depth, count, steps, weight)
                    if (top - sbase == K) {
                        // ring full: the oldest kChunk records go to global memory
#pragma unroll
                        for (int i = 0; i < kChunk; ++i) {
                            const int idx = sbase + i;
                            gmeta[idx] = smeta[(uint32_t)(idx & (K - 1)) * ST + lane];
                            gwt[idx] = sw[(uint32_t)(idx & (K - 1)) * ST + lane];
                        }
                        sbase += kChunk;
                    }
                    if (top >= P.n_max) {
                        set_status(P.status, PERM_EOVERFLOW);
                    } else {
                        const uint32_t rest = (o.dirs >> 3) & ((1u << (3 * (c - 1))) - 1u);
                        const int ti = top & (K - 1);
                        smeta[(uint32_t)ti * ST + lane] = (uint32_t)n | ((uint32_t)(c - 1) << 16) | (rest << 19);
                        sw[(uint32_t)ti * ST + lane] = o.child_w;
                        ++top;
                        my_max_stack = top - bot > my_max_stack ? top - bot : my_max_stack;
                    }
                }
                const int dir0 = (int)(o.dirs & 7u);
                const int s0 = select_slot<D>(eslot, dir0);
                step_coords(dir0, cx, cy, cz);
                back = dir0 ^ 1;
                n += 1;
                if (n < P.n_max) {
                    hash[(uint32_t)s0 * ST + lane] = KeyCodec<D, Key>::encode(cx, cy, cz);
                    sites[(uint32_t)n * ST + lane] = (uint16_t)s0;
                }
                W = o.child_w;
                if (snapshot && P.share && don_cell < 0 && top - bot >= 2 && *(volatile int *)&head->want_don > 0) {
                    // hand the oldest waiting copy record to an idle walk: its subtree
                    // grows there, and its weights still go to this tour's row `own`.
                    // The header is written now; the walk's sites 0..bdp go into the
                    // cell after the node passes, copied by the whole warp
                    const uint32_t bi = (uint32_t)(bot & (K - 1)) * ST + lane;
                    const uint32_t bm = bot < sbase ? gmeta[bot] : smeta[bi];
                    const double bw = bot < sbase ? gwt[bot] : sw[bi];
                    const int bdp = (int)(bm & 0xFFFFu);
                    // at most P.share parts of one tour grow at once (a soft cap: the
                    // parts of a tour stay few, so each still sees its siblings' samples)
                    bool room = true;
                    if (!(did == 0u && !donated))
                        room = *(volatile unsigned int *)(P.outst + own) < (unsigned)*(volatile int *)&head->cap;
                    if (room && P.n_max - bdp >= kMinShareGap && atomicSub(&head->want_don, 1) > 0) {
                        unsigned long long pos = 0ull;
                        bool got = false;
                        for (int attempt = 0; attempt < 8; ++attempt) {
                            const unsigned long long t0 = *(volatile unsigned long long *)P.dq_tail;
                            const uint32_t c0 = (uint32_t)t0 & dq_mask;
                            if (*(volatile unsigned int *)(P.dq_free + c0) != (uint32_t)(t0 >> P.dq_log2cap)) break;
                            if (atomicCAS(P.dq_tail, t0, t0 + 1ull) == t0) { pos = t0; got = true; break; }
                        }
                        if (got) {
                            if (did == 0u && !donated) { P.outst[own] = 2u; donated = true; }
                            else atomicAdd(P.outst + own, 1u);
                            const uint32_t cell = (uint32_t)pos & dq_mask;
                            unsigned char *cb = P.dq_cells + (size_t)cell * (size_t)P.dq_cell_bytes;
                            *reinterpret_cast<uint4 *>(cb) = make_uint4((uint32_t)own, seq, tour, (uint32_t)bdp);
                            *reinterpret_cast<uint2 *>(cb + 16) = make_uint2(bm, 0u);
                            *reinterpret_cast<double *>(cb + 24) = bw;
                            don_cell = (int)cell;
                            don_round = (uint32_t)(pos >> P.dq_log2cap);
                            don_bdp = bdp;
                            bot += 1;
                            if (sbase < bot) sbase = bot;
                        } else {
                            atomicAdd(&head->want_don, 1);
                        }
                    }
                }
            } else {
                // leaf: resume the most recent waiting copy, or end the tour
                if (top == sbase && sbase > bot) {
                    // ring empty: bring back up to kChunk records, all loads in flight
                    // before the first store (one round trip to L2, not kChunk)
                    const int lo = sbase - kChunk > bot ? sbase - kChunk : bot;
                    uint32_t fmeta[kChunk];
                    double fw[kChunk];
#pragma unroll
                    for (int i = 0; i < kChunk; ++i) {
                        const int idx = lo + i;
                        fmeta[i] = idx < sbase ? __ldcg(gmeta + idx) : 0u;
                        fw[i] = idx < sbase ? __ldcg(gwt + idx) : 0.0;
                    }
#pragma unroll
                    for (int i = 0; i < kChunk; ++i) {
                        const int idx = lo + i;
                        if (idx < sbase) {
                            smeta[(uint32_t)(idx & (K - 1)) * ST + lane] = fmeta[i];
                            sw[(uint32_t)(idx & (K - 1)) * ST + lane] = fw[i];
                        }
                    }
                    sbase = lo;
                }
                const int hi = n < P.n_max - 1 ? n : P.n_max - 1;
                if (top == bot) {
                    un_lo = 0; un_hi = hi; tour_end = true;
                } else {
                    const int ti = (top - 1) & (K - 1);
                    const uint32_t meta = smeta[(uint32_t)ti * ST + lane];
                    const int dp = (int)(meta & 0xFFFFu);
                    const int cnt = (int)((meta >> 16) & 7u);
                    const uint32_t dirs = meta >> 19;
                    pend_dir = (int)(dirs & 7u);
                    pend_w = sw[(uint32_t)ti * ST + lane];
                    pend_depth = dp;
                    if (cnt <= 1) --top;
                    else smeta[(uint32_t)ti * ST + lane] = (uint32_t)dp | ((uint32_t)(cnt - 1) << 16) | ((dirs >> 3) << 19);
                    un_lo = dp + 1; un_hi = hi; tour_end = false;
                }
                state = kUnwindState;
            }
        }
        }

        // ---------------- hand-overs: the whole warp copies each donor's sites ----------------
        // A donor's sites 0..bdp are still in its hash (this iteration's deletions come
        // below), each in the slot an in-order rebuild would give it, so the cell holds
        // (key, slot) per site and the taker places them without probing.
        if (P.share) {
            unsigned dm = __ballot_sync(kFull, don_cell >= 0);
            if (dm) __syncwarp();          // every lane sees the donors' sites
            while (dm) {
                const int src = __ffs(dm) - 1;
                dm &= dm - 1u;
                const int scell = __shfl_sync(kFull, don_cell, src);
                const int sbdp = __shfl_sync(kFull, don_bdp, src);
                unsigned char *cb = P.dq_cells + (size_t)scell * (size_t)P.dq_cell_bytes;
                Key *ck = reinterpret_cast<Key *>(cb + 32);
                uint16_t *cs = reinterpret_cast<uint16_t *>(cb + 32 + cell_key_bytes);
                copy_sites_to_cell<Key>(hash, sites, ST, src, sbdp, ck, cs, lane);
                __syncwarp();
                if (lane == src) {
                    __threadfence();
                    *(volatile unsigned int *)(P.dq_ready + scell) = don_round + 1u;
                }
            }
            don_cell = -1;
        }

        // ---------------- backtrack: LIFO deletions, then resume ----------------
        if (state == kUnwindState) {
#pragma unroll
            for (int i = 0; i < kUnwind; ++i) {
                const int k = un_hi - i;
                if (k >= un_lo) hash[(uint32_t)sites[(uint32_t)k * ST + lane] * ST + lane] = (Key)0;
            }
            un_hi -= kUnwind;
            if (un_hi < un_lo) {
                if (tour_end) {
                    state = kFlush;
                } else {
                    const int dp = pend_depth;
                    KeyCodec<D, Key>::decode(hash[(uint32_t)sites[(uint32_t)dp * ST + lane] * ST + lane], cx, cy, cz);
                    step_coords(pend_dir, cx, cy, cz);
                    back = pend_dir ^ 1;
                    n = dp + 1;
                    if (n < P.n_max) {
                        const int s = hash_insert<Key>(hash, ST, lane, P.log2h, KeyCodec<D, Key>::encode(cx, cy, cz));
                        if (s < 0) { set_status(P.status, PERM_EOVERFLOW); state = kDone; }
                        else sites[(uint32_t)n * ST + lane] = (uint16_t)s;
                    }
                    W = pend_w;
                    if (state != kDone) state = kNode;
                }
            }
        }

        // ---------------- end of a tour (part): per-tour sums into Q (whole warp) ----------------
        if (__any_sync(kFull, state == kFlush)) {
            if (state == kFlush) {
                if (did == 0u && !donated) {
                    // the whole tour grew on this walk
                    frow = own; fmaxn = maxn; do_flush = true; shared_flush = false;
                } else {
                    // parts of the tour grew elsewhere: the last part to end flushes
                    const unsigned om = atomicMax(P.tmaxn + own, (unsigned)maxn);
                    __threadfence();
                    const unsigned left = atomicSub(P.outst + own, 1u);
                    do_flush = (left == 1u);
                    shared_flush = true;
                    frow = own;
                    fmaxn = (int)(om > (unsigned)maxn ? om : (unsigned)maxn);
                    if (!do_flush && did == 0u) {
                        // the row stays with the parts still growing: the next tour
                        // takes the walk's other row, if that one is free
                        myrow ^= rows_per_walk - 1;
                        xbusy = *(volatile unsigned int *)(P.outst + myrow) != kRowFree;
                    }
                }
            }
            unsigned fm = __ballot_sync(kFull, state == kFlush && do_flush);
            __threadfence();
            __syncwarp();
            while (fm) {
                const int src = __ffs(fm) - 1;
                fm &= fm - 1u;
                const int s_slot = __shfl_sync(kFull, frow, src);
                const int s_maxn = __shfl_sync(kFull, fmaxn, src);
                const int s_seq = __shfl_sync(kFull, cur_seq, src);
                double *Xr = P.X + (size_t)s_slot * L;
                double *Qr = (P.alg == PERM_ALG1) ? P.Qn + (size_t)(s_seq < 0 ? 0 : s_seq) * L : P.Qn;
                // eight loads in flight per lane, then the squares go straight to Q_n
                for (int k0 = 0; k0 <= s_maxn; k0 += 32 * 8) {
                    double x[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = k0 + u * 32 + lane;
                        x[u] = (k <= s_maxn) ? __ldcg(Xr + k) : 0.0;
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = k0 + u * 32 + lane;
                        if (__double_as_longlong(x[u]) != 0ll) {     // (an integer test: no -0.0 here)
                            atomicAdd(&Qr[k], __dmul_rn(x[u], x[u]));
                            __stcg(Xr + k, 0.0);
                        }
                    }
                }
            }
            __threadfence();
            __syncwarp();
            if (state == kFlush) {
                if (do_flush) {
                    if (shared_flush) {
                        P.tmaxn[frow] = 0u;
                        __threadfence();
                        *(volatile unsigned int *)(P.outst + frow) = kRowFree;
                    }
                    atomicAdd(P.finished, 1ull);
                    if (P.alg == PERM_ALG1) {
                        seq_t += 1;
                        P.seq_M[cur_seq] = (unsigned long long)seq_t;
                    }
                }
                own = myrow; did = 0u; donated = false; do_flush = false;
                state = kNeed;
            }
        }
    }
    if (P.share && lane == 0 && my_hungry != 0) atomicAdd(P.hungry, -my_hungry);

    // statistics, then tell the refresher this warp is done
    unsigned long long tot = my_steps, cps = my_copies, exn = my_exact;
    int ms = my_max_stack;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        tot += __shfl_xor_sync(kFull, tot, off);
        cps += __shfl_xor_sync(kFull, cps, off);
        exn += __shfl_xor_sync(kFull, exn, off);
        const int o = __shfl_xor_sync(kFull, ms, off);
        ms = o > ms ? o : ms;
    }
    if (lane == 0) {
        atomicAdd(P.steps, tot);
        atomicAdd(P.copies, cps);
        if (exn) atomicAdd(P.exact_steps, exn);
        atomicAdd(P.iterations, my_iters);
        atomicMax(P.max_stack, (unsigned long long)ms);
        __threadfence_block();
        atomicAdd(&head->done_warps, 1);
    }
    }   // worker warps
}

template <int D, typename Key, int MODE>
__global__ void __launch_bounds__(32 * 9, 1) grow_kernel(const __grid_constant__ RunDev P) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (P.arena_mode == kArenaNone) grow_run<D, Key, MODE, true>(P, smem, nullptr, P.worker_warps * P.S);
    else grow_run<D, Key, MODE, false>(P, smem, nullptr, P.worker_warps * P.S);
}

// ---------------------------------------------------------------------------
// Batch launch: R runs grown by one persistent grid.  Each CTA picks the open
// run (tours left to start, walks left to grant) with the most tours left to
// start per CTA already on it, weighted by n_max + 1, copies its descriptor to
// shared memory, lays its shared memory out for that run and grows it until
// the run is complete, or until its walks have no tickets left while another
// run is open; then it picks again.  A run's tour-growing walks (at most one per
// sequence, as in a single launch) are granted to the CTAs that join it.  With
// no run open, a CTA joins an unfinished run (a stalled one first) as a helper
// whose walks take waiting copies only.
// ---------------------------------------------------------------------------
// Returns the run to join (walks: how many of the CTA's walks grow tours), -1
// when no run can take the CTA now, -2 when every run has finished or failed.
__device__ int pick_run(const BatchDev &B, int &walks, bool &helper) {
    int best = -1, stall = -1;
    double best_s = -1.0, stall_s = -1.0;
    bool best_open = false, unfinished = false;
    for (int r = 0; r < B.R; ++r) {
        const RunDev &Q = B.runs[r];
        if (*(volatile int *)Q.status != 0) continue;
        const long long lim = Q.tour_limit;
        const long long f = (long long)*(volatile unsigned long long *)Q.finished;
        if (f >= lim) continue;
        unfinished = true;
        const long long t = (long long)*(volatile unsigned long long *)Q.tickets;
        const int a = *(volatile int *)(B.active + r);
        const int g = *(volatile int *)(B.granted + r);
        const double len = (double)(Q.n_max + 1);
        // a run stalled on a large tour is the batch's critical path: among runs
        // that take helpers it comes first, up to the CTAs its parts can use
        const int fl = *(volatile int *)(B.closed + r);
        if ((fl & kStalledBit) && Q.share && a * Q.worker_warps * Q.S < Q.share_boost) {
            const double sc = (double)(lim - f) * len / (double)(a + 1);
            if (sc > stall_s) { stall = r; stall_s = sc; }
        }
        if (t < lim) {
            if (g < Q.n_seq) {
                const double sc = (double)(lim - t) * len / (double)(a + 1);
                if (!best_open || sc > best_s) { best = r; best_s = sc; best_open = true; }
            }
        } else if (!best_open && Q.share) {
            const double sc = (double)(lim - f) * len / (double)(a + 1);
            if (sc > best_s) { best = r; best_s = sc; }
        }
    }
    walks = 0;
    helper = false;
    if (stall >= 0 && !best_open) best = stall;
    if (best < 0) return unfinished ? -1 : -2;
    const RunDev &Q = B.runs[best];
    const int cap = Q.worker_warps * Q.S;
    if (best_open) {
        // grant up to a CTA's worth of walks, never more than one per sequence
        for (int attempt = 0; attempt < 64; ++attempt) {
            const int g = *(volatile int *)(B.granted + best);
            const int k = Q.n_seq - g < cap ? Q.n_seq - g : cap;
            if (k <= 0) break;
            if (atomicCAS(B.granted + best, g, g + k) == g) {
                walks = k;
                if (g + k >= Q.n_seq && (atomicOr(B.closed + best, 2) & 3) == 0) atomicSub(B.runs_open, 1);
                break;
            }
        }
        if (walks == 0) return -1;
    } else {
        walks = cap;                    // helper
        helper = true;
    }
    atomicAdd(B.active + best, 1);
    return best;
}

template <int MODE>
__global__ void __launch_bounds__(32 * 9, 1) batch_kernel(const BatchDev B) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ RunDev Ps;
    __shared__ int cur, walks, helping;
    const long long t0 = global_ns();
    for (;;) {
        if (threadIdx.x == 0) {
            int w = 0;
            bool hp = false;
            int r = pick_run(B, w, hp);
            helping = hp ? 1 : 0;
            if (r == -1 && global_ns() - t0 > B.max_ns) {
                // the batch's time is up: every run not finished fails
                for (int q = 0; q < B.R; ++q) {
                    const RunDev &Q = B.runs[q];
                    if ((long long)*(volatile unsigned long long *)Q.finished < Q.tour_limit)
                        set_status(Q.status, PERM_ETIMEOUT);
                }
                r = -2;
            }
            cur = r;
            walks = w;
        }
        __syncthreads();
        const int r = cur;
        if (r == -2) break;
        if (r == -1) {
            __nanosleep(8000);
            __syncthreads();
            continue;
        }
        const uint32_t *src = reinterpret_cast<const uint32_t *>(B.runs + r);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&Ps);
        for (int i = threadIdx.x; i < (int)(sizeof(RunDev) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
        __syncthreads();
        const BatchLeave bl{B.runs_open, B.closed, B.active + r, helping != 0};
        const int cw = walks;
        // a batch member's walks are laid out in shared memory (never the arena)
        if (Ps.d == 2) grow_run<2, uint32_t, MODE, true>(Ps, smem, &bl, cw);
        else if (Ps.n_max > 512) grow_run<3, unsigned long long, MODE, true>(Ps, smem, &bl, cw);
        else grow_run<3, uint32_t, MODE, true>(Ps, smem, &bl, cw);
        __syncthreads();
        if (threadIdx.x == 0) atomicSub(B.active + r, 1);
        __syncthreads();
    }
}

// Scheduling counters of a batch launch: nothing granted, no CTA on a run; a run
// with no tours left to start counts as closed.
__global__ void batch_init_kernel(const BatchDev B) {
    __shared__ int open;
    if (threadIdx.x == 0) open = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < B.R; r += blockDim.x) {
        // a run grows in this launch if it has tours left to start (a continued
        // batch leaves retired runs with none)
        const bool grows = B.runs[r].tour_limit > (long long)*(volatile unsigned long long *)B.runs[r].tickets;
        B.active[r] = 0;
        B.granted[r] = 0;
        B.closed[r] = grows ? 0 : 3;
        if (grows) atomicAdd(&open, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *B.runs_open = open;
}

// ---------------------------------------------------------------------------
// Growth step on caller-given snapshot states (one thread per state).
// ---------------------------------------------------------------------------
template <int D, typename Key>
__global__ void __launch_bounds__(32) debug_step_kernel(int n_max, int log2h, int B,
        const int32_t *coords, const int32_t *len, const double *Wv, const double *Wsv,
        const uint64_t *Mv, const uint64_t *ordv, const uint32_t *seqv, const uint32_t *tourv,
        uint32_t k0, uint32_t k1, int force_exact, int32_t *out_i, double *out_r, double *out_w) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = 1 << log2h;
    Key *hash = reinterpret_cast<Key *>(smem);
    double *aoc = reinterpret_cast<double *>(smem + (size_t)H * kStride * sizeof(Key));
    const int lane = threadIdx.x;
    fill_aoc(aoc, D, lane, 32);
    for (int s = 0; s < H; ++s) hash[(size_t)s * kStride + lane] = (Key)0;
    __syncwarp();
    const int b = blockIdx.x * 32 + lane;
    if (b >= B) return;
    int32_t *oi = out_i + (size_t)b * 11;
    const int n = len[b];
    if (n < 0 || n > n_max) { oi[0] = -1; return; }
    const int32_t *cb = coords + (size_t)b * (n_max + 1) * D;
    bool ovf = false;
    const int top = n < n_max - 1 ? n : n_max - 1;
    for (int k = 0; k <= top; ++k) {
        const Key key = KeyCodec<D, Key>::encode(cb[k * D], cb[k * D + 1], D == 3 ? cb[k * D + 2] : 0);
        if (hash_insert<Key>(hash, kStride, lane, log2h, key) < 0) ovf = true;
    }
    const int cx = cb[n * D], cy = cb[n * D + 1], cz = (D == 3) ? cb[n * D + 2] : 0;
    int eslot[2 * D];
    const Cutoffs none{nullptr, 1, 1.0, 1.0, 0ull};
    const NodeOut o = grow_node<D, Key>(hash, kStride, lane, log2h, n, n_max, cx, cy, cz, Wv[b],
                                        Wsv[b], Mv[b], ordv[b], seqv[b], tourv[b], k0, k1, aoc, eslot,
                                        none, 0.0, -1, force_exact != 0);
    oi[0] = (ovf || o.overflow) ? -2 : o.outcome;
    oi[1] = o.a;
    oi[2] = o.mask;
    oi[3] = o.c;
    for (int i = 0; i < 6; ++i) oi[4 + i] = (i < o.c) ? (int)((o.dirs >> (3 * i)) & 7u) : -1;
    oi[10] = o.exact ? 1 : 0;
    out_r[b] = o.r;
    out_w[b] = o.child_w;
}

__global__ void philox_kernel(int B, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const Philox4 w = philox4x32_10(ctr[4 * b], ctr[4 * b + 1], ctr[4 * b + 2], ctr[4 * b + 3], k0, k1);
    out[4 * b] = w.x; out[4 * b + 1] = w.y; out[4 * b + 2] = w.z; out[4 * b + 3] = w.w;
}

__global__ void finalize_kernel(unsigned long long *tickets, long long limit) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if ((long long)*tickets > limit) *tickets = (unsigned long long)limit;
    }
}

}  // namespace

size_t cta_smem_bytes(int d, bool key64, int n_max, int log2h, int stack_cache, int worker_warps,
                      bool snapshot, int stride) {
    (void)d;
    return head_region_bytes(n_max, snapshot) +
           warp_region_bytes(n_max, log2h, stack_cache, key64 ? 8 : 4, stride) * (size_t)worker_warps;
}

size_t cta_head_bytes(int n_max, bool snapshot) { return head_region_bytes(n_max, snapshot); }

size_t cta_warp_bytes(bool key64, int n_max, int log2h, int stack_cache, int stride) {
    return warp_region_bytes(n_max, log2h, stack_cache, key64 ? 8 : 4, stride);
}

namespace {
template <int D, typename Key, int MODE>
cudaError_t allow_smem() {
    // the largest opt-in shared memory per block, set once per instantiation
    static int done = 0;
    if (done) return cudaSuccess;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(grow_kernel<D, Key, MODE>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) done = 1;
    return e;
}

template <int D, typename Key, int MODE>
cudaError_t launch_one(const RunDev &P, int ctas, cudaStream_t stream) {
    const bool snapshot = (MODE == kSnapshot);
    // shared memory holds what the arena does not
    const size_t smem = P.arena_mode == kArenaAll ? 0
                      : (P.arena_mode == kArenaWalks ? head_region_bytes(P.n_max, snapshot)
                                                     : cta_smem_bytes(D, sizeof(Key) == 8, P.n_max, P.log2h,
                                                                      P.stack_cache, P.worker_warps, snapshot,
                                                                      P.stride));
    cudaError_t e = allow_smem<D, Key, MODE>();
    if (e != cudaSuccess) return e;
    const int threads = 32 * (P.worker_warps + (snapshot ? 1 : 0));
    grow_kernel<D, Key, MODE><<<ctas, threads, smem, stream>>>(P);
    return cudaGetLastError();
}
}  // namespace

cudaError_t batch_smem_budget(size_t *dynamic_max) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, batch_kernel<kSnapshot>);
    if (e != cudaSuccess) return e;
    const long long dyn = (long long)optin - (long long)fa.sharedSizeBytes;
    if (dyn <= 0) return cudaErrorInvalidValue;
    *dynamic_max = (size_t)dyn;
    return cudaFuncSetAttribute(batch_kernel<kSnapshot>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t batch_grid(int threads, size_t smem, int *ctas) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<kSnapshot>, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *ctas = sms * per_sm;
    return cudaSuccess;
}

cudaError_t launch_batch(const BatchDev &B, int ctas, int threads, size_t smem, cudaStream_t stream) {
    batch_init_kernel<<<1, 256, 0, stream>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    batch_kernel<kSnapshot><<<ctas, threads, smem, stream>>>(B);
    return cudaGetLastError();
}

cudaError_t set_smem_limits() {
    cudaError_t e = allow_smem<2, uint32_t, kSnapshot>();
    if (e == cudaSuccess) e = allow_smem<2, uint32_t, kFresh>();
    if (e == cudaSuccess) e = allow_smem<3, uint32_t, kSnapshot>();
    if (e == cudaSuccess) e = allow_smem<3, uint32_t, kFresh>();
    if (e == cudaSuccess) e = allow_smem<3, unsigned long long, kSnapshot>();
    if (e == cudaSuccess) e = allow_smem<3, unsigned long long, kFresh>();
    return e;
}

cudaError_t launch_grow(const RunDev &P, int thresh_mode, bool key64, int ctas, cudaStream_t stream) {
    if (P.d == 2) {
        return thresh_mode == kSnapshot ? launch_one<2, uint32_t, kSnapshot>(P, ctas, stream)
                                        : launch_one<2, uint32_t, kFresh>(P, ctas, stream);
    }
    if (key64) {
        return thresh_mode == kSnapshot ? launch_one<3, unsigned long long, kSnapshot>(P, ctas, stream)
                                        : launch_one<3, unsigned long long, kFresh>(P, ctas, stream);
    }
    return thresh_mode == kSnapshot ? launch_one<3, uint32_t, kSnapshot>(P, ctas, stream)
                                    : launch_one<3, uint32_t, kFresh>(P, ctas, stream);
}

cudaError_t launch_finalize(unsigned long long *tickets, long long limit, cudaStream_t stream) {
    finalize_kernel<<<1, 32, 0, stream>>>(tickets, limit);
    return cudaGetLastError();
}

cudaError_t launch_debug_step(int d, int n_max, int B, const int32_t *coords, const int32_t *len,
                              const double *W, const double *Wsum, const uint64_t *M,
                              const uint64_t *ordinal, const uint32_t *seq, const uint32_t *tour,
                              uint32_t key0, uint32_t key1, int force_exact, int32_t *out_i,
                              double *out_r, double *out_w, cudaStream_t stream) {
    int log2h = 4;
    while ((1 << log2h) < 2 * n_max) ++log2h;
    const int blocks = (B + 31) / 32;
    if (blocks == 0) return cudaSuccess;
    const size_t key_b = 4;
    const size_t smem = ((size_t)1 << log2h) * kStride * key_b + 128 * 8;
    if (d == 2) {
        cudaError_t e = cudaFuncSetAttribute(debug_step_kernel<2, uint32_t>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        debug_step_kernel<2, uint32_t><<<blocks, 32, smem, stream>>>(n_max, log2h, B, coords, len, W, Wsum,
                M, ordinal, seq, tour, key0, key1, force_exact, out_i, out_r, out_w);
    } else {
        cudaError_t e = cudaFuncSetAttribute(debug_step_kernel<3, uint32_t>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        debug_step_kernel<3, uint32_t><<<blocks, 32, smem, stream>>>(n_max, log2h, B, coords, len, W, Wsum,
                M, ordinal, seq, tour, key0, key1, force_exact, out_i, out_r, out_w);
    }
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(int B, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                cudaStream_t stream) {
    if (B <= 0) return cudaSuccess;
    philox_kernel<<<(B + 127) / 128, 128, 0, stream>>>(B, ctr, k0, k1, out);
    return cudaGetLastError();
}

}  // namespace perm
