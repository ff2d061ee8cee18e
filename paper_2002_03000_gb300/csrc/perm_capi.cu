// perm_capi.cu -- C ABI of libperm.so (declared in include/perm.h).
//
// Host side of the interacting flatPERM run: argument checks, the layout of
// walks on the device (slots per warp, warps per CTA, CTAs), device memory,
// launches, and the estimates of Sec. 1, eq. (4) (Alg. 1: eq. (7)) computed
// from the tables the kernels fill.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "perm.h"
#include "perm_kernels.cuh"

using perm::RunDev;

struct perm_run_s {
    perm_config cfg;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    bool key64 = false;
    int thresh = perm::kSnapshot;
    int log2h = 0, slots = 0, ctas = 0, worker_warps = 0, lanes = 0, stride = 32, stack_cache = 16;
    size_t smem = 0;
    int arena_mode = 0;            // perm::ArenaMode
    long long arena_cta_bytes = 0;
    unsigned char *arena = nullptr;
    int ntab = 1;
    int xrows = 0;                 // tour-sum rows: one per walk, two with shared copies
    int tour_slots = 0;            // walks that start tours; the other slots are helpers
    // device buffers
    double *Wn = nullptr, *Qn = nullptr, *X = nullptr, *gstk_w = nullptr, *Rn = nullptr;
    unsigned long long *Sn = nullptr, *tickets = nullptr, *seq_M = nullptr;
    unsigned long long *steps = nullptr, *max_stack = nullptr, *copies = nullptr, *refreshes = nullptr, *trace_count = nullptr;
    unsigned long long *iterations = nullptr, *finished = nullptr, *exact_steps = nullptr;
    uint32_t *gstk_meta = nullptr;
    int *status = nullptr;
    // shared copies
    bool share = false;
    int share_cap = 0;
    int dq_log2cap = 0, dq_cell_bytes = 0;
    unsigned char *dq_cells = nullptr;
    unsigned long long *dq_head = nullptr, *dq_tail = nullptr;
    unsigned int *dq_ready = nullptr, *dq_free = nullptr, *outst = nullptr, *tmaxn = nullptr;
    int *hungry = nullptr;
    double2 *cut = nullptr;        // original PERM's cut-offs (nullptr: flatPERM)
    int cut_copies = 1;
    double cut_q = 1.0;
    perm_trace_record *trace = nullptr;
    int32_t *trace_coords = nullptr;
    int trace_cap = 0;
    long long trace_every = 0, trace_tour_every = 1;
    // host bookkeeping
    long long tour_limit = 0;      // Alg. 2 tickets handed out so far (cumulative)
    long long seq_target = 0;      // Alg. 1 tours per sequence (cumulative)
    long long device_bytes = 0;
    int last_status = PERM_OK;
};

namespace {

int to_code(cudaError_t e) {
    if (e == cudaSuccess) return PERM_OK;
    if (e == cudaErrorMemoryAllocation) return PERM_ENOMEM;
    return PERM_EDEVICE;
}

template <typename T>
int dalloc(perm_handle h, T **p, size_t count) {
    const size_t bytes = count * sizeof(T);
    if (bytes == 0) { *p = nullptr; return PERM_OK; }
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) { *p = nullptr; return to_code(e); }
    h->device_bytes += (long long)bytes;
    e = cudaMemsetAsync(*p, 0, bytes, h->stream);
    return to_code(e);
}

void free_all(perm_handle h) {
    void *ptrs[] = {h->Wn, h->Qn, h->Rn, h->X, h->gstk_w, h->Sn, h->tickets, h->seq_M, h->steps,
                    h->max_stack, h->copies, h->refreshes, h->iterations, h->finished, h->exact_steps,
                    h->trace_count, h->gstk_meta, h->status, h->trace,
                    h->trace_coords, h->dq_cells, h->dq_head, h->dq_tail, h->dq_ready, h->dq_free, h->outst,
                    h->tmaxn, h->hungry, h->cut, h->arena};
    for (void *p : ptrs) if (p) cudaFree(p);
}

// Parts of one tour that may grow on other walks at once (shared copies), and the
// larger bound used once no tour of the run has finished for kStallNs.
constexpr int kDefaultShareCap = 4;
constexpr int kBoostShareCap = 1024;
constexpr long long kStallNs = 5000000;

int scale_exp_host(int d, int n) { return d == 2 ? (11 * n) >> 3 : (9 * n) >> 2; }

int max_n_for(int d, bool key64) {
    if (d == 2) return 32766;
    return key64 ? (1 << 20) - 2 : 512;
}

}  // namespace

extern "C" {

void perm_config_init(perm_config *cfg, int d, int n_max, int n_seq, uint64_t seed) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->d = d;
    cfg->n_max = n_max;
    cfg->n_seq = n_seq;
    cfg->seed = seed;
    cfg->run_id = 0u;
    cfg->alg = PERM_ALG2;
    cfg->threshold = PERM_THRESH_SNAPSHOT;
    cfg->slots = 0;
    cfg->lanes_per_warp = 0;
    cfg->refresh_ns = 0;
    cfg->max_seconds = 0.0;
    cfg->ramp_c0 = 0;
    cfg->ramp_gamma = 0.0;
    cfg->max_ctas = 0;
    cfg->hash_scale = 0;
    cfg->share_copies = 0;
    cfg->stack_ring = 0;
    cfg->observables = 0;
    cfg->walk_memory = 0;
    cfg->helper_walks = 0;
}

const char *perm_strerror(int code) {
    switch (code) {
        case PERM_OK: return "ok";
        case PERM_EINVAL: return "invalid argument";
        case PERM_ENOMEM: return "out of memory";
        case PERM_EOVERFLOW: return "stack or hash bound exceeded in a kernel";
        case PERM_EDEVICE: return "CUDA device error";
        case PERM_ETIMEOUT: return "bounded device wait ran out";
        case PERM_EUNSUPPORTED: return "configuration not supported";
        case PERM_ESCRATCH: return "requested walks need more scratch than the static buffer holds";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// A layout forced by a batch launch: `ctas` CTAs (the batch grid) within
// smem_budget bytes of shared memory each.
struct ForcedLayout {
    int ctas;
    size_t smem_budget;
};

int create_impl(perm_handle *out, const perm_config *cfg, const ForcedLayout *force) {
    if (!out || !cfg) return PERM_EINVAL;
    *out = nullptr;
    const int d = cfg->d, n_max = cfg->n_max, n_seq = cfg->n_seq;
    if ((d != 2 && d != 3) || n_max < 1 || n_seq < 1) return PERM_EINVAL;
    if (cfg->alg != PERM_ALG1 && cfg->alg != PERM_ALG2) return PERM_EINVAL;
    if (cfg->threshold != PERM_THRESH_SNAPSHOT && cfg->threshold != PERM_THRESH_FRESH) return PERM_EINVAL;
    if (cfg->slots < 0 || cfg->refresh_ns < 0 || !(cfg->max_seconds >= 0.0)) return PERM_EINVAL;
    if (!(cfg->ramp_gamma >= 0.0) || cfg->ramp_gamma > 1e6) return PERM_EINVAL;
    if (cfg->max_ctas < -1 || cfg->hash_scale < 0 || cfg->hash_scale > 2) return PERM_EINVAL;
    if (cfg->share_copies < -1 || cfg->share_copies > 1024) return PERM_EINVAL;
    if (cfg->observables != 0 && cfg->observables != 1) return PERM_EINVAL;
    if (cfg->walk_memory < 0 || cfg->walk_memory > 2) return PERM_EINVAL;
    // helper walks take waiting copies only: they need shared copies
    if (cfg->helper_walks < -1 || cfg->helper_walks > (1 << 20)) return PERM_EINVAL;
    if (cfg->helper_walks > 0 && !(cfg->share_copies >= 0 && cfg->alg == PERM_ALG2 &&
                                   cfg->threshold == PERM_THRESH_SNAPSHOT))
        return PERM_EINVAL;
    if (cfg->stack_ring != 0 && cfg->stack_ring != 16 && cfg->stack_ring != 32 &&
        cfg->stack_ring != 64 && cfg->stack_ring != 128) return PERM_EINVAL;
    const int lpw = cfg->lanes_per_warp;
    if (lpw != 0 && (lpw < 1 || lpw > 32)) return PERM_EINVAL;
    const bool key64 = (d == 3 && n_max > 512);
    if (n_max > max_n_for(d, key64)) return PERM_EUNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PERM_EDEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return PERM_EDEVICE;

    perm_handle h = new (std::nothrow) perm_run_s();
    if (!h) return PERM_ENOMEM;
    h->cfg = *cfg;
    if (cfg->stack_ring) h->stack_cache = cfg->stack_ring;
    if (h->cfg.refresh_ns == 0) h->cfg.refresh_ns = 8000;
    if (h->cfg.refresh_ns > 1000000) h->cfg.refresh_ns = 1000000;
    if (h->cfg.max_seconds == 0.0) h->cfg.max_seconds = 600.0;
    if (h->cfg.ramp_c0 == 0) h->cfg.ramp_c0 = 2;
    if (h->cfg.ramp_gamma == 0.0) h->cfg.ramp_gamma = 0.25;
    h->device = dev;
    h->num_sms = prop.multiProcessorCount;
    if (cfg->max_ctas > 0 && cfg->max_ctas < h->num_sms) h->num_sms = cfg->max_ctas;
    h->key64 = key64;
    // Algorithm 1 reads its private rows directly (no snapshot needed)
    h->thresh = (cfg->alg == PERM_ALG1) ? perm::kFresh
              : (cfg->threshold == PERM_THRESH_FRESH ? perm::kFresh : perm::kSnapshot);
    int log2h = 4;
    while ((1 << log2h) < 2 * n_max) ++log2h;
    log2h += cfg->hash_scale;
    if (log2h > 16) log2h = 16;                 // site slots are 16-bit
    h->log2h = log2h;
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return PERM_EDEVICE;
    }
    h->own_stream = true;

    // layout: walks per warp (lanes), worker warps per CTA, CTAs.  Each thread
    // grows one walk; the walks of an SM are spread over about four warps so
    // that every scheduler has a walk's dependent chain to issue from.
    const bool snap = (h->thresh == perm::kSnapshot);
    const size_t budget = force ? force->smem_budget : prop.sharedMemPerBlockOptin;
    auto pow2_at_least = [](int v) { int p = 1; while (p < v) p <<= 1; return p; };
    // where the walks' hashes, site lists and stack rings live: shared memory, or a
    // global arena when asked for or when not one walk per CTA fits beside the head
    const size_t head_b = perm::cta_head_bytes(n_max, snap);
    auto arena_for = [&](int wm) {
        if (wm != 2) return (int)perm::kArenaNone;
        return head_b <= budget ? (int)perm::kArenaWalks : (int)perm::kArenaAll;
    };
    int arena_mode = arena_for(force ? 1 : cfg->walk_memory);
    if (!force && cfg->walk_memory == 0 &&
        perm::cta_smem_bytes(d, key64, n_max, log2h, h->stack_cache, 1, snap, 1) > budget)
        arena_mode = arena_for(2);
    auto smem_for = [&](int warps, int stride) {
        if (arena_mode == perm::kArenaWalks) return head_b;
        if (arena_mode == perm::kArenaAll) return (size_t)0;
        return perm::cta_smem_bytes(d, key64, n_max, log2h, h->stack_cache, warps, snap, stride);
    };
    if (!force && cfg->max_ctas == -1) {
        // dense packing: the fewest CTAs (of up to 8 x 32 walks) that hold one walk
        // per sequence, so that runs sharing the device take few SMs each
        long long per_cta = 0;
        for (int w = 1; w <= 8; ++w)
            for (int l = 32; l >= 1; --l)
                if (smem_for(w, pow2_at_least(l)) <= budget) {
                    per_cta = std::max(per_cta, (long long)w * l);
                    break;
                }
        if (per_cta > 0) {
            const long long need = ((long long)n_seq + per_cta - 1) / per_cta;
            h->num_sms = (int)std::max(1LL, std::min((long long)h->num_sms, need));
        }
    }
    long long tslots = cfg->slots ? cfg->slots : (long long)n_seq;   // walks that grow tours
    if (tslots > n_seq) tslots = n_seq;
    // and helper walks: as asked (none by default), or (-1) the walks the automatic
    // layout has room for beyond the tour walks (4 warps of 8 per SM), when shared
    // copies are on
    const bool can_help = cfg->share_copies >= 0 && cfg->alg == PERM_ALG2 &&
                          cfg->threshold == PERM_THRESH_SNAPSHOT && !force;
    long long helpers = cfg->helper_walks;
    if (helpers < 0) helpers = can_help && !lpw ? std::max(0LL, (long long)h->num_sms * 32 - tslots) : 0;
    long long slots = tslots + helpers;
    const long long slots_wanted = slots;
    int warps = 0, lanes = 0, stride = 0;
    if (force) {
        // every CTA of the batch grid may join this run: the most walks up to
        // 4 warps x 8 (the automatic layout's bound) that fit the shared memory
        for (int w = 4; w >= 1 && !warps; --w)
            for (int l = 8; l >= 1; --l)
                if (smem_for(w, pow2_at_least(l)) <= budget) { warps = w; lanes = l; stride = pow2_at_least(l); break; }
        slots = (long long)force->ctas * warps * lanes;
        if (!warps || slots > (1LL << 30)) { cudaStreamDestroy(h->stream); delete h; return PERM_EUNSUPPORTED; }
        h->num_sms = force->ctas;
    }
    for (; !force;) {
        const long long per_cta = (slots + h->num_sms - 1) / h->num_sms;
        int best_w = 0, best_l = 0, best_s = 0;
        for (int w = 1; w <= 8; ++w) {
            int l = (int)((per_cta + w - 1) / w);
            if (lpw) { if (l > lpw) continue; l = lpw < l ? lpw : l; }
            // automatic: at most 4 walk warps of 8 walks.  A warp's walks take
            // different paths through the step, so its iteration time grows with its
            // walks, and past about 32 walks per SM more walks buy little and lengthen
            // the start-up (cubic lattice, n_max 512, 8192 sequences: 4 x 8 walks per
            // SM run in 0.57 s, 5 x 8 in 0.63 s)
            else if (l > 8 || w > 4) continue;
            if (l > 32 || (long long)w * l < per_cta) continue;
            const int st = pow2_at_least(l);
            if (smem_for(w, st) > budget) continue;
            // prefer about four warps; among fitting choices keep the first that reaches it
            if (best_w == 0 || (best_w < 4 && w <= 4) || (lpw && w < best_w)) {
                best_w = w; best_l = l; best_s = st;
            }
            if (!lpw && w >= 4) break;
        }
        if (best_w) { warps = best_w; lanes = best_l; stride = best_s; break; }
        if (slots <= 1) break;
        slots = slots - (slots + 7) / 8;        // does not fit: fewer concurrent walks
    }
    if (!warps) { cudaStreamDestroy(h->stream); delete h; return PERM_EUNSUPPORTED; }
    const long long per_cta_eff = (long long)warps * lanes;
    // with the layout fixed, use every SM (sequences beyond it wait at tour boundaries)
    if (!force && slots < slots_wanted) {
        const long long cap = (long long)h->num_sms * per_cta_eff;
        slots = slots_wanted < cap ? slots_wanted : cap;
    }
    h->ctas = (int)((slots + per_cta_eff - 1) / per_cta_eff);
    // helpers are the walks beyond the tour walks (fewer when not all fit).  A batch
    // member is laid out for the whole grid and its walks are granted per sequence by
    // the batch kernel, so none of its walks is a helper by position
    h->tour_slots = force ? (int)slots : (int)std::min(tslots, slots);
    h->worker_warps = warps;
    h->lanes = lanes;
    h->stride = stride;
    h->slots = (int)slots;
    h->smem = smem_for(warps, stride);
    // the batch kernel grows its members with the shared-memory body only
    if (force && arena_mode != perm::kArenaNone) { cudaStreamDestroy(h->stream); delete h; return PERM_EUNSUPPORTED; }
    h->arena_mode = arena_mode;
    if (arena_mode != perm::kArenaNone) {
        const size_t wb = perm::cta_warp_bytes(key64, n_max, log2h, h->stack_cache, stride);
        h->arena_cta_bytes = (long long)(wb * (size_t)warps + (arena_mode == perm::kArenaAll ? head_b : 0));
        h->arena_cta_bytes = (h->arena_cta_bytes + 255) & ~255LL;
        // at most 64 GB of walk state
        if ((double)h->arena_cta_bytes * h->ctas > 64e9) { cudaStreamDestroy(h->stream); delete h; return PERM_ENOMEM; }
    }

    const size_t L = (size_t)n_max + 1;
    h->ntab = (cfg->alg == PERM_ALG1) ? n_seq : 1;
    int rc = PERM_OK;
    if (rc == PERM_OK) rc = dalloc(h, &h->Wn, L * h->ntab);
    if (rc == PERM_OK) rc = dalloc(h, &h->Qn, L * h->ntab);
    if (rc == PERM_OK) rc = dalloc(h, &h->Sn, L * h->ntab);
    if (rc == PERM_OK && cfg->observables) rc = dalloc(h, &h->Rn, L * h->ntab);
    if (rc == PERM_OK) rc = dalloc(h, &h->tickets, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->seq_M, (size_t)n_seq);
    h->share = cfg->share_copies >= 0 && cfg->alg == PERM_ALG2 && h->thresh == perm::kSnapshot;
    h->xrows = h->slots * (h->share ? 2 : 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->X, L * (size_t)h->xrows);
    if (rc == PERM_OK) rc = dalloc(h, &h->gstk_meta, (size_t)n_max * h->slots);
    if (rc == PERM_OK) rc = dalloc(h, &h->gstk_w, (size_t)n_max * h->slots);
    if (rc == PERM_OK && h->arena_mode != perm::kArenaNone)
        rc = dalloc(h, &h->arena, (size_t)h->arena_cta_bytes * (size_t)h->ctas);
    if (rc == PERM_OK) rc = dalloc(h, &h->steps, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->max_stack, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->copies, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->refreshes, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->iterations, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->finished, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->exact_steps, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->trace_count, 1);
    if (rc == PERM_OK) rc = dalloc(h, &h->status, 1);
    // shared copies: a ring of cells, each one waiting copy record plus the keys of the
    // walk up to its branch point
    h->share_cap = cfg->share_copies > 0 ? cfg->share_copies : kDefaultShareCap;
    if (rc == PERM_OK && h->share) {
        int lc = 6;
        while ((1 << lc) < h->slots && lc < 12) ++lc;
        h->dq_log2cap = lc;
        // header, the keys of sites 0..n_max, their hash slots (u16)
        h->dq_cell_bytes = (int)(32 + ((((size_t)n_max + 1) * (key64 ? 8 : 4) + 15) & ~(size_t)15) +
                                 ((((size_t)n_max + 1) * 2 + 15) & ~(size_t)15));
        const size_t cap = (size_t)1 << lc;
        rc = dalloc(h, &h->dq_cells, cap * (size_t)h->dq_cell_bytes);
        if (rc == PERM_OK) rc = dalloc(h, &h->dq_ready, cap);
        if (rc == PERM_OK) rc = dalloc(h, &h->dq_free, cap);
        if (rc == PERM_OK) rc = dalloc(h, &h->dq_head, 1);
        if (rc == PERM_OK) rc = dalloc(h, &h->dq_tail, 1);
        if (rc == PERM_OK) rc = dalloc(h, &h->outst, (size_t)h->xrows);
        if (rc == PERM_OK) rc = to_code(cudaMemsetAsync(h->outst, 0xFF, sizeof(unsigned int) * h->xrows, h->stream));
        if (rc == PERM_OK) rc = dalloc(h, &h->tmaxn, (size_t)h->xrows);
        if (rc == PERM_OK) rc = dalloc(h, &h->hungry, 1);
    }
    if (rc == PERM_OK) rc = to_code(cudaStreamSynchronize(h->stream));
    if (rc != PERM_OK) {
        free_all(h);
        cudaStreamDestroy(h->stream);
        delete h;
        return rc;
    }
    *out = h;
    return PERM_OK;
}

}  // namespace

extern "C" {

int perm_create_ex(perm_handle *out, const perm_config *cfg) { return create_impl(out, cfg, nullptr); }

int perm_create(perm_handle *out, int d, int n_max, int n_seq, uint64_t seed) {
    perm_config cfg;
    perm_config_init(&cfg, d, n_max, n_seq, seed);
    return perm_create_ex(out, &cfg);
}

int perm_set_stream(perm_handle h, void *stream) {
    if (!h) return PERM_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PERM_EDEVICE;
    if (h->own_stream) cudaStreamDestroy(h->stream);
    h->stream = (cudaStream_t)stream;
    h->own_stream = false;
    return PERM_OK;
}

static RunDev make_params(perm_handle h) {
    RunDev P;
    std::memset(&P, 0, sizeof(P));
    P.d = h->cfg.d; P.n_max = h->cfg.n_max; P.n_seq = h->cfg.n_seq; P.alg = h->cfg.alg;
    P.log2h = h->log2h; P.S = h->lanes; P.stride = h->stride;
    P.worker_warps = h->worker_warps; P.slots = h->slots; P.tour_slots = h->tour_slots;
    P.stack_cache = h->stack_cache;
    P.arena_mode = h->arena_mode; P.arena = h->arena; P.arena_cta_bytes = h->arena_cta_bytes;
    P.key0 = (uint32_t)h->cfg.seed ^ h->cfg.run_id;
    P.key1 = (uint32_t)(h->cfg.seed >> 32);
    P.tour_limit = h->tour_limit;
    P.seq_target = h->seq_target;
    P.refresh_ns = h->cfg.refresh_ns;
    P.max_ns = (long long)(h->cfg.max_seconds * 1e9);
    P.Wn = h->Wn; P.Sn = h->Sn; P.Qn = h->Qn; P.Rn = h->Rn; P.tickets = h->tickets; P.seq_M = h->seq_M;
    P.X = h->X; P.gstk_meta = h->gstk_meta; P.gstk_w = h->gstk_w;
    P.steps = h->steps; P.max_stack = h->max_stack; P.copies = h->copies; P.refreshes = h->refreshes; P.iterations = h->iterations;
    P.exact_steps = h->exact_steps;
    P.finished = h->finished;
    P.ramp_c0 = h->cfg.ramp_c0 < 0 ? -1 : (long long)h->cfg.ramp_c0;
    P.ramp_gamma_q16 = (unsigned long long)(h->cfg.ramp_gamma * 65536.0);
    P.share = h->share ? h->share_cap : 0;
    P.share_boost = h->share ? std::max(h->share_cap, kBoostShareCap) : 0;
    P.stall_ns = kStallNs;
    P.dq_log2cap = h->dq_log2cap; P.dq_cell_bytes = h->dq_cell_bytes; P.dq_cells = h->dq_cells;
    P.dq_head = h->dq_head; P.dq_tail = h->dq_tail; P.dq_ready = h->dq_ready; P.dq_free = h->dq_free;
    P.outst = h->outst; P.tmaxn = h->tmaxn; P.hungry = h->hungry;
    P.status = h->status;
    P.cut = h->cut;
    P.cut_copies = h->cut_copies;
    P.cut_q = h->cut_q;
    P.cut_inv_q = 1.0 / h->cut_q;
    // survive iff u0 < 1/q, i.e. w0 < 2^32 fl(1/q), i.e. w0 < ceil(2^32 fl(1/q)) (w0 integer)
    P.cut_K = (unsigned long long)std::ceil(P.cut_inv_q * 4294967296.0);
    P.trace = (h->trace_every > 0) ? h->trace : nullptr;
    P.trace_coords = h->trace_coords; P.trace_count = h->trace_count; P.trace_cap = h->trace_cap;
    P.trace_every = h->trace_every > 0 ? h->trace_every : 1;
    P.trace_tour_every = h->trace_tour_every > 0 ? h->trace_tour_every : 1;
    return P;
}

int perm_set_cutoffs(perm_handle h, const double *T_hi, const double *t_lo, int copies, double q) {
    if (!h) return PERM_EINVAL;
    if (!T_hi && !t_lo) {                                   // back to flatPERM
        if (h->cut) {
            if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PERM_EDEVICE;
            cudaFree(h->cut);
            h->device_bytes -= (long long)(sizeof(double2) * ((size_t)h->cfg.n_max + 1));
        }
        h->cut = nullptr;
        return PERM_OK;
    }
    if (!T_hi || !t_lo || copies < 1 || copies > 2 * h->cfg.d || !(q >= 1.0) || q > 4294967296.0)
        return PERM_EINVAL;
    const size_t L = (size_t)h->cfg.n_max + 1;
    std::vector<double2> host(L);
    for (size_t k = 0; k < L; ++k) host[k] = make_double2(T_hi[k], t_lo[k]);
    if (!h->cut) {
        const int rc = dalloc(h, &h->cut, L);
        if (rc != PERM_OK) return rc;
    }
    // the copy is ordered on the handle's stream, after any launch already queued
    cudaError_t e = cudaMemcpyAsync(h->cut, host.data(), sizeof(double2) * L, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return to_code(e);
    h->cut_copies = copies;
    h->cut_q = q;
    return PERM_OK;
}

int perm_run(perm_handle h, int64_t tours_per_seq) {
    if (!h || tours_per_seq < 0) return PERM_EINVAL;
    if (tours_per_seq == 0) return PERM_OK;
    cudaError_t e;
    if (h->cfg.alg == PERM_ALG2) {
        h->tour_limit += tours_per_seq * (long long)h->cfg.n_seq;
    } else {
        h->seq_target += tours_per_seq;
        e = cudaMemsetAsync(h->tickets, 0, sizeof(unsigned long long), h->stream);
        if (e != cudaSuccess) return to_code(e);
    }
    const RunDev P = make_params(h);
    e = perm::launch_grow(P, h->thresh, h->key64, h->ctas, h->stream);
    if (e != cudaSuccess) return to_code(e);
    if (h->cfg.alg == PERM_ALG2) {
        e = perm::launch_finalize(h->tickets, h->tour_limit, h->stream);
        if (e != cudaSuccess) return to_code(e);
    }
    return PERM_OK;
}

// Copy device -> host on the handle's own stream and wait for that stream only
// (other streams, e.g. other runs served concurrently, keep running).
static cudaError_t copy_out(perm_handle h, void *dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e;
}

static int sync_status(perm_handle h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return to_code(e);
    int st = 0;
    e = copy_out(h, &st, h->status, sizeof(int));
    if (e != cudaSuccess) return to_code(e);
    h->last_status = st;
    return st;
}

int perm_run_sync(perm_handle h, int64_t tours_per_seq) {
    int rc = perm_run(h, tours_per_seq);
    if (rc != PERM_OK) return rc;
    return sync_status(h);
}

int perm_tables(perm_handle h, double *W_n, double *S_n, double *Q_n, int64_t *M) {
    if (!h) return PERM_EINVAL;
    int st = sync_status(h);
    if (st < 0 && st != PERM_EOVERFLOW && st != PERM_ETIMEOUT) return st;
    const size_t L = (size_t)h->cfg.n_max + 1, cnt = L * h->ntab;
    cudaError_t e = cudaSuccess;
    if (W_n) e = copy_out(h, W_n, h->Wn, cnt * sizeof(double));
    if (e == cudaSuccess && Q_n) e = copy_out(h, Q_n, h->Qn, cnt * sizeof(double));
    if (e == cudaSuccess && S_n) {
        std::vector<unsigned long long> s(cnt);
        e = copy_out(h, s.data(), h->Sn, cnt * sizeof(unsigned long long));
        for (size_t i = 0; i < cnt; ++i) S_n[i] = (double)s[i];
    }
    if (e == cudaSuccess && M) {
        if (h->cfg.alg == PERM_ALG2) {
            M[0] = h->tour_limit;
        } else {
            std::vector<unsigned long long> m(h->cfg.n_seq);
            e = copy_out(h, m.data(), h->seq_M, m.size() * sizeof(unsigned long long));
            for (size_t i = 0; i < m.size(); ++i) M[i] = (int64_t)m[i];
        }
    }
    if (e != cudaSuccess) return to_code(e);
    return st;
}

int perm_reset(perm_handle h) {
    if (!h) return PERM_EINVAL;
    const size_t L = (size_t)h->cfg.n_max + 1, cnt = L * h->ntab;
    cudaError_t e = cudaMemsetAsync(h->Wn, 0, cnt * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Qn, 0, cnt * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Sn, 0, cnt * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess && h->Rn) e = cudaMemsetAsync(h->Rn, 0, cnt * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->tickets, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->seq_M, 0, sizeof(unsigned long long) * h->cfg.n_seq, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->steps, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->copies, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->refreshes, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->iterations, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->finished, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->exact_steps, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->max_stack, 0, sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
    if (e == cudaSuccess && h->last_status != PERM_OK)   // a stopped run may leave tour sums behind
        e = cudaMemsetAsync(h->X, 0, L * (size_t)h->xrows * sizeof(double), h->stream);
    if (e == cudaSuccess && h->share) {
        const size_t cap = (size_t)1 << h->dq_log2cap;
        e = cudaMemsetAsync(h->dq_head, 0, sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dq_tail, 0, sizeof(unsigned long long), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dq_ready, 0, sizeof(unsigned int) * cap, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->dq_free, 0, sizeof(unsigned int) * cap, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->hungry, 0, sizeof(int), h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->outst, 0xFF, sizeof(unsigned int) * h->xrows, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(h->tmaxn, 0, sizeof(unsigned int) * h->xrows, h->stream);
    }
    if (e != cudaSuccess) return to_code(e);
    h->tour_limit = 0;
    h->seq_target = 0;
    h->last_status = PERM_OK;
    return PERM_OK;
}

int perm_estimates_from_tables(int d, int n_max, int rows, const double *W_n, const double *Q_n,
                               const int64_t *M, int combine, double *log_cn, double *relvar_n) {
    if ((d != 2 && d != 3) || n_max < 0 || rows < 1 || !W_n || !M) return PERM_EINVAL;
    if (combine != PERM_COMBINE_MEAN && combine != PERM_COMBINE_GEOMETRIC) return PERM_EINVAL;
    const size_t L = (size_t)n_max + 1;
    const double log2 = std::log(2.0);
    for (size_t n = 0; n < L; ++n) {
        // per row: the sample average c = W_n / M (eq. 4, any M >= 1) and the
        // per-tour variance of it, (Q_n / M - c^2) / (M - 1) (M >= 2)
        double mean = 0.0, mlog = 0.0, var = 0.0, rvar = 0.0;
        bool ok = Q_n != nullptr, any_zero = false;
        for (int t = 0; t < rows; ++t) {
            const int64_t m = M[t];
            if (m < 1) return PERM_EINVAL;
            const double c = W_n[(size_t)t * L + n] / (double)m;
            mean += c;
            if (c > 0.0) mlog += std::log(c); else any_zero = true;
            if (m < 2 || !Q_n) { ok = false; continue; }
            double v = (Q_n[(size_t)t * L + n] / (double)m - c * c) / (double)(m - 1);
            if (v < 0.0) v = 0.0;
            var += v;
            if (c > 0.0) rvar += v / (c * c);
        }
        const double R = (double)rows;
        const double shift = scale_exp_host(d, (int)n) * log2;
        double lc, rv;
        if (combine == PERM_COMBINE_MEAN) {
            // the average of the rows' sample averages (Sec. 3; one row: eq. 4)
            mean /= R;
            lc = mean > 0.0 ? std::log(mean) + shift : -INFINITY;
            rv = (ok && mean > 0.0) ? (var / (R * R)) / (mean * mean) : INFINITY;
        } else {
            // the mean of the rows' log sample averages (the geometric combination of
            // Sec. 4); its variance to first order is the mean relative variance / rows
            lc = any_zero ? -INFINITY : mlog / R + shift;
            rv = (ok && !any_zero) ? rvar / (R * R) : INFINITY;
        }
        if (log_cn) log_cn[n] = lc;
        if (relvar_n) relvar_n[n] = rv;
    }
    return PERM_OK;
}

int perm_estimates(perm_handle h, double *log_cn, double *S_n, double *relvar_n) {
    if (!h) return PERM_EINVAL;
    const size_t L = (size_t)h->cfg.n_max + 1, cnt = L * h->ntab;
    std::vector<double> W(cnt), S(cnt), Q(cnt);
    std::vector<int64_t> M(h->ntab);
    int rc = perm_tables(h, W.data(), S.data(), Q.data(), M.data());
    if (rc != PERM_OK) return rc;
    for (int t = 0; t < h->ntab; ++t) {
        if (M[t] < 1) {                          // no tour yet: nothing estimated
            for (size_t n = 0; n < L; ++n) {
                if (log_cn) log_cn[n] = -INFINITY;
                if (relvar_n) relvar_n[n] = INFINITY;
                if (S_n) S_n[n] = 0.0;
            }
            return PERM_OK;
        }
    }
    rc = perm_estimates_from_tables(h->cfg.d, h->cfg.n_max, h->ntab, W.data(), Q.data(), M.data(),
                                    PERM_COMBINE_MEAN, log_cn, relvar_n);
    if (rc != PERM_OK) return rc;
    if (S_n) {
        for (size_t n = 0; n < L; ++n) {
            double s = 0.0;
            for (int t = 0; t < h->ntab; ++t) s += S[(size_t)t * L + n];
            S_n[n] = s;
        }
    }
    return PERM_OK;
}

int perm_observable_r2(perm_handle h, double *mean_r2, double *R_n) {
    if (!h || !mean_r2 || !h->Rn) return PERM_EINVAL;
    const size_t L = (size_t)h->cfg.n_max + 1, cnt = L * h->ntab;
    std::vector<double> W(cnt), R(cnt);
    std::vector<int64_t> M(h->ntab);
    int rc = perm_tables(h, W.data(), nullptr, nullptr, M.data());
    if (rc != PERM_OK) return rc;
    if (copy_out(h, R.data(), h->Rn, cnt * sizeof(double)) != cudaSuccess) return PERM_EDEVICE;
    for (size_t n = 0; n < L; ++n) {
        double num = 0.0, den = 0.0;
        for (int t = 0; t < h->ntab; ++t) {
            if (M[t] < 1) continue;
            num += R[(size_t)t * L + n] / (double)M[t];
            den += W[(size_t)t * L + n] / (double)M[t];
        }
        mean_r2[n] = den > 0.0 ? num / den : NAN;
    }
    if (R_n) for (size_t i = 0; i < cnt; ++i) R_n[i] = R[i];
    return PERM_OK;
}

int perm_stats(perm_handle h, perm_stats_t *out) {
    if (!h || !out) return PERM_EINVAL;
    int st = sync_status(h);
    if (st < 0 && st != PERM_EOVERFLOW && st != PERM_ETIMEOUT) return st;
    unsigned long long steps = 0, ms = 0, cp = 0, rf = 0, it = 0, fin = 0, shr = 0, ex = 0;
    if (copy_out(h, &steps, h->steps, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &cp, h->copies, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &rf, h->refreshes, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &it, h->iterations, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &ms, h->max_stack, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &fin, h->finished, 8) != cudaSuccess) return PERM_EDEVICE;
    if (copy_out(h, &ex, h->exact_steps, 8) != cudaSuccess) return PERM_EDEVICE;
    if (h->share && copy_out(h, &shr, h->dq_tail, 8) != cudaSuccess) return PERM_EDEVICE;
    out->steps = (int64_t)steps;
    out->tours = h->cfg.alg == PERM_ALG2 ? h->tour_limit : h->seq_target * h->cfg.n_seq;
    out->max_stack = (int64_t)ms;
    out->copies = (int64_t)cp;
    out->refreshes = (int64_t)rf;
    out->iterations = (int64_t)it;
    out->slots = h->slots;
    out->ctas = h->ctas;
    out->lanes_per_warp = h->lanes;
    out->warps_per_cta = h->worker_warps;
    out->hash_slots = 1 << h->log2h;
    out->status = st;
    out->device_bytes = h->device_bytes;
    out->tours_finished = (int64_t)fin;
    out->shared = (int64_t)shr;
    out->exact_steps = (int64_t)ex;
    out->walk_memory = h->arena_mode == perm::kArenaNone ? 1 : 2;
    out->pad = 0;
    return PERM_OK;
}

int perm_trace_enable(perm_handle h, int64_t every, int64_t tour_every, int capacity) {
    if (!h || every < 0 || tour_every < 0 || capacity < 0) return PERM_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PERM_EDEVICE;
    if (h->trace) { cudaFree(h->trace); h->trace = nullptr; }
    if (h->trace_coords) { cudaFree(h->trace_coords); h->trace_coords = nullptr; }
    h->trace_every = every;
    h->trace_tour_every = tour_every > 0 ? tour_every : 1;
    h->trace_cap = 0;
    if (every == 0 || capacity == 0) { h->trace_every = 0; return PERM_OK; }
    const size_t L = (size_t)h->cfg.n_max + 1;
    if (cudaMalloc((void **)&h->trace, sizeof(perm_trace_record) * (size_t)capacity) != cudaSuccess ||
        cudaMalloc((void **)&h->trace_coords, sizeof(int32_t) * (size_t)capacity * L * h->cfg.d) != cudaSuccess) {
        h->trace_every = 0;
        return PERM_ENOMEM;
    }
    h->trace_cap = capacity;
    if (cudaMemset(h->trace_count, 0, 8) != cudaSuccess) return PERM_EDEVICE;
    return PERM_OK;
}

int perm_trace_read(perm_handle h, int64_t *count, perm_trace_record *recs, int32_t *coords) {
    if (!h) return PERM_EINVAL;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return PERM_EDEVICE;
    unsigned long long c = 0;
    if (cudaMemcpy(&c, h->trace_count, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return PERM_EDEVICE;
    if (count) *count = (int64_t)c;
    const size_t kept = c < (unsigned long long)h->trace_cap ? (size_t)c : (size_t)h->trace_cap;
    const size_t L = (size_t)h->cfg.n_max + 1;
    if (recs && kept && cudaMemcpy(recs, h->trace, kept * sizeof(perm_trace_record), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PERM_EDEVICE;
    if (coords && kept && cudaMemcpy(coords, h->trace_coords, kept * L * h->cfg.d * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return PERM_EDEVICE;
    return PERM_OK;
}

void perm_destroy(perm_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

int perm_debug_step(int d, int n_max, int B, const int32_t *coords, const int32_t *len,
                    const double *W, const double *Wsum, const uint64_t *M,
                    const uint64_t *ordinal, const uint32_t *seq, const uint32_t *tour,
                    uint64_t seed, uint32_t run_id, int force_exact, int32_t *out_i,
                    double *out_r, double *out_w, void *stream) {
    if ((d != 2 && d != 3) || n_max < 1 || n_max > 512 || B < 0) return PERM_EINVAL;
    if (force_exact != 0 && force_exact != 1) return PERM_EINVAL;
    if (B > 0 && (!coords || !len || !W || !Wsum || !M || !ordinal || !seq || !tour || !out_i ||
                  !out_r || !out_w))
        return PERM_EINVAL;
    cudaError_t e = perm::launch_debug_step(d, n_max, B, coords, len, W, Wsum, M, ordinal, seq, tour,
                                            (uint32_t)seed ^ run_id, (uint32_t)(seed >> 32), force_exact,
                                            out_i, out_r, out_w, (cudaStream_t)stream);
    return to_code(e);
}

int perm_debug_philox(int B, const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    if (B < 0 || (B > 0 && (!ctr || !key || !out))) return PERM_EINVAL;
    cudaError_t e = perm::launch_debug_philox(B, ctr, key[0], key[1], out, nullptr);
    if (e != cudaSuccess) return to_code(e);
    return to_code(cudaDeviceSynchronize());
}

}  // extern "C"

namespace perm {

int member_create(perm_handle *out, const perm_config *cfg, int ctas, size_t smem_budget) {
    if (!cfg || ctas < 1) return PERM_EINVAL;
    if (cfg->alg != PERM_ALG2 || cfg->threshold != PERM_THRESH_SNAPSHOT) return PERM_EUNSUPPORTED;
    const ForcedLayout f{ctas, smem_budget};
    return create_impl(out, cfg, &f);
}

int member_params(perm_handle h, int64_t tours_per_seq, int run_index, RunDev *P, size_t *smem,
                  int *worker_warps) {
    if (!h || !P || tours_per_seq < 0) return PERM_EINVAL;
    h->tour_limit = tours_per_seq * (long long)h->cfg.n_seq;
    *P = make_params(h);
    P->run_index = run_index;
    if (smem) *smem = h->smem;
    if (worker_warps) *worker_warps = h->worker_warps;
    return PERM_OK;
}

int member_extend(perm_handle h, int64_t extra_tours_per_seq, int run_index, RunDev *P) {
    if (!h || !P || extra_tours_per_seq < 0) return PERM_EINVAL;
    h->tour_limit += extra_tours_per_seq * (long long)h->cfg.n_seq;
    *P = make_params(h);
    P->run_index = run_index;
    return PERM_OK;
}

int member_reset(perm_handle h) {
    int rc = perm_reset(h);
    if (rc != PERM_OK) return rc;
    const size_t L = (size_t)h->cfg.n_max + 1;
    return to_code(cudaMemsetAsync(h->X, 0, L * (size_t)h->xrows * sizeof(double), h->stream));
}

}  // namespace perm

// ---------------------------------------------------------------------------
// Checkpoint and resume at a tour boundary.  Between launches every tour of the
// handle has ended: the per-walk tour sums are zero, the stacks are empty and
// no copy waits in the donation ring, so the run's state is its tables, its
// tour counters and its statistics.  The random streams are counter-based
// (sequence, tour, node), so a resumed run draws what the uninterrupted run
// would have drawn.
// ---------------------------------------------------------------------------
namespace {

constexpr char kCkptMagic[8] = {'P', 'E', 'R', 'M', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkptVersion = 3;

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    perm_config cfg;               // as the handle holds it (defaults filled in)
    int64_t tour_limit, seq_target;
    int32_t ntab, has_rn, has_cut, cut_copies;
    double cut_q;
    uint64_t steps, max_stack, copies, refreshes, iterations, finished, exact_steps;
};

// Bytes of the arrays after the header, or 0 when the sizes make no sense.
uint64_t ckpt_payload(const CkptHeader &hd) {
    const uint64_t L = (uint64_t)hd.cfg.n_max + 1;
    if (hd.cfg.n_max < 1 || hd.cfg.n_seq < 1 || hd.cfg.n_max > (1 << 20)) return 0;
    const uint64_t ntab = hd.cfg.alg == PERM_ALG1 ? (uint64_t)hd.cfg.n_seq : 1;
    if ((uint64_t)hd.ntab != ntab || L * ntab > (1ull << 34)) return 0;
    const uint64_t cnt = L * ntab;
    return cnt * 8 * (3 + (hd.has_rn ? 1 : 0)) + (uint64_t)hd.cfg.n_seq * 8 + (hd.has_cut ? L * 16 : 0);
}

}  // namespace

extern "C" {

int perm_save(perm_handle h, const char *path) {
    if (!h || !path) return PERM_EINVAL;
    const int st = sync_status(h);
    if (st != PERM_OK) return st < 0 ? st : PERM_EINVAL;     // a failed run is not saved
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kCkptMagic, 8);
    hd.version = kCkptVersion;
    hd.header_bytes = (uint32_t)sizeof(CkptHeader);
    hd.cfg = h->cfg;
    hd.tour_limit = h->tour_limit;
    hd.seq_target = h->seq_target;
    hd.ntab = h->ntab;
    hd.has_rn = h->Rn != nullptr;
    hd.has_cut = h->cut != nullptr;
    hd.cut_copies = h->cut_copies;
    hd.cut_q = h->cut_q;
    const size_t L = (size_t)h->cfg.n_max + 1, cnt = L * h->ntab;
    std::vector<double> W(cnt), Q(cnt), R(hd.has_rn ? cnt : 0);
    std::vector<unsigned long long> S(cnt), sM(h->cfg.n_seq);
    std::vector<double2> cut(hd.has_cut ? L : 0);
    cudaError_t e = copy_out(h, W.data(), h->Wn, cnt * 8);
    if (e == cudaSuccess) e = copy_out(h, Q.data(), h->Qn, cnt * 8);
    if (e == cudaSuccess) e = copy_out(h, S.data(), h->Sn, cnt * 8);
    if (e == cudaSuccess && hd.has_rn) e = copy_out(h, R.data(), h->Rn, cnt * 8);
    if (e == cudaSuccess) e = copy_out(h, sM.data(), h->seq_M, sM.size() * 8);
    if (e == cudaSuccess && hd.has_cut) e = copy_out(h, cut.data(), h->cut, L * sizeof(double2));
    unsigned long long *cnts[7] = {h->steps, h->max_stack, h->copies, h->refreshes, h->iterations, h->finished,
                                   h->exact_steps};
    uint64_t *dst[7] = {&hd.steps, &hd.max_stack, &hd.copies, &hd.refreshes, &hd.iterations, &hd.finished,
                        &hd.exact_steps};
    for (int i = 0; e == cudaSuccess && i < 7; ++i) e = copy_out(h, dst[i], cnts[i], 8);
    if (e != cudaSuccess) return to_code(e);
    // write beside the target, then rename: a crash never leaves half a checkpoint
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return PERM_EINVAL;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && std::fwrite(W.data(), 8, cnt, f) == cnt;
    ok = ok && std::fwrite(Q.data(), 8, cnt, f) == cnt;
    ok = ok && std::fwrite(S.data(), 8, cnt, f) == cnt;
    if (hd.has_rn) ok = ok && std::fwrite(R.data(), 8, cnt, f) == cnt;
    ok = ok && std::fwrite(sM.data(), 8, sM.size(), f) == sM.size();
    if (hd.has_cut) ok = ok && std::fwrite(cut.data(), sizeof(double2), L, f) == L;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return PERM_EINVAL;
    }
    return PERM_OK;
}

int perm_get_config(perm_handle h, perm_config *out) {
    if (!h || !out) return PERM_EINVAL;
    *out = h->cfg;
    return PERM_OK;
}

int perm_load(perm_handle *out, const char *path) {
    if (!out || !path) return PERM_EINVAL;
    *out = nullptr;
    FILE *f = std::fopen(path, "rb");
    if (!f) return PERM_EINVAL;
    CkptHeader hd;
    bool ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kCkptMagic, 8) == 0 &&
              hd.version == kCkptVersion && hd.header_bytes == (uint32_t)sizeof(CkptHeader);
    const uint64_t payload = ok ? ckpt_payload(hd) : 0;
    ok = ok && payload > 0;
    std::vector<unsigned char> body(ok ? (size_t)payload : 0);
    ok = ok && std::fread(body.data(), 1, body.size(), f) == body.size();
    ok = ok && std::fgetc(f) == EOF;                        // nothing after the arrays
    std::fclose(f);
    if (!ok) return PERM_EINVAL;
    perm_handle h = nullptr;
    int rc = perm_create_ex(&h, &hd.cfg);
    if (rc != PERM_OK) return rc;
    if (hd.has_rn != (h->Rn != nullptr)) { perm_destroy(h); return PERM_EINVAL; }
    const size_t L = (size_t)hd.cfg.n_max + 1, cnt = L * (size_t)hd.ntab;
    const unsigned char *p = body.data();
    auto put = [&](void *dev, size_t bytes) {
        cudaError_t e = cudaMemcpyAsync(dev, p, bytes, cudaMemcpyHostToDevice, h->stream);
        p += bytes;
        return e;
    };
    cudaError_t e = put(h->Wn, cnt * 8);
    if (e == cudaSuccess) e = put(h->Qn, cnt * 8);
    if (e == cudaSuccess) e = put(h->Sn, cnt * 8);
    if (e == cudaSuccess && hd.has_rn) e = put(h->Rn, cnt * 8);
    if (e == cudaSuccess) e = put(h->seq_M, (size_t)hd.cfg.n_seq * 8);
    if (e == cudaSuccess && hd.has_cut) {
        rc = dalloc(h, &h->cut, L);
        if (rc != PERM_OK) { perm_destroy(h); return rc; }
        e = put(h->cut, L * sizeof(double2));
        h->cut_copies = hd.cut_copies;
        h->cut_q = hd.cut_q;
    }
    // the tour counter: Alg. 2 hands out tickets from the tours started so far
    const unsigned long long tickets = hd.cfg.alg == PERM_ALG2 ? (unsigned long long)hd.tour_limit : 0ull;
    const uint64_t vals[8] = {hd.steps, hd.max_stack, hd.copies, hd.refreshes, hd.iterations, hd.finished,
                              hd.exact_steps, tickets};
    unsigned long long *dev[8] = {h->steps, h->max_stack, h->copies, h->refreshes, h->iterations, h->finished,
                                  h->exact_steps, h->tickets};
    for (int i = 0; e == cudaSuccess && i < 8; ++i)
        e = cudaMemcpyAsync(dev[i], &vals[i], 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { perm_destroy(h); return to_code(e); }
    h->tour_limit = hd.tour_limit;
    h->seq_target = hd.seq_target;
    *out = h;
    return PERM_OK;
}

}  // extern "C"
