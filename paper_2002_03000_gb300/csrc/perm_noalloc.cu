// perm_noalloc.cu -- perm_run_static: one complete growth run that allocates
// nothing.
//
// Some callers cannot call cudaMalloc or cudaFree:
//   - a host program whose device memory is already owned by another
//     allocator (a framework's caching pool that holds the whole device);
//   - a plugin loaded into such a process;
//   - a serving or real-time loop that must not allocate, because
//     cudaMalloc/cudaFree can synchronise the device and stall work queued on
//     other streams.
// For them this entry point keeps all of the run's scratch in a fixed
// file-scope device array instead of memory allocated per handle.  Scratch
// here means the tour counters, the status word, the per-walk tour sums and
// the per-walk stack spill areas.  The caller still passes the output tables.
//
// The array is PERM_STATIC_SCRATCH_BYTES long.  Every GPU that loads the
// library holds it until the process exits.  All calls share it and it keeps
// the last call's contents; each call clears what must start at zero.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on it and both results are then invalid.
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "perm.h"
#include "perm_kernels.cuh"

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[PERM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the static array for the current device; looked up once
// per device (the host-side name is only a stand-in, not a device address).
int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PERM_EDEVICE;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return PERM_EDEVICE;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PERM_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int perm_run_static(const perm_config *cfg, int64_t tours_per_seq, double *W_n,
                               unsigned long long *S_n, double *Q_n, int64_t *steps,
                               void *stream) {
    if (!cfg || !W_n || !S_n || !Q_n || tours_per_seq < 0) return PERM_EINVAL;
    const int d = cfg->d, n_max = cfg->n_max, n_seq = cfg->n_seq;
    if ((d != 2 && d != 3) || n_max < 1 || n_seq < 1) return PERM_EINVAL;
    if (cfg->alg != PERM_ALG2) return PERM_EINVAL;
    if (cfg->threshold != PERM_THRESH_SNAPSHOT && cfg->threshold != PERM_THRESH_FRESH) return PERM_EINVAL;
    if (cfg->slots < 0 || cfg->refresh_ns < 0 || !(cfg->max_seconds >= 0.0)) return PERM_EINVAL;
    if (!(cfg->ramp_gamma >= 0.0) || cfg->ramp_gamma > 1e6) return PERM_EINVAL;
    // settings this entry point does not carry out are refused, not ignored: the
    // eq. 5 sums, a chosen layout (walks per warp, hash size, stack ring, CTA cap,
    // walk memory) and shared copies (the run grows every copy on the walk that
    // made it)
    if (cfg->observables != 0 || cfg->hash_scale != 0 || cfg->lanes_per_warp != 0 ||
        cfg->stack_ring != 0 || cfg->max_ctas != 0 || cfg->share_copies > 0 || cfg->walk_memory != 0 ||
        cfg->helper_walks > 0)
        return PERM_EUNSUPPORTED;
    const bool key64 = (d == 3 && n_max > 512);
    if (n_max > (d == 2 ? 32766 : (key64 ? (1 << 20) - 2 : 512))) return PERM_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;

    // scratch: counters, then per-walk tour sums and stack spill areas
    const size_t L = (size_t)n_max + 1;
    const size_t counters = round256(16 * sizeof(unsigned long long));
    const size_t per_slot = L * sizeof(double) + (size_t)n_max * (sizeof(uint32_t) + sizeof(double));
    if (counters + 3 * 256 + per_slot > PERM_STATIC_SCRATCH_BYTES) return PERM_ESCRATCH;
    const long long fit = (long long)((PERM_STATIC_SCRATCH_BYTES - counters - 3 * 256) / per_slot);
    // an explicit walk count beyond the sequences is clamped first (one walk per
    // sequence at most), then checked against what the buffer holds
    const long long asked = cfg->slots > n_seq ? n_seq : cfg->slots;
    if (asked > 0 && asked > fit) return PERM_ESCRATCH;

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PERM_OK) return rc;
    int dev = 0, smem_optin = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PERM_EDEVICE;
    const size_t optin = (size_t)smem_optin;

    // layout: one walk per thread, 32 walks per warp at most, as many warps per
    // CTA as shared memory allows, one CTA per SM
    const bool snap = (cfg->threshold == PERM_THRESH_SNAPSHOT);
    int log2h = 4;
    while ((1 << log2h) < 2 * n_max) ++log2h;
    const int K = 16;
    int stride = 32;
    size_t head = 0, per_warp = 0;
    for (;; stride /= 2) {
        head = perm::cta_smem_bytes(d, key64, n_max, log2h, K, 0, snap, stride);
        per_warp = perm::cta_smem_bytes(d, key64, n_max, log2h, K, 1, snap, stride) - head;
        if (head + per_warp <= optin || stride == 1) break;
    }
    if (head + per_warp > optin) return PERM_EUNSUPPORTED;
    int max_warps = (int)((optin - head) / per_warp);
    if (max_warps > 4) max_warps = 4;

    long long slots = cfg->slots ? cfg->slots : n_seq;
    if (slots > n_seq) slots = n_seq;
    if (slots > fit) slots = fit;
    const long long cap = (long long)num_sms * max_warps * stride;
    if (slots > cap) slots = cap;
    const long long per_cta = (slots + num_sms - 1) / num_sms;
    int warps = (int)((per_cta + stride - 1) / stride);
    if (warps > max_warps) warps = max_warps;
    if (warps < 1) warps = 1;
    int lanes = (int)((per_cta + warps - 1) / warps);
    if (lanes > stride) lanes = stride;
    const int ctas = (int)((slots + (long long)warps * lanes - 1) / ((long long)warps * lanes));

    unsigned char *p = static_cast<unsigned char *>(base);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(p);
    double *X = reinterpret_cast<double *>(p + counters);
    uint32_t *gmeta = reinterpret_cast<uint32_t *>(p + counters + round256(L * sizeof(double) * slots));
    double *gw = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(gmeta) +
                                            round256((size_t)n_max * sizeof(uint32_t) * slots));

    // what must start at zero: counters, tour sums and the output tables
    cudaError_t e = cudaMemsetAsync(cnt, 0, counters, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(X, 0, L * sizeof(double) * slots, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(W_n, 0, L * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S_n, 0, L * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Q_n, 0, L * sizeof(double), st);
    if (e != cudaSuccess) return PERM_EDEVICE;
    if (tours_per_seq == 0) {
        if (steps) *steps = 0;
        return cudaStreamSynchronize(st) == cudaSuccess ? PERM_OK : PERM_EDEVICE;
    }

    perm::RunDev P;
    std::memset(&P, 0, sizeof(P));
    P.d = d; P.n_max = n_max; P.n_seq = n_seq; P.alg = PERM_ALG2;
    P.log2h = log2h; P.S = lanes; P.stride = stride; P.worker_warps = warps;
    P.slots = (int)slots; P.tour_slots = (int)slots; P.stack_cache = K;
    P.key0 = (uint32_t)cfg->seed ^ cfg->run_id;
    P.key1 = (uint32_t)(cfg->seed >> 32);
    P.tour_limit = tours_per_seq * (long long)n_seq;
    P.refresh_ns = cfg->refresh_ns ? (cfg->refresh_ns > 1000000 ? 1000000 : cfg->refresh_ns) : 8000;
    P.max_ns = (long long)((cfg->max_seconds > 0.0 ? cfg->max_seconds : 600.0) * 1e9);
    P.Wn = W_n; P.Sn = S_n; P.Qn = Q_n;
    P.tickets = cnt + 0; P.seq_M = nullptr;
    P.X = X; P.gstk_meta = gmeta; P.gstk_w = gw;
    P.steps = cnt + 1; P.max_stack = cnt + 2; P.copies = cnt + 3; P.refreshes = cnt + 4;
    P.iterations = cnt + 5; P.finished = cnt + 6; P.exact_steps = cnt + 9;
    P.status = reinterpret_cast<int *>(cnt + 7);
    P.ramp_c0 = cfg->ramp_c0 < 0 ? -1 : (cfg->ramp_c0 == 0 ? 2 : cfg->ramp_c0);
    P.ramp_gamma_q16 = (unsigned long long)((cfg->ramp_gamma == 0.0 ? 0.25 : cfg->ramp_gamma) * 65536.0);
    P.trace = nullptr; P.trace_coords = nullptr; P.trace_count = cnt + 8;
    P.trace_cap = 0; P.trace_every = 1; P.trace_tour_every = 1;

    e = perm::launch_grow(P, snap ? perm::kSnapshot : perm::kFresh, key64, ctas, st);
    if (e != cudaSuccess) return PERM_EDEVICE;
    e = perm::launch_finalize(P.tickets, P.tour_limit, st);
    if (e != cudaSuccess) return PERM_EDEVICE;
    // the counters come back on the caller's stream, which is then waited for (no
    // blocking copy on the legacy default stream, which would wait for every stream)
    unsigned long long host_cnt[8];
    if (cudaMemcpyAsync(host_cnt, cnt, sizeof(host_cnt), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PERM_EDEVICE;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PERM_EDEVICE;
    if (steps) *steps = (int64_t)host_cnt[1];
    int status = 0;
    std::memcpy(&status, &host_cnt[7], sizeof(int));
    return status;
}
