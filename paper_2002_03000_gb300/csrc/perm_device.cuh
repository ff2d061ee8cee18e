// perm_device.cuh -- device building blocks of the flatPERM growth step.
//
// Paper: Campbell and Janse van Rensburg, "Parallel PERM".
//   Sec. 1, eqs. (1)-(2): a_+ free neighbours of the end-point; the next step is
//     uniform among them; W = prod a_+.
//   Sec. 2, eq. (6) and the two paragraphs after it: r = W/[W_n]^sample with the
//     own weight included; r >= 1 enriches into c copies (c = floor r with
//     probability ceil r - r, else ceil r) of weight W/c; r < 1 prunes with
//     probability 1 - r, a survivor carries W/r.
//
// Layout conventions shared by the kernels:
//   - A walk's occupancy hash and its per-site slot list live in shared memory,
//     interleaved by lane: element i of lane l is at [i * S + l] (S = lanes per
//     warp), so that every lane always hits its own bank.
//   - Keys pack the lattice coordinates of a site; 0 is the empty slot.
//   - Directions: j = 0..2d-1 -> axis j/2, sign + for even j (+x,-x,+y,-y,+z,-z).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace perm {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with round keys bumped by the Weyl constants.
// ---------------------------------------------------------------------------
struct Philox4 { uint32_t x, y, z, w; };

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
    const uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
    const uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t hi0 = __umulhi(kM0, c0), lo0 = kM0 * c0;
        const uint32_t hi1 = __umulhi(kM1, c2), lo1 = kM1 * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += kW0;
        k1 += kW1;
    }
    return {c0, c1, c2, c3};
}

// ---------------------------------------------------------------------------
// Site keys.  Key32<2>: 16-bit fields x+32768 | (y+32768)<<16, |x|,|y| <= 32766.
// Key32<3>: 10-bit fields (c+512) mod 1024, for walks with n_max <= 512: every
// stored site has |c| <= 511 (field 1..1023, never 0); a probe at |c| = 512
// gives field 0 and cannot match a stored site.  Key64<3>: 21-bit fields.
// ---------------------------------------------------------------------------
template <int D, typename Key> struct KeyCodec;

template <> struct KeyCodec<2, uint32_t> {
    __device__ __forceinline__ static uint32_t encode(int x, int y, int) {
        return (uint32_t)(x + 32768) | ((uint32_t)(y + 32768) << 16);
    }
    __device__ __forceinline__ static void decode(uint32_t k, int &x, int &y, int &z) {
        x = (int)(k & 0xFFFFu) - 32768;
        y = (int)(k >> 16) - 32768;
        z = 0;
    }
};

template <> struct KeyCodec<3, uint32_t> {
    __device__ __forceinline__ static uint32_t encode(int x, int y, int z) {
        return ((uint32_t)(x + 512) & 1023u) | (((uint32_t)(y + 512) & 1023u) << 10) |
               (((uint32_t)(z + 512) & 1023u) << 20);
    }
    __device__ __forceinline__ static void decode(uint32_t k, int &x, int &y, int &z) {
        x = (int)(k & 1023u) - 512;
        y = (int)((k >> 10) & 1023u) - 512;
        z = (int)((k >> 20) & 1023u) - 512;
    }
};

template <> struct KeyCodec<3, unsigned long long> {
    __device__ __forceinline__ static unsigned long long encode(int x, int y, int z) {
        return (unsigned long long)(uint32_t)(x + (1 << 20)) |
               ((unsigned long long)(uint32_t)(y + (1 << 20)) << 21) |
               ((unsigned long long)(uint32_t)(z + (1 << 20)) << 42);
    }
    __device__ __forceinline__ static void decode(unsigned long long k, int &x, int &y, int &z) {
        x = (int)(k & 0x1FFFFFull) - (1 << 20);
        y = (int)((k >> 21) & 0x1FFFFFull) - (1 << 20);
        z = (int)((k >> 42) & 0x1FFFFFull) - (1 << 20);
    }
};

__device__ __forceinline__ uint32_t hash_home(uint32_t k, int log2h) {
    return (k * 0x9E3779B1u) >> (32 - log2h);
}
__device__ __forceinline__ uint32_t hash_home(unsigned long long k, int log2h) {
    const uint32_t f = (uint32_t)k ^ (uint32_t)(k >> 29) ^ (uint32_t)(k >> 53);
    return (f * 0x9E3779B1u) >> (32 - log2h);
}

// Neighbour j of (x, y, z).
__device__ __forceinline__ void step_coords(int j, int &x, int &y, int &z) {
    const int s = (j & 1) ? -1 : 1;
    if (j < 2) x += s; else if (j < 4) y += s; else z += s;
}

// Insert a key known to be absent; returns its slot, or -1 if the probe
// sequence wrapped around (table full: impossible at load factor <= 1/2).
template <typename Key>
__device__ __forceinline__ int hash_insert(Key *tab, int S, int lane, int log2h, Key k) {
    const uint32_t mask = (1u << log2h) - 1u;
    uint32_t s = hash_home(k, log2h);
    for (int it = 0; it <= (int)mask; ++it) {
        Key *p = tab + (s * (uint32_t)S + (uint32_t)lane);
        if (*p == (Key)0) { *p = k; return (int)s; }
        s = (s + 1) & mask;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// a_+ (Sec. 1): probe the 2d neighbours of the end-point with linear probing.
// Returns the free mask; slot[j] is the empty slot that ended the probe of a
// free direction j (its insertion slot while the table is unchanged).  Each
// round loads all 2d slots and updates the probes with selects (no branches);
// at load factor <= 1/2 almost every probe ends in the first round.
// ---------------------------------------------------------------------------
template <int D, typename Key>
__device__ __forceinline__ int probe_neighbours(const Key *tab, int S, int lane, int log2h,
                                                int x, int y, int z, int (&slot)[2 * D],
                                                bool &overflow) {
    const uint32_t mask = (1u << log2h) - 1u;
    Key key[2 * D];
    uint32_t s[2 * D];
#pragma unroll
    for (int j = 0; j < 2 * D; ++j) {
        int xx = x, yy = y, zz = z;
        step_coords(j, xx, yy, zz);
        key[j] = KeyCodec<D, Key>::encode(xx, yy, zz);
        s[j] = hash_home(key[j], log2h);
        slot[j] = 0;
    }
    uint32_t pending = (1u << (2 * D)) - 1u, freem = 0u;
    for (int it = 0; it <= (int)mask; ++it) {
        Key v[2 * D];
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) v[j] = tab[s[j] * (uint32_t)S + (uint32_t)lane];
#pragma unroll
        for (int j = 0; j < 2 * D; ++j) {
            const bool pend = (pending >> j) & 1u;
            const bool hit = v[j] == key[j];
            const bool emp = v[j] == (Key)0;          // keys are never 0
            slot[j] = (pend && emp) ? (int)s[j] : slot[j];
            freem |= (uint32_t)(pend && emp) << j;
            pending &= ~((uint32_t)(pend && (hit || emp)) << j);
            s[j] = (s[j] + 1u) & mask;                // harmless for resolved probes
        }
        if (pending == 0u) break;
    }
    overflow = pending != 0u;
    return (int)freem;
}

// ---------------------------------------------------------------------------
// The ratio r of Sec. 2 in single precision.  Doubles enter through their
// mantissa rounded to 24 bits (nearest, ties to even; a carry bumps the
// exponent) and their exponent.  The running average T (before the node's own
// weight) is carried packed: low word = FP32 bits of the rounded mantissa in
// [1, 2) (0 if T is zero or subnormal), high word = the biased exponent.
// r = 1 / (T/W + 1/M): the own weight enters through 1/M, since
// [W_n] = T + W/M.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mant24_bits(unsigned long long b, int &ef) {
    const uint32_t hi = (uint32_t)(b >> 32) & 0xFFFFFu, lo = (uint32_t)b;
    uint32_t keep = (hi << 3) | (lo >> 29);          // top 23 fraction bits
    const uint32_t rem = lo & 0x1FFFFFFFu;           // the 29 bits dropped
    if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) keep += 1u;
    if (keep == (1u << 23)) { keep = 0u; ef += 1; }
    return (127u << 23) | keep;
}

__device__ __forceinline__ unsigned long long pack_threshold(double T) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(T);
    int ef = (int)((b >> 52) & 0x7FFull);
    if (ef == 0) return 0ull;
    const uint32_t fm = mant24_bits(b, ef);
    return (unsigned long long)fm | ((unsigned long long)(uint32_t)ef << 32);
}

__device__ __forceinline__ double unpack_threshold(unsigned long long p) {
    const uint32_t fm = (uint32_t)p;
    if (fm == 0u) return 0.0;
    const uint32_t ef = (uint32_t)(p >> 32);
    const unsigned long long b = ((unsigned long long)ef << 52) |
                                 ((unsigned long long)(fm & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ float ratio_r(int n, double W, unsigned long long Tp,
                                         unsigned long long M) {
    // 1/M in FP32 (M rounded to nearest first; 32-bit conversion when it fits)
    const float Mf = (M >> 32) ? __ull2float_rn(M) : __uint2float_rn((uint32_t)M);
    const float inv_m = __frcp_rn(Mf);
    const uint32_t tm = (uint32_t)Tp;
    const unsigned long long wb = (unsigned long long)__double_as_longlong(W);
    const int ew0 = (int)((uint32_t)(wb >> 52) & 0x7FFu);
    int ew = ew0;
    const float fm_w = __uint_as_float(mant24_bits(wb, ew));
    const float q = __fdiv_rn(__uint_as_float(tm | (tm == 0u ? (127u << 23) : 0u)), fm_w);
    int e = (int)(uint32_t)(Tp >> 32) - ew;
    e = e > 100 ? 100 : (e < -100 ? -100 : e);
    float rho = __fmul_rn(q, __uint_as_float((uint32_t)(e + 127) << 23));
    rho = (ew0 == 0) ? 1.2676506e30f : rho;          // W zero or subnormal: 2^100
    rho = (tm == 0u) ? 0.0f : rho;                  // T zero: 0 (checked first)
    const float r = __frcp_rn(__fadd_rn(rho, inv_m));
    return n == 0 ? 1.0f : r;
}

// Stored-weight scale: weight of a length-n walk is kept divided by 2^E(n).
__device__ __forceinline__ int scale_exp(int d, int n) {
    return d == 2 ? (11 * n) >> 3 : (9 * n) >> 2;
}

// ---------------------------------------------------------------------------
// Decision of one node (Sec. 2).  Inputs: a_+ (>= 1), free list packed 3 bits
// per entry in direction order, r, Philox words w0 (decision) and w1 (steps).
// Output: c (0 = pruned), the chosen directions packed 3 bits each (first =
// the copy grown now), and the weight factor F with child weight = W * F at
// the stored scale of length n+1.  aoc[dE_index][a*8+c] = (a/c) 2^-dE.
// ---------------------------------------------------------------------------
struct NodeDecision {
    int c;
    uint32_t dirs;
    double F;        // enrichment: child weight factor (a/c) 2^-dE
    double Fs;       // survival: 1/K = Fs (1 + e) with Fs = y0 the FP32 reciprocal of K ...
    float e;         // ... and e = 1 - K y0 in FP32 (K has at most 24 significant bits)
    bool survive;
};

// Exact float -> double widening by bit manipulation (normal floats).
__device__ __forceinline__ double widen(float f) {
    const uint32_t b = __float_as_uint(f);
    if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
    const unsigned long long e = ((b >> 23) & 0xFFu) + (1023u - 127u);
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) | (e << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// w < ceil(x) for an integer w in [0, 2^32) and a float x in [0, 2^32], exactly,
// with integer operations only (u0 < x/2^32  <=>  w < ceil(x)).
__device__ __forceinline__ bool below_ceil(uint32_t w, float x) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)(b >> 23) - 127;
    const uint32_t m = (b & 0x7FFFFFu) | 0x800000u;
    const int sh = 23 - e;
    const uint32_t c_small = (m + ((1u << (sh & 31)) - 1u)) >> (sh & 31);   // 0 <= e < 23
    const uint32_t c_big = m << ((e - 23) & 31);                             // 23 <= e < 32
    const uint32_t c = (e >= 23) ? c_big : c_small;
    return (b == 0u) ? false : (e >= 32 ? true : (e < 0 ? (w == 0u) : (w < c)));
}

// ceil(x) for a float x in [0, 2^32] as a 64-bit integer (exact).
__device__ __forceinline__ unsigned long long ceil_u64(float x) {
    const uint32_t b = __float_as_uint(x);
    if (b == 0u) return 0ull;
    const int e = (int)(b >> 23) - 127;
    const unsigned long long m = (b & 0x7FFFFFu) | 0x800000u;
    if (e < 0) return 1ull;
    if (e >= 23) return m << (e - 23);
    const int sh = 23 - e;
    return (m + ((1ull << sh) - 1ull)) >> sh;
}

// K = ceil(r 2^32), the integer survival threshold of a pruning decision (r < 1);
// 0 when r >= 1.  Only test records carry it.
__device__ __forceinline__ unsigned long long survive_K(float r) {
    return r >= 1.0f ? 0ull : ceil_u64(ceilf(__fmul_rn(r, 4294967296.0f)));
}

__device__ __forceinline__ NodeDecision decide(int a, uint32_t freelist, float r, uint32_t w0,
                                               uint32_t w1, const double *aoc_row, int dE) {
    NodeDecision o;
    o.F = 0.0;
    o.Fs = 0.0;
    o.e = 0.0f;
    o.survive = false;
    (void)dE;
    // enrichment: p = ceil(r) - r; c = floor(r) iff u0 < p; at most a_+ copies
    const float fl = floorf(r), ce = ceilf(r);
    const float xp = __fmul_rn(__fsub_rn(ce, r), 4294967296.0f);   // p 2^32, exact
    const float craw = below_ceil(w0, xp) ? fl : ce;
    const int c_en = (craw >= (float)a) ? a : (int)craw;
    // pruning: survive iff u0 < r, i.e. w0 < K = ceil(r 2^32)
    const float kf = ceilf(__fmul_rn(r, 4294967296.0f));           // K, at most 24 bits
    const bool surv = below_ceil(w0, kf);
    const bool enrich = r >= 1.0f;
    o.c = enrich ? c_en : (surv ? 1 : 0);
    o.survive = !enrich && surv;
    o.F = aoc_row[a * 8 + (enrich ? c_en : 0)];
    // 1/K = y0 (1 + e) to ~2^-46: y0 the FP32 reciprocal, e its FP32 residual
    const float y0 = __frcp_rn(kf);
    o.e = __fmaf_rn(-kf, y0, 1.0f);
    o.Fs = widen(y0);
    // partial Fisher-Yates: c distinct free steps, draws by multiply-high on w1
    // (the draws form one dependent chain, so it stops after c of them)
    uint32_t x = w1, list = freelist;
    for (int i = 0; i < o.c; ++i) {
        const uint32_t m = (uint32_t)(a - i);
        const unsigned long long prod = (unsigned long long)x * m;
        const int j = i + (int)(prod >> 32);
        x = (uint32_t)prod;
        const uint32_t vi = (list >> (3 * i)) & 7u, vj = (list >> (3 * j)) & 7u;
        const uint32_t t = vi ^ vj;
        list ^= (t << (3 * i)) | (t << (3 * j));
    }
    o.dirs = (o.c == 0) ? 0u : list;
    return o;
}

}  // namespace perm
