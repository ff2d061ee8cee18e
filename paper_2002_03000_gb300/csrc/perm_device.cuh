// perm_device.cuh -- device building blocks of the flatPERM growth step.
//
// Paper: Campbell and Janse van Rensburg, "Parallel PERM".
//   Sec. 1, eqs. (1)-(2): a_+ free neighbours of the end-point; the next step is
//     uniform among them; W = prod a_+.
//   Sec. 2, eq. (6) and the two paragraphs after it: r = W/[W_n]^sample with the
//     own weight included; r >= 1 enriches into c copies (c = floor r with
//     probability ceil r - r, else ceil r) of weight W/c; r < 1 prunes with
//     probability 1 - r, a survivor's weight is multiplied by 1/r.
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

// Open addressing with triangular probing: the i-th probe of key k is slot
// home(k) + i(i+1)/2 mod 2^log2h, which visits every slot once in the first
// 2^log2h probes.  Against linear probing it breaks up the runs of occupied
// slots that a walk's clustered sites leave, so the longest probe of a warp's
// walks (the warp waits for it) is shorter: on random square-lattice walks of up
// to 511 steps, 3.5 rounds against 4.6 for the longest of six walks' neighbour
// probes.  Deletion in LIFO order stays exact for any fixed probe sequence.
//
// Insert a key known to be absent; returns its slot, or -1 if the probe
// sequence ran through the whole table (full: impossible at load factor <= 1/2).
template <typename Key>
__device__ __forceinline__ int hash_insert(Key *tab, int S, int lane, int log2h, Key k) {
    const uint32_t mask = (1u << log2h) - 1u;
    uint32_t s = hash_home(k, log2h);
    for (int it = 0; it <= (int)mask; ++it) {
        Key *p = tab + (s * (uint32_t)S + (uint32_t)lane);
        if (*p == (Key)0) { *p = k; return (int)s; }
        s = (s + (uint32_t)it + 1u) & mask;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// a_+ (Sec. 1): probe the 2d neighbours of the end-point (triangular probing).
// Returns the free mask; slot[j] is the empty slot that ended the probe of a
// free direction j (its insertion slot while the table is unchanged).  Each
// round loads all 2d slots and updates the probes with selects (no branches);
// at load factor <= 1/2 almost every probe ends in the first round.
// ---------------------------------------------------------------------------
template <int D, typename Key>
__device__ __forceinline__ int probe_neighbours(const Key *tab, int S, int lane, int log2h,
                                                int x, int y, int z, int (&slot)[2 * D],
                                                bool &overflow, int back = -1) {
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
    // direction `back` leads to the walk's previous site, occupied by definition:
    // no probe
    uint32_t pending = ((1u << (2 * D)) - 1u) & ~(back >= 0 ? 1u << back : 0u), freem = 0u;
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
            s[j] = (s[j] + (uint32_t)it + 1u) & mask; // harmless for resolved probes
        }
        if (pending == 0u) break;
    }
    overflow = pending != 0u;
    return (int)freem;
}

// ---------------------------------------------------------------------------
// The ratio r of Sec. 2 (eq. 6): r = W / [W_n]^sample, [W_n]^sample =
// (Wsum + W) / M with Wsum the sum of the weights recorded at length n before
// the node and M the tours started.
//
// The decision needs r only through comparisons (r >= 1, floor and ceil of r,
// u0 < ceil(r) - r, u0 < r), so each node first takes them on a single-
// precision estimate x of r and falls back to r evaluated exactly as defined,
// in double precision, when x lies too close to a comparison's boundary to
// settle it.  The decision then equals the one taken on the double-precision
// r at every node.
//
// The estimate: x = M / (1 + Wsum/W), with the two doubles entering through
// their mantissas rounded to 24 bits (nearest, ties to even; a carry bumps the
// exponent) and their exponents.  Each quotient is a product with the
// hardware's approximate reciprocal (rcp.approx, at most one unit in the last
// place, i.e. relative error <= 2^-23) rounded once more; the other operations
// are correctly rounded single-precision ones.  Relative errors: the two
// mantissas 2^-24 each, the quotient 3 2^-24, the sum 1 + rho 2^-24 (plus rho's
// own 5 2^-24 scaled by rho/(1 + rho) < 1), M 2^-24 and the final quotient
// 3 2^-24, with the three roundings of the double-precision r (<= 4 2^-53):
// |x - r| <= 10.02 2^-24 x.  Every margin below allows at least 15 2^-24 x.
// Doubles with no such bound (W zero, negative, subnormal or not finite; Wsum
// negative, subnormal or not finite; Wsum/W above 2^100) set `odd` and take
// the exact path, and so does M of 2^32 or more (M enters through a 32-bit
// conversion: a 64-bit one costs as much as a double-precision operation).
// Every operation here is single-precision or integer arithmetic: a double-
// precision one takes 64 cycles or more on this part.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mant24_bits(unsigned long long b, int &ef) {
    const uint32_t hi = (uint32_t)(b >> 32) & 0xFFFFFu, lo = (uint32_t)b;
    uint32_t keep = (hi << 3) | (lo >> 29);          // top 23 fraction bits
    const uint32_t rem = lo & 0x1FFFFFFFu;           // the 29 bits dropped
    if (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) keep += 1u;
    if (keep == (1u << 23)) { keep = 0u; ef += 1; }
    return (127u << 23) | keep;
}

// 1/v to within one unit in the last place (v normal and positive).
__device__ __forceinline__ float rcp_approx(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ float ratio_estimate(double W, double Wsum, unsigned long long M, bool &odd) {
    const unsigned long long wb = (unsigned long long)__double_as_longlong(W);
    const unsigned long long sb = (unsigned long long)__double_as_longlong(Wsum);
    int ew = (int)((uint32_t)(wb >> 52) & 0x7FFu), es = (int)((uint32_t)(sb >> 52) & 0x7FFu);
    const bool s_zero = (sb == 0ull);
    bool bad = (wb >> 63) != 0ull || (sb >> 63) != 0ull || ew == 0 || ew == 0x7FF || es == 0x7FF ||
               (es == 0 && !s_zero);
    const float mw = __uint_as_float(mant24_bits(wb, ew));
    const float ms = __uint_as_float(mant24_bits(sb, es));
    const float q = __fmul_rn(ms, rcp_approx(mw));    // in (0.5, 2)
    int e = es - ew;
    bad = bad || (!s_zero && e > 100);
    // below 2^-100 the ratio only moves 1 + rho by less than 2^-99
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    float rho = __fmul_rn(q, __uint_as_float((uint32_t)(e + 127) << 23));   // exact scaling
    rho = s_zero ? 0.0f : rho;
    const float s = __fadd_rn(1.0f, rho);
    const float Mf = __uint2float_rn((uint32_t)M);
    odd = bad || (M >> 32) != 0ull;
    return __fmul_rn(Mf, rcp_approx(s));
}

// r exactly as defined, in double precision: three correctly rounded operations
// in the definition's order.
__device__ __forceinline__ double ratio_exact(double W, double Wsum, unsigned long long M) {
    const double avg = __ddiv_rn(__dadd_rn(Wsum, W), __ull2double_rn(M));
    return __ddiv_rn(W, avg);
}

// Stored-weight scale: weight of a length-n walk is kept divided by 2^E(n).
__device__ __forceinline__ int scale_exp(int d, int n) {
    return d == 2 ? (11 * n) >> 3 : (9 * n) >> 2;
}

// Exact float -> double widening by bit manipulation (normal floats and zero).
__device__ __forceinline__ double widen(float f) {
    const uint32_t b = __float_as_uint(f);
    if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
    const unsigned long long e = ((b >> 23) & 0xFFu) + (1023u - 127u);
    const unsigned long long d = ((unsigned long long)(b >> 31) << 63) | (e << 52) |
                                 ((unsigned long long)(b & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// ---------------------------------------------------------------------------
// The decision of Sec. 2 on the estimate x (enrichment: c = floor r iff
// u0 < ceil(r) - r, at most a_+ copies; pruning: survive iff u0 < r, with
// u0 = w0 2^-32).  Sets `amb` when x cannot settle it:
//  - the branch: x >= 1 + 2^-19 gives r > 1, x <= 1 - 2^-19 gives r < 1;
//  - x (1 - 2^-20) >= a_+ + 1 gives floor r > a_+, so c = a_+ whatever u0;
//  - floor and ceil: x farther than x 2^-20 from an integer gives
//    floor r = floor x;
//  - the u0 comparisons, on w0 against the threshold P = (ceil x - x) 2^32 or
//    P = x 2^32 (exact in single precision), which is within 2565 x of the
//    threshold of r: |w0 - P| > 4096 x + 512 settles them (the 512 covers the
//    rounding of w0 to single precision and of the difference, 128 each).
// Returns c (0: pruned); `surv` marks a survivor of pruning.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int decide_estimate(float x, int a, uint32_t w0, bool &surv, bool &amb) {
    const float w0f = __uint2float_rn(w0);
    const float margin = __fmaf_rn(x, 4096.0f, 512.0f);
    int c = 0;
    surv = false;
    amb = false;
    if (x >= 1.0f + 0x1p-19f) {
        if (__fmul_rn(x, 1.0f - 0x1p-20f) >= (float)(a + 1)) {
            c = a;
        } else {
            const float fl = floorf(x), ce = __fadd_rn(fl, 1.0f);
            const float fr = __fsub_rn(x, fl), p = __fsub_rn(ce, x);          // both exact
            const float dlt = __fsub_rn(w0f, __fmul_rn(p, 4294967296.0f));
            amb = fminf(fr, p) <= __fmul_rn(x, 0x1p-20f) || fabsf(dlt) <= margin;
            const float craw = dlt < 0.0f ? fl : ce;
            c = (craw >= (float)a) ? a : (int)craw;
        }
    } else if (x <= 1.0f - 0x1p-19f) {
        const float dlt = __fsub_rn(w0f, __fmul_rn(x, 4294967296.0f));
        amb = fabsf(dlt) <= margin;
        surv = dlt < 0.0f;
        c = surv ? 1 : 0;
    } else {
        amb = true;
    }
    return c;
}

// The same decision on the double-precision r, with the comparisons taken on
// doubles exactly as defined.
__device__ __forceinline__ int decide_exact(double r, int a, uint32_t w0, bool &surv) {
    const double u0 = __dmul_rn(__uint2double_rn(w0), 0x1p-32);             // exact
    surv = false;
    if (r >= 1.0) {
        const double fl = floor(r), ce = ceil(r);
        const double p = __dsub_rn(ce, r);
        const double craw = (u0 < p) ? fl : ce;
        return (craw >= (double)a) ? a : (int)craw;
    }
    surv = u0 < r;
    return surv ? 1 : 0;
}

// Partial Fisher-Yates: c distinct free steps from the free list (3 bits per
// entry), draws by multiply-high on w1 (one dependent chain, stopped after c).
__device__ __forceinline__ uint32_t choose_steps(int c, int a, uint32_t freelist, uint32_t w1) {
    uint32_t x = w1, list = freelist;
    for (int i = 0; i < c; ++i) {
        const uint32_t m = (uint32_t)(a - i);
        const unsigned long long prod = (unsigned long long)x * m;
        const int j = i + (int)(prod >> 32);
        x = (uint32_t)prod;
        const uint32_t vi = (list >> (3 * i)) & 7u, vj = (list >> (3 * j)) & 7u;
        const uint32_t t = vi ^ vj;
        list ^= (t << (3 * i)) | (t << (3 * j));
    }
    return (c == 0) ? 0u : list;
}

}  // namespace perm
