// device.cuh -- per-event device arithmetic of the Independent algorithm.
//
// All of it is integer arithmetic except the event-time sums (binary64 adds
// and compares): B300 issues binary64 at a small fraction of its 32-bit
// integer rate, so the inverse-transform logarithm, the Gaussian and the
// alias draws run on the integer pipes.
#pragma once

#include <cstdint>

namespace indep {

constexpr uint32_t TAG_INTERVAL = 1u;
constexpr uint32_t TAG_EVENT = 2u;
constexpr uint32_t TAG_MAP = 3u;
constexpr uint32_t TAG_SAMPLE = 4u;

constexpr int KIND_NONSPATIAL = 0;
constexpr int KIND_TORUS = 1;
constexpr int KIND_MAP = 2;
constexpr int KIND_IMPLICIT = 3;  // local community + static metacommunity

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11): ten rounds, multipliers 0xD2511F53 / 0xCD9E8D57,
// Weyl key increments 0x9E3779B9 / 0xBB67AE85.
// ---------------------------------------------------------------------------
struct u32x4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                                      uint32_t& c3, uint32_t k0, uint32_t k1) {
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
    uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
}

__host__ __device__ __forceinline__ u32x4 philox10(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                                   uint32_t c2, uint32_t c3) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(c0, c1, c2, c3, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Block j of the stream primed at (location, time key, tag): the location
// is folded into the key, (time key, j, tag) is the counter.  Returns draws
// 2j (lo) and 2j + 1 (hi).
struct u64x2 {
    uint64_t lo, hi;
};

__host__ __device__ __forceinline__ u64x2 stream_block(uint32_t sk0, uint32_t sk1, uint64_t loc,
                                                       uint64_t tkey, uint32_t j, uint32_t tag) {
    u32x4 o = philox10(sk0 ^ (uint32_t)loc, sk1 ^ (uint32_t)(loc >> 32), (uint32_t)tkey,
                       (uint32_t)(tkey >> 32), j, tag);
    return {(uint64_t)o.x | ((uint64_t)o.y << 32), (uint64_t)o.z | ((uint64_t)o.w << 32)};
}

__host__ __device__ __forceinline__ uint64_t umulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// floor(a b / 2^64) for a 32-bit b, by two 32-bit products: with
// a = h 2^32 + l, floor(a b / 2^64) = floor((h b + floor(l b / 2^32)) / 2^32)
// (the sum stays below 2^64); shorter than a 64 x 64 high product
__host__ __device__ __forceinline__ uint64_t mulhi_u64_u32(uint64_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    const uint64_t hb = (uint64_t)(uint32_t)(a >> 32) * b;
    return (hb + __umulhi((uint32_t)a, b)) >> 32;
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// ---------------------------------------------------------------------------
// Exp(1) by inverse transform of U = (r + 1) 2^-53, r the top 53 bits of a
// draw: -ln U = (53 - e) ln 2 - ln m for r + 1 = m 2^e, m in [1, 2).
// ln m = ln(2^32 / R_j) + ln(1 + s), with j the 12 bits after the leading one
// of m, R_j = round(2^45 / (8193 + 2 j)) and 1 + s = m R_j / 2^32
// (|s| < 2^-12.9); ln(1 + s) = s - s^2 (1/2 - s/3 + s^2/4) with s in signed
// Q0.64 and the bracket in Q2.62.  Result in Q6.58, rounded half up.
// ---------------------------------------------------------------------------
constexpr int LN_BITS = 12;
constexpr uint32_t LN_N = 1u << LN_BITS;

struct __align__(16) LnTables {
    uint64_t L[LN_N];    // round(2^62 ln(2^32 / R_j))
    uint32_t R[LN_N];    // R_j
    uint64_t ln2_q64;    // round(2^64 ln 2)
    int64_t c3;          // round(2^64 / 3)
};

// 32-bit leading zeros and funnel shift, on the device by intrinsic, on the
// host (tests) in plain C++
__host__ __device__ __forceinline__ int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz((int)x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}

// high 32 bits of (hi:lo) << sh, 0 <= sh < 32
__host__ __device__ __forceinline__ uint32_t funnel_l(uint32_t lo, uint32_t hi, int sh) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, (unsigned)sh);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) << sh >> 32);
#endif
}


// floor(log2 x) for x >= 1: on the device the exponent of x converted to
// binary32 rounding toward zero (shorter than a leading-zero count on B300)
__host__ __device__ __forceinline__ int ilog2_32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return (int)(__float_as_uint(__uint2float_rz(x)) >> 23) - 127;
#else
    return 31 - __builtin_clz(x);
#endif
}

// Signed high products by one unsigned high product and a correction that
// depends only on the sign (formed beside the product): a signed a < 0 read
// as unsigned is a + 2^64, so
//   floor(a b / 2^64) = hi(a b) - b          (b >= 0),
//   floor(a^2 / 2^64) = hi(a a) - 2 a  mod 2^64.
__host__ __device__ __forceinline__ int64_t mulhi64s_pos(int64_t a, uint64_t b) {
    return (int64_t)(umulhi64((uint64_t)a, b) - (a < 0 ? b : 0ull));
}
__host__ __device__ __forceinline__ uint64_t sqrhi64s(int64_t a) {
    return umulhi64((uint64_t)a, (uint64_t)a) - (a < 0 ? 2ull * (uint64_t)a : 0ull);
}

__host__ __device__ __forceinline__ int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// One exponential draw of the event search, in units of the grid the
// running event time lives on.  In the interval's binade binary64 values are
// the multiples of 2^sft units of 2^-58, so the search's draw lands on that
// grid rounded twice: -ln U to binary64 (rn53 of X58), then the sum to the
// grid.  Away from a grid midpoint (further than half the draw's binary64
// ulp from one) the two roundings equal one rounding of X58 itself, which
// needs neither the draw's binade nor the first rounding on the chain.
// Returns
//   x58:  X58, -ln U in units of 2^-58 (the value exp1_q58 returns);
//   a:    X58 rounded to the grid, half down: (X58 + 2^(sft-1) - 1) >> sft;
//   near: X58 lies within half its binary64 ulp (an upper bound of it) of a
//         grid midpoint, or that ulp is not finer than the grid; the caller
//         then rounds rn53(x58) to the grid itself.
//
// X58 follows the logarithm's definition step by step up to the series'
// products; the last steps are regrouped (exactly):
//   LN1P = S - 4 Q, LNM = L_j + floor(LN1P / 4) = L_j + floor(S / 4) - Q,
//   X58 = floor((X64 + 32) / 64), X64 = (53 - e) LN2 - 4 LNM
//       = floor((A0 - 4 floor(S / 4) + 4 Q) / 64),  A0 = (53 - e) LN2 + 32 - 4 L_j
//       = U + floor((u - floor(S / 4) + Q) / 16),
//   U = floor(A0 / 64), u = floor(A0 / 4) mod 16,
// so that U, u and the bound of the ulp come from the table entry while the
// series' products run, and three adds and a shift follow the last product.
// X64 + 32 >= 28 for every draw (X64 = -4 at U = 1, its only negative
// value), so the definition's clamp of X64 at 0 never changes X58.
//
// The rest of the chain is built for latency too (each choice measured as a
// dependent chain on B300): the normalising shift works on the high word
// (n >= 2^32 for all but 2^-21 of the draws), takes its length from a
// binary32 conversion's exponent and handles n < 2^32 by selects, not a
// branch; the two high products that feed the bracket run in parallel, each
// an unsigned product whose sign correction is formed beside it.
struct GridDraw {
    uint64_t x58;
    uint64_t a;
    bool near;
};

__host__ __device__ __forceinline__ GridDraw exp1_grid(uint64_t r53, const uint64_t* __restrict__ Ltab,
                                                       const uint32_t* __restrict__ Rtab, uint64_t ln2_q64,
                                                       int64_t c3, int sft) {
    const uint64_t n = r53 + 1ull;
    const uint32_t nh = (uint32_t)(n >> 32), nl = (uint32_t)n;
    // m 2^63 = n << lz as two words, lz the leading zeros of n (10 .. 63);
    // selects rather than a branch for the rare n < 2^32
    const bool big = nh != 0u;
    const int l = 31 - ilog2_32(big ? nh : nl);
    const int lz = big ? l : 32 + l;
    const uint32_t Mh = big ? funnel_l(nl, nh, l) : nl << l;
    const uint32_t Ml = big ? nl << l : 0u;
    const uint32_t j = (Mh >> (31 - LN_BITS)) & (LN_N - 1u);
    const uint32_t R = Rtab[j];   // plain loads: the tables may sit in shared or global memory
    const uint64_t Lj = Ltab[j];
    // A0 = (53 - e) LN2 + 32 - 4 L_j, 128-bit two's complement; U and u
    const uint64_t k = (uint64_t)(lz - 10);  // 53 - e
    const uint64_t klo = k * ln2_q64;
    const uint64_t khi = umulhi64(k, ln2_q64);
    const uint64_t b0 = klo + 32ull;
    const uint64_t l4 = Lj << 2;
    const uint64_t alo = b0 - l4;
    const uint64_t ahi = khi + (b0 < klo ? 1ull : 0ull) - (b0 < l4 ? 1ull : 0ull);
    const uint64_t U = (ahi << 58) | (alo >> 6);
    const int64_t u = (int64_t)((alo >> 2) & 15ull);
    // the draw's binary64 ulp is at most 2^shu units: X58 <= (53 - e) LN2 / 64 + 1
    const uint64_t xb = ((khi << 58) | (klo >> 6)) + 2ull;
    const int shu = 11 - clz64(xb) > 0 ? 11 - clz64(xb) : 0;
    // P = M R = (Mh R) 2^32 + Ml R; S = low 64 bits of P >> 31
    const uint64_t pl = (uint64_t)Ml * R;
    const uint64_t ph = (uint64_t)Mh * R;
    const int64_t s = (int64_t)((ph << 1) + (pl >> 31));
    const int64_t v = u - (s >> 2);
    const int64_t s2 = (int64_t)sqrhi64s(s);
    const int64_t s3 = mulhi64s_pos(s, (uint64_t)c3);
    const int64_t t = (1ll << 61) - (s3 >> 2) + (s2 >> 4);
    const int64_t q = (int64_t)umulhi64((uint64_t)s2, (uint64_t)t);
    const uint64_t w = (uint64_t)((v + q) >> 4);
    // the grid: 2^sft units, midpoint M, zone [M - H, M + H] around it
    const uint64_t half = sft > 0 ? 1ull << (sft - 1) : 0ull;
    const uint64_t gmask = (1ull << sft) - 1ull;
    const uint64_t hu = shu > 0 ? 1ull << (shu - 1) : 0ull;
    GridDraw g;
    g.x58 = U + w;
    g.a = ((U + half - 1ull) + w) >> sft;
    g.near = sft <= shu || (((U - half + hu) + w) & gmask) <= 2ull * hu;
    return g;
}

// Exp(1) of the draw r53 in Q6.58 (the grid parts of exp1_grid unused)
__host__ __device__ __forceinline__ uint64_t exp1_q58(uint64_t r53, const uint64_t* __restrict__ Ltab,
                                                      const uint32_t* __restrict__ Rtab, uint64_t ln2_q64,
                                                      int64_t c3) {
    return exp1_grid(r53, Ltab, Rtab, ln2_q64, c3, 1).x58;
}

// q rounded to 53 significant bits, to nearest, ties to even (q < 2^63.5):
// the multiple of 2^-58 that the binary64 value of q 2^-58 equals.  One add
// and a mask: adding half an ulp less one, plus the ulp bit, carries exactly
// when the rounding goes up.
__host__ __device__ __forceinline__ uint64_t rn53(uint64_t q) {
    const uint32_t qh = (uint32_t)(q >> 32);
    const int sh = qh >= (1u << 21) ? 11 - clz32(qh) : 0;  // bits below the 53rd significant one
    const uint64_t mask = (1ull << sh) - 1ull;
    const uint64_t odd = (uint64_t)(((uint32_t)q >> sh) & (uint32_t)mask & 1u);  // 0 when sh = 0
    return (q + (mask >> 1) + odd) & ~mask;
}

// round-to-nearest-even binary64 of q 2^-58 (q < 2^64), by integer assembly
__device__ __forceinline__ double q58_to_double(uint64_t q) {
    if (q == 0ull) return 0.0;
    const int lz = __clzll((long long)q);
    const uint64_t m = q << lz;                       // bit 63 set
    uint64_t mant = m >> 11;                          // 53 bits
    const uint64_t rem = m & 0x7FFull;
    mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    int64_t E = 5 - lz;                               // q 2^-58 = (m / 2^63) 2^(5 - lz)
    if (mant >> 53) {
        mant >>= 1;
        E += 1;
    }
    return __longlong_as_double((long long)(((uint64_t)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// binary64 of q 2^e for q < 2^53 (exact), by integer assembly: keeps the
// conversion on the integer pipes (B300's FP64 pipe is narrow)
__device__ __forceinline__ double q53_scaled(uint64_t q, int e) {
    if (q == 0ull) return 0.0;
    const int lz = __clzll((long long)q);                 // >= 11
    const uint64_t mant = q << (lz - 11);                  // bit 52 set
    return __longlong_as_double((long long)(((uint64_t)(63 - lz + e + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull)));
}

// ---------------------------------------------------------------------------
// exact integer forms of the event-time bookkeeping (delta_t = 2^d)
// ---------------------------------------------------------------------------
// floor(tau / 2^d) for tau >= 0 given by its bits; tau < 2^(53 + d)
__device__ __forceinline__ uint64_t floor_div_pow2(uint64_t tau_bits, int d) {
    const int E = (int)((tau_bits >> 52) & 0x7FF) - 1023 - d;
    if (E < 0) return 0ull;
    const uint64_t mant = (tau_bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return E >= 52 ? mant << (E - 52) : mant >> (52 - E);
}

// bits of the binary64 value k 2^d (exact for k < 2^53)
__device__ __forceinline__ uint64_t k_times_pow2_bits(uint64_t k, int d) {
    if (k == 0ull) return 0ull;
    const int lz = __clzll((long long)k);
    const uint64_t mant = (k << lz) >> 11;            // exact: k < 2^53
    return ((uint64_t)(63 - lz + d + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFull);
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t pack_loc(uint64_t x, uint64_t y, uint64_t i) {
    return x | (y << 20) | (i << 40);
}
__host__ __device__ __forceinline__ uint32_t loc_x(uint64_t l) { return (uint32_t)(l & 0xFFFFFu); }
__host__ __device__ __forceinline__ uint32_t loc_y(uint64_t l) { return (uint32_t)((l >> 20) & 0xFFFFFu); }
__host__ __device__ __forceinline__ uint32_t loc_i(uint64_t l) { return (uint32_t)(l >> 40); }

// spatially implicit model: local individual i at (0, 0, i); metacommunity
// individual i at y = 1 with i's low 20 bits in x and the rest in the deme
// index
__host__ __device__ __forceinline__ bool in_meta(uint64_t l) { return loc_y(l) != 0u; }
__host__ __device__ __forceinline__ uint64_t meta_loc(uint64_t i) { return pack_loc(i & 0xFFFFFu, 1, i >> 20); }
__host__ __device__ __forceinline__ uint64_t meta_index(uint64_t l) {
    return ((uint64_t)loc_i(l) << 20) | loc_x(l);
}

__device__ __forceinline__ uint32_t wrap_add(uint32_t x, int32_t d, uint32_t n) {
    // (x + d) mod n for |d| < 2^24, x < n <= 2^20
    const int32_t v = (int32_t)x + d;
    if ((uint32_t)v < n) return (uint32_t)v;
    const int32_t w = v < 0 ? v + (int32_t)n : v - (int32_t)n;  // one lap
    if ((uint32_t)w < n) return (uint32_t)w;
    const int32_t r = v % (int32_t)n;
    return (uint32_t)(r < 0 ? r + (int32_t)n : r);
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace indep
