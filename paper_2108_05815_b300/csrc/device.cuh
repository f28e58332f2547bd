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

// ---------------------------------------------------------------------------
// Exp(1) by inverse transform of U = (r + 1) 2^-53, r the top 53 bits of a
// draw: -ln U = (53 - e) ln 2 - ln m for r + 1 = m 2^e, m in [1, 2).
// ln m = ln(2^16 / R_j) + ln(1 + s), with j the 8 bits after the leading one
// of m, R_j = round(2^25 / (513 + 2 j)) and 1 + s = m R_j / 2^16
// (|s| < 2^-8.9), the series to s^6 evaluated in signed Q2.62.  Result in
// Q6.58, rounded half up, then converted to binary64.
// ---------------------------------------------------------------------------
struct LnTables {
    uint64_t L[256];     // round(2^62 ln(2^16 / R_j))
    uint32_t R[256];     // R_j
    uint64_t ln2_q64;    // round(2^64 ln 2)
    int64_t c[7];        // round(2^62 / k), k = 1..6
};

// floor(a b / 2^62) for signed a, b whose product fits in 2^125
__device__ __forceinline__ int64_t q62_mul(int64_t a, int64_t b) {
    uint64_t lo = (uint64_t)a * (uint64_t)b;
    int64_t hi = __mul64hi(a, b);
    return (int64_t)(((uint64_t)hi << 2) | (lo >> 62));
}

__device__ __forceinline__ uint64_t exp1_q58(uint64_t r53, const uint64_t* __restrict__ Ltab,
                                             const uint32_t* __restrict__ Rtab, uint64_t ln2_q64,
                                             const int64_t* c) {
    const uint64_t n = r53 + 1ull;
    const int lz = __clzll((long long)n);            // 10 .. 63
    const uint64_t M = n << lz;                      // m 2^63
    const uint32_t j = (uint32_t)(M >> 55) & 0xFFu;
    const uint64_t R = Rtab[j];
    const uint64_t plo = M * R;
    const uint64_t phi = __umul64hi(M, R);           // (1 + s) 2^79 = phi:plo
    const int64_t s = (int64_t)((phi << 47) | (plo >> 17)) - (int64_t)(1ull << 62);
    int64_t P = c[6];
    P = c[5] - q62_mul(s, P);
    P = c[4] - q62_mul(s, P);
    P = c[3] - q62_mul(s, P);
    P = c[2] - q62_mul(s, P);
    P = c[1] - q62_mul(s, P);
    const int64_t lnm = (int64_t)Ltab[j] + q62_mul(s, P);    // Q62, |lnm| < 1
    // x = k ln2 (Q64, 128-bit) - 4 lnm, k = 53 - e = lz - 10
    const uint64_t k = (uint64_t)(lz - 10);
    uint64_t xlo = k * ln2_q64;
    uint64_t xhi = __umul64hi(k, ln2_q64);
    const uint64_t slo = (uint64_t)lnm << 2;
    const uint64_t shi = (uint64_t)(lnm >> 62);      // sign extension of 4 lnm
    const uint64_t borrow = xlo < slo ? 1ull : 0ull;
    xlo -= slo;
    xhi = xhi - shi - borrow;
    if ((int64_t)xhi < 0) return 0ull;
    const uint64_t rlo = xlo + 32ull;
    const uint64_t rhi = xhi + (rlo < xlo ? 1ull : 0ull);
    return (rhi << 58) | (rlo >> 6);
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

__device__ __forceinline__ uint32_t wrap_add(uint32_t x, int32_t d, uint32_t n) {
    // (x + d) mod n for |d| < 2^24, x < n <= 2^20
    int32_t v = (int32_t)x + d;
    if ((uint32_t)v < n) return (uint32_t)v;
    v %= (int32_t)n;
    return (uint32_t)(v < 0 ? v + (int32_t)n : v);
}

// number of table entries <= r (table nondecreasing, length n)
__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* __restrict__ t, uint32_t n, uint64_t r) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (t[lo + half] <= r) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo;
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace indep
