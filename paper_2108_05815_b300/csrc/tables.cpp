// tables.cpp -- host-side integer tables of the library, computed in binary128
// (libquadmath).  They are roundings of real-valued definitions:
//   ln tables   L_j = round(2^62 ln(2^32 / R_j)), R_j = round(2^45/(8193+2j)),
//               ln2 = round(2^64 ln 2), c3 = round(2^64 / 3)  (inverse
//               transform -ln U of the appendix "Inverse Transform: Uniform
//               and Exponential")
//   Gaussian    C_k = round(2^64 Phi((k - half + 1/2) / sigma)), clamped to
//               [0, 2^64 - 1], half = ceil(10 sigma) in binary64: the
//               per-axis discretised normal of section "Normal Dispersal"
//   kernel      K[d2] = round(2^32 exp(-d2 / (2 sigma^2))): Gaussian weights
//               of the habitat-map dispersal
//   Poisson     round(2^64 P(Poi(mu) <= n)), clamped, n < ceil(mu + 12 sqrt(mu)
//               + 24): point counts of the Poisson event-time sampler
// binary128 carries about 113 bits, far more than the 64 needed, so ties of
// the rounding cannot flip (the tables' distance to the rounding boundary is
// asserted in the test suite).
#include <cmath>
#include <cstdint>
#include <vector>

extern "C" {
#include <quadmath.h>
}

namespace indep {

static uint64_t round_q(__float128 x) {
    __float128 f = floorq(x + (__float128)0.5);
    if (f <= 0) return 0;
    if (f >= ldexpq((__float128)1, 64) - 1) return ~0ull;
    return (uint64_t)f;
}

void host_ln_tables(uint64_t* L, uint32_t* R, int n, uint64_t* ln2_q64, int64_t* c3) {
    for (int j = 0; j < n; ++j) {
        uint64_t d = 8193u + 2u * (uint64_t)j;
        R[j] = (uint32_t)(((1ull << 46) + d) / (2u * d));
        __float128 v = logq(ldexpq((__float128)1, 32) / (__float128)R[j]);
        L[j] = round_q(ldexpq(v, 62));
    }
    *ln2_q64 = round_q(ldexpq(logq((__float128)2), 64));
    *c3 = (int64_t)((((unsigned __int128)1 << 65) + 3) / 6);  // round(2^64 / 3)
}

int host_gauss_half(double sigma) { return (int)std::ceil(10.0 * sigma); }

std::vector<uint64_t> host_gauss_cdf(double sigma) {
    int half = host_gauss_half(sigma);
    std::vector<uint64_t> out(2 * (size_t)half);
    __float128 s = (__float128)sigma;
    __float128 rt2 = sqrtq((__float128)2);
    for (int k = 0; k < 2 * half; ++k) {
        __float128 z = ((__float128)(k - half) + (__float128)0.5) / s;
        __float128 phi = erfcq(-z / rt2) / 2;
        out[k] = round_q(ldexpq(phi, 64));
    }
    return out;
}

std::vector<uint64_t> host_kernel_weights(double sigma, int radius) {
    std::vector<uint64_t> out((size_t)radius * radius + 1);
    __float128 s = (__float128)sigma;
    for (int d2 = 0; d2 <= radius * radius; ++d2)
        out[d2] = round_q(ldexpq(expq(-(__float128)d2 / (2 * s * s)), 32));
    return out;
}

int host_poisson_n(double mu) { return (int)std::ceil(mu + 12.0 * std::sqrt(mu) + 24.0); }

// round(2^64 P(Poi(mu) <= n)), clamped, n = 0 .. host_poisson_n(mu) - 1
std::vector<uint64_t> host_poisson_cdf(double mu) {
    const int n = host_poisson_n(mu);
    std::vector<uint64_t> out(n);
    __float128 m = (__float128)mu;
    __float128 term = expq(-m), acc = 0;
    for (int i = 0; i < n; ++i) {
        if (i > 0) term = term * m / (__float128)i;
        acc += term;
        out[i] = round_q(ldexpq(acc, 64));
    }
    return out;
}

}  // namespace indep
