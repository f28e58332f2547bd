"""Integer tables of the oracle, computed in arbitrary precision with mpmath.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  These are the oracle's
own tables; the CUDA library computes its copies independently.

Every table is a rounding of a real-valued definition to integers:

* ``ln_tables`` -- the fixed-point natural logarithm behind the inverse
  transform Exp(1) = -ln U (appendix "Inverse Transform: Uniform and
  Exponential"): L_j = round(2^62 ln(2^32 / R_j)) with
  R_j = round(2^45 / (8193 + 2j)), ln2_q64 = round(2^64 ln 2) and
  round(2^64 / 3).
* ``gauss_cdf`` -- the per-axis discretised normal N(0, sigma^2) used for
  Gaussian dispersal (section "Normal Dispersal" compares against exactly
  this discretisation): entry k is round(2^64 Phi((k - half + 1/2) / sigma)),
  clamped to [0, 2^64 - 1], half = ceil(10 sigma) in binary64.
* ``kernel_weights`` -- the Gaussian dispersal weights of the habitat-map
  model, round(2^32 exp(-d2 / (2 sigma^2))) for squared offsets d2.
* ``poisson_cdf`` -- the point count of a re-prime interval in the Poisson
  event-time method (section "Homogeneous Poisson Point Process"):
  entry n is round(2^64 P(Poi(mu) <= n)), clamped to [0, 2^64 - 1], for
  n < ceil(mu + 12 sqrt(mu) + 24) (binary64), mu = lambda delta_t.

Each value also comes with its distance (in units of the last place) from
the nearest rounding boundary, so that tests can show that an independent
computation with a smaller error bound must round to the same integer.
"""
import functools
import math

import mpmath

_DPS = 60


def _round_with_margin(x):
    """round-half-up of an mpf to an int, plus |frac(x) - 1/2| as float"""
    fl = mpmath.floor(x)
    frac = x - fl
    value = int(fl) + (1 if frac >= mpmath.mpf("0.5") else 0)
    return value, float(abs(frac - mpmath.mpf("0.5")))


LN_TABLE_BITS = 12


def ln_recip(j):
    """R_j = round(2^45 / (8193 + 2 j)), ties up (integer arithmetic): 2^32
    over the midpoint (8193 + 2j) / 8192 of bucket j of m in [1, 2)"""
    d = 8193 + 2 * j
    return ((1 << 46) + d) // (2 * d)


@functools.lru_cache(maxsize=None)
def ln_tables():
    """(ln_tab[4096], ln2_q64, c3_q64, min_margin):
    ln_tab[j] = round(2^62 ln(2^32 / R_j)), ln2_q64 = round(2^64 ln 2),
    c3_q64 = round(2^64 / 3)"""
    with mpmath.workdps(_DPS):
        tab, margins = [], []
        for j in range(1 << LN_TABLE_BITS):
            v, mg = _round_with_margin(mpmath.ldexp(mpmath.log(mpmath.mpf(2) ** 32 / ln_recip(j)), 62))
            tab.append(v)
            margins.append(mg)
        ln2, mg = _round_with_margin(mpmath.ldexp(mpmath.log(2), 64))
        margins.append(mg)
    c3 = ((1 << 65) + 3) // 6  # round(2^64 / 3)
    return tuple(tab), ln2, c3, min(margins)


def gauss_half(sigma):
    """ceil(10 sigma) evaluated in binary64"""
    return int(math.ceil(10.0 * float(sigma)))


@functools.lru_cache(maxsize=None)
def gauss_cdf(sigma):
    """(cdf[2*half], half, min_margin) of the per-axis discretised normal"""
    sigma = float(sigma)
    half = gauss_half(sigma)
    out, margins = [], []
    with mpmath.workdps(_DPS):
        s = mpmath.mpf(sigma)
        for k in range(2 * half):
            z = (mpmath.mpf(k - half) + mpmath.mpf("0.5")) / s
            phi = mpmath.erfc(-z / mpmath.sqrt(2)) / 2
            v, mg = _round_with_margin(mpmath.ldexp(phi, 64))
            out.append(min(max(v, 0), (1 << 64) - 1))
            margins.append(mg)
    return tuple(out), half, min(margins)


@functools.lru_cache(maxsize=None)
def kernel_weights(sigma, radius):
    """(kw[0..radius^2], min_margin): round(2^32 exp(-d2 / (2 sigma^2)))"""
    sigma = float(sigma)
    out, margins = [], []
    with mpmath.workdps(_DPS):
        s = mpmath.mpf(sigma)
        for d2 in range(radius * radius + 1):
            v, mg = _round_with_margin(mpmath.ldexp(mpmath.exp(-mpmath.mpf(d2) / (2 * s * s)), 32))
            out.append(v)
            margins.append(mg)
    return tuple(out), min(margins)


def poisson_n(mu):
    """number of CDF entries, ceil(mu + 12 sqrt(mu) + 24) in binary64"""
    mu = float(mu)
    return int(math.ceil(mu + 12.0 * math.sqrt(mu) + 24.0))


@functools.lru_cache(maxsize=None)
def poisson_cdf(mu):
    """(cdf[n], min_margin): round(2^64 P(Poi(mu) <= n)), clamped"""
    mu = float(mu)
    out, margins = [], []
    with mpmath.workdps(_DPS):
        m = mpmath.mpf(mu)
        term = mpmath.exp(-m)
        acc = mpmath.mpf(0)
        for n in range(poisson_n(mu)):
            if n > 0:
                term = term * m / n
            acc += term
            v, mg = _round_with_margin(mpmath.ldexp(acc, 64))
            out.append(min(max(v, 0), (1 << 64) - 1))
            margins.append(mg if v < (1 << 64) - 1 else 0.5)
    return tuple(out), min(margins)
