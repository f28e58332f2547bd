"""The logarithm of the inverse transform, stated as a definition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Nothing in the product
path imports this module.

The paper draws each exponential inter-event time by inverse transform,
X = -ln(U) (appendix "Inverse Transform: Uniform and Exponential"), and
fixes no particular logarithm.  Bit-exact reproducibility needs one, so the
build fixes it here: X58(r), the value of -ln((r + 1) 2^-53) in units of
2^-58, is *defined* by the steps below.  The oracle's C function
``or_exp1_q58`` and the CUDA library each compute this same function with
word-size arithmetic (64-bit words, 128-bit products, a table in memory);
this module states it plainly, with Python integers of unbounded size,
exact rationals for every division, and every constant computed in place
from its definition (mpmath for the two real logarithms).  A test compares
``or_exp1_q58`` with ``x58`` on every bucket edge of every binade.

The definition is frozen: a change to it changes every seed's random
streams, and it is made only for a new reading of the paper, never to suit
a kernel.

The steps (all quantities are integers unless said otherwise; floor(a / b)
of integers is exact):

  1. n = r + 1 (1 <= n <= 2^53); e = floor(log2 n); m = n / 2^e in [1, 2).
  2. j = floor((m - 1) 2^12): the bucket of m, 0 <= j < 4096.
  3. R_j = round(2^45 / (8193 + 2 j)), ties up: 2^32 over the bucket's
     midpoint 1 + (j + 1/2) / 4096.
  4. 1 + s = m R_j / 2^32 (exact, |s| < 2^-12.9); S = floor(s 2^64).
  5. ln(1 + s) by the series s - s^2 (1/2 - s/3 + s^2/4) in fixed point:
        S2 = floor(S^2 / 2^64)                   s^2        in units 2^-64
        S3 = floor(S C3 / 2^64), C3 = round(2^64 / 3)       s/3
        T  = 2^61 - floor(S3 / 4) + floor(S2 / 16)    the bracket, units 2^-62
        Q  = floor(S2 T / 2^64)                  s^2 x bracket, units 2^-62
        LN1P = S - 4 Q                           ln(1 + s), units 2^-64
  6. L_j = round(2^62 ln(2^32 / R_j)), the real logarithm rounded to nearest.
  7. LNM = L_j + floor(LN1P / 4): ln m in units 2^-62.
  8. X64 = (53 - e) round(2^64 ln 2) - 4 LNM: -ln U in units 2^-64; a
     negative X64 (only at n = 2^53, U = 1) is taken as 0.
  9. X58 = floor((X64 + 32) / 64): rounded half up to units of 2^-58.

The error of X58 2^-58 against the exact -ln U is below 2^-57 (the s^5/5
term left out of the series is below 2^-66; each floor costs at most one
unit of its scale); the oracle's tests check that against mpmath.
"""
import functools

import mpmath

BUCKET_BITS = 12


def bucket_reciprocal(j):
    """step 3: R_j = round(2^45 / (8193 + 2 j)), ties up"""
    num, den = 1 << 45, 8193 + 2 * j
    return (2 * num + den) // (2 * den)


@functools.lru_cache(maxsize=None)
def bucket_log(j):
    """step 6: L_j = round(2^62 ln(2^32 / R_j)) (to nearest; mpmath at 60 digits)"""
    with mpmath.workdps(60):
        v = mpmath.ldexp(mpmath.log(mpmath.mpf(2) ** 32 / bucket_reciprocal(j)), 62)
        return int(mpmath.nint(v))


@functools.lru_cache(maxsize=None)
def ln2_units():
    """round(2^64 ln 2)"""
    with mpmath.workdps(60):
        return int(mpmath.nint(mpmath.ldexp(mpmath.log(2), 64)))


def third_units():
    """C3 = round(2^64 / 3)"""
    return (2 * (1 << 64) + 3) // 6


def x58(r):
    """X58(r) for 0 <= r < 2^53, by steps 1-9"""
    assert 0 <= r < (1 << 53)
    n = r + 1                                        # 1
    e = n.bit_length() - 1
    j = ((n - (1 << e)) << BUCKET_BITS) >> e         # 2: floor((m - 1) 2^12), m = n / 2^e
    R = bucket_reciprocal(j)                         # 3
    # 4: s = n R / 2^(e + 32) - 1, so s 2^64 = (n R 2^32 - 2^(e + 64)) / 2^e
    S = (n * R * (1 << 32) - (1 << (e + 64))) >> e   # floor (Python's >> floors negatives)
    S2 = (S * S) >> 64                               # 5
    S3 = (S * third_units()) >> 64
    T = (1 << 61) - (S3 >> 2) + (S2 >> 4)
    Q = (S2 * T) >> 64
    LN1P = S - 4 * Q
    LNM = bucket_log(j) + (LN1P >> 2)                # 6, 7
    X64 = (53 - e) * ln2_units() - 4 * LNM           # 8
    if X64 < 0:
        X64 = 0
    return (X64 + 32) >> 6                           # 9


def bucket_edges(e):
    """for the binade [2^e, 2^(e+1)) of n: the first and the last n of every
    non-empty bucket j, with the value just outside each edge that lies in
    the binade; returned as r = n - 1 values (sorted, distinct)"""
    lo, hi = 1 << e, 1 << (e + 1)
    out = set()
    for j in range(1 << BUCKET_BITS):
        first = lo + (((j << e) + (1 << BUCKET_BITS) - 1) >> BUCKET_BITS)   # ceil(j 2^e / 4096)
        nxt = lo + ((((j + 1) << e) + (1 << BUCKET_BITS) - 1) >> BUCKET_BITS)
        if first >= nxt:
            continue  # bucket j holds no integer n in this binade
        for n in (first - 1, first, nxt - 1, nxt):
            if lo <= n < hi and n <= (1 << 53):
                out.add(n - 1)
    return sorted(out)
