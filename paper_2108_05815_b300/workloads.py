"""Seeded synthetic workloads: the parameters of each simulation only.

This module holds none of the method's arithmetic; it draws configuration
parameters (sizes, speciation probabilities, dispersal widths, arrival
times) with numpy's seeded generator.  The CUDA path and the oracle both
take their inputs from here.

  config 1  non-spatial deme, J = 10,000, all sampled, nu = 1e-3, seed 42
  config 2  256 x 256 torus, one individual per cell, Gaussian sigma = 2,
            nu = 1e-4, seed 42
  config 3  1024 x 1024 percolation map (60% habitable, deme uniform 1..8,
            map seed 7), alias dispersal over radius 16 from sigma = 4,
            nu = 1e-5, seed 42
  config 4  256 simulations: sizes log-uniform 1e3..1e6, nu log-uniform
            1e-6..1e-2, half non-spatial (J = size) and half torus
            (side = round(sqrt(size)), deme 1, sigma uniform in [1, 8])
  config 5  Poisson arrivals (mean 50 per second) of torus requests: side
            log-uniform 128..4096, deme uniform 1..4, sample fraction uniform
            0.01..1, nu log-uniform 1e-7..1e-3, sigma uniform in [1, 8]
"""
import math

import numpy as np

NONSPATIAL, TORUS, MAP, IMPLICIT = 0, 1, 2, 3


def config1(seed=42):
    return dict(kind=NONSPATIAL, width=1, height=1, deme=10000, nu=1e-3, seed=seed, fraction=1.0)


def config2(seed=42):
    return dict(kind=TORUS, width=256, height=256, deme=1, sigma=2.0, nu=1e-4, seed=seed, fraction=1.0)


def config3(seed=42, side=1024):
    return dict(kind=MAP, width=side, height=side, map_seed=7, p_habitable=0.6, max_deme=8, sigma=4.0,
                radius=16, nu=1e-5, seed=seed, fraction=1.0)


def implicit(seed=42):
    """spatially implicit stand-in: a local community of 10^5 individuals (all
    sampled), migration probability 0.01 per event, a static metacommunity of
    10^9 individuals with speciation probability 10^-4, no local speciation"""
    return dict(kind=IMPLICIT, width=1, height=1, deme=100000, nu=0.0, seed=seed, fraction=1.0, migration=0.01,
                meta_size=10 ** 9, meta_nu=1e-4)


def _loguniform(rng, lo, hi, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def config4(master_seed=42, n=256, size_lo=1e3, size_hi=1e6, nu_lo=1e-6, nu_hi=1e-2):
    rng = np.random.default_rng(master_seed)
    sizes = _loguniform(rng, size_lo, size_hi, n)
    nus = _loguniform(rng, nu_lo, nu_hi, n)
    sigmas = rng.uniform(1.0, 8.0, n)
    seeds = rng.integers(1, 1 << 62, n)
    out = []
    for k in range(n):
        if k % 2 == 0:
            out.append(dict(kind=NONSPATIAL, width=1, height=1, deme=int(round(sizes[k])), nu=float(nus[k]),
                            seed=int(seeds[k]), fraction=1.0))
        else:
            side = max(1, int(round(math.sqrt(sizes[k]))))
            out.append(dict(kind=TORUS, width=side, height=side, deme=1, sigma=float(sigmas[k]),
                            nu=float(nus[k]), seed=int(seeds[k]), fraction=1.0))
    return out


def config5(master_seed=42, rate=50.0, window_s=60.0, side_lo=128, side_hi=4096, nu_lo=1e-7, nu_hi=1e-3):
    rng = np.random.default_rng(master_seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= window_s:
            break
        side = int(round(_loguniform(rng, side_lo, side_hi)))
        reqs.append(dict(arrival=t, kind=TORUS, width=side, height=side, deme=int(rng.integers(1, 5)),
                         sigma=float(rng.uniform(1.0, 8.0)), nu=float(_loguniform(rng, nu_lo, nu_hi)),
                         fraction=float(rng.uniform(0.01, 1.0)), seed=int(rng.integers(1, 1 << 62)),
                         sample_seed=int(rng.integers(1, 1 << 62))))
    return reqs
