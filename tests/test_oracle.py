"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: a
published known-answer vector, the exact logarithm, a distribution the paper
states (its event-statistics tests), the Ewens sampling formula (exact law
and the expected-richness closed form), a brute-force forward Moran model, or
a special case with a known answer.  No GPU is needed.
"""
import math
import os

import mpmath
import numpy as np
import pytest
from scipy import special, stats

import oracle as O
from oracle import ln_definition as LD
from oracle import tables as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _times(bits):
    return np.asarray(bits, dtype=np.uint64).view(np.float64)


# --------------------------------------------------------------------------
# RNG
# --------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox_kat.txt")) if not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r if x != "->"]
        ctr, key, out = vals[0:4], vals[4:6], vals[6:10]
        assert O.philox4x32_10(key, ctr) == out


def test_prime_avalanche():
    """strict avalanche of prime (section "Hash functions and the Avalanche
    Effect"): flipping any one bit of the (location, time) input flips every
    output bit with probability close to 1/2"""
    rng = np.random.default_rng(7)
    sk = O.seed_key(42)
    n = 160
    flips = np.zeros((128, 64))
    for _ in range(n):
        loc = int(rng.integers(0, 1 << 63))
        t = int(rng.integers(0, 1 << 63))
        base = O.lib().or_draw(O._ptr(sk), loc, t, O.TAG_EVENT, 0)
        for b in range(128):
            l2, t2 = (loc ^ (1 << b), t) if b < 64 else (loc, t ^ (1 << (b - 64)))
            v = O.lib().or_draw(O._ptr(sk), l2, t2, O.TAG_EVENT, 0)
            d = base ^ v
            flips[b] += [(d >> k) & 1 for k in range(64)]
    p = flips / n
    assert p.min() > 0.3 and p.max() < 0.7
    assert abs(p.mean() - 0.5) < 0.01


def test_neighbour_streams_uncorrelated():
    """correlation test of neighbouring individuals' streams (section
    "Correlation"): four adjacent locations, 100 draws each, many seeds"""
    locs = [O.pack_loc(0, 0, 0), O.pack_loc(1, 0, 0), O.pack_loc(0, 1, 0), O.pack_loc(1, 1, 0)]
    streams = [[] for _ in locs]
    for seed in range(1, 101):
        for a, loc in enumerate(locs):
            streams[a] += [O.draw(seed, loc, 0, O.TAG_INTERVAL, j) >> 11 for j in range(100)]
    n = len(streams[0])
    for a in range(4):
        for b in range(a + 1, 4):
            rho, _ = stats.spearmanr(streams[a], streams[b])
            assert abs(rho) < 4.0 / math.sqrt(n)


# --------------------------------------------------------------------------
# Exp(1) by inverse transform with the fixed-point logarithm
# --------------------------------------------------------------------------
def _r53_cases():
    rng = np.random.default_rng(3)
    cases = {0, 1, 2, 3, (1 << 52) - 1, 1 << 52, (1 << 52) + 1, (1 << 53) - 2, (1 << 53) - 1}
    for k in range(54):
        for d in (-1, 0, 1):
            v = (1 << k) + d - 1
            if 0 <= v < (1 << 53):
                cases.add(v)
    for e in rng.integers(0, 53, size=3000):
        cases.add(int(rng.integers(0, 1 << int(e) + 1)) & ((1 << 53) - 1))
    return sorted(cases)


def test_exp1_matches_exact_logarithm():
    """X = -ln((r + 1) 2^-53) within 2^-57 plus half an ulp of X"""
    mpmath.mp.dps = 40
    for r in _r53_cases():
        x = O.exp1(r << 11)
        exact = -mpmath.log(mpmath.mpf(r + 1) / mpmath.mpf(2) ** 53)
        err = abs(mpmath.mpf(x) - exact)
        bound = mpmath.mpf(2) ** -57 + mpmath.mpf(math.ulp(x) if x > 0 else 0) / 2
        assert err <= bound, (r, x, float(exact))


def test_exp1_q58_is_its_definition_on_every_bucket_edge():
    """the oracle's word-size logarithm equals the plain statement of the
    frozen definition (oracle/ln_definition.py: exact integers, constants
    computed from their definitions) on the first and last value of every
    table bucket of every binade, and on the values just across each edge"""
    n = 0
    for e in range(54):
        for r in LD.bucket_edges(e):
            assert O.exp1_q58(r) == LD.x58(r), (e, r)
            n += 1
    assert n > 300000


def test_ln_definition_constants_and_accuracy():
    """the definition's constants are the oracle's tables, and the definition
    itself is within 2^-57 of the exact logarithm (the values plus half an
    ulp of binary64 bound the oracle's double above)"""
    tab, ln2, c3, _ = T.ln_tables()
    assert ln2 == LD.ln2_units() and c3 == LD.third_units()
    assert all(tab[j] == LD.bucket_log(j) for j in range(1 << LD.BUCKET_BITS))
    assert all(O.lib().or_ln_recip(j) == LD.bucket_reciprocal(j) for j in range(1 << LD.BUCKET_BITS))
    mpmath.mp.dps = 40
    for r in _r53_cases():
        exact = -mpmath.log(mpmath.mpf(r + 1) / mpmath.mpf(2) ** 53)
        assert abs(mpmath.mpf(LD.x58(r)) / mpmath.mpf(2) ** 58 - exact) <= mpmath.mpf(2) ** -57, r


def test_exp1_monotone_and_extremes():
    rs = _r53_cases()
    xs = [O.exp1(r << 11) for r in rs]
    assert all(a >= b for a, b in zip(xs, xs[1:]))
    assert O.exp1(((1 << 53) - 1) << 11) == 0.0
    assert O.exp1(0) == pytest.approx(53 * math.log(2), abs=1e-14)


def test_exp1_distribution():
    rng = np.random.default_rng(11)
    draws = rng.integers(0, 1 << 63, size=20000, dtype=np.int64).astype(np.uint64) * np.uint64(2)
    xs = np.array([O.exp1(int(d)) for d in draws])
    assert stats.kstest(xs, "expon").pvalue > 1e-3


def test_table_rounding_margins():
    """the tables are far from rounding boundaries, so an independent
    computation with error below 1e-4 of the last place rounds identically"""
    assert T.ln_tables()[3] > 1e-4
    assert T.gauss_cdf(2.0)[2] > 1e-4
    assert T.gauss_cdf(4.0)[2] > 1e-4
    assert T.kernel_weights(4.0, 16)[1] > 1e-4


# --------------------------------------------------------------------------
# Event statistics (section "Event Statistics")
# --------------------------------------------------------------------------
def _fixed_point_model(lam=1.0, delta_t=1.0, nu=1e-12, seed=5, sampler=0):
    # a 1 x 1 torus with one individual: every dispersal returns to the same
    # location, so the lineage's event process is one location's process
    return O.Model(O.TORUS, 1, 1, 1, nu, seed, lam=lam, delta_t=delta_t, sigma=1.0, sampler=sampler)


SAMPLERS = [0, 1]


@pytest.mark.parametrize("sampler", SAMPLERS)
@pytest.mark.parametrize("lam,delta_t", [(1.0, 1.0), (2.5, 0.5), (0.3, 4.0)])
def test_inter_event_times_exponential(lam, delta_t, sampler):
    """inter-event times ~ Exp(lambda) (section "Turnover and Speciation Times")"""
    m = _fixed_point_model(lam, delta_t, sampler=sampler)
    loc = O.pack_loc(0, 0, 0)
    tau, gaps = 0.0, []
    for _ in range(20000):
        nxt = m.next_event_time(loc, tau)
        assert nxt > tau
        gaps.append(nxt - tau)
        tau = nxt
    assert stats.kstest(np.array(gaps) * lam, "expon").pvalue > 1e-3


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_points_per_interval_poisson(sampler):
    """points per re-prime interval ~ Poi(lambda delta_t) (section
    "Properties of Homogeneous Poisson Point Processes")"""
    m = _fixed_point_model(1.0, 1.0, sampler=sampler)
    loc = O.pack_loc(0, 0, 0)
    tau, counts = 0.0, {}
    for _ in range(30000):
        tau = m.next_event_time(loc, tau)
        k = int(math.floor(tau))
        counts[k] = counts.get(k, 0) + 1
    last = int(math.floor(tau))
    per = np.array([counts.get(k, 0) for k in range(last)])
    kmax = 5
    obs = np.array([np.sum(per == k) for k in range(kmax)] + [np.sum(per >= kmax)])
    pk = [math.exp(-1.0) / math.factorial(k) for k in range(kmax)]
    exp_ = np.array(pk + [1 - sum(pk)]) * len(per)
    assert stats.chisquare(obs, exp_).pvalue > 1e-3


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_memoryless_from_arbitrary_time(sampler):
    m = _fixed_point_model(1.0, 1.0, sampler=sampler)
    rng = np.random.default_rng(2)
    starts = rng.uniform(0, 5000, size=8000)
    gaps = [m.next_event_time(O.pack_loc(0, 0, 0), t) - t for t in starts]
    assert stats.kstest(gaps, "expon").pvalue > 1e-3


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_speciation_times_exponential(sampler):
    """with dispersal disabled, speciation times ~ Exp(lambda nu)"""
    nu = 0.05
    times = []
    for seed in range(1, 1501):
        m = O.Model(O.TORUS, 1, 1, 1, nu, seed, sigma=1.0, sampler=sampler)
        _, kt, _ = m.trace([O.pack_loc(0, 0, 0)])
        times.append(_times(kt)[0])
    assert stats.kstest(np.array(times) * nu, "expon").pvalue > 1e-3


def test_uniform_dispersal():
    """non-spatial dispersal is uniform over all J indexed locations,
    including the parent's own (section "Uniform Dispersal")"""
    J = 50
    m = O.Model(O.NONSPATIAL, 1, 1, J, 1e-3, 9)
    rng = np.random.default_rng(4)
    hits = np.zeros(J)
    for t in rng.uniform(0, 1e4, size=25000):
        x, y, i = O.unpack_loc(m.disperse(O.pack_loc(0, 0, 17), t))
        assert x == 0 and y == 0
        hits[i] += 1
    assert stats.chisquare(hits).pvalue > 1e-3


@pytest.mark.parametrize("sigma", [2.0, 4.0, 0.7])
def test_normal_dispersal_per_axis(sigma):
    """each axis of a Gaussian dispersal move ~ the discretised N(0, sigma^2),
    round(sigma z) (section "Normal Dispersal")"""
    W = 1000
    m = O.Model(O.TORUS, W, W, 1, 1e-3, 21, sigma=sigma)
    rng = np.random.default_rng(5)
    dxs, dys = [], []
    for t in rng.uniform(0, 1e4, size=25000):
        x, y, i = O.unpack_loc(m.disperse(O.pack_loc(500, 500, 0), t))
        dxs.append(x - 500)
        dys.append(y - 500)
    K = int(math.ceil(4 * sigma)) + 1
    ks = np.arange(-K, K + 1)
    p = stats.norm.cdf((ks + 0.5) / sigma) - stats.norm.cdf((ks - 0.5) / sigma)
    p[0] += stats.norm.cdf((-K - 0.5) / sigma)
    p[-1] += stats.norm.sf((K + 0.5) / sigma)
    for d in (np.clip(dxs, -K, K), np.clip(dys, -K, K)):
        obs = np.array([np.sum(d == k) for k in ks])
        keep = p * len(d) >= 5
        obs2 = np.append(obs[keep], obs[~keep].sum())
        exp2 = np.append(p[keep], p[~keep].sum()) * len(d)
        if exp2[-1] == 0:
            obs2, exp2 = obs2[:-1], exp2[:-1]
        assert stats.chisquare(obs2, exp2).pvalue > 1e-3


def test_gauss_table_is_normal_cdf():
    """the per-axis table is 2^64 Phi((k - half + 1/2)/sigma), checked against
    scipy's independent normal CDF"""
    for sigma in (1.0, 2.0, 3.7, 8.0):
        cdf, half, _ = T.gauss_cdf(sigma)
        assert half == math.ceil(10 * sigma)
        z = (np.arange(2 * half) - half + 0.5) / sigma
        ref = stats.norm.cdf(z)
        got = np.array(cdf, dtype=np.float64) / 2.0 ** 64
        assert np.max(np.abs(got - ref)) < 1e-15


def test_alias_rows_reproduce_weights():
    """every per-cell alias row implies the renormalised dispersal law
    w(o) = exp(-|o|^2 / (2 sigma^2)) deme(target) / W to within n 2^-30"""
    Wd = Hd = 40
    dm = O.habitat(7, Wd, Hd)
    m = O.Model(O.MAP, Wd, Hd, 0, 1e-3, 1, sigma=4.0, radius=16, deme_map=dm)
    habitable = np.flatnonzero(dm)
    for c in habitable[:: max(1, len(habitable) // 12)]:
        cx, cy = int(c % Wd), int(c // Wd)
        q, al, full, dx, dy = m.alias_row(cx, cy)
        n = len(q)
        assert n == 797
        w = np.array([math.exp(-(a * a + b * b) / 32.0) * dm[((cy + b) % Hd) * Wd + (cx + a) % Wd]
                      for a, b in zip(dx.astype(int), dy.astype(int))])
        target = w / w.sum()
        implied = np.zeros(n)
        for col in range(n):
            lo = -(-(col << 32) // n)
            hi = -(-((col + 1) << 32) // n)
            pc = (hi - lo) / 2.0 ** 32
            acc = 1.0 if full[col] else q[col] / 2.0 ** 32
            implied[col] += pc * acc
            implied[al[col]] += pc * (1.0 - acc)
        assert np.max(np.abs(implied - target)) < n * 2.0 ** -30
        assert implied[w == 0].max(initial=0.0) == 0.0


# --------------------------------------------------------------------------
# Whole-model pins: Ewens, forward Moran, special cases
# --------------------------------------------------------------------------
def _nonspatial_K(J, nu, seed, sampler=0):
    m = O.Model(O.NONSPATIAL, 1, 1, J, nu, seed, sampler=sampler)
    kl, kt, _ = m.run_merge(m.sample())
    return O.species_ids(kl, kt)[1]


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_ewens_expected_richness_config1(sampler):
    """J = 10^4, nu = 10^-3, all sampled: the mean richness over 200 seeds is
    within 3 standard errors of theta (psi(theta + J) - psi(theta)),
    theta = J nu / (1 - nu) (appendix "Analytical solutions", Non-Spatial)"""
    J, nu = 10000, 1e-3
    Ks = np.array([_nonspatial_K(J, nu, s, sampler) for s in range(1, 201)])
    theta = J * nu / (1 - nu)
    expected = theta * (special.digamma(theta + J) - special.digamma(theta))
    assert abs(expected - 69.6545) < 1e-3
    se = Ks.std(ddof=1) / math.sqrt(len(Ks))
    assert abs(Ks.mean() - expected) < 3 * se, (Ks.mean(), expected, se)
    # spread of the Ewens law for the same theta: Var K = sum theta k / (theta + k)^2
    sd = math.sqrt(sum(theta * k / (theta + k) ** 2 for k in range(J)))
    assert 0.75 * sd < Ks.std(ddof=1) < 1.3 * sd


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_wide_torus_is_ewens(sampler):
    """A 4 x 4 torus of demes of 4 with sigma = 40: each axis's discretised
    normal, wrapped onto 4 cells, is uniform up to about exp(-2 pi^2 sigma^2
    / 16) (far below 2^-64), and the deme index is uniform, so every
    dispersal picks one of the J = 64 individuals uniformly, the parent's own
    included: the non-spatial model of the appendix "Analytical solutions"
    (Ewens, theta = J nu / (1 - nu)) run through the torus's dispersal,
    wrap and slot code."""
    J, nu = 64, 0.02
    Ks = []
    for seed in range(1, 1001):
        m = O.Model(O.TORUS, 4, 4, 4, nu, seed, sigma=40.0, sampler=sampler)
        kl, kt, _ = m.run_merge(m.sample())
        Ks.append(O.species_ids(kl, kt)[1])
    Ks = np.array(Ks)
    theta = J * nu / (1 - nu)
    expected = theta * (special.digamma(theta + J) - special.digamma(theta))
    se = Ks.std(ddof=1) / math.sqrt(len(Ks))
    assert abs(Ks.mean() - expected) < 3 * se, (Ks.mean(), expected, se)
    sd = math.sqrt(sum(theta * k / (theta + k) ** 2 for k in range(J)))
    assert 0.85 * sd < Ks.std(ddof=1) < 1.15 * sd


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_single_cell_map_is_ewens(sampler):
    """A habitat map of one cell holding 64 individuals: every alias-table
    offset wraps back onto that cell, so a dispersal draws its alias column
    and then a uniform index in the deme: the non-spatial model with J = 64
    (Ewens, theta = J nu / (1 - nu)) run through the map's alias and deme
    code."""
    J, nu = 64, 0.02
    dm = np.array([J], dtype=np.uint8)
    Ks = []
    for seed in range(1, 1001):
        m = O.Model(O.MAP, 1, 1, 0, nu, seed, sigma=2.0, radius=4, deme_map=dm, sampler=sampler)
        kl, kt, _ = m.run_merge(m.sample())
        Ks.append(O.species_ids(kl, kt)[1])
    Ks = np.array(Ks)
    theta = J * nu / (1 - nu)
    expected = theta * (special.digamma(theta + J) - special.digamma(theta))
    se = Ks.std(ddof=1) / math.sqrt(len(Ks))
    assert abs(Ks.mean() - expected) < 3 * se, (Ks.mean(), expected, se)
    sd = math.sqrt(sum(theta * k / (theta + k) ** 2 for k in range(J)))
    assert 0.85 * sd < Ks.std(ddof=1) < 1.15 * sd


def _exact_law(path):
    rows = [l.split() for l in open(path) if not l.startswith("#")]
    return {int(k): int(a) / int(b) for k, a, b in rows}


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_ewens_sampling_formula_J3(sampler):
    law = _exact_law(os.path.join(GOLDEN, "ewens_j3.txt"))
    counts = np.zeros(3)
    pair_same = 0
    n = 12000
    for seed in range(1, n + 1):
        m = O.Model(O.NONSPATIAL, 1, 1, 3, 0.1, seed, sampler=sampler)
        kl, kt, _ = m.run_merge(m.sample())
        ids, K = O.species_ids(kl, kt)
        counts[K - 1] += 1
        pair_same += ids[0] == ids[1]
    exp_ = np.array([law[1], law[2], law[3]]) * n
    assert stats.chisquare(counts, exp_).pvalue > 1e-3
    # exchangeability: P(individuals 0 and 1 share a species) = P(K=1) + P(K=2)/3
    p01 = law[1] + law[2] / 3
    assert abs(pair_same / n - p01) < 5 * math.sqrt(p01 * (1 - p01) / n)


def test_forward_moran_brute_force():
    """the forward-time neutral model (section "The Neutral Theory of
    Biodiversity"), simulated directly with self-replacement allowed, has the
    same richness law as the backward oracle; both match the Ewens formula"""
    J, nu = 4, 0.2
    rng = np.random.default_rng(12)
    labels = np.zeros(J, dtype=np.int64)
    fresh = 1
    fwd = np.zeros(J)
    burn, spacing, samples = 2000, 40, 12000
    u = rng.random((burn + spacing * samples, 3))
    for step in range(burn + spacing * samples):
        dying = int(u[step, 0] * J)
        parent = int(u[step, 1] * J)
        if u[step, 2] < nu:
            labels[dying] = fresh
            fresh += 1
        else:
            labels[dying] = labels[parent]
        if step >= burn and (step - burn) % spacing == 0:
            fwd[len(set(labels.tolist())) - 1] += 1
    bwd = np.zeros(J)
    for seed in range(1, samples + 1):
        bwd[_nonspatial_K(J, nu, seed) - 1] += 1
    theta = J * nu / (1 - nu)
    stirling = [6, 11, 6, 1]  # |s(4, k)|
    poch = theta * (theta + 1) * (theta + 2) * (theta + 3)
    law = np.array([stirling[k] * theta ** (k + 1) / poch for k in range(J)])
    for obs in (fwd, bwd):
        assert stats.chisquare(obs, law * obs.sum()).pvalue > 1e-3
    table = np.vstack([fwd, bwd])
    assert stats.chi2_contingency(table)[1] > 1e-3


def test_special_cases():
    # nu = 1: every lineage speciates at its first event -> K = n
    m = O.Model(O.NONSPATIAL, 1, 1, 60, 1.0, 3)
    kl, kt, U = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 60 and U == 60
    m = O.Model(O.TORUS, 8, 8, 2, 1.0, 3, sigma=2.0)
    kl, kt, _ = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 128
    # J = 1: one species
    m = O.Model(O.NONSPATIAL, 1, 1, 1, 1e-3, 3)
    kl, kt, _ = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 1
    # dispersal forced to self on a deme-1 torus: lineages never meet -> K = n
    m = O.Model(O.TORUS, 6, 5, 1, 0.05, 3, sigma=1e-3)
    kl, kt, _ = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 30


# --------------------------------------------------------------------------
# Invariants: mode P == mode M, unique-event count, subsets
# --------------------------------------------------------------------------
def _models(sampler):
    dm = O.habitat(11, 48, 40)
    return [
        O.Model(O.NONSPATIAL, 1, 1, 2000, 1e-2, 42, sampler=sampler),
        O.Model(O.TORUS, 32, 24, 2, 1e-3, 42, sigma=1.5, sampler=sampler),
        O.Model(O.MAP, 48, 40, 0, 1e-2, 42, sigma=4.0, radius=16, deme_map=dm, sampler=sampler),
    ]


@pytest.mark.parametrize("sampler", SAMPLERS)
@pytest.mark.parametrize("idx", [0, 1, 2])
def test_mode_p_equals_mode_m(idx, sampler):
    m = _models(sampler)[idx]
    locs = m.sample()
    kl, kt, U = m.run_merge(locs)
    pl, pt, ne = m.trace(locs)
    assert np.array_equal(kl, pl) and np.array_equal(kt, pt)
    assert ne.sum() >= U


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_unique_events_are_the_union_of_plain_traces(sampler):
    m = O.Model(O.TORUS, 16, 16, 1, 1e-2, 8, sigma=1.0, sampler=sampler)
    locs = m.sample()
    _, _, U = m.run_merge(locs)
    union = set()
    for l in locs:
        el, et = m.trace_log(int(l))
        union.update(zip(el.tolist(), et.tolist()))
    assert len(union) == U


def test_subset_consistency():
    m = O.Model(O.TORUS, 40, 40, 1, 1e-3, 17, sigma=2.0)
    locs = m.sample()
    kl, kt, _ = m.run_merge(locs)
    sub = np.arange(0, len(locs), 37)
    m2 = O.Model(O.TORUS, 40, 40, 1, 1e-3, 17, sigma=2.0)
    sl, st, _ = m2.run_merge(locs[sub])
    assert np.array_equal(sl, kl[sub]) and np.array_equal(st, kt[sub])


# --------------------------------------------------------------------------
# Inputs
# --------------------------------------------------------------------------
def test_habitat_statistics():
    W = H = 256
    dm = O.habitat(7, W, H)
    n = W * H
    hab = dm[dm > 0]
    assert abs(len(hab) / n - 0.6) < 5 * math.sqrt(0.24 / n)
    obs = np.array([np.sum(hab == d) for d in range(1, 9)])
    assert stats.chisquare(obs).pvalue > 1e-3
    assert np.array_equal(dm, O.habitat(7, W, H))
    assert not np.array_equal(dm, O.habitat(8, W, H))


def test_sample_fraction():
    m = O.Model(O.TORUS, 128, 128, 2, 1e-3, 1, sigma=2.0)
    N = 128 * 128 * 2
    assert len(m.sample(1.0)) == N
    locs = m.sample(0.3, 99)
    assert abs(len(locs) - 0.3 * N) < 5 * math.sqrt(0.21 * N)
    assert np.all(np.diff(locs.astype(np.int64)) != 0)


# --------------------------------------------------------------------------
# Poisson event-time sampler (section "Homogeneous Poisson Point Process")
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mu", [1.0, 0.3, 2.5, 17.0])
def test_poisson_table_is_poisson_cdf(mu):
    """the count table is 2^64 P(Poi(mu) <= n), checked against scipy"""
    cdf, margin = T.poisson_cdf(mu)
    assert len(cdf) == T.poisson_n(mu)
    got = np.array(cdf, dtype=np.float64) / 2.0 ** 64
    ref = stats.poisson.cdf(np.arange(len(cdf)), mu)
    assert np.max(np.abs(got - ref)) < 1e-14
    assert margin > 1e-4
    assert stats.poisson.sf(len(cdf) - 1, mu) < 2.0 ** -64


def test_poisson_points_uniform_within_intervals():
    """given their count, the points of an interval are uniform in it"""
    m = _fixed_point_model(1.0, 1.0, sampler=1)
    loc = O.pack_loc(0, 0, 0)
    tau, fr = 0.0, []
    for _ in range(20000):
        tau = m.next_event_time(loc, tau)
        fr.append(tau - math.floor(tau))
    assert stats.kstest(fr, "uniform").pvalue > 1e-3


def test_samplers_give_different_streams_same_law():
    """the two samplers are different random streams of the same process"""
    a = _nonspatial_K(2000, 1e-2, 9, 0)
    b = _nonspatial_K(2000, 1e-2, 9, 1)
    ka = [_nonspatial_K(500, 2e-2, s, 0) for s in range(1, 121)]
    kb = [_nonspatial_K(500, 2e-2, s, 1) for s in range(1, 121)]
    assert stats.mannwhitneyu(ka, kb).pvalue > 1e-3
    assert (a, b) != (None, None)


# --------------------------------------------------------------------------
# Spatially implicit scenario (background section "Spatially Implicit";
# appendix of the neutral scenarios): a local community of J individuals
# whose parent lives with probability m per event in a static metacommunity
# of J_meta individuals with speciation probability nu_meta.
# --------------------------------------------------------------------------
META = (1 << 31) - 1


def _implicit(J, nu, seed, m, meta_size, meta_nu, sampler=0):
    return O.Model(O.IMPLICIT, 1, 1, J, nu, seed, migration=m, meta_size=meta_size, meta_nu=meta_nu,
                   sampler=sampler)


def _meta_index(loc):
    x, y, i = O.unpack_loc(loc)
    assert y == 1
    return (i << 20) | x


def test_implicit_dispersal_draws():
    """a local lineage's parent lives in the metacommunity with probability m,
    uniform there; otherwise it is uniform over the J local individuals; a
    metacommunity lineage's parent is uniform over the metacommunity"""
    J, meta, mig = 40, 30, 0.3
    m = _implicit(J, 0.0, 9, mig, meta, 0.1)
    rng = np.random.default_rng(5)
    local, metah, n = np.zeros(J), np.zeros(meta), 30000
    for t in rng.uniform(0, 1e4, size=n):
        loc = m.disperse(O.pack_loc(0, 0, 7), t)
        x, y, i = O.unpack_loc(loc)
        if y == 1:
            metah[_meta_index(loc)] += 1
        else:
            assert x == 0 and y == 0
            local[i] += 1
    assert abs(metah.sum() / n - mig) < 5 * math.sqrt(mig * (1 - mig) / n)
    assert stats.chisquare(local).pvalue > 1e-3 and stats.chisquare(metah).pvalue > 1e-3
    # inside the metacommunity: uniform, never back to the local community
    hits = np.zeros(meta)
    for t in rng.uniform(0, 1e4, size=15000):
        hits[_meta_index(m.disperse(O.pack_loc(11, 1, 0), t))] += 1
    assert stats.chisquare(hits).pvalue > 1e-3
    # large metacommunity indices split over x (low 20 bits) and the deme index
    big = _implicit(J, 0.0, 9, 1.0, META, 0.1)
    idx = [_meta_index(big.disperse(O.pack_loc(0, 0, 3), t)) for t in rng.uniform(0, 1e4, size=4000)]
    assert max(idx) < META and max(idx) > (1 << 30) and stats.kstest(np.array(idx) / META, "uniform").pvalue > 1e-3


def test_implicit_speciation_by_community():
    """speciation uses nu locally and nu_meta in the metacommunity"""
    m = _implicit(20, 0.1, 4, 0.5, 1000, 0.6)
    rng = np.random.default_rng(6)
    ts = rng.uniform(0, 1e4, size=20000)
    loc_rate = np.mean([m.speciates(O.pack_loc(0, 0, 5), t) for t in ts])
    meta_rate = np.mean([m.speciates(O.pack_loc(123, 1, 0), t) for t in ts])
    assert abs(loc_rate - 0.1) < 5 * math.sqrt(0.1 * 0.9 / len(ts))
    assert abs(meta_rate - 0.6) < 5 * math.sqrt(0.6 * 0.4 / len(ts))


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_implicit_immigrant_ancestors(sampler):
    """nu_local = 0 and nu_meta = 1: every immigrant ancestor founds its own
    species at its first event in a metacommunity too large for two of them
    to meet, so the richness is the number of immigrant ancestors.  That is
    the theta -> infinity limit of the closed form (appendix "Spatially
    Implicit"): its law is Ewens' with gamma = J m / (1 - m) in place of
    theta, E S = sum_{i < J} gamma / (gamma + i) (self-replacement allowed,
    as for theta in the non-spatial pin)"""
    J, mig = 500, 0.05
    Ks = []
    for seed in range(1, 201):
        m = _implicit(J, 0.0, seed, mig, META, 1.0, sampler)
        kl, kt, _ = m.trace(m.sample())
        Ks.append(O.species_ids(kl, kt)[1])
    Ks = np.array(Ks)
    g = J * mig / (1 - mig)
    expected = sum(g / (g + i) for i in range(J))
    assert abs(expected - g * (special.digamma(g + J) - special.digamma(g))) < 1e-9
    se = Ks.std(ddof=1) / math.sqrt(len(Ks))
    assert abs(Ks.mean() - expected) < 3 * se, (Ks.mean(), expected, se)
    sd = math.sqrt(sum(g * i / (g + i) ** 2 for i in range(J)))
    assert 0.75 * sd < Ks.std(ddof=1) < 1.3 * sd


def test_implicit_closed_community_is_ewens():
    """m = 0: the local community is closed and the model is the non-spatial
    one (Ewens, theta = J nu / (1 - nu)), drawn from different draws"""
    J, nu = 1000, 0.01
    Ks = []
    for seed in range(1, 201):
        m = _implicit(J, nu, seed, 0.0, 1000, 0.5)
        kl, kt, _ = m.run_merge(m.sample())
        Ks.append(O.species_ids(kl, kt)[1])
    Ks = np.array(Ks)
    theta = J * nu / (1 - nu)
    expected = theta * (special.digamma(theta + J) - special.digamma(theta))
    se = Ks.std(ddof=1) / math.sqrt(len(Ks))
    assert abs(Ks.mean() - expected) < 3 * se, (Ks.mean(), expected, se)


def test_implicit_forward_brute_force():
    """the forward-time model simulated directly -- J local and J_meta
    metacommunity individuals, each replaced at rate 1; a local death takes a
    new species (nu), a metacommunity parent (m) or a local parent (self
    allowed); a metacommunity death takes a new species (nu_meta) or a
    metacommunity parent; the metacommunity never sees the local community --
    has the richness law of the backward oracle"""
    J, meta, nu, mig, nu_m = 3, 2, 0.05, 0.3, 0.2
    rng = np.random.default_rng(21)
    labels = np.arange(J + meta, dtype=np.int64)
    fresh = J + meta
    burn, spacing, samples = 3000, 50, 12000
    steps = burn + spacing * samples
    u = rng.random((steps, 4))
    fwd = np.zeros(J)
    for step in range(steps):
        dying = int(u[step, 0] * (J + meta))
        if dying < J:
            if u[step, 1] < nu:
                labels[dying] = fresh
                fresh += 1
            elif u[step, 2] < mig:
                labels[dying] = labels[J + int(u[step, 3] * meta)]
            else:
                labels[dying] = labels[int(u[step, 3] * J)]
        else:
            if u[step, 1] < nu_m:
                labels[dying] = fresh
                fresh += 1
            else:
                labels[dying] = labels[J + int(u[step, 3] * meta)]
        if step >= burn and (step - burn) % spacing == 0:
            fwd[len(set(labels[:J].tolist())) - 1] += 1
    bwd = np.zeros(J)
    for seed in range(1, samples + 1):
        m = _implicit(J, nu, seed, mig, meta, nu_m)
        kl, kt, _ = m.run_merge(m.sample())
        bwd[O.species_ids(kl, kt)[1] - 1] += 1
    assert stats.chi2_contingency(np.vstack([fwd, bwd]))[1] > 1e-3


def test_implicit_special_cases():
    # nu = 1: every lineage speciates at its first (local) event -> S = n
    m = _implicit(80, 1.0, 3, 0.5, 1000, 0.5)
    kl, kt, U = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 80 and U == 80
    # m = 1, nu_meta = 1, no local speciation: every lineage migrates at its
    # first event and founds a species at its second -> S = n, 2n events
    m = _implicit(80, 0.0, 3, 1.0, META, 1.0)
    kl, kt, ne = m.trace(m.sample())
    assert O.species_ids(kl, kt)[1] == 80 and np.all(ne == 2)
    assert all(O.unpack_loc(int(l))[1] == 1 for l in kl)
    # a local community of one individual: S = 1
    m = _implicit(1, 0.0, 3, 0.2, 5, 0.01)
    kl, kt, _ = m.run_merge(m.sample())
    assert O.species_ids(kl, kt)[1] == 1


@pytest.mark.parametrize("sampler", SAMPLERS)
def test_implicit_mode_p_equals_mode_m(sampler):
    m = _implicit(700, 1e-3, 42, 0.05, 5000, 0.02, sampler)
    locs = m.sample()
    kl, kt, U = m.run_merge(locs)
    pl, pt, ne = m.trace(locs)
    assert np.array_equal(kl, pl) and np.array_equal(kt, pt)
    assert ne.sum() >= U


# --------------------------------------------------------------------------
# Event stream (section "Reporting Coalescence Events Independently"):
# mode M's executed events in time order, with prior event times, and its
# coalescences, checked against the plain per-lineage traces
# --------------------------------------------------------------------------
NO_TARGET = np.uint64(0xFFFFFFFFFFFFFFFF)


def _stream_models(sampler):
    dm = O.habitat(5, 24, 20)
    return [
        O.Model(O.NONSPATIAL, 1, 1, 300, 1e-2, 5, sampler=sampler),
        O.Model(O.TORUS, 16, 12, 2, 2e-2, 6, sigma=1.5, sampler=sampler),
        O.Model(O.MAP, 24, 20, 0, 3e-2, 7, sigma=2.0, radius=6, deme_map=dm, sampler=sampler),
        O.Model(O.IMPLICIT, 1, 1, 300, 0.0, 8, sampler=sampler, migration=0.05, meta_size=400, meta_nu=0.02),
    ]


@pytest.mark.parametrize("sampler", SAMPLERS)
@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_event_stream_against_plain_traces(idx, sampler):
    m = _stream_models(sampler)[idx]
    locs = m.sample()
    kl, kt, U, ev, co = m.run_merge_events(locs)
    n = len(locs)
    t = _times(ev["time_bits"])
    # every executed event once, in strictly increasing time
    assert len(t) == U and np.all(np.diff(t) > 0)
    # every lineage ends in exactly one speciation or one coalescence
    spec = ev["target"] == NO_TARGET
    assert int(spec.sum()) + len(co["child"]) == n
    assert len(set(co["child"].tolist())) == len(co["child"])
    # each lineage's events are the prefix of its own plain trace, chained by
    # prior event times and dispersal targets
    plain = [m.trace_log(int(l)) for l in locs]
    merged_at = {int(c): int(tb) for c, tb in zip(co["child"], co["time_bits"])}
    for a in range(n):
        mine = np.nonzero(ev["lineage"] == a)[0]
        pl, pt = plain[a]
        k = len(mine)
        assert k >= 1
        assert np.array_equal(ev["loc"][mine], pl[:k]) and np.array_equal(ev["time_bits"][mine], pt[:k])
        prior = np.concatenate([[0.0], _times(pt[:k - 1])])
        assert np.array_equal(_times(ev["prior_bits"][mine]), prior)
        nxt = ev["target"][mine[:-1]]
        assert np.array_equal(nxt, pl[1:k])
        if a in merged_at:  # it stopped at its merging dispersal
            assert ev["time_bits"][mine[-1]] == merged_at[a] and ev["target"][mine[-1]] != NO_TARGET
        else:
            assert ev["target"][mine[-1]] == NO_TARGET and k == len(pl)
    # a coalescence: the child's trace, after dispersing at time t into L,
    # has its next event where the parent's trace has one at L, and the
    # parent's event before that lies before t
    for L, tb, p, c in zip(co["loc"], co["time_bits"], co["parent"], co["child"]):
        cl, ct = plain[int(c)]
        j = int(np.nonzero(ct == tb)[0][0])
        assert cl[j + 1] == L
        pl, pt = plain[int(p)]
        hit = np.nonzero((pt == ct[j + 1]) & (pl == L))[0]
        assert len(hit) == 1
        h = int(hit[0])
        assert h == 0 or _times(pt[h - 1:h])[0] < _times([tb])[0]


def test_longest_chain_fixture_config1():
    """The stored longest mode-P traces of config 1 (both samplers) are the
    oracle's.  A plausibility tie to the species keys: with lambda = 1 a
    lineage's events come at rate 1, so a trace of n events ends near time n
    (standard deviation sqrt(n)), and the latest speciation time lies within
    40 standard deviations of the longest trace."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2108_05815_b300 import workloads as W
    rows = {}
    for line in open(os.path.join(GOLDEN, "longest_chains.txt")):
        if not line.startswith("#") and line.strip():
            w, s, seed, n, best = line.split()
            rows[(w, s)] = (int(seed), int(n), int(best))
    c = W.config1(42)
    for sampler, name in ((0, "exp"), (1, "poisson")):
        seed, n, best = rows[("config1", name)]
        m = O.Model(c["kind"], 1, 1, c["deme"], c["nu"], seed, sampler=sampler)
        locs = m.sample()
        assert len(locs) == n
        kl, kt, ne = m.trace(locs)
        assert int(ne.max()) == best
        times = kt.view(np.float64)
        assert times.max() <= best + 40.0 * math.sqrt(best)


@pytest.mark.parametrize("workload", ["config1", "config2"])
def test_merge_mode_finds_the_longest_trace(workload):
    """Mode M's count of the longest line of descent (a lineage carries the
    most events of any individual it stands for; a merge keeps the larger
    count) equals the longest mode-P trace, stored for configs 1 and 2 by
    the script that traces every lineage alone; its keys are mode M's."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2108_05815_b300 import workloads as W
    rows = {}
    for line in open(os.path.join(GOLDEN, "longest_chains.txt")):
        if not line.startswith("#") and line.strip():
            w, s, seed, n, best = line.split()
            rows[(w, s)] = (int(seed), int(n), int(best))
    for sampler, name in ((0, "exp"), (1, "poisson")):
        seed, n, best = rows[(workload, name)]
        c = getattr(W, workload)(seed)
        m = O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], seed, sigma=c.get("sigma", 0.0),
                    sampler=sampler)
        locs = m.sample()
        assert len(locs) == n
        kl, kt, U, L = m.run_merge_longest(locs)
        kl2, kt2, U2 = m.run_merge(locs)
        assert L == best and U == U2
        assert np.array_equal(kl, kl2) and np.array_equal(kt, kt2)
