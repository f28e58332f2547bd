"""Full-size parity of the batched and served forms.

Config 4 (256 uneven simulations in one batch, sizes up to 10^6, nu down to
10^-6): every simulation's speciation keys against the digest of the oracle's
event-ordered run (mode M, stored by tests/golden/make_config4.py), with its
species count and unique events.  Served requests of config 5's shapes are
too large for the oracle's event-ordered mode, so each request is checked on
a few sampled individuals that the oracle traces alone (mode P: the
individual's lineage followed to its speciation, section "The Independent
Algorithm"), plus two properties that hold at any size: the species
identities are the dense ranks of the speciation keys (the oracle's
definition applied to the device's keys), and the species count is the
number of distinct keys.  Every comparison is bit-exact.
"""
import hashlib
import os

import numpy as np
import pytest

import oracle as O
import paper_2108_05815_b300 as ind
from paper_2108_05815_b300 import workloads as W

pytestmark = pytest.mark.gpu

# the launch configuration the batch benchmark's autotuner chose on B300
TUNED = dict(block_threads=256, blocks_per_sm=8, lineages_per_lane=1, events_per_visit=8, coop_lineages=16384,
             occupancy_step=1.0, tail_events=32.0)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_05815_b300 import build
    build.build()
    yield


def _sim(c, sampler):
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c["deme"],
                          sigma=c.get("sigma", 0.0), sampler=sampler)


def _model(c, sampler):
    return O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], c["seed"], sigma=c.get("sigma"),
                   sampler=sampler)


def _check(c, s, sampler, rng, picks, fraction=1.0, sample_seed=0):
    ids, K = s.species()
    kl, kt = s.species_keys()
    # identities: the oracle's dense ranking of the device's keys
    oids, oK = O.species_ids(kl, kt)
    assert K == oK and np.array_equal(ids, oids)
    # sampled individuals: the oracle traces their lineages alone
    m = _model(c, sampler)
    locs = m.sample(fraction, sample_seed)
    assert len(locs) == s.n_sampled
    if len(locs) == 0:
        return
    pick = rng.choice(len(locs), size=min(picks, len(locs)), replace=False)
    okl, okt, _ = m.trace(locs[pick])
    assert np.array_equal(kl[pick], okl) and np.array_equal(kt[pick], okt)


def _config4_digest():
    """the oracle's event-ordered result of every simulation of config 4
    (tests/golden/make_config4.py): {(sampler, index): row}"""
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "config4_digest.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w, s, k, kind, n, U, K, L, h = line.split()
        rows[(0 if s == "exp" else 1, int(k))] = dict(kind=kind, n=int(n), U=int(U), K=int(K), L=int(L), sha=h)
    return rows


@pytest.mark.parametrize("sampler", [0, 1])
def test_config4_full_size_sampled_parity(sampler):
    """The whole batch of 256 simulations at full size: every simulation's
    speciation keys hash to the digest of the oracle's event-ordered run, with
    its species count and unique events; the batch's critical events are never
    below any simulation's longest line of descent; and two individuals of
    each simulation equal the oracle's lone traces"""
    specs = W.config4()
    want = _config4_digest()
    sims = [_sim(c, sampler) for c in specs]
    try:
        for s in sims:
            s.sample()
        st = ind.batch_run(sims, count_unique=1, **TUNED)
        rng = np.random.default_rng(11 + sampler)
        longest = 0
        for k, (c, s) in enumerate(zip(specs, sims)):
            w = want[(sampler, k)]
            kl, kt = s.species_keys()
            assert s.n_sampled == w["n"]
            h = hashlib.sha256(kl.astype("<u8").tobytes() + kt.astype("<u8").tobytes()).hexdigest()
            assert h == w["sha"], "simulation %d differs from the oracle" % k
            assert st[k]["unique_events"] == w["U"]
            longest = max(longest, w["L"])
            _check(c, s, sampler, rng, picks=2)
            assert s.species()[1] == w["K"]
        assert st[0]["critical_events"] >= longest
    finally:
        for s in sims:
            s.close()


def test_served_config5_shapes_sampled_parity():
    """Requests of config 5's shapes (torus sides log-uniform 128..4096,
    deme 1..4, sample fractions 0.01..1), those with nu >= 1e-5 among the
    first three seconds of arrivals, all submitted at once to a server
    whose budget admits them in waves."""
    reqs = [r for r in W.config5(window_s=3.0) if r["nu"] >= 1e-5][:24]
    assert len(reqs) >= 12
    srv = ind.Server(8 * 10 ** 9, max_sims=16)
    sims, tickets, done = {}, {}, set()
    try:
        for k, r in enumerate(reqs):
            s = _sim(r, 0)
            s.sample(r["fraction"], r["sample_seed"])
            sims[k] = s
            tickets[srv.submit(s)] = k
        steps = 0
        while len(done) < len(reqs):
            for t in srv.step(4):
                done.add(tickets[t])
            steps += 1
            assert steps < 1000000
        rng = np.random.default_rng(17)
        for k, r in enumerate(reqs):
            _check(r, sims[k], 0, rng, picks=3, fraction=r["fraction"], sample_seed=r["sample_seed"])
    finally:
        for s in sims.values():
            s.close()
        srv.close()


@pytest.mark.parametrize("sampler", [0, 1])
def test_served_small_nu_sampled_parity(sampler):
    """The requests that set config 5's latency: speciation probabilities
    in [1e-7, 1e-5), whose last lineages run 10^5 to 10^7 events before they
    speciate.  From the first ten seconds of arrivals: the request of the
    smallest nu (1.0e-7), the three smallest (by sampled individuals) with
    nu below 1e-6 and the two smallest with nu in [1e-6, 1e-5) share a
    server; three individuals of each are traced alone by the oracle, for
    both event-time samplers."""
    arr = W.config5(window_s=10.0)

    def size(r):
        return r["width"] * r["height"] * r["deme"] * r["fraction"]
    lowest = min(arr, key=lambda r: r["nu"])
    low = sorted([r for r in arr if r["nu"] < 1e-6 and r is not lowest], key=size)[:3]
    mid = sorted([r for r in arr if 1e-6 <= r["nu"] < 1e-5], key=size)[:2]
    reqs = [lowest] + low + mid
    assert len(reqs) == 6 and lowest["nu"] < 1.1e-7
    srv = ind.Server(8 * 10 ** 9, max_sims=16)
    sims, tickets, done = {}, {}, set()
    try:
        for k, r in enumerate(reqs):
            s = _sim(r, sampler)
            s.sample(r["fraction"], r["sample_seed"])
            sims[k] = s
            tickets[srv.submit(s)] = k
        steps = 0
        while len(done) < len(reqs):
            for t in srv.step(8):
                done.add(tickets[t])
            steps += 1
            assert steps < 10000000
        rng = np.random.default_rng(29 + sampler)
        for k, r in enumerate(reqs):
            _check(r, sims[k], sampler, rng, picks=3, fraction=r["fraction"], sample_seed=r["sample_seed"])
    finally:
        for s in sims.values():
            s.close()
        srv.close()


@pytest.mark.parametrize("sampler", [0, 1])
def test_implicit_full_size_sampled_parity(sampler):
    """The spatially implicit workload at full size (a local community of
    10^5, a static metacommunity of 10^9): too many metacommunity slots for
    the oracle's event-ordered mode, so 32 sampled lineages are traced alone."""
    c = W.implicit()
    s = ind.Simulation(c["kind"], c["nu"], c["seed"], width=1, height=1, deme=c["deme"], sampler=sampler,
                       migration=c["migration"], meta_size=c["meta_size"], meta_nu=c["meta_nu"])
    try:
        s.sample()
        assert s.run()
        ids, K = s.species()
        kl, kt = s.species_keys()
        oids, oK = O.species_ids(kl, kt)
        assert K == oK and np.array_equal(ids, oids)
        m = O.Model(c["kind"], 1, 1, c["deme"], c["nu"], c["seed"], sampler=sampler, migration=c["migration"],
                    meta_size=c["meta_size"], meta_nu=c["meta_nu"])
        locs = m.sample()
        assert len(locs) == s.n_sampled
        pick = np.random.default_rng(23 + sampler).choice(len(locs), size=32, replace=False)
        okl, okt, _ = m.trace(locs[pick])
        assert np.array_equal(kl[pick], okl) and np.array_equal(kt[pick], okt)
    finally:
        s.close()
