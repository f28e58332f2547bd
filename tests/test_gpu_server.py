"""Continuous batching: every request's species are identical whether it runs
alone or in the served mix (admitted while others are on the GPU, sharing the
persistent advance kernel), and identical to the oracle."""
import numpy as np
import pytest

import oracle as O
import paper_2108_05815_b300 as ind
from paper_2108_05815_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_05815_b300 import build
    build.build()


REQUESTS = [
    dict(kind=W.TORUS, width=64, height=64, deme=2, sigma=2.0, nu=1e-3, seed=11, fraction=0.5, sample_seed=3),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=3000, nu=5e-3, seed=12, fraction=1.0, sample_seed=0),
    dict(kind=W.TORUS, width=128, height=96, deme=1, sigma=5.0, nu=2e-3, seed=13, fraction=0.2, sample_seed=4),
    dict(kind=W.TORUS, width=30, height=30, deme=4, sigma=1.0, nu=1e-2, seed=14, fraction=1.0, sample_seed=0),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=1, nu=1e-3, seed=15, fraction=1.0, sample_seed=0),
    dict(kind=W.TORUS, width=200, height=200, deme=1, sigma=3.0, nu=3e-4, seed=16, fraction=0.05, sample_seed=5),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=20000, nu=1e-3, seed=17, fraction=0.3, sample_seed=6),
    dict(kind=W.TORUS, width=50, height=40, deme=3, sigma=7.5, nu=5e-2, seed=18, fraction=1.0, sample_seed=0),
    dict(kind=W.IMPLICIT, width=1, height=1, deme=1500, nu=0.0, seed=19, fraction=0.7, sample_seed=2,
         migration=0.03, meta_size=4000, meta_nu=4e-3),
]


def make(r):
    s = ind.Simulation(r["kind"], r["nu"], r["seed"], width=r["width"], height=r["height"], deme=r["deme"],
                       sigma=r.get("sigma", 0.0), migration=r.get("migration", 0.0),
                       meta_size=r.get("meta_size", 0), meta_nu=r.get("meta_nu", 0.0),
                       sampler=r.get("sampler", ind.SAMPLER_EXP))
    s.sample(r["fraction"], r["sample_seed"])
    return s


def alone(r):
    s = make(r)
    assert s.run()
    ids, K = s.species()
    kl, kt = s.species_keys()
    s.close()
    return ids, K, kl, kt


def serve(reqs, budget, max_sims, rounds, arrivals):
    """submit request k at step arrivals[k]; step until all finished"""
    srv = ind.Server(budget, max_sims)
    sims, tickets, done = {}, {}, set()
    step = 0
    while len(done) < len(reqs):
        for k, r in enumerate(reqs):
            if arrivals[k] == step:
                sims[k] = make(r)
                tickets[srv.submit(sims[k])] = k
        for t in srv.step(rounds):
            done.add(tickets[t])
        step += 1
        assert step < 200000
    out = {}
    for k, s in sims.items():
        ids, K = s.species()
        kl, kt = s.species_keys()
        out[k] = (ids, K, kl, kt)
        s.close()
    st = srv.stats()
    srv.close()
    return out, st


def test_served_mix_equals_alone():
    ref = [alone(r) for r in REQUESTS]
    arrivals = [0, 0, 1, 3, 3, 5, 8, 13, 4]
    got, st = serve(REQUESTS, budget=1 << 33, max_sims=64, rounds=4, arrivals=arrivals)
    assert st["finished"] == len(REQUESTS) and st["resident"] == 0 and st["queued"] == 0
    for k in range(len(REQUESTS)):
        ids, K, kl, kt = got[k]
        rid, rK, rkl, rkt = ref[k]
        assert K == rK and np.array_equal(ids, rid)
        assert np.array_equal(kl, rkl) and np.array_equal(kt, rkt)


def test_served_matches_oracle_under_tight_budget():
    # a budget that holds about two of these requests at a time: the rest queue
    reqs = REQUESTS[:5]
    sizes = []
    for r in reqs:
        s = make(r)
        sizes.append(s.n_sampled)
        s.close()
    budget = int(2.2 * max(sizes) * 160 + (1 << 20))
    got, st = serve(reqs, budget=budget, max_sims=3, rounds=2, arrivals=[0] * len(reqs))
    assert st["finished"] == len(reqs)
    for k, r in enumerate(reqs):
        m = O.Model(r["kind"], r["width"], r["height"], r["deme"], r["nu"], r["seed"], sigma=r.get("sigma"),
                    migration=r.get("migration", 0.0), meta_size=r.get("meta_size", 0), meta_nu=r.get("meta_nu", 0.0))
        kl, kt, _ = m.run_merge(m.sample(r["fraction"], r["sample_seed"]))
        oids, oK = O.species_ids(kl, kt)
        ids, K, gkl, gkt = got[k]
        assert K == oK and np.array_equal(ids, oids)
        assert np.array_equal(gkl, kl) and np.array_equal(gkt, kt)


@pytest.mark.parametrize("sampler", [ind.SAMPLER_EXP, ind.SAMPLER_POISSON])
def test_served_uniform_requests_use_the_specialised_kernel(sampler):
    """Requests that all share one landscape kind and search form are run by
    the warp kernel specialised for them (chosen from the resident requests
    between chunks); a non-spatial request arriving later switches the form
    back to the general one and then away again.  Every result equals the
    request run alone and the oracle's."""
    tori = [r for r in REQUESTS if r["kind"] == W.TORUS]
    reqs = [dict(r, sampler=sampler) for r in tori] + [dict(REQUESTS[1], sampler=sampler)]
    ref = [alone(r) for r in reqs]
    arrivals = [0, 0, 2, 2, 3, 6][:len(reqs)]
    assert len(reqs) == 6
    got, st = serve(reqs, budget=1 << 33, max_sims=16, rounds=3, arrivals=arrivals)
    assert st["finished"] == len(reqs)
    for k in range(len(reqs)):
        ids, K, kl, kt = got[k]
        rid, rK, rkl, rkt = ref[k]
        assert K == rK and np.array_equal(ids, rid)
        assert np.array_equal(kl, rkl) and np.array_equal(kt, rkt)
    r = reqs[0]
    m = O.Model(r["kind"], r["width"], r["height"], r["deme"], r["nu"], r["seed"], sigma=r.get("sigma"),
                sampler=sampler)
    kl, kt, _ = m.run_merge(m.sample(r["fraction"], r["sample_seed"]))
    assert np.array_equal(got[0][2], kl) and np.array_equal(got[0][3], kt)


def test_served_empty_request_finishes_without_species():
    """A request whose sample is empty is admitted and reported finished at
    once; the requests around it are unaffected."""
    empty = dict(kind=W.TORUS, width=8, height=8, deme=1, sigma=2.0, nu=1e-2, seed=20, fraction=1e-9,
                 sample_seed=3)
    reqs = [REQUESTS[0], empty, REQUESTS[3]]
    ref = [alone(r) for r in reqs]
    assert ref[1][1] == 0 and ref[1][0].size == 0
    got, st = serve(reqs, budget=1 << 33, max_sims=8, rounds=2, arrivals=[0, 1, 1])
    assert st["finished"] == len(reqs)
    for k in range(len(reqs)):
        ids, K, kl, kt = got[k]
        rid, rK, rkl, rkt = ref[k]
        assert K == rK and np.array_equal(ids, rid)
        assert np.array_equal(kl, rkl) and np.array_equal(kt, rkt)


def test_server_rejects_what_cannot_fit():
    srv = ind.Server(1 << 20, 4)
    s = make(dict(kind=W.NONSPATIAL, width=1, height=1, deme=100000, nu=1e-3, seed=1, fraction=1.0, sample_seed=0))
    with pytest.raises(ind.IndError):
        srv.submit(s)
    s.close()
    srv.close()
