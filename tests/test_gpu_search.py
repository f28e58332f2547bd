"""GPU parity of the event-time searches, one query at a time.

Every search form of the device (one lane per lineage, one or two draw
blocks per step, as the one-lane kernel runs them with integer sums; the
warp-cooperative general search; the short warp search in binary64; the
short warp search as the tail kernel runs it, with integer sums for lambda
= 1; the one-lane search in binary64 throughout) must return, for any (location, tau), the first point
of that location's event process strictly after tau: the oracle's
next_event_time, bit for bit.  The queries mix times in the first interval,
small interval indices (where the integer sums meet rounding ties most
often), exact interval boundaries, large times, and chains of event times
(each query is the previous answer, or one ulp below it).
"""
import numpy as np
import pytest

import oracle as O
import paper_2108_05815_b300 as ind
from paper_2108_05815_b300 import workloads as W

pytestmark = pytest.mark.gpu

FORMS = (0, 1, 2, 3, 4, 5)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_05815_b300 import build
    build.build()
    yield


def queries(model, dt, seed, n_chain=8, chain_len=250):
    rng = np.random.default_rng(seed)
    locs, taus = [], []

    def add(loc, tau):
        locs.append(int(loc))
        taus.append(float(tau))

    def rand_loc():
        x, y, i = rng.integers(0, 1 << 20), rng.integers(0, 1 << 20), rng.integers(0, 1 << 24)
        return O.pack_loc(int(x), int(y), int(i))

    for _ in range(200):  # first interval
        add(rand_loc(), rng.random() * dt)
    for k in range(1, 17):  # small interval indices
        for _ in range(128):
            add(rand_loc(), (k + rng.random()) * dt)
    for k in range(0, 64):  # exact interval boundaries
        add(rand_loc(), k * dt)
    for e in range(8, 46, 2):  # large times
        for _ in range(12):
            k = int(rng.integers(1 << e, 1 << (e + 1)))
            add(rand_loc(), (k + rng.random()) * dt)
    for _ in range(n_chain):  # chains of event times, and one ulp below each
        loc, tau = rand_loc(), 0.0
        for _ in range(chain_len):
            add(loc, tau)
            nxt = model.next_event_time(loc, tau)
            assert nxt > tau
            add(loc, np.nextafter(nxt, 0.0))
            tau = nxt
    return np.array(locs, dtype=np.uint64), np.array(taus, dtype=np.float64)


CASES = [
    dict(sampler=0, lam=1.0, delta_t=1.0),
    dict(sampler=0, lam=1.0, delta_t=0.25),
    dict(sampler=0, lam=1.0, delta_t=4.0),
    dict(sampler=0, lam=1.0, delta_t=2.0 ** -7),
    dict(sampler=0, lam=1.0, delta_t=64.0),
    dict(sampler=0, lam=2.5, delta_t=0.5),
    dict(sampler=0, lam=0.3, delta_t=4.0),
    dict(sampler=1, lam=1.0, delta_t=1.0),
    dict(sampler=1, lam=0.3, delta_t=4.0),
    dict(sampler=1, lam=2.5, delta_t=0.5),
    dict(sampler=1, lam=40.0, delta_t=1.0),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "s%d-lam%g-dt%g" % (c["sampler"], c["lam"], c["delta_t"]))
def test_search_forms_match_oracle(case):
    seed = 11
    model = O.Model(W.NONSPATIAL, 1, 1, 1000, 1e-3, seed, lam=case["lam"], delta_t=case["delta_t"],
                    sampler=case["sampler"])
    locs, taus = queries(model, case["delta_t"], seed=int(case["lam"] * 1000) + case["sampler"])
    want = np.array([model.next_event_time(int(l), float(t)) for l, t in zip(locs, taus)], dtype=np.float64)
    assert np.all(want > taus)
    s = ind.Simulation(W.NONSPATIAL, 1e-3, seed, deme=1000, lam=case["lam"], delta_t=case["delta_t"],
                       sampler=case["sampler"])
    try:
        for form in FORMS:
            got = s.selftest_search(form, locs, taus)
            bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
            assert bad.size == 0, "form %d: %d of %d differ, first at tau=%r loc=%d: %r vs %r" % (
                form, bad.size, locs.size, taus[bad[0]], int(locs[bad[0]]), got[bad[0]], want[bad[0]])
    finally:
        s.close()


def test_search_probe_rejects_bad_arguments():
    s = ind.Simulation(W.NONSPATIAL, 1e-3, 1, deme=10)
    try:
        with pytest.raises(ind.IndError):
            s.selftest_search(6, np.zeros(1, np.uint64), np.zeros(1))
        with pytest.raises(ind.IndError):
            s.selftest_search(0, np.zeros(0, np.uint64), np.zeros(0))
    finally:
        s.close()
