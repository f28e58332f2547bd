"""The event stream (section "Reporting Coalescence Events Independently")
computed on the device equals the oracle's: the distinct events with their
prior event times and outcomes, in time order, and the coalescences.  Which
lineage of a merged group is named is not unique; it is checked to be a
lineage whose own plain trace holds the event."""
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


DM = None


def deme_map():
    global DM
    if DM is None:
        DM = O.habitat(5, 24, 20)
    return DM


CFGS = [
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=300, nu=1e-2, seed=5),
    dict(kind=W.TORUS, width=16, height=12, deme=2, sigma=1.5, nu=2e-2, seed=6),
    dict(kind=W.MAP, width=24, height=20, sigma=2.0, radius=6, nu=3e-2, seed=7),
    dict(kind=W.IMPLICIT, width=1, height=1, deme=300, nu=0.0, seed=8, migration=0.05, meta_size=400, meta_nu=0.02),
    dict(kind=W.TORUS, width=64, height=64, deme=1, sigma=2.0, nu=1e-3, seed=9),
]


def oracle(cfg, sampler):
    m = O.Model(cfg["kind"], cfg.get("width", 1), cfg.get("height", 1), cfg.get("deme", 1), cfg["nu"], cfg["seed"],
                sigma=cfg.get("sigma"), radius=cfg.get("radius"),
                deme_map=deme_map() if cfg["kind"] == W.MAP else None, sampler=sampler,
                migration=cfg.get("migration", 0.0), meta_size=cfg.get("meta_size", 0),
                meta_nu=cfg.get("meta_nu", 0.0))
    locs = m.sample()
    kl, kt, U, ev, co = m.run_merge_events(locs)
    return m, locs, kl, kt, U, ev, co


def gpu(cfg, sampler, tuning, cap=None):
    if cap is None:
        # raw events (copies included) are the same on every run of a tuning;
        # a culled lineage adds one entry
        _, _, _, _, st = gpu(cfg, sampler, tuning, cap=0)
        cap = st["raw_events"] + st["n_sampled"] + 64
    s = ind.Simulation(cfg["kind"], cfg["nu"], cfg["seed"], width=cfg.get("width", 1), height=cfg.get("height", 1),
                       deme=cfg.get("deme", 1), sigma=cfg.get("sigma", 0.0), radius=cfg.get("radius", 0),
                       deme_map=deme_map() if cfg["kind"] == W.MAP else None, sampler=sampler,
                       migration=cfg.get("migration", 0.0), meta_size=cfg.get("meta_size", 0),
                       meta_nu=cfg.get("meta_nu", 0.0), tuning=tuning)
    s.set_event_log(cap)
    s.sample()
    assert s.run()
    ev, co = s.events() if cap else (None, None)
    kl, kt = s.species_keys()
    st = s.stats()
    s.close()
    return ev, co, kl, kt, st


def check(cfg, sampler, tuning):
    m, locs, okl, okt, U, oev, oco = oracle(cfg, sampler)
    gev, gco, gkl, gkt, st = gpu(cfg, sampler, tuning)
    # logging changes nothing else
    assert np.array_equal(gkl, okl) and np.array_equal(gkt, okt)
    # the distinct events, in time order, with prior times and outcomes
    assert len(gev) == U
    assert np.array_equal(gev["time_bits"], oev["time_bits"])
    assert np.array_equal(gev["loc"], oev["loc"])
    assert np.array_equal(gev["prior_bits"], oev["prior_bits"])
    assert np.array_equal(gev["target"], oev["target"])
    # the coalescences: same (location, time) records
    assert len(gco) == len(oco["loc"])
    g = sorted(zip(gco["time_bits"].tolist(), gco["loc"].tolist()))
    o = sorted(zip(oco["time_bits"].tolist(), oco["loc"].tolist()))
    assert g == o
    # the lineages named are valid: an event's lineage trace holds the event;
    # a coalescence's child disperses at its time into loc, whose next event
    # the parent's trace also holds
    traces = {}

    def trace(a):
        if a not in traces:
            traces[a] = m.trace_log(int(locs[a]))
        return traces[a]

    rng = np.random.default_rng(0)
    for k in rng.choice(len(gev), size=min(200, len(gev)), replace=False):
        tl, tt = trace(int(gev["lineage"][k]))
        assert np.any((tt == gev["time_bits"][k]) & (tl == gev["loc"][k]))
    for k in range(min(100, len(gco))):
        cl, ct = trace(int(gco["child"][k]))
        j = int(np.nonzero(ct == gco["time_bits"][k])[0][0])
        assert cl[j + 1] == gco["loc"][k]
        pl, pt = trace(int(gco["parent"][k]))
        assert np.any((pt == ct[j + 1]) & (pl == gco["loc"][k]))
    return st


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("idx", range(len(CFGS)))
def test_event_stream_matches_oracle(idx, sampler):
    check(CFGS[idx], sampler, None)


@pytest.mark.parametrize("tuning", [dict(coop_lineages=0), dict(coop_lineages=1 << 30), dict(dedup=0),
                                    dict(occupancy_step=0.05, min_events_per_lineage=0.05, tail_events=2.0,
                                         busy_lineages=1e9),
                                    dict(occupancy_step=8.0, tail_events=4096.0)])
def test_event_stream_under_tunings(tuning):
    """every advance form and dedup cadence gives the same stream, the one
    where lineages are culled often included (a culled lineage's copy keeps
    its coalescence visible)"""
    check(CFGS[4], 0, tuning)


def test_event_log_capacity_and_state():
    cfg = CFGS[0]
    s = ind.Simulation(cfg["kind"], cfg["nu"], cfg["seed"], deme=cfg["deme"])
    s.sample()
    with pytest.raises(ind.IndError):
        s.events()  # not run yet
    assert s.run()
    with pytest.raises(ind.IndError):
        s.events()  # run without a log
    s.set_event_log(16)  # far too small
    s.sample()
    with pytest.raises(ind.IndError):
        s.run()
    s.close()
    # a batch mixing logged and unlogged simulations is refused, and so is a
    # logged simulation by the server
    a = ind.Simulation(cfg["kind"], cfg["nu"], 1, deme=cfg["deme"])
    b = ind.Simulation(cfg["kind"], cfg["nu"], 2, deme=cfg["deme"])
    a.set_event_log(1 << 20)
    a.sample()
    b.sample()
    with pytest.raises(ind.IndError):
        ind.batch_run([a, b])
    srv = ind.Server(1 << 30, 4)
    with pytest.raises(ind.IndError):
        srv.submit(a)
    srv.close()
    a.close()
    b.close()


def verify(cfg, sampler, gev, gco, gkl, gkt):
    """check() for a stream obtained another way (a batch)"""
    m, locs, okl, okt, U, oev, oco = oracle(cfg, sampler)
    assert np.array_equal(gkl, okl) and np.array_equal(gkt, okt)
    assert len(gev) == U
    for f in ("time_bits", "loc", "prior_bits", "target"):
        assert np.array_equal(gev[f], oev[f]), f
    g = sorted(zip(gco["time_bits"].tolist(), gco["loc"].tolist()))
    o = sorted(zip(oco["time_bits"].tolist(), oco["loc"].tolist()))
    assert g == o
    rng = np.random.default_rng(1)
    for k in rng.choice(len(gev), size=min(100, len(gev)), replace=False):
        tl, tt = m.trace_log(int(locs[int(gev["lineage"][k])]))
        assert np.any((tt == gev["time_bits"][k]) & (tl == gev["loc"][k]))
    for k in range(min(50, len(gco))):
        cl, ct = m.trace_log(int(locs[int(gco["child"][k])]))
        j = int(np.nonzero(ct == gco["time_bits"][k])[0][0])
        assert cl[j + 1] == gco["loc"][k]


@pytest.mark.parametrize("sampler", [0, 1])
def test_event_stream_of_a_batch(sampler):
    """a batch of logged simulations of every landscape kind: each receives
    the stream the oracle gives it alone, lineages numbered as it samples
    them"""
    cfgs = CFGS[:4]
    caps = []
    for cfg in cfgs:
        _, _, _, _, st = gpu(cfg, sampler, None, cap=0)
        caps.append(st["raw_events"] + st["n_sampled"] + 64)
    sims = []
    for cfg, cap in zip(cfgs, caps):
        s = ind.Simulation(cfg["kind"], cfg["nu"], cfg["seed"], width=cfg.get("width", 1),
                           height=cfg.get("height", 1), deme=cfg.get("deme", 1), sigma=cfg.get("sigma", 0.0),
                           radius=cfg.get("radius", 0), deme_map=deme_map() if cfg["kind"] == W.MAP else None,
                           sampler=sampler, migration=cfg.get("migration", 0.0), meta_size=cfg.get("meta_size", 0),
                           meta_nu=cfg.get("meta_nu", 0.0))
        s.set_event_log(cap)
        s.sample()
        sims.append(s)
    ind.batch_run(sims)
    try:
        for cfg, s in zip(cfgs, sims):
            ev, co = s.events()
            kl, kt = s.species_keys()
            verify(cfg, sampler, ev, co, kl, kt)
    finally:
        for s in sims:
            s.close()

