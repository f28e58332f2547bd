"""GPU parity: the CUDA path, called through the C ABI, against the oracle.

Every comparison is bit-exact: speciation keys (location, IEEE bits of the
time), dense species identities and species counts are integers, so the
tolerance is zero.  Inputs are seeded and synthetic (see workloads.py).
"""
import math
import os

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
    yield


def gpu_sim(cfg, deme_map=None, tuning=None):
    kw = dict(width=cfg.get("width", 1), height=cfg.get("height", 1), deme=cfg.get("deme", 1),
              sigma=cfg.get("sigma", 0.0), radius=cfg.get("radius", 0), lam=cfg.get("lam", 1.0),
              delta_t=cfg.get("delta_t", 1.0), tuning=tuning, sampler=cfg.get("sampler", 0),
              migration=cfg.get("migration", 0.0), meta_size=cfg.get("meta_size", 0),
              meta_nu=cfg.get("meta_nu", 0.0))
    if cfg["kind"] == W.MAP:
        kw["deme_map"] = deme_map
    return ind.Simulation(cfg["kind"], cfg["nu"], cfg["seed"], **kw)


def oracle_model(cfg, deme_map=None):
    return O.Model(cfg["kind"], cfg.get("width", 1), cfg.get("height", 1), cfg.get("deme", 1), cfg["nu"],
                   cfg["seed"], lam=cfg.get("lam", 1.0), delta_t=cfg.get("delta_t", 1.0),
                   sigma=cfg.get("sigma"), radius=cfg.get("radius"), deme_map=deme_map,
                   sampler=cfg.get("sampler", 0), migration=cfg.get("migration", 0.0),
                   meta_size=cfg.get("meta_size", 0), meta_nu=cfg.get("meta_nu", 0.0))


def run_gpu(cfg, deme_map=None, tuning=None, fraction=1.0, sample_seed=0):
    s = gpu_sim(cfg, deme_map, tuning)
    n = s.sample(fraction, sample_seed)
    assert s.run()
    ids, K = s.species()
    kl, kt = s.species_keys()
    st = s.stats()
    s.close()
    return dict(n=n, ids=ids, K=K, kl=kl, kt=kt, stats=st)


def run_oracle(cfg, deme_map=None, fraction=1.0, sample_seed=0):
    m = oracle_model(cfg, deme_map)
    locs = m.sample(fraction, sample_seed)
    kl, kt, U = m.run_merge(locs)
    ids, K = O.species_ids(kl, kt)
    return dict(n=len(locs), ids=ids, K=K, kl=kl, kt=kt, U=U, locs=locs, model=m)


def assert_same(g, o):
    assert g["n"] == o["n"]
    assert np.array_equal(g["kl"], o["kl"])
    assert np.array_equal(g["kt"], o["kt"])
    assert g["K"] == o["K"]
    assert np.array_equal(g["ids"], o["ids"])


# --------------------------------------------------------------------------
# device arithmetic, bit for bit
# --------------------------------------------------------------------------
def test_device_exp_and_philox_bitexact():
    rng = np.random.default_rng(123)
    v = rng.integers(0, np.iinfo(np.int64).max, size=200000, dtype=np.int64).astype(np.uint64)
    v[:54] = [(np.uint64(1) << np.uint64(k)) << np.uint64(11) for k in range(54)]
    v[54] = np.uint64(0xFFFFFFFFFFFFFFFF)
    v[55] = np.uint64(0)
    e, p = ind.selftest(v)
    for i in range(0, len(v), 97):
        assert int(e[i]) == O.exp1_q58(int(v[i]) >> 11), i
    # every value of a set aimed at the logarithm's table buckets: U = (r + 1)
    # 2^-53 just around bucket edges m = 1 + j 2^-12 for every binade
    edges = []
    for ex in range(0, 53):
        for j in rng.integers(0, 4096, size=40):
            base = (1 << ex) + ((int(j) << ex) >> 12)
            for dlt in (-2, -1, 0, 1, 2):
                r = base + dlt - 1
                if 0 <= r < (1 << 53):
                    edges.append(r << 11)
    ev = np.array(edges, dtype=np.uint64)
    ee, _ = ind.selftest(ev, want_philox=False)
    want = np.array([O.exp1_q58(int(x) >> 11) for x in ev], dtype=np.uint64)
    assert np.array_equal(ee, want)
    for i in range(0, len(v), 211):
        w, z = int(v[(i + 1) % len(v)]), int(v[(i + 2) % len(v)])
        key = [int(v[i]) & 0xFFFFFFFF, int(v[i]) >> 32]
        ctr = [w & 0xFFFFFFFF, w >> 32, z & 0xFFFFFFFF, z >> 32]
        assert O.philox4x32_10(key, ctr) == [int(x) for x in p[i]]


def test_device_habitat_matches_oracle():
    for (seed, Wd, Hd, p, md) in [(7, 300, 200, 0.6, 8), (3, 64, 1, 0.25, 3), (11, 1, 1, 1.0, 255)]:
        g = ind.habitat(seed, Wd, Hd, p, md)
        o = O.habitat(seed, Wd, Hd, p, md)
        assert np.array_equal(g, o)


# --------------------------------------------------------------------------
# whole simulations: full parity on small and mid-size workloads
# --------------------------------------------------------------------------
def test_config1_nonspatial_full_parity():
    cfg = W.config1()
    o = run_oracle(cfg)
    g = run_gpu(cfg)
    assert_same(g, o)
    assert g["stats"]["raw_events"] >= o["U"]
    assert g["stats"]["n_sampled"] == 10000


def test_config2_torus_full_parity():
    cfg = W.config2()
    o = run_oracle(cfg)
    g = run_gpu(cfg)
    assert_same(g, o)


@pytest.mark.parametrize("cfg", [
    dict(kind=W.TORUS, width=64, height=48, deme=2, sigma=1.5, nu=1e-3, seed=5),
    dict(kind=W.TORUS, width=37, height=23, deme=3, sigma=6.3, nu=3e-3, seed=6),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=777, nu=2e-2, seed=9),
])
def test_small_models_full_parity(cfg):
    assert_same(run_gpu(cfg), run_oracle(cfg))


@pytest.mark.parametrize("side,nu,sigma,radius", [(96, 1e-2, 4.0, 16), (50, 3e-3, 2.5, 7), (40, 5e-2, 9.0, 20)])
def test_map_full_parity(side, nu, sigma, radius):
    dm = O.habitat(13, side, side)
    cfg = dict(kind=W.MAP, width=side, height=side, sigma=sigma, radius=radius, nu=nu, seed=17)
    assert_same(run_gpu(cfg, deme_map=dm), run_oracle(cfg, deme_map=dm))


def test_sampled_fraction_parity():
    cfg = dict(kind=W.TORUS, width=80, height=60, deme=4, sigma=2.0, nu=2e-3, seed=21)
    o = run_oracle(cfg, fraction=0.3, sample_seed=77)
    g = run_gpu(cfg, fraction=0.3, sample_seed=77)
    assert_same(g, o)
    dm = O.habitat(4, 70, 50)
    cfgm = dict(kind=W.MAP, width=70, height=50, sigma=3.0, radius=10, nu=4e-3, seed=22)
    assert_same(run_gpu(cfgm, dm, fraction=0.45, sample_seed=5), run_oracle(cfgm, dm, fraction=0.45, sample_seed=5))


# --------------------------------------------------------------------------
# unique-event counting is exact
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", [W.config1(),
                                 dict(kind=W.TORUS, width=64, height=64, deme=1, sigma=2.0, nu=1e-3, seed=3)])
def test_unique_event_count_matches_oracle(cfg):
    o = run_oracle(cfg)
    g = run_gpu(cfg, tuning=dict(count_unique=1))
    assert_same(g, o)
    assert g["stats"]["unique_events"] == o["U"]


def test_dedup_insert_counts():
    """the exact-counting mode also counts the horizon dedup's inserts: all,
    those whose slot was already entered, and those shadowed by a lower lane
    of the same warp with the same slot in the same instruction (each of
    which finds its slot entered); without counting, and with the dedup off,
    nothing is counted"""
    cfg = dict(kind=W.TORUS, width=64, height=64, deme=1, sigma=2.0, nu=1e-3, seed=3)
    st = run_gpu(cfg, tuning=dict(count_unique=1, coop_lineages=0))["stats"]
    assert st["dedup_inserts"] > 0 and st["dedup_inserts"] >= st["dedup_repeats"] >= st["dedup_warp_repeats"] >= 0
    assert st["dedup_repeats"] > 0  # lineages meet on a 64 x 64 torus
    for tun in (dict(), dict(count_unique=1, dedup=0)):
        st = run_gpu(cfg, tuning=tun)["stats"]
        assert st["dedup_inserts"] == st["dedup_repeats"] == st["dedup_warp_repeats"] == 0


# --------------------------------------------------------------------------
# invariants: tuning, dedup, graphs, batching, resumption
# --------------------------------------------------------------------------
TUNINGS = [
    dict(dedup=0),
    dict(use_graph=0, rounds_per_check=3),
    dict(block_threads=64, blocks_per_sm=1, lineages_per_lane=1),
    dict(block_threads=512, blocks_per_sm=2, lineages_per_lane=16),
    dict(events_per_round=500.0, min_events_per_lineage=0.5, tail_events=0.5, occupancy_step=0.05),
    dict(events_per_round=1e9, min_events_per_lineage=1e6),
    dict(busy_lineages=0.0),
    dict(busy_lineages=1e12),
    dict(coop_lineages=0),              # one lineage per lane throughout
    dict(coop_lineages=1 << 30),        # one lineage per warp throughout
    dict(coop_lineages=200, events_per_visit=1, lineages_per_lane=2),
    dict(max_step_events=3.0, tail_events=8.0),
    dict(advance_variant=0, coop_lineages=0),   # convergent state machine throughout
    dict(advance_variant=1, coop_lineages=0),   # one-lane loop throughout
]


_TUNING_CFG = dict(kind=W.TORUS, width=48, height=40, deme=2, sigma=2.0, nu=2e-3, seed=31)
_tuning_oracle = {}


@pytest.mark.parametrize("tuning", [None] + TUNINGS)
def test_results_do_not_depend_on_tuning(tuning):
    """every tuning gives the oracle's result (not merely the default
    tuning's), including dedup off, no graphs, one-lane and one-warp forms
    throughout, and extreme water levels"""
    if "o" not in _tuning_oracle:
        _tuning_oracle["o"] = run_oracle(_TUNING_CFG)
    assert_same(run_gpu(_TUNING_CFG, tuning=tuning), _tuning_oracle["o"])


def test_round_budget_resumes():
    cfg = dict(kind=W.TORUS, width=48, height=48, deme=1, sigma=2.0, nu=1e-3, seed=8)
    ref = run_gpu(cfg)
    s = gpu_sim(cfg, tuning=dict(events_per_round=2000.0, min_events_per_lineage=1.0, tail_events=1.0,
                                  rounds_per_check=2))
    s.sample()
    calls = 0
    while not s.run(round_budget=3):
        calls += 1
        assert calls < 100000
    assert calls > 1
    ids, K = s.species()
    kl, kt = s.species_keys()
    assert np.array_equal(kl, ref["kl"]) and np.array_equal(kt, ref["kt"]) and K == ref["K"]
    s.close()


def test_batch_equals_alone():
    dm = O.habitat(2, 60, 60)
    cfgs = [W.config1(),
            dict(kind=W.TORUS, width=100, height=90, deme=1, sigma=3.0, nu=1e-3, seed=4),
            dict(kind=W.NONSPATIAL, width=1, height=1, deme=3, nu=0.5, seed=5),
            dict(kind=W.MAP, width=60, height=60, sigma=4.0, radius=16, nu=1e-2, seed=6),
            dict(kind=W.TORUS, width=20, height=20, deme=4, sigma=1.0, nu=1e-1, seed=7),
            dict(kind=W.NONSPATIAL, width=1, height=1, deme=1, nu=1e-4, seed=8),
            dict(kind=W.TORUS, width=70, height=50, deme=2, sigma=2.0, nu=2e-3, seed=9, sampler=1),
            dict(kind=W.NONSPATIAL, width=1, height=1, deme=5000, nu=1e-3, seed=10, sampler=1),
            dict(kind=W.IMPLICIT, width=1, height=1, deme=3000, nu=0.0, seed=11, migration=0.02,
                 meta_size=4000, meta_nu=3e-3),
            dict(kind=W.IMPLICIT, width=1, height=1, deme=800, nu=1e-3, seed=12, migration=0.1,
                 meta_size=(1 << 31), meta_nu=0.5, sampler=1)]
    alone = [run_gpu(c, dm if c["kind"] == W.MAP else None) for c in cfgs]
    sims = [gpu_sim(c, dm if c["kind"] == W.MAP else None) for c in cfgs]
    for s in sims:
        s.sample()
    stats = ind.batch_run(sims)
    for s, a, st in zip(sims, alone, stats):
        ids, K = s.species()
        kl, kt = s.species_keys()
        assert np.array_equal(kl, a["kl"]) and np.array_equal(kt, a["kt"])
        assert K == a["K"] and np.array_equal(ids, a["ids"])
        assert st["raw_events"] == a["stats"]["raw_events"]
        s.close()


@pytest.mark.parametrize("sampler", [0, 1])
def test_single_cell_map_parity(sampler):
    """A habitat map of one cell of 64 individuals: every alias offset wraps
    back onto the cell."""
    dm = np.array([64], dtype=np.uint8)
    for seed in (3, 4, 5):
        cfg = dict(kind=W.MAP, width=1, height=1, sigma=2.0, radius=4, nu=0.02, seed=seed, sampler=sampler)
        assert_same(run_gpu(cfg, dm), run_oracle(cfg, dm))


def test_empty_sample():
    """A sampling fraction that draws nobody: the run ends at once with no
    species, as in the oracle."""
    cfg = dict(kind=W.TORUS, width=8, height=8, deme=1, sigma=2.0, nu=1e-2, seed=5)
    o = run_oracle(cfg, fraction=1e-9, sample_seed=3)
    g = run_gpu(cfg, fraction=1e-9, sample_seed=3)
    assert o["n"] == 0 and g["n"] == 0
    assert o["K"] == 0 and g["K"] == 0
    assert g["ids"].size == 0 and g["kl"].size == 0


def test_batch_with_an_empty_member():
    """A simulation whose sample is empty shares a batch with others: it
    finishes with no species and leaves the others' results unchanged."""
    cfgs = [dict(kind=W.TORUS, width=40, height=30, deme=1, sigma=2.0, nu=3e-3, seed=21),
            dict(kind=W.TORUS, width=8, height=8, deme=1, sigma=2.0, nu=1e-2, seed=22),
            dict(kind=W.NONSPATIAL, width=1, height=1, deme=700, nu=2e-3, seed=23)]
    fractions = [1.0, 1e-9, 0.5]
    alone = [run_gpu(c, fraction=f, sample_seed=3) for c, f in zip(cfgs, fractions)]
    assert alone[1]["n"] == 0 and alone[1]["K"] == 0
    sims = [gpu_sim(c) for c in cfgs]
    for s, f in zip(sims, fractions):
        s.sample(f, 3)
    ind.batch_run(sims)
    for s, a in zip(sims, alone):
        ids, K = s.species()
        kl, kt = s.species_keys()
        assert K == a["K"] and np.array_equal(ids, a["ids"])
        assert np.array_equal(kl, a["kl"]) and np.array_equal(kt, a["kt"])
        s.close()


# --------------------------------------------------------------------------
# edge and degenerate cases
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", [
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=500, nu=1.0, seed=1),      # nu = 1: K = n
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=1, nu=1e-3, seed=2),       # J = 1: K = 1
    dict(kind=W.TORUS, width=1, height=1, deme=1, sigma=3.0, nu=1e-2, seed=3), # a single cell
    dict(kind=W.TORUS, width=31, height=17, deme=1, sigma=1e-3, nu=0.05, seed=4),  # no movement: K = n
    dict(kind=W.TORUS, width=40, height=30, deme=2, sigma=2.0, nu=3e-3, seed=5, lam=2.5, delta_t=0.5),
    dict(kind=W.TORUS, width=40, height=30, deme=2, sigma=2.0, nu=3e-3, seed=6, lam=0.3, delta_t=4.0),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=2000, nu=1e-2, seed=7, lam=7.0, delta_t=0.125),
    dict(kind=W.TORUS, width=4, height=4, deme=4, sigma=40.0, nu=0.02, seed=8),   # kernel wider than the torus
    dict(kind=W.TORUS, width=4, height=4, deme=4, sigma=40.0, nu=0.02, seed=9, sampler=1),
])
def test_edge_cases_parity(cfg):
    o = run_oracle(cfg)
    g = run_gpu(cfg)
    assert_same(g, o)
    if cfg["nu"] == 1.0 or cfg.get("sigma") == 1e-3:
        assert g["K"] == g["n"]
    if cfg.get("deme") == 1 and cfg["kind"] == W.NONSPATIAL:
        assert g["K"] == 1


# --------------------------------------------------------------------------
# full-size habitat map (config 3): every individual against the oracle's
# stored result, sampled individuals against its lone traces
# --------------------------------------------------------------------------
def _config3_digest():
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "config3_digest.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w, s, seed, n, U, K, L, h = line.split()
        rows[s] = dict(seed=int(seed), n=int(n), U=int(U), K=int(K), L=int(L), sha=h)
    return rows


_c3 = {}


def _config3_gpu(sampler):
    """config 3 at full size on the GPU, once per sampler per module"""
    if sampler not in _c3:
        cfg = dict(W.config3(), sampler=sampler)
        dm = ind.habitat(cfg["map_seed"], cfg["width"], cfg["height"], cfg["p_habitable"], cfg["max_deme"])
        g = run_gpu(cfg, deme_map=dm, tuning=dict(count_unique=1))
        _c3[sampler] = (cfg, dm, g)
    return _c3[sampler]


@pytest.mark.parametrize("sampler", [0, 1])
def test_config3_full_size_equals_oracle(sampler):
    """Every one of config 3's 2,829,667 individuals: the speciation keys of
    the whole sample hash to the digest of the oracle's event-ordered run
    (written by tests/golden/make_config3.py), and the species count, the
    unique-event count and the longest line of descent agree with it."""
    import hashlib
    want = _config3_digest()["exp" if sampler == 0 else "poisson"]
    cfg, dm, g = _config3_gpu(sampler)
    assert np.array_equal(dm, O.habitat(cfg["map_seed"], cfg["width"], cfg["height"], cfg["p_habitable"],
                                        cfg["max_deme"]))
    assert g["n"] == want["n"] == int(dm.astype(np.int64).sum())
    h = hashlib.sha256(g["kl"].astype("<u8").tobytes() + g["kt"].astype("<u8").tobytes()).hexdigest()
    assert h == want["sha"]
    assert g["K"] == want["K"]
    assert g["stats"]["unique_events"] == want["U"]
    assert g["stats"]["critical_events"] >= want["L"]
    # identities: the dense ranks of the keys (the oracle's definition)
    keys = np.stack([g["kl"], g["kt"]], axis=1)
    uniq, inv = np.unique(keys, axis=0, return_inverse=True)
    assert len(uniq) == g["K"] and np.array_equal(g["ids"], inv.reshape(-1).astype(np.uint64))


@pytest.mark.parametrize("sampler", [0, 1])
def test_config3_full_size_sampled_parity(sampler):
    """256 individuals of config 3 picked at random, each traced alone by the
    oracle (mode P) to its speciation: their keys equal the device's"""
    cfg, dm, g = _config3_gpu(sampler)
    m = oracle_model(cfg, dm)
    locs = m.sample()
    assert len(locs) == g["n"]
    pick = np.random.default_rng(100 + sampler).choice(g["n"], size=256, replace=False)
    kl, kt, _ = m.trace(locs[pick])
    assert np.array_equal(kl, g["kl"][pick]) and np.array_equal(kt, g["kt"][pick])


# --------------------------------------------------------------------------
# Poisson event-time sampler
# --------------------------------------------------------------------------
@pytest.mark.parametrize("cfg", [
    dict(W.config1(), sampler=1),
    dict(W.config2(), sampler=1),
    dict(kind=W.TORUS, width=40, height=30, deme=3, sigma=2.5, nu=3e-3, seed=5, sampler=1, lam=2.5, delta_t=0.5),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=2000, nu=1e-2, seed=7, sampler=1, lam=0.3, delta_t=4.0),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=300, nu=1.0, seed=8, sampler=1),
    dict(kind=W.TORUS, width=25, height=25, deme=1, sigma=1.0, nu=1e-2, seed=9, sampler=1, lam=40.0, delta_t=1.0),
])
def test_poisson_sampler_parity(cfg):
    assert_same(run_gpu(cfg), run_oracle(cfg))


def test_poisson_sampler_map_parity_and_count():
    dm = O.habitat(21, 64, 64)
    cfg = dict(kind=W.MAP, width=64, height=64, sigma=4.0, radius=16, nu=5e-3, seed=23, sampler=1)
    o = run_oracle(cfg, dm)
    g = run_gpu(cfg, dm, tuning=dict(count_unique=1))
    assert_same(g, o)
    assert g["stats"]["unique_events"] == o["U"]


@pytest.mark.parametrize("variant", [0, 1])
def test_advance_variants_match_oracle(variant):
    for cfg in [dict(W.config1(), sampler=1), dict(kind=W.TORUS, width=60, height=50, deme=2, sigma=3.0, nu=2e-3,
                                                   seed=12, lam=40.0), dict(W.config2())]:
        o = run_oracle(cfg)
        g = run_gpu(cfg, tuning=dict(advance_variant=variant, coop_lineages=0, count_unique=1))
        assert_same(g, o)
        assert g["stats"]["unique_events"] == o["U"]


@pytest.mark.parametrize("coop", [0, 1 << 30])
@pytest.mark.parametrize("cfg", [
    dict(W.config1(), sampler=1),
    dict(kind=W.TORUS, width=40, height=30, deme=3, sigma=2.5, nu=3e-3, seed=5, sampler=1, lam=2.5, delta_t=0.5),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=2000, nu=1e-2, seed=7, lam=0.3, delta_t=4.0),
    dict(kind=W.TORUS, width=25, height=25, deme=1, sigma=1.0, nu=1e-2, seed=9, lam=40.0, delta_t=1.0),
    dict(kind=W.TORUS, width=25, height=25, deme=1, sigma=1.0, nu=1e-2, seed=9, sampler=1, lam=40.0),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=700, nu=3e-3, seed=4, lam=0.05, delta_t=2.0),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=700, nu=3e-3, seed=4, sampler=1, lam=0.05, delta_t=2.0),
    # lambda dt = 2: the four-interval searches, with intervals of more than 8 points
    dict(kind=W.TORUS, width=30, height=30, deme=2, sigma=2.0, nu=5e-3, seed=21, lam=2.0),
    dict(kind=W.TORUS, width=30, height=30, deme=2, sigma=2.0, nu=5e-3, seed=21, sampler=1, lam=2.0),
    dict(kind=W.TORUS, width=3, height=2, deme=1, sigma=6.0, nu=1e-3, seed=22, lam=0.5, delta_t=1.0),
    dict(kind=W.TORUS, width=3, height=2, deme=1, sigma=6.0, nu=1e-3, seed=22, sampler=1, lam=0.5),
])
def test_cooperative_tail_parity(cfg, coop):
    """the warp-cooperative advance kernel gives the oracle's results for both
    samplers and both search forms, including long and nearly empty re-prime
    intervals and tori narrower than the dispersal kernel"""
    o = run_oracle(cfg)
    g = run_gpu(cfg, tuning=dict(coop_lineages=coop, count_unique=1))
    assert_same(g, o)
    assert g["stats"]["unique_events"] == o["U"]


def test_cooperative_map_parity():
    dm = O.habitat(31, 50, 50)
    for sampler in (0, 1):
        cfg = dict(kind=W.MAP, width=50, height=50, sigma=3.0, radius=9, nu=8e-3, seed=33, sampler=sampler)
        assert_same(run_gpu(cfg, dm, tuning=dict(coop_lineages=1 << 30)), run_oracle(cfg, dm))


# --------------------------------------------------------------------------
# spatially implicit scenario (local community + static metacommunity)
# --------------------------------------------------------------------------
IMPLICIT_CFGS = [
    # immigrant-ancestor regime of the oracle pin (every ancestor its own species)
    dict(kind=W.IMPLICIT, width=1, height=1, deme=500, nu=0.0, seed=7, migration=0.05, meta_size=(1 << 31) - 1,
         meta_nu=1.0),
    # coalescence in a small metacommunity, local speciation too
    dict(kind=W.IMPLICIT, width=1, height=1, deme=2000, nu=1e-4, seed=8, migration=0.02, meta_size=5000,
         meta_nu=2e-3),
    # metacommunity indices above 2^20 (split over x and the deme index)
    dict(kind=W.IMPLICIT, width=1, height=1, deme=3000, nu=0.0, seed=9, migration=0.3, meta_size=3 << 28,
         meta_nu=1e-3),
    # closed local community (m = 0), and every lineage leaving at once (m = 1)
    dict(kind=W.IMPLICIT, width=1, height=1, deme=1500, nu=2e-3, seed=10, migration=0.0, meta_size=10, meta_nu=0.5),
    dict(kind=W.IMPLICIT, width=1, height=1, deme=400, nu=0.0, seed=11, migration=1.0, meta_size=600, meta_nu=1e-2),
    # other rates and re-prime intervals
    dict(kind=W.IMPLICIT, width=1, height=1, deme=700, nu=5e-4, seed=12, migration=0.05, meta_size=900, meta_nu=5e-3,
         lam=2.5, delta_t=0.5),
]


@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("idx", range(len(IMPLICIT_CFGS)))
def test_implicit_parity(idx, sampler):
    """species identities, keys and the exact unique-event count equal the
    oracle's, for both event-time samplers"""
    cfg = dict(IMPLICIT_CFGS[idx], sampler=sampler)
    if cfg["meta_size"] > (1 << 24):
        # too many indexed locations for the oracle's event-ordered mode:
        # compare with its per-lineage traces
        m = oracle_model(cfg)
        locs = m.sample()
        kl, kt, _ = m.trace(locs)
        ids, K = O.species_ids(kl, kt)
        o = dict(n=len(locs), ids=ids, K=K, kl=kl, kt=kt)
        assert_same(run_gpu(cfg), o)
        return
    o = run_oracle(cfg)
    g = run_gpu(cfg, tuning=dict(count_unique=1))
    assert_same(g, o)
    assert g["stats"]["unique_events"] == o["U"]


@pytest.mark.parametrize("tuning", [dict(coop_lineages=0), dict(coop_lineages=1 << 30),
                                    dict(advance_variant=0, coop_lineages=0), dict(dedup=0),
                                    dict(occupancy_step=4.0, tail_events=4096.0)])
def test_implicit_tunings(tuning):
    cfg = IMPLICIT_CFGS[1]
    assert_same(run_gpu(cfg, tuning=tuning), run_oracle(cfg))


def test_implicit_sampled_fraction():
    cfg = IMPLICIT_CFGS[1]
    assert_same(run_gpu(cfg, fraction=0.3, sample_seed=5), run_oracle(cfg, fraction=0.3, sample_seed=5))



def test_alias_rows_equal_oracle():
    """The device's alias rows (k_alias_build) against the oracle's alias
    construction, entry by entry: threshold, the alias column's offset, the
    always-taken mark, and the demes of both target cells that the packed
    entry carries."""
    W_, H_ = 97, 83
    dm = O.habitat(5, W_, H_)
    cfg = dict(kind=W.MAP, width=W_, height=H_, sigma=4.0, radius=16, nu=1e-3, seed=3)
    s = gpu_sim(cfg, dm)
    m = oracle_model(cfg, dm)
    rng = np.random.default_rng(9)
    cells = np.flatnonzero(dm.reshape(-1) > 0)
    pick = rng.choice(cells, size=min(250, cells.size), replace=False)
    try:
        for cell in pick:
            cx, cy = int(cell % W_), int(cell // W_)
            e = s.alias_row(cx, cy)
            q, al, full, dx, dy = m.alias_row(cx, cy)
            assert e.size == q.size
            assert np.array_equal(e & 0xFFFFFFFF, q.astype(np.uint64))
            full_b = full.astype(bool)
            al_eff = np.where(full_b, np.arange(q.size), al.astype(np.int64))  # a full column is its own alias
            sx = (((e >> 32) & 0x7F).astype(np.int64) ^ 0x40) - 0x40  # 7-bit two's complement
            sy = (((e >> 39) & 0x7F).astype(np.int64) ^ 0x40) - 0x40
            assert np.array_equal(sx, dx[al_eff].astype(np.int64)) and np.array_equal(sy, dy[al_eff].astype(np.int64))
            assert np.array_equal(e >> 63, full.astype(np.uint64))
            tdeme = dm.reshape(H_, W_)[(cy + dy.astype(np.int64)) % H_, (cx + dx.astype(np.int64)) % W_]
            assert np.array_equal((e >> 46) & 0xFF, tdeme.astype(np.uint64))
            assert np.array_equal((e >> 54) & 0xFF, tdeme[al_eff].astype(np.uint64))
        with pytest.raises(ind.IndError):  # a cell without habitat has no row
            empty = np.flatnonzero(dm.reshape(-1) == 0)[0]
            s.alias_row(int(empty % W_), int(empty // W_))
    finally:
        s.close()


def _longest_chains():
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "longest_chains.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w, s, seed, n, best = line.split()
        rows[(w, s)] = (int(seed), int(n), int(best))
    return rows


@pytest.mark.parametrize("tuning", [None, dict(coop_lineages=0), dict(coop_lineages=1 << 30),
                                    dict(max_step_events=3.0, tail_events=8.0)])
@pytest.mark.parametrize("sampler", [0, 1])
@pytest.mark.parametrize("workload", ["config1", "config2"])
def test_critical_chain_not_below_longest_lineage(workload, sampler, tuning):
    """Between horizons a lineage's events are run by one lineage of the
    round (merges happen only at horizons), so the events of any one
    sampled individual's trace that fall in a round are at most the round's
    most events on one lineage.  The run's critical-event count (the sum of
    those maxima) is therefore never below the longest trace of the oracle's
    mode P, stored with its writer script beside the other fixtures."""
    seed, n, best = _longest_chains()[(workload, "exp" if sampler == 0 else "poisson")]
    cfg = dict(getattr(W, workload)(seed), sampler=sampler)
    g = run_gpu(cfg, tuning=tuning)
    assert g["n"] == n
    assert g["stats"]["critical_events"] >= best
