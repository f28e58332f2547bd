"""Isolated partitions (the paper's IsolatedIndividuals and IsolatedLandscape
strategies) on one GPU: each part of a simulation's sample runs alone, and
the merge of the parts' distinct speciation keys gives every individual the
identity it has in the one-piece run and in the oracle.  Bit-exact."""
import numpy as np
import pytest

import oracle as O
import paper_2108_05815_b300 as ind
from paper_2108_05815_b300 import partition as PT
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


def _sim(c, dm=None):
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c.get("deme", 1),
                          sigma=c.get("sigma", 0.0), radius=c.get("radius", 0), deme_map=dm,
                          sampler=c.get("sampler", 0))


def _part_indices(locs, height, part, n_parts, scheme):
    """the documented partition rule on the whole sample's order"""
    j = np.arange(len(locs))
    if scheme == ind.PARTITION_INDIVIDUALS:
        return j[j % n_parts == part]
    y = (locs.astype(np.uint64) >> np.uint64(20)) & np.uint64(0xFFFFF)
    return j[(y.astype(np.int64) * n_parts) // height == part]


CASES = [
    dict(kind=W.TORUS, width=96, height=80, deme=2, sigma=2.0, nu=2e-3, seed=5),
    dict(kind=W.TORUS, width=64, height=64, deme=1, sigma=3.0, nu=1e-3, seed=6, sampler=1),
    dict(kind=W.MAP, width=60, height=50, sigma=3.0, radius=9, nu=4e-3, seed=7),
    dict(kind=W.NONSPATIAL, width=1, height=1, deme=5000, nu=1e-3, seed=8),
]


@pytest.mark.parametrize("n_parts", [2, 3])
@pytest.mark.parametrize("scheme", [ind.PARTITION_LANDSCAPE, ind.PARTITION_INDIVIDUALS])
@pytest.mark.parametrize("idx", range(len(CASES)))
def test_partitions_merge_to_the_one_piece_run(idx, scheme, n_parts):
    c = CASES[idx]
    dm = O.habitat(3, c["width"], c["height"]) if c["kind"] == W.MAP else None
    m = O.Model(c["kind"], c["width"], c["height"], c.get("deme", 1), c["nu"], c["seed"], sigma=c.get("sigma"),
                radius=c.get("radius"), deme_map=dm, sampler=c.get("sampler", 0))
    locs = m.sample()
    okl, okt, _ = m.run_merge(locs)
    oids, oK = O.species_ids(okl, okt)
    whole = _sim(c, dm)
    whole.sample()
    assert whole.run()
    wids, wK = whole.species()
    whole.close()
    assert wK == oK and np.array_equal(wids, oids)

    keys, idxs, raw = [], [], 0
    for p in range(n_parts):
        s = _sim(c, dm)
        kl, kt = PT.run_part(s, p, n_parts, scheme)
        raw += s.stats()["raw_events"]
        s.close()
        want = _part_indices(locs, c["height"], p, n_parts, scheme)
        assert kl.numel() == len(want)
        # an individual's key is the same in its part as in the whole run
        assert np.array_equal(kl.cpu().numpy(), okl[want]) and np.array_equal(kt.cpu().numpy(), okt[want])
        keys.append((kl, kt))
        idxs.append(want)
    ids = np.zeros(len(locs), dtype=np.uint64)
    for (kl, kt), want in zip(keys, idxs):
        g, K = PT.merge_species(kl, kt, part_keys=keys)
        assert K == oK
        ids[want] = g.cpu().numpy()
    assert np.array_equal(ids, oids)


def test_keys_unique_and_rank():
    import torch
    rng = np.random.default_rng(4)
    kl = rng.integers(0, 50, size=30000, dtype=np.uint64) << np.uint64(40)
    kt = rng.integers(0, 7, size=30000, dtype=np.uint64)
    kl[:3] = np.uint64(0xFFFFFFFFFFFFFFFF)
    kt[:3] = np.uint64(0xFFFFFFFFFFFFFFFF)  # the all-ones key sorts last, like the padding
    dl = torch.from_numpy(kl.view(np.int64)).cuda().view(torch.uint64)
    dt = torch.from_numpy(kt.view(np.int64)).cuda().view(torch.uint64)
    ul, ut = ind.keys_unique(dl, dt)
    want = np.unique(np.stack([kl, kt], axis=1), axis=0)
    assert np.array_equal(ul.cpu().numpy(), want[:, 0]) and np.array_equal(ut.cpu().numpy(), want[:, 1])
    r = ind.keys_rank(dl, dt, ul, ut).cpu().numpy()
    _, inv = np.unique(np.stack([kl, kt], axis=1), axis=0, return_inverse=True)
    assert np.array_equal(r, inv.reshape(-1).astype(np.uint64))
    # a key outside the reference is an argument error
    with pytest.raises(ind.IndError):
        ind.keys_rank(dl, dt, ul[1:], ut[1:])
    # one key, and keys that are all equal
    e0, e1 = ind.keys_unique(dl[:1], dt[:1])
    assert e0.numel() == 1
    z = torch.zeros(5000, dtype=torch.uint64, device="cuda")
    z0, z1 = ind.keys_unique(z, z)
    assert z0.numel() == 1 and int(ind.keys_rank(z, z, z0, z1).cpu().numpy().max()) == 0


def test_partition_arguments():
    s = ind.Simulation(ind.TORUS, 1e-2, 1, width=8, height=8, deme=1, sigma=1.0)
    try:
        for part, n_parts, scheme in ((2, 2, 0), (0, 0, 0), (0, 2, 5)):
            with pytest.raises(ind.IndError):
                s.sample_partition(part, n_parts, scheme)
        assert s.sample_partition(0, 1, 0) == 64
        # more bands than rows: some parts are empty, and they still run
        sizes = [s.sample_partition(p, 16, ind.PARTITION_LANDSCAPE) for p in range(16)]
        assert sum(sizes) == 64 and 0 in sizes
        s.sample_partition(1, 16, ind.PARTITION_LANDSCAPE)
        assert s.run()
    finally:
        s.close()
