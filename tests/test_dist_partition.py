"""The exchange of isolated partitions across ranks, on CPU: two gloo ranks
each hold one part of a simulation's sample (the paper's isolated
partitioning), traced by the oracle alone on the rank (as a GPU would run
its part), and gather their distinct speciation keys with the library's
exchange helper.  The identities each rank derives from the gathered keys
equal the one-rank run of the oracle, for both partition schemes.  The
ranking itself runs on the GPU in the product (ind_keys_rank, tested in
test_gpu_partition.py); here the test ranks the gathered keys with numpy."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

CFG = dict(width=40, height=30, deme=2, sigma=2.0, nu=5e-3, seed=17)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _part(locs, height, part, n_parts, scheme):
    j = np.arange(len(locs))
    if scheme == 1:
        return j[j % n_parts == part]
    y = (locs.astype(np.uint64) >> np.uint64(20)) & np.uint64(0xFFFFF)
    return j[(y.astype(np.int64) * n_parts) // height == part]


def _rank(rank, world, port, scheme, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist
    import oracle as O
    from paper_2108_05815_b300 import partition as PT
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = O.Model(O.TORUS, CFG["width"], CFG["height"], CFG["deme"], CFG["nu"], CFG["seed"], sigma=CFG["sigma"])
    locs = m.sample()
    mine = _part(locs, CFG["height"], rank, world, scheme)
    kl, kt, _ = m.trace(locs[mine])
    u = np.unique(np.stack([kl, kt], axis=1), axis=0)
    ul = torch.from_numpy(u[:, 0].copy().view(np.int64)).view(torch.uint64)
    ut = torch.from_numpy(u[:, 1].copy().view(np.int64)).view(torch.uint64)
    al, at = PT.gather_keys(dist, ul, ut)
    g = np.unique(np.stack([al.view(torch.int64).numpy().view(np.uint64),
                            at.view(torch.int64).numpy().view(np.uint64)], axis=1), axis=0)
    # each individual's rank among the gathered distinct keys
    order = np.lexsort((g[:, 1], g[:, 0]))
    assert np.array_equal(order, np.arange(len(g)))
    pos = {tuple(k): r for r, k in enumerate(g.tolist())}
    ids = np.array([pos[(a, b)] for a, b in zip(kl.tolist(), kt.tolist())], dtype=np.uint64)
    out[rank] = (mine.tolist(), ids.tolist(), len(g), int(al.numel()))
    dist.destroy_process_group()


@pytest.mark.parametrize("scheme", [0, 1])
def test_two_gloo_ranks_merge_partitions(scheme):
    import oracle as O
    m = O.Model(O.TORUS, CFG["width"], CFG["height"], CFG["deme"], CFG["nu"], CFG["seed"], sigma=CFG["sigma"])
    locs = m.sample()
    okl, okt, _ = m.run_merge(locs)
    oids, oK = O.species_ids(okl, okt)
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        ctx = mp.get_context("spawn")
        ps = [ctx.Process(target=_rank, args=(r, 2, port, scheme, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(300)
            assert p.exitcode == 0
        ids = np.full(len(locs), np.iinfo(np.uint64).max, dtype=np.uint64)
        for r in range(2):
            mine, rids, K, gathered = out[r]
            assert K == oK
            ids[np.array(mine, dtype=np.int64)] = np.array(rids, dtype=np.uint64)
        # both ranks gathered the same union, and every individual got its id
        assert out[0][3] == out[1][3]
        assert np.array_equal(ids, oids)
