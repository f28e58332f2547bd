"""The allocation-free species ranking (ind_species_rank_static) gives the same
species identities and counts as sim_species.

It serves callers that must not allocate device memory while they run (for
example a process that plans all of its device memory at start-up), so its
scratch is a fixed device array inside the library.  Two calls in a row on
different inputs check that a call does not see the previous call's leftovers.
This file is collected last on purpose.
"""
import ctypes
import gc

import numpy as np
import pytest

import paper_2108_05815_b300 as ind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_05815_b300 import build
    build.build()
    return torch


def _reference(kind, nu, seed, **kw):
    s = ind.Simulation(kind, nu, seed, **kw)
    s.sample()
    assert s.run()
    ids, K = s.species()
    kl, kt = s.species_keys()
    s.close()
    return ids, K, kl, kt


def test_static_rank_matches_sim_species_twice(torch_cuda):
    torch = torch_cuda
    cases = [
        dict(kind=ind.TORUS, nu=1e-3, seed=3, width=96, height=80, deme=2, sigma=2.0),   # 15,360 individuals
        dict(kind=ind.NONSPATIAL, nu=1e-3, seed=42, deme=10000),                        # config 1
    ]
    for c in cases:
        ids_ref, K_ref, kl, kt = _reference(**c)
        dl = torch.from_numpy(kl.view(np.int64)).cuda()
        dt = torch.from_numpy(kt.view(np.int64)).cuda()
        out = torch.full((kl.size,), -1, dtype=torch.int64, device="cuda")
        K = ind.species_rank_static(dl, dt, out)
        torch.cuda.synchronize()
        assert K == K_ref
        assert np.array_equal(out.cpu().numpy().view(np.uint64), ids_ref)


def test_static_rank_rejects_too_many_and_handles_empty(torch_cuda):
    torch = torch_cuda
    big = torch.zeros(65537, dtype=torch.int64, device="cuda")
    with pytest.raises(ind.IndError) as e:
        ind.species_rank_static(big, big, big)
    assert e.value.status == -1
    empty = torch.zeros(0, dtype=torch.int64, device="cuda")
    assert ind.species_rank_static(empty, empty, empty) == 0


def test_static_rank_allocates_nothing(torch_cuda):
    """its defining property: with an allocator hook that counts every call
    and refuses every request installed, the call still succeeds, the hook is
    never called, and torch's allocated device memory is unchanged"""
    torch = torch_cuda
    ids_ref, K_ref, kl, kt = _reference(kind=ind.TORUS, nu=2e-3, seed=5, width=64, height=48, deme=1, sigma=2.0)
    dl = torch.from_numpy(kl.view(np.int64)).cuda()
    dt = torch.from_numpy(kt.view(np.int64)).cuda()
    out = torch.full((kl.size,), -1, dtype=torch.int64, device="cuda")
    calls = {"n": 0}

    def alloc(nbytes, stream, ctx):
        calls["n"] += 1
        return None

    def release(ptr, nbytes, stream, ctx):
        calls["n"] += 1

    refusing = ind.Allocator(ind._ALLOC(alloc), ind._RELEASE(release), None)
    # tensors of earlier tests that only the cyclic collector frees must not
    # be freed inside the measured window: collect first, then hold it off
    gc.collect()
    gc.disable()
    try:
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        assert ind.lib().ind_set_allocator(ctypes.byref(refusing)) == 0
        try:
            K = ind.species_rank_static(dl, dt, out)
            torch.cuda.synchronize()
        finally:
            assert ind.lib().ind_set_allocator(ctypes.byref(ind._torch_alloc)) == 0
        after = torch.cuda.memory_allocated()
    finally:
        gc.enable()
    assert calls["n"] == 0
    assert after == before
    assert K == K_ref and np.array_equal(out.cpu().numpy().view(np.uint64), ids_ref)
