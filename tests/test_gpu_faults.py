"""Failure paths without any GPU fault: allocation failures injected on the
host through the allocator hook, invalid calls, and recovery afterwards."""
import ctypes

import numpy as np
import pytest

import paper_2108_05815_b300 as ind

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2108_05815_b300 import build
    build.build()


def _failing_allocator(fail_after):
    import torch
    state = {"n": 0}

    def alloc(nbytes, stream, ctx):
        state["n"] += 1
        if state["n"] > fail_after:
            return None
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))

    def release(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    return ind.Allocator(ind._ALLOC(alloc), ind._RELEASE(release), None)


@pytest.mark.parametrize("fail_after", [0, 1, 3, 6, 12])
def test_allocation_failure_is_reported_and_recoverable(fail_after):
    ind.use_torch_allocator()
    a = _failing_allocator(fail_after)
    assert ind.lib().ind_set_allocator(ctypes.byref(a)) == 0
    got = None
    try:
        s = ind.Simulation(ind.TORUS, 1e-2, 3, width=40, height=30, deme=2, sigma=2.0)
        s.sample()
        s.run()
        got = s.species()[1]
        s.close()
    except ind.IndError as e:
        assert e.status == -2  # IND_ERR_OOM, never a crash
    finally:
        ind._torch_alloc = None
        ind.use_torch_allocator()
    # the library keeps working after the failures
    s = ind.Simulation(ind.TORUS, 1e-2, 3, width=40, height=30, deme=2, sigma=2.0)
    s.sample()
    assert s.run()
    K = s.species()[1]
    s.close()
    if got is not None:
        assert got == K


def test_out_of_order_calls():
    s = ind.Simulation(ind.NONSPATIAL, 1e-2, 3, deme=100)
    with pytest.raises(ind.IndError) as e:
        s.run()
    assert e.value.status == -5  # not sampled
    s.sample()
    with pytest.raises(ind.IndError) as e:
        s.species()
    assert e.value.status == -5  # not finished
    assert s.run()
    s.close()


def test_round_budget_leaves_state_resumable_and_species_waits():
    s = ind.Simulation(ind.NONSPATIAL, 1e-3, 5, deme=2000, tuning=dict(max_step_events=1.0, tail_events=1.0,
                                                                      rounds_per_check=1))
    s.sample()
    assert s.run(round_budget=1) is False
    with pytest.raises(ind.IndError):
        s.species()
    while not s.run(round_budget=50):
        pass
    ids, K = s.species()
    assert K >= 1 and ids.max() == K - 1
    s.close()
