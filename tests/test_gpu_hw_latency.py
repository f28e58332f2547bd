"""The hardware latency microbenchmark behind the event-chain floor.

Checks that every measured dependent latency is a plausible number of SM
cycles, that the compound steps order as their parts do, and that the floor
of one event lies below what the library's warp kernel takes per event on a
lone lineage (a floor above a measured time would mean a wrong chain).
"""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import hw_latency as H  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    return H.measure(reps=2, dram_ring_mib=256, dram_steps=2000)


def test_latencies_plausible(lat):
    for name in H.CLASSES:
        assert 1.0 <= lat[name] <= 400.0, (name, lat[name])
    assert lat["philox_round"] >= lat["imad_hi"]
    assert lat["hi_xor"] >= lat["imad_hi"]
    assert lat["lds"] < lat["ldg_dram"] and lat["ldg_l1"] < lat["ldg_dram"]
    assert 200.0 < lat["ldg_dram"] < 5000.0
    assert 0.5 * lat["ldg_dram"] < lat["bulk_row"] < 20000.0
    assert 300.0 < lat["clock_mhz"] < 2200.0


def test_floor_below_lone_lineage_event(lat):
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build
    build.build()
    s = ind.Simulation(ind.TORUS, 1e-4, 1, width=1, height=1, deme=1, sigma=2.0, tuning=dict(profile=1))
    s.sample()
    assert s.run()
    st = s.stats()
    s.close()
    cycles_per_event = st["advance_ms"] * 1e-3 * lat["clock_mhz"] * 1e6 / st["raw_events"]
    for sampler in ("exp", "poisson"):
        f = H.event_floor(lat, sampler, "torus")
        assert 100.0 < f < cycles_per_event, (sampler, f, cycles_per_event)


def test_integer_throughput_plausible(lat):
    """the measured integer peak of the Philox mix is of the order of every
    lane issuing one integer instruction per cycle at the measured clock"""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    lanes_peak = sms * 128 * lat["clock_mhz"] * 1e6 / 1e12
    # (a block counts 100 ops for about 45 instructions: a wide product is a
    # high and a low product, a three-input xor two xors)
    assert 0.05 * lanes_peak < lat["philox_tput_tops"] < 3.0 * lanes_peak, (lat["philox_tput_tops"], lanes_peak)
