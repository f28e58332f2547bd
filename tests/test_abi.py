"""The C-ABI library loads, exports every symbol include/indep.h declares,
and rejects invalid arguments before touching the GPU.  No GPU needed."""
import ctypes
import os
import re

import pytest

import paper_2108_05815_b300 as ind
from paper_2108_05815_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "indep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:[A-Za-z_][A-Za-z0-9_ \*]*?[\s\*])([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ind.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sim_create", "sim_sample", "sim_run", "sim_species", "sim_species_keys", "sim_destroy",
              "sim_batch_run", "sim_mem_estimate", "ind_habitat", "ind_set_allocator"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(ind.EXPORTS)


def test_status_strings(lib):
    for code, name in ind.STATUS.items():
        assert lib.ind_status_string(code).decode() == name


def test_default_tuning(lib):
    t = ind.default_tuning()
    assert t["block_threads"] % 32 == 0 and t["dedup"] == 1 and t["count_unique"] == 0
    # the server's defaults: the same, with the busy requests' water level raised
    sv = ind.server_default_tuning()
    assert sv["occupancy_step"] == 1.0 and sv["min_events_per_lineage"] == 1.0
    assert sv["events_per_round"] == float(1 << 24)
    assert {k: v for k, v in sv.items() if k not in ("occupancy_step", "min_events_per_lineage",
                                                      "events_per_round")} == \
        {k: v for k, v in t.items() if k not in ("occupancy_step", "min_events_per_lineage", "events_per_round")}


def _create(lib, L, D, nu):
    h = ctypes.c_void_p()
    return lib.sim_create(ctypes.byref(L), ctypes.byref(D), nu, 1, None, ctypes.byref(h))


@pytest.mark.parametrize("case", [
    dict(kind=ind.NONSPATIAL, width=1, height=1, deme=0, dk=0, nu=0.1),          # empty deme
    dict(kind=ind.NONSPATIAL, width=1, height=1, deme=10, dk=0, nu=0.0),         # nu = 0
    dict(kind=ind.NONSPATIAL, width=1, height=1, deme=10, dk=0, nu=1.5),         # nu > 1
    dict(kind=ind.NONSPATIAL, width=2, height=1, deme=10, dk=0, nu=0.1),         # non-spatial needs 1 x 1
    dict(kind=ind.NONSPATIAL, width=1, height=1, deme=1 << 23, dk=0, nu=0.1),    # deme too large
    dict(kind=ind.TORUS, width=8, height=8, deme=1, dk=1, sigma=0.0, nu=0.1),    # sigma = 0
    dict(kind=ind.TORUS, width=8, height=8, deme=1, dk=0, sigma=1.0, nu=0.1),    # wrong dispersal kind
    dict(kind=ind.TORUS, width=1 << 21, height=8, deme=1, dk=1, sigma=1.0, nu=0.1),
    dict(kind=ind.TORUS, width=8, height=8, deme=1, dk=1, sigma=1.0, nu=0.1, delta_t=3.0),  # not 2^k
    dict(kind=ind.TORUS, width=8, height=8, deme=1, dk=1, sigma=1.0, nu=0.1, lam=0.0),
    dict(kind=ind.MAP, width=8, height=8, deme=0, dk=2, sigma=1.0, radius=4, nu=0.1),      # no map
    dict(kind=7, width=8, height=8, deme=1, dk=1, sigma=1.0, nu=0.1),
])
def test_invalid_arguments_are_rejected(lib, case):
    L, _ = ind.landscape(case["kind"], case["width"], case["height"], case["deme"], None,
                         case.get("lam", 1.0), case.get("delta_t", 1.0))
    D = ind.dispersal(case["dk"], case.get("sigma", 0.0), case.get("radius", 0))
    assert _create(lib, L, D, case["nu"]) == -1


@pytest.mark.parametrize("case", [
    dict(nu=0.0, migration=0.0, meta_size=10, meta_nu=0.5),              # no lineage could ever end
    dict(nu=1e-3, migration=0.1, meta_size=0, meta_nu=0.5),              # empty metacommunity
    dict(nu=1e-3, migration=0.1, meta_size=(1 << 31) + 1, meta_nu=0.5),  # metacommunity too large
    dict(nu=1e-3, migration=1.5, meta_size=10, meta_nu=0.5),             # migration > 1
    dict(nu=1e-3, migration=-0.1, meta_size=10, meta_nu=0.5),
    dict(nu=1e-3, migration=0.1, meta_size=10, meta_nu=0.0),             # meta_nu = 0
    dict(nu=-1e-3, migration=0.1, meta_size=10, meta_nu=0.5),
    dict(nu=1e-3, migration=0.1, meta_size=10, meta_nu=0.5, width=2),    # the local community is 1 x 1
    dict(nu=1e-3, migration=0.1, meta_size=10, meta_nu=0.5, dk=1),       # dispersal must be uniform
])
def test_implicit_invalid_arguments_are_rejected(lib, case):
    L, _ = ind.landscape(ind.IMPLICIT, case.get("width", 1), 1, 100, None, 1.0, 1.0, 0, case["migration"],
                         case["meta_size"], case["meta_nu"])
    D = ind.dispersal(case.get("dk", 0), 1.0)
    assert _create(lib, L, D, case["nu"]) == -1


def test_null_arguments(lib):
    assert lib.sim_create(None, None, 0.5, 1, None, None) == -1
    assert lib.sim_sample(None, 1.0, 0, None) == -1
    assert lib.sim_run(None, 0, None) == -1
    assert lib.sim_species(None, None, None) == -1
    assert lib.sim_batch_run(None, 0, None, None) == -1
    assert lib.sim_sample_partition(None, 1.0, 0, 0, 2, 0, None) == -1
    lib.sim_destroy(None)


def test_partition_merge_arguments(lib):
    """the merge entry points reject bad sizes and null outputs before any
    device work, and accept empty inputs without touching the GPU"""
    n = ctypes.c_uint64(7)
    assert lib.ind_keys_unique(None, None, 0, None, None, None, None) == -1      # no count output
    assert lib.ind_keys_unique(None, None, 0, None, None, ctypes.byref(n), None) == 0 and n.value == 0
    assert lib.ind_keys_unique(None, None, 5, None, None, ctypes.byref(n), None) == -1
    assert lib.ind_keys_unique(ctypes.c_void_p(8), ctypes.c_void_p(8), (1 << 31) + 1, ctypes.c_void_p(8),
                               ctypes.c_void_p(8), ctypes.byref(n), None) == -1
    assert lib.ind_keys_rank(None, None, 0, None, None, 0, None, None) == 0
    assert lib.ind_keys_rank(None, None, 3, None, None, 0, None, None) == -1


def test_mem_estimate_is_host_only_and_monotone(lib):
    a = ind.mem_estimate(ind.TORUS, 256, 256, 1, sigma=2.0)
    b = ind.mem_estimate(ind.TORUS, 512, 512, 1, sigma=2.0)
    c = ind.mem_estimate(ind.TORUS, 512, 512, 1, sigma=2.0, fraction=0.1)
    assert 0 < a < b and c < b
    assert ind.mem_estimate(ind.TORUS, 8, 8, 1, sigma=0.0) == 0


def test_build_targets_sm_103a():
    cmd = B.command()
    assert "arch=compute_103a,code=sm_103a" in cmd
    assert "-fmad=false" in cmd
