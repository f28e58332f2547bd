"""The oracle-written fixtures under tests/golden and the benchmark's readers
of them (CPU): every row belongs to the workload the seeded generator
defines, and bench.py picks the longest line of descent the binding
roofline divides by."""
import importlib.util
import os

from paper_2108_05815_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)  # main() runs only as a script
    return mod


def _rows(name):
    return [l.split() for l in open(os.path.join(GOLD, name)) if l.strip() and not l.startswith("#")]


def test_config4_digest_rows_match_the_generator():
    specs = W.config4()
    rows = _rows("config4_digest.txt")
    assert len(rows) == 2 * len(specs)
    for sampler in ("exp", "poisson"):
        mine = sorted((r for r in rows if r[1] == sampler), key=lambda r: int(r[2]))
        assert [int(r[2]) for r in mine] == list(range(len(specs)))
        for r, c in zip(mine, specs):
            _, _, _, kind, n, U, K, L, sha = r
            assert kind == ("nonspatial" if c["kind"] == W.NONSPATIAL else "torus")
            assert int(n) == c["width"] * c["height"] * c["deme"]  # every individual sampled
            # at least one event per individual; species between 1 and n;
            # the longest line of descent at most the unique events
            assert int(U) >= int(n) and 1 <= int(K) <= int(n) and 1 <= int(L) <= int(U)
            assert len(sha) == 64 and int(sha, 16) >= 0


def test_bench_reads_the_longest_lines_of_descent():
    b = _bench()
    rows = _rows("config4_digest.txt")
    for sampler in ("exp", "poisson"):
        mine = [r for r in rows if r[1] == sampler]
        top = max(mine, key=lambda r: int(r[7]))
        assert b.config4_longest(sampler) == (int(top[7]), int(top[2]), top[3])
    c3 = {r[1]: r for r in _rows("config3_digest.txt")}
    for sampler in ("exp", "poisson"):
        assert b.longest_descent("config3", sampler) == int(c3[sampler][6])
    chains = {(r[0], r[1]): int(r[4]) for r in _rows("longest_chains.txt")}
    assert b.longest_descent("config2", "exp") == chains[("config2", "exp")]
    assert b.longest_descent("config5", "exp") is None


def test_chain_floor_fraction_prefers_the_longest_line_of_descent():
    b = _bench()
    hw = {"frac_of_longest_floor": 0.46, "step_over_critical_floor": 2.0}
    assert b.chain_floor_frac({"hw_floor": hw}) == 0.46
    assert b.chain_floor_frac({"hw_floor": {"step_over_critical_floor": 2.0}}) == 0.5
    assert b.chain_floor_frac({}) is None
