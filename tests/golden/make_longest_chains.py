"""Writes longest_chains.txt: for config 1 and config 2 (seed 42, all
individuals sampled), with each event-time sampler, the most events any one
sampled lineage runs before it speciates.

The lineages of the Independent algorithm are traced alone (the paper's
per-individual loop of section "The Independent Algorithm"): lineage i's
trace is a chain of ne_i dependent events, each keyed by the location and
time the previous one produced.  Merging at a horizon only hands the rest of
a chain to another lineage, so no schedule finishes a simulation in fewer
dependent events than max_i ne_i.  A device run's critical-event count (the
sum over rounds of the most events one lineage ran in the round) is never
below it.

Calls only the oracle (mode P traces) and the seeded parameter generators.
Run from the repository root:  python tests/golden/make_longest_chains.py
(about 90 s on one core).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2108_05815_b300 import workloads as W  # noqa: E402


def longest_chain(cfg, sampler):
    m = O.Model(cfg["kind"], cfg["width"], cfg["height"], cfg["deme"], cfg["nu"], cfg["seed"],
                sigma=cfg.get("sigma", 0.0), sampler=sampler)
    locs = m.sample()
    best = 0
    for a in range(0, len(locs), 4096):
        _, _, ne = m.trace(locs[a:a + 4096])
        best = max(best, int(ne.max()))
    return len(locs), best


def main():
    rows = []
    for name, cfg in (("config1", W.config1(42)), ("config2", W.config2(42))):
        for sampler, sname in ((0, "exp"), (1, "poisson")):
            n, best = longest_chain(cfg, sampler)
            rows.append("%s %s %d %d %d" % (name, sname, cfg["seed"], n, best))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "longest_chains.txt")
    with open(path, "w") as f:
        f.write("# Most events one sampled lineage runs before it speciates (mode P traces of the\n"
                "# oracle, all individuals sampled), written by make_longest_chains.py.\n"
                "# workload sampler seed lineages max_events\n")
        for r in rows:
            f.write(r + "\n")
    print("\n".join(rows))


if __name__ == "__main__":
    main()
