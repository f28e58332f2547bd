"""Writes config4_digest.txt: the oracle's full result for every simulation of
config 4 (256 uneven simulations, master seed 42, every individual sampled),
one line per (event-time sampler, simulation): its landscape kind,
individuals, unique events, species, the longest line of descent, and the
SHA-256 of the speciation keys of every individual (location words, then
time-bit words, little-endian uint64, in sample order).

Each result comes from the oracle's event-ordered mode (mode M), as for
config 3.  A GPU test runs the whole batch and checks every simulation's keys
against its digest; the benchmark sets the batch's time against the longest
line of descent of any of its simulations (the batch cannot end before that
chain of dependent events has run).

Calls only the oracle and the seeded parameter generators.  Run from the
repository root:  python tests/golden/make_config4.py  (a process pool over
the host's cores; about 80 s on 8 cores).
"""
import hashlib
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config4_digest.txt")
KIND_NAME = {0: "nonspatial", 1: "torus"}


def one(task):
    sampler, k = task
    import numpy as np
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = W.config4()[k]
    m = O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], c["seed"], sigma=c.get("sigma"),
                sampler=sampler)
    locs = m.sample()
    kl, kt, U, L = m.run_merge_longest(locs)
    K = len(np.unique(np.stack([kl, kt], axis=1), axis=0))
    digest = hashlib.sha256(kl.astype("<u8").tobytes() + kt.astype("<u8").tobytes()).hexdigest()
    return sampler, k, "config4 %s %d %s %d %d %d %d %s" % (
        "exp" if sampler == 0 else "poisson", k, KIND_NAME[c["kind"]], len(locs), U, K, L, digest)


def main():
    from paper_2108_05815_b300 import workloads as W
    specs = W.config4()
    # the smallest speciation probabilities run the longest: start those first
    order = sorted(range(len(specs)), key=lambda k: specs[k]["nu"])
    tasks = [(s, k) for k in order for s in (0, 1)]
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        rows = pool.map(one, tasks, chunksize=1)
    rows.sort(key=lambda r: (r[0], r[1]))
    with open(PATH, "w") as f:
        f.write("# Oracle result of every simulation of config 4 (mode M), written by make_config4.py.\n"
                "# workload sampler index kind individuals unique_events species longest_descent "
                "sha256(key_loc|key_time)\n")
        for r in rows:
            f.write(r[2] + "\n")
    print("%d rows written to %s" % (len(rows), PATH))


if __name__ == "__main__":
    main()
