"""Writes config3_digest.txt: the oracle's full result for config 3 (the
1024 x 1024 habitat map, seed 42, every individual sampled), one line per
event-time sampler: individuals, unique events, species, the longest line of
descent, and the SHA-256 of the speciation keys of every individual
(location words, then time-bit words, little-endian uint64, in sample order).

The result comes from the oracle's event-ordered mode (mode M, equal to the
per-lineage traces of the Independent algorithm by the argument in the
oracle's header), which also counts the unique events and finds the most
events any one individual's lineage runs before it speciates.  A GPU test
runs config 3 at full size and checks its keys against the digest, and the
benchmark sets its step time against the longest line of descent.

Calls only the oracle and the seeded parameter generators.  Run from the
repository root:  python tests/golden/make_config3.py  (one process per
sampler, about 15 minutes each on one core of a 2.7 GHz Xeon).
"""
import hashlib
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config3_digest.txt")


def one(sampler):
    import numpy as np
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = W.config3(42)
    dm = O.habitat(c["map_seed"], c["width"], c["height"], c["p_habitable"], c["max_deme"])
    m = O.Model(c["kind"], c["width"], c["height"], 0, c["nu"], c["seed"], sigma=c["sigma"], radius=c["radius"],
                deme_map=dm, sampler=sampler)
    locs = m.sample()
    kl, kt, U, L = m.run_merge_longest(locs)
    K = len(np.unique(np.stack([kl, kt], axis=1), axis=0))
    digest = hashlib.sha256(kl.astype("<u8").tobytes() + kt.astype("<u8").tobytes()).hexdigest()
    return "config3 %s %d %d %d %d %d %s" % ("exp" if sampler == 0 else "poisson", c["seed"], len(locs), U, K, L,
                                              digest)


def main():
    with mp.get_context("spawn").Pool(2) as pool:
        rows = pool.map(one, [0, 1])
    with open(PATH, "w") as f:
        f.write("# Oracle result of config 3 (mode M), written by make_config3.py.\n"
                "# workload sampler seed individuals unique_events species longest_descent sha256(key_loc|key_time)\n")
        for r in rows:
            f.write(r + "\n")
    print("\n".join(rows))


if __name__ == "__main__":
    main()
