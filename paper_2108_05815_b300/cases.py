"""Small named runs of the engine for profilers (ncu) and latency checks.

  python -m paper_2108_05815_b300.cases config2 [--sampler exp|poisson] [--events]
      the 256 x 256 torus workload once, without CUDA graphs, so that every
      advance launch is a separate kernel launch a profiler can select;
      --events also logs the run and reduces it to the event stream
  python -m paper_2108_05815_b300.cases busy [--sampler ...] [--rounds 6]
      a 1024 x 1024 torus (1,048,576 lineages, sigma 2, nu 1e-3) for a few
      rounds: the throughput-bound phase, all lineages active
  python -m paper_2108_05815_b300.cases tail [--sampler ...] [--only nonspatial|torus]
         [--reps 3] [--block-threads T --blocks-per-sm B]
      one lineage, nu 1e-4 (about 10^4 events), on a non-spatial deme of one
      and on a 1 x 1 torus with sigma 2: the latency-bound phase; prints the
      device time per event (fastest of --reps runs).  A small launch shape
      (--block-threads 64 --blocks-per-sm 1) leaves few idle warps beside the
      working one, so that a profiler's per-warp figures are its own

  python -m paper_2108_05815_b300.cases implicit [--sampler ...]
      the spatially implicit workload (local community of 10^5, migration
      0.01, metacommunity of 10^9 with nu 1e-4) once, without CUDA graphs
  python -m paper_2108_05815_b300.cases alias [--reps 3]
      config 3's habitat map (1024 x 1024, 60 % habitable, demes 1..8) and
      its dispersal tables: sim_create builds one alias row of 797 offsets
      per habitable cell (k_alias_build); prints the wall time of each
      sim_create

Every run prints one JSON line with what it did.  The device memory held is
well under 1 GB in all cases.
"""
import argparse
import json
import time

from . import workloads as W

SAMPLERS = {"exp": 0, "poisson": 1}


def _sim(ind, kind, nu, seed, sampler, tuning, **kw):
    return ind.Simulation(kind, nu, seed, sampler=sampler, tuning=tuning, **kw)


def run_config2(ind, sampler, events=False):
    c = W.config2()
    s = _sim(ind, c["kind"], c["nu"], c["seed"], sampler, dict(use_graph=0, profile=1),
             width=c["width"], height=c["height"], deme=c["deme"], sigma=c["sigma"])
    if events:
        s.set_event_log(8 << 20)  # raw events of the workload: about 4.1 M
    s.sample()
    assert s.run()
    _, K = s.species()
    st = s.stats()
    out = dict(case="config2", species=K, **{k: st[k] for k in ("rounds", "raw_events", "advance_launches")})
    if events:
        ev, co = s.events()
        out.update(distinct_events=len(ev), coalescences=len(co))
    s.close()
    return out


def run_implicit(ind, sampler):
    c = W.implicit()
    s = _sim(ind, c["kind"], c["nu"], c["seed"], sampler, dict(use_graph=0), deme=c["deme"],
             migration=c["migration"], meta_size=c["meta_size"], meta_nu=c["meta_nu"])
    s.sample()
    assert s.run()
    _, K = s.species()
    st = s.stats()
    s.close()
    return dict(case="implicit", species=K, **{k: st[k] for k in ("rounds", "raw_events", "critical_events")})


def run_busy(ind, sampler, rounds):
    s = _sim(ind, W.TORUS, 1e-3, 42, sampler, dict(use_graph=0), width=1024, height=1024, deme=1, sigma=2.0)
    s.sample()
    done = s.run(round_budget=rounds)
    st = s.stats()
    s.close()
    return dict(case="busy", finished=bool(done), rounds=st["rounds"], raw_events=st["raw_events"])


def run_tail(ind, sampler, only=None, reps=3, launch=None):
    out = {}
    for name, kw in (("nonspatial_deme1", dict(kind=W.NONSPATIAL, deme=1)),
                     ("torus_1x1_sigma2", dict(kind=W.TORUS, width=1, height=1, deme=1, sigma=2.0))):
        if only and not name.startswith(only):
            continue
        best = None
        for _ in range(reps):
            kind = kw["kind"]
            args = {k: v for k, v in kw.items() if k != "kind"}
            s = _sim(ind, kind, 1e-4, 1, sampler, dict(profile=1, **(launch or {})), **args)
            s.sample()
            t0 = time.perf_counter()
            assert s.run()
            t1 = time.perf_counter()
            st = s.stats()
            s.close()
            per = dict(events=st["raw_events"], rounds=st["rounds"], us_per_event_wall=(t1 - t0) * 1e6 / st["raw_events"],
                       us_per_event_device=st["advance_ms"] * 1e3 / st["raw_events"])
            if best is None or per["us_per_event_device"] < best["us_per_event_device"]:
                best = per
        out[name] = best
    return dict(case="tail", **out)


def run_alias(ind, reps):
    import torch
    c = W.config3()
    dm = ind.habitat(c["map_seed"], c["width"], c["height"], c["p_habitable"], c["max_deme"])
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], sigma=c["sigma"],
                           radius=c["radius"], deme_map=dm)
        torch.cuda.synchronize()
        times.append(round((time.perf_counter() - t0) * 1e3, 2))
        s.close()
    return dict(case="alias", habitable_cells=int((dm > 0).sum()), sim_create_ms=times)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["config2", "busy", "tail", "alias", "implicit"])
    ap.add_argument("--sampler", default="exp", choices=sorted(SAMPLERS))
    ap.add_argument("--rounds", type=int, default=6)
    ap.add_argument("--events", action="store_true")
    ap.add_argument("--only", choices=["nonspatial", "torus"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--block-threads", type=int)
    ap.add_argument("--blocks-per-sm", type=int)
    ap.add_argument("--tail-events", type=float, help="tail: events per lineage per round (fewer, longer launches)")
    a = ap.parse_args(argv)
    import torch  # noqa: F401  (device memory comes from torch's allocator)
    import paper_2108_05815_b300 as ind
    from . import build
    build.build()
    sampler = SAMPLERS[a.sampler]
    if a.case == "config2":
        r = run_config2(ind, sampler, a.events)
    elif a.case == "busy":
        r = run_busy(ind, sampler, a.rounds)
    elif a.case == "alias":
        r = run_alias(ind, a.reps)
    elif a.case == "implicit":
        r = run_implicit(ind, sampler)
    else:
        launch = {}
        if a.block_threads:
            launch["block_threads"] = a.block_threads
        if a.blocks_per_sm:
            launch["blocks_per_sm"] = a.blocks_per_sm
        if a.tail_events:
            launch["tail_events"] = a.tail_events
        r = run_tail(ind, sampler, a.only, a.reps, launch)
    r["sampler"] = a.sampler
    print(json.dumps(r))


if __name__ == "__main__":
    main()
