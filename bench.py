#!/usr/bin/env python
"""Benchmark: lineage events per second of the Independent algorithm on B300.

Workload (default): a 256 x 256 torus with one individual per cell (65,536
sampled lineages), discretised-normal dispersal sigma = 2, nu = 1e-4,
seed 42.  One step = sim_sample (all lineages back to the present) +
sim_run (every lineage to its speciation event) + sim_species (dense species
identities), i.e. every step of the hot path.  The unique-event count U of
the workload comes from an untimed pass of the same simulation with exact
event counting (the trajectories are bit-identical with and without it);
value = U / (device time per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own replica on its own GPU (the
simulation is not sharded); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "lineage events/sec and species-count latency p50/p99; batched vs plain, bit-exact"
UNIT = "events/s"
WORKLOAD = ("config2: torus 256x256, 1 individual per cell (65536 sampled lineages), Gaussian dispersal "
            "sigma=2 (discretised per axis), nu=1e-4, lambda=1, delta_t=1, seed=42")
# Algorithmic 32-bit integer operations of one event of the spec (the integer
# work the spec itself defines, not the instructions a compiler emits):
PHILOX_OPS = 100          # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key adds)
EXP_DRAW_OPS = 110        # fixed-point -ln U of one draw, incl. conversion to binary64
EVENT_FIXED_OPS = 40      # speciation compare, dispersal index arithmetic, wrap, bookkeeping
INT32_LANES_PER_SM = 128  # Blackwell: 128 INT32-capable lanes per SM per clock
# DRAM bytes (read + write) of the advance launches of one round of the
# default workload, measured with ncu on this kernel build:
#   ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum \
#       --clock-control none -k regex:k_advance -c 400 --csv \
#       python -m paper_2108_05815_b300.cases config2 [--sampler poisson]
# (17.05 MB over the 29 rounds with exponential sums, 15.11 MB over 29 with
# Poisson points, default tuning).
TRAFFIC_PER_ROUND = {"exp": 588e3, "poisson": 521e3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="simulations in the batched-vs-plain comparison")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
    ap.add_argument("--workload", default="config2", choices=["config2", "batch", "served", "implicit"])
    ap.add_argument("--sampler", default="exp", choices=["exp", "poisson"],
                    help="event-time sampler of the headline (the other is reported beside it)")
    ap.add_argument("--window", type=float, default=60.0, help="served: arrival window in seconds")
    ap.add_argument("--plain-subset", type=int, default=32, help="batch: simulations timed one by one")
    ap.add_argument("--served-plain", type=int, default=16,
                    help="served: requests re-run one by one on the plain path (0: none)")
    ap.add_argument("--events", action="store_true",
                    help="single workloads: every step also produces the full event stream (distinct events and "
                         "coalescences) on the device")
    return ap.parse_args()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce_max(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# our implementation
# --------------------------------------------------------------------------
SAMPLER = {"exp": 0, "poisson": 1}
_sampler = 0


IMPLICIT_WORKLOAD = ("implicit: spatially implicit local community of 100000 individuals (all sampled), "
                     "migration 0.01 per event, static metacommunity of 1e9 individuals with nu_meta=1e-4, "
                     "local nu=0, lambda=1, delta_t=1, seed=42")
# the single-simulation workload of this run: (parameters of seed, description,
# sampled individuals, host-to-device bytes of the tables and parameters)
_single = {}


def single_workload(name):
    from paper_2108_05815_b300 import workloads as W
    if name == "implicit":
        return dict(params=W.implicit, desc=IMPLICIT_WORKLOAD, n=100000, h2d=400, dataset="implicit")
    # discretised-normal table (2 x 20 x 8 B) + simulation parameters
    return dict(params=W.config2, desc=WORKLOAD, n=65536, h2d=8 * 2 * 20 + 400, dataset="config2")


def make_sim(ind, seed=42, tuning=None, sampler=None):
    c = _single["params"](seed)
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c["deme"],
                          sigma=c.get("sigma", 0.0), migration=c.get("migration", 0.0),
                          meta_size=c.get("meta_size", 0), meta_nu=c.get("meta_nu", 0.0), tuning=tuning,
                          sampler=_sampler if sampler is None else sampler)


def unique_events(ind, seed, sampler=None):
    s = make_sim(ind, seed, tuning=dict(count_unique=1), sampler=sampler)
    s.sample()
    assert s.run()
    st = s.stats()
    s.close()
    return st["unique_events"], st["raw_events"]


def run_ours(args, rank, world, local, pg):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    U, R = unique_events(ind, 42)

    sim = make_sim(ind, 42, tuning=dict(profile=1))
    # event log capacity: the raw events of the workload (the same on every
    # run) and one entry per lineage the dedup removes
    log_cap = int(R) + _single["n"] + 4096 if args.events else 0
    if log_cap:
        sim.set_event_log(log_cap)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    n_ind = _single["n"]
    ids = torch.empty(n_ind, dtype=torch.int64, device=dev)

    def step():
        sim.sample()
        ok = sim.run()
        _, k = sim.species(out=ids)
        return ok, k

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    base_stats = sim.stats()
    launches0 = ind.kernel_launches()
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize()
    step_ms, lat_ms, adv_ms, adv_n, raw = [], [], 0.0, 0, 0
    best = None
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        e0.record(stream)
        ok, K = step()
        e1.record(stream)
        e1.synchronize()
        h1 = time.perf_counter()
        assert ok
        step_ms.append(e0.elapsed_time(e1))
        lat_ms.append((h1 - h0) * 1e3)
        st = sim.stats()
        adv_ms += st["advance_ms"]
        adv_n += st["advance_launches"]
        raw += st["raw_events"]
        if st["busiest_launch_ms"] and (best is None or st["busiest_launch_events"] / st["busiest_launch_ms"] >
                                        best["busiest_launch_events"] / best["busiest_launch_ms"]):
            best = st
    torch.cuda.synchronize()
    barrier(pg)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = ind.kernel_launches() - launches0
    ms_step = sum(step_ms) / len(step_ms)
    ms_step_max = allreduce_max(pg, ms_step)
    value = U * world / (ms_step_max * 1e-3)

    # end to end through the public API with host buffers
    host_ids = torch.empty(n_ind, dtype=torch.int64, pin_memory=True)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        s2 = make_sim(ind, 42)
        if log_cap:
            s2.set_event_log(log_cap)
        s2.sample()
        s2.run()
        s2.species(out=host_ids)
        if log_cap:
            ev_host, co_host = s2.events()
        h1 = time.perf_counter()
        s2.close()
        e2e_ms.append((h1 - h0) * 1e3)
    e2e_ms_max = allreduce_max(pg, statistics.median(e2e_ms))
    h2d = _single["h2d"]
    d2h = n_ind * 8 + 64    # species identities + completion flags
    stream_line = None
    if log_cap:
        d2h += ev_host.nbytes + co_host.nbytes  # the event stream
        stream_line = {"distinct_events": int(len(ev_host)), "coalescences": int(len(co_host)),
                       "log_capacity": log_cap, "bytes_to_host": int(ev_host.nbytes + co_host.nbytes),
                       "what": "every step also sorts its raw event log on the device into the distinct events "
                               "(with prior times and outcomes) and the coalescences"}
        assert len(ev_host) == U

    # batched vs plain on `batch` independent replicas of the workload
    seeds = [42 + k for k in range(args.batch)]
    Us = [unique_events(ind, s)[0] for s in seeds]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in seeds:
        x = make_sim(ind, s)
        x.sample()
        x.run()
        x.species(out=ids)
        x.close()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    sims = [make_sim(ind, s) for s in seeds]
    for x in sims:
        x.sample()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ind.batch_run(sims)
    for x in sims:
        x.species(out=ids)
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t0
    for x in sims:
        x.close()

    # the other event-time sampler on the same workload (same protocol, fewer steps)
    other = 1 - _sampler
    U_o, _ = unique_events(ind, 42, sampler=other)
    so = make_sim(ind, 42, sampler=other)
    o_ms = []
    for k in range(args.warmup + max(3, args.steps // 2)):
        flush.fill_(1)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        so.sample()
        so.run()
        so.species(out=ids)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            o_ms.append(e0.elapsed_time(e1))
    so.close()
    other_line = {"sampler": [n for n, v in SAMPLER.items() if v == other][0], "unique_events_per_step": U_o,
                  "ms_per_step": sum(o_ms) / len(o_ms), "value": U_o / (sum(o_ms) / len(o_ms) * 1e-3)}

    # The dependent chain: a round lasts as long as its busiest lineage, so a
    # step takes at least (critical events) x (the time of one event of a
    # lineage that runs alone).  Eight lineages sampled on the same landscape
    # give that time (device time of their advance launches / their critical
    # events).
    crit = st["critical_events"]
    lone = make_sim(ind, 42, tuning=dict(profile=1))
    lone.sample(8.0 / n_ind, 1)
    assert lone.run()
    ls = lone.stats()
    lone.close()
    lone_ns = ls["advance_ms"] * 1e6 / max(ls["critical_events"], 1)
    crit_ns = ms_step * 1e6 / max(crit, 1)
    latency = {"critical_events_per_step": crit, "ns_per_critical_event": crit_ns,
               "lone_lineage_ns_per_event": lone_ns, "lone_lineages": ls["n_sampled"],
               "frac": lone_ns / crit_ns,
               "what": "step time / (sum over rounds of the most events one lineage ran in the round), against "
                       "the advance-kernel time per event of a few lineages alone on the same landscape"}
    longest = longest_chain(args.workload, args.sampler)
    if longest:
        # no schedule runs the workload in fewer dependent events than its
        # longest lineage: that many lone-lineage events is the step's floor
        latency.update({"longest_lineage_events": longest, "chain_floor_ms": longest * lone_ns * 1e-6,
                        "frac_of_chain_floor": longest * lone_ns * 1e-6 / ms_step})

    # roofline of the advance kernel (events per launch / its CUDA-event time)
    raw_per_step = raw / args.steps
    events_per_launch = raw / max(adv_n, 1)
    ops_per_event = ops_per_raw_event()
    avg_launch_ms = adv_ms / max(adv_n, 1)
    achieved = events_per_launch * ops_per_event / (avg_launch_ms * 1e-3) / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * INT32_LANES_PER_SM * 2032e6 / 1e12
    cpu = None
    if rank == 0:
        cpu = cpu_baseline_traces(args.cpu_seconds) if _single["dataset"] == "implicit" else cpu_baseline(args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": _single["desc"] + (" + full event stream" if log_cap else ""),
                   "event_sampler": args.sampler,
                   "parallelism": "replicas (one independent simulation per GPU)",
                   "l2": "flushed by a 256 MiB write between timed steps",
                   "unique_events_per_step": U, "raw_events_per_step": raw_per_step,
                   "species": K, "tuning": ind.default_tuning()},
        "latency_ms": {"p50": pct(lat_ms, 50), "p99": pct(lat_ms, 99), "what": "step start to species count on host"},
        "raw_events_per_s": raw_per_step * world / (ms_step_max * 1e-3),
        "roofline": {"bound": "alu", "kernel": "k_advance_coop + k_advance (one round: both launched, one works)",
                     "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (32-bit integer)", "frac": achieved / peak,
                     "traffic": TRAFFIC_PER_ROUND.get(args.sampler) if _single["dataset"] == "config2" else None,
                     "ops_per_event": ops_per_event, "events_per_launch": events_per_launch,
                     "avg_launch_ms": avg_launch_ms, "launches_timed": adv_n,
                     "dominant": ("k_advance_coop, %s of the step (ncu launch list): latency-bound, see latency_bound"
                                  % {"exp": "95 %", "poisson": "93 %"}[args.sampler]
                                  if _single["dataset"] == "config2" else None),
                     "busiest_launch": busiest(best or {}, ops_per_event, peak),
                     "peak_source": "148 SMs x 128 INT32 lanes x 2032 MHz max SM clock (derived)"},
        "latency_bound": latency,
        "event_stream": stream_line,
        "cpu_baseline": cpu,
        "e2e": {"value": U * world / (e2e_ms_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max,
                "what": "sim_create + sim_sample + sim_run + sim_species into pinned host memory"},
        "batched": {"sims": args.batch, "workload": "%s replicas, seeds 42..%d" % (_single["dataset"], 41 + args.batch),
                    "unique_events": sum(Us), "batched_events_per_s": sum(Us) / batch_s,
                    "plain_events_per_s": sum(Us) / plain_s, "speedup": plain_s / batch_s},
        "other_sampler": other_line,
        "gpu_launches": launches, "clocks": clk, "wall_s_timed": t_wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    f = int(k)
    c = min(f + 1, len(xs) - 1)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


POINT_OPS = 15            # Poisson sampler: one uniform point (conversion, rounded add, compare)
COUNT_OPS = 20            # Poisson sampler: guided inversion of the point count


def ops_per_raw_event(sampler=None):
    """integer operations per executed event (spec-derived): the event's own
    Philox blocks (two for Gaussian dispersal) and bookkeeping, plus the
    next-event search at lambda dt = 1: sums of exponentials draw on average
    2.7 exponentials from 1.35 blocks; the Poisson sampler visits 1.6
    intervals of one block, one count and on average one point each"""
    sampler = _sampler if sampler is None else sampler
    event = 2 * PHILOX_OPS + EVENT_FIXED_OPS
    if sampler == 1:
        return event + 1.6 * (PHILOX_OPS + COUNT_OPS + 1.0 * POINT_OPS)
    return event + 1.35 * PHILOX_OPS + 2.7 * EXP_DRAW_OPS


def longest_chain(workload, sampler):
    """the most events one sampled lineage of the workload (seed 42, all
    sampled) runs before it speciates: the oracle's mode P traces, stored
    in the test fixtures by the script that wrote them; None if not stored"""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", "longest_chains.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) == 5 and f[0] == workload and f[1] == sampler and f[2] == "42":
            return int(f[4])
    return None


def busiest(st, ops, peak):
    ms, ev = st.get("busiest_launch_ms", 0.0), st.get("busiest_launch_events", 0)
    if not ms:
        return None
    a = ev * ops / (ms * 1e-3) / 1e12
    return {"events": ev, "ms": ms, "achieved": a, "frac": a / peak,
            "what": "the advance launch with the highest event rate (throughput-bound phase)"}


# --------------------------------------------------------------------------
# config 4: 256 uneven simulations in one batch
# --------------------------------------------------------------------------
def _make_from(ind, c, tuning=None, sampler=0):
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c["deme"],
                          sigma=c.get("sigma", 0.0), tuning=tuning, sampler=sampler)


def run_batch(args, rank, world, local, pg):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import autotune, build, workloads as W
    build.build()
    torch.cuda.set_device(local)
    specs = W.config4()

    def make_all(specs_, tuning=None):
        sims = [_make_from(ind, c, tuning, _sampler) for c in specs_]
        for x in sims:
            x.sample()
        return sims

    # exact distinct events of every simulation (untimed counting pass)
    sims = make_all(specs)
    st = ind.batch_run(sims, count_unique=1)
    U = sum(x["unique_events"] for x in st)
    for x in sims:
        x.close()
    # autotuning on a probe of the same batch with short speciation times
    probe = [dict(c, nu=max(c["nu"], 2e-3)) for c in specs]
    trials = []
    tuned, probe_s, n_trials = autotune.tune(lambda: make_all(probe), passes=1, log=trials)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    for _ in range(args.warmup):
        sims = make_all(specs)
        ind.batch_run(sims, **tuned)
        for x in sims:
            x.close()
    launches0 = ind.kernel_launches()
    clocks.start()
    step_ms, adv_ms, adv_n, raw = [], 0.0, 0, 0
    best = None
    for _ in range(args.steps):
        sims = make_all(specs)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ind.batch_run(sims, profile=1, **tuned)
        for x in sims:
            x.species()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        adv_ms += st[0]["advance_ms"]
        adv_n += st[0]["advance_launches"]
        raw += sum(x["raw_events"] for x in st)
        if st[0]["busiest_launch_ms"] and (best is None or st[0]["busiest_launch_events"] / st[0]["busiest_launch_ms"]
                                           > best["busiest_launch_events"] / best["busiest_launch_ms"]):
            best = st[0]
        for x in sims:
            x.close()
    clk = clocks.stop()
    launches = ind.kernel_launches() - launches0
    ms = sum(step_ms) / len(step_ms)
    # the plain path (one simulation per sim_run) on a stratified subset
    order = sorted(range(len(specs)), key=lambda k: specs[k]["nu"])
    stride = max(1, len(specs) // args.plain_subset)
    subset = order[::stride][: args.plain_subset]
    plain_s = 0.0
    for k in subset:
        x = _make_from(ind, specs[k], tuned, _sampler)
        x.sample()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.run()
        x.species()
        torch.cuda.synchronize()
        plain_s += time.perf_counter() - t0
        x.close()
    plain_est_s = plain_s * len(specs) / len(subset)
    ops = ops_per_raw_event()
    avg_launch_ms = adv_ms / max(adv_n, 1)
    ev_per_launch = raw / max(adv_n, 1)
    achieved = ev_per_launch * ops / (avg_launch_ms * 1e-3) / 1e12
    peak = torch.cuda.get_device_properties(local).multi_processor_count * INT32_LANES_PER_SM * 2032e6 / 1e12
    line = {
        "metric": METRIC, "value": U / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": "config4: 256 simulations in one batch (sizes log-uniform 1e3..1e6, nu log-uniform "
                               "1e-6..1e-2, half non-spatial, half torus with sigma uniform 1..8; master seed 42)",
                   "event_sampler": args.sampler, "unique_events_per_step": U, "raw_events_per_step": raw / args.steps,
                   "tuning": tuned, "autotune": {"trials": n_trials, "probe_seconds": probe_s}},
        "batched": {"events_per_s": U / (ms * 1e-3), "plain_events_per_s_estimated": U / plain_est_s,
                    "speedup": plain_est_s / (ms * 1e-3),
                    "plain": "sim_run one simulation at a time on %d of the 256 (stratified by nu), scaled"
                             % len(subset)},
        "roofline": {"bound": "alu", "kernel": "k_advance", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (32-bit integer)", "frac": achieved / peak, "traffic": None,
                     "events_per_launch": ev_per_launch, "avg_launch_ms": avg_launch_ms, "launches_timed": adv_n,
                     "ops_per_event": ops, "busiest_launch": busiest(best or {}, ops, peak)},
        "latency_bound": {"critical_events_per_step": st[0]["critical_events"],
                          "ns_per_critical_event": ms * 1e6 / max(st[0]["critical_events"], 1),
                          "what": "step time / (sum over rounds of the most events one lineage of the batch ran "
                                  "in the round): the batch lasts as long as its longest dependent chain"},
        "gpu_launches": launches, "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# config 5: served Poisson arrivals with continuous batching
# --------------------------------------------------------------------------
def run_served(args, rank, world, local, pg):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build, workloads as W
    build.build()
    torch.cuda.set_device(local)
    reqs = W.config5(window_s=args.window)
    srv_stream = torch.cuda.Stream()
    prep_stream = torch.cuda.Stream()
    srv = ind.Server(150 * 10 ** 9, max_sims=4096, stream=srv_stream)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ind.kernel_launches()
    sims, lat, arrival, index, lat_of = {}, [], {}, {}, {}
    nxt, done = 0, 0
    t0 = time.perf_counter()
    raw = 0
    while done < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
            r = reqs[nxt]
            with torch.cuda.stream(prep_stream):
                x = _make_from(ind, r, None, _sampler)
                x.sample(r["fraction"], r["sample_seed"])
            tk = srv.submit(x)
            sims[tk] = x
            arrival[tk] = r["arrival"]
            index[tk] = nxt
            nxt += 1
        fin = srv.step(4)
        t_now = time.perf_counter() - t0
        for tk in fin:
            x = sims.pop(tk)
            x.species()
            raw += x.stats()["raw_events"]
            lat.append(time.perf_counter() - t0 - arrival[tk])
            lat_of[index[tk]] = lat[-1]
            x.close()
            done += 1
        if not fin and srv.stats()["resident"] == 0 and nxt < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[nxt]["arrival"] - t_now)))
    total = time.perf_counter() - t0
    clk = clocks.stop()
    st = srv.stats()
    srv.close()
    plain = served_plain(ind, torch, reqs, lat_of, total, args.served_plain) if args.served_plain > 0 else None
    line = {
        "metric": METRIC, "value": raw / total, "unit": "raw events/s", "n_gpus": world, "steps": 1,
        "warmup": 0, "ms_per_step": total * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": "config5: Poisson arrivals 50/s over %.0f s, torus side log-uniform 128..4096, deme "
                               "1..4, fraction 0.01..1, nu log-uniform 1e-7..1e-3, sigma 1..8, HBM budget 150 GB"
                               % args.window, "requests": len(reqs), "event_sampler": args.sampler},
        "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat),
                      "what": "arrival to species identities on the device"},
        "plain": plain, "server": st, "clocks": clk, "gpu_launches": ind.kernel_launches() - launches0,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def served_plain(ind, torch, reqs, lat_of, total_s, n):
    """the plain path on a subset of the served requests, stratified by nu:
    each request alone, sim_create + sim_sample + sim_run + sim_species one
    after another on an idle GPU.  Scaled to all requests, the sum of these
    times is how long a server running one simulation at a time would need
    for the same work; per request, the served latency over the time alone
    is what sharing the GPU cost it"""
    order = sorted(range(len(reqs)), key=lambda k: reqs[k]["nu"])
    stride = max(1, len(reqs) // n)
    subset = order[stride // 2::stride][:n]
    alone, ratio = 0.0, []
    for k in subset:
        r = reqs[k]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = _make_from(ind, r, None, _sampler)
        x.sample(r["fraction"], r["sample_seed"])
        x.run()
        x.species()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        x.close()
        alone += dt
        ratio.append(lat_of[k] / dt)
    est = alone * len(reqs) / len(subset)
    return {"requests_timed": len(subset), "seconds_alone": alone, "seconds_all_estimated": est,
            "speedup": est / total_s, "served_over_alone": {"p50": pct(ratio, 50), "max": max(ratio)},
            "what": "each request alone on the plain path (sample, run, species), %d of %d stratified by nu; "
                    "speedup = their summed time scaled to all requests / the served run's wall time; "
                    "served_over_alone = a request's served latency / its time alone" % (len(subset), len(reqs))}


# --------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------
def oracle_run(seed=42):
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = W.config2(seed)
    m = O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], c["seed"], sigma=c["sigma"], sampler=_sampler)
    locs = m.sample()
    t0 = time.perf_counter()
    kl, kt, U = m.run_merge(locs)
    O.species_ids(kl, kt)
    return U, time.perf_counter() - t0


def cpu_baseline(seconds):
    total_u, total_t, runs = 0, 0.0, 0
    while total_t < seconds or runs == 0:
        U, dt = oracle_run(42 + runs)
        total_u += U
        total_t += dt
        runs += 1
    return {"value": total_u / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full config2 simulations (seeds 42..%d), event-ordered merge mode, one thread"
                      % (runs, 41 + runs)}


def cpu_baseline_traces(seconds):
    """the oracle on the spatially implicit workload: its event-ordered mode
    would need a slot per metacommunity individual (10^9), so lineages are
    traced alone (mode P), 64 at a time in order until the time is used; each
    traced event costs what a unique event costs in the event-ordered mode.
    The oracle's trace loop runs its 64 lineages on OpenMP's default team
    (the host's cores), so the line reports that many threads"""
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = W.implicit(42)
    m = O.Model(c["kind"], 1, 1, c["deme"], c["nu"], c["seed"], sampler=_sampler, migration=c["migration"],
                meta_size=c["meta_size"], meta_nu=c["meta_nu"])
    locs = m.sample()
    events, lineages, t = 0, 0, 0.0
    while (t < seconds or lineages == 0) and lineages < len(locs):
        chunk = locs[lineages:lineages + 64]
        t0 = time.perf_counter()
        _, _, ne = m.trace(chunk)
        t += time.perf_counter() - t0
        events += int(ne.sum())
        lineages += len(chunk)
    threads = min(O.max_threads(), 64)
    return {"value": events / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of the %d lineages traced alone (mode P, %d events), 64 at a time on %d threads"
                      % (lineages, len(locs), events, threads)}


def run_reference(args, rank, world, local, pg):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_run(42)
    times, us = [], []
    for k in range(args.steps):
        U, dt = oracle_run(42 + k)
        times.append(dt)
        us.append(U)
    value = sum(us) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "parallelism": "one CPU thread"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "one full config2 simulation per step (seeds 42..%d)" % (41 + args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    global _sampler, _single
    _sampler = SAMPLER[args.sampler]
    _single = single_workload(args.workload)
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only; other ranks exit
        rank = int(os.environ.get("RANK", "0"))
        if rank == 0:
            run_reference(args, 0, int(os.environ.get("WORLD_SIZE", "1")), 0, None)
        return
    rank, world, local, pg = dist_setup(args)
    if args.workload == "batch":
        run_batch(args, rank, world, local, pg)
    elif args.workload == "served":
        run_served(args, rank, world, local, pg)
    else:
        run_ours(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
