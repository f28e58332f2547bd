#!/usr/bin/env python
"""Benchmark: lineage events per second and species-count latency of the
Independent algorithm on B300, batched vs plain, bit-exact.

Default run (one JSON line):
  headline  config 3, the largest single simulation: a 1024 x 1024 seeded
            percolation habitat map (60 % habitable, demes 1..8, 2,829,667
            sampled lineages), alias dispersal over radius 16 from sigma = 4,
            nu = 1e-5, seed 42.  One step = sim_sample + sim_run +
            sim_species, every step of the hot path.  value = U / (device
            time per step), U = the workload's unique events, counted exactly
            by an untimed pass of the same simulation (the trajectories are
            bit-identical with and without counting).
  batched   config 4: 256 uneven simulations in one persistent batch
            (autotuned launch shape, CUDA-graph chunks) against the plain
            path (one simulation per sim_run), in unique events per second.
  served    config 5: Poisson arrivals of torus requests into the
            continuous-batching server at the highest rate it sustains
            on one B300 (10 requests/s: the requests in the system stay
            bounded), and at the specified 50 requests/s over a short
            window (beyond capacity); latency p50/p99 from arrival to
            species identities, offered and achieved request rates, drain
            time, requests in the system once a second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload all|config2|config3|implicit|batch|served]
  python bench.py --case NAME   named runs for profilers (see run_case)

Under torchrun every rank runs its own replica on its own GPU (replicas
only: the simulation is not sharded); rank 0 prints the line.
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
SAMPLER = {"exp": 0, "poisson": 1}

# Algorithmic 32-bit integer operations of one event of the spec (the
# integer work the spec itself defines, not the instructions a compiler emits)
PHILOX_OPS = 100          # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key adds)
EXP_DRAW_OPS = 110        # fixed-point -ln U of one draw, incl. conversion to binary64
EVENT_FIXED_OPS = 40      # speciation compare, dispersal index arithmetic, wrap, bookkeeping
ALIAS_OPS = 20            # map dispersal: column, take-or-alias choice, offset, deme index
POINT_OPS = 15            # Poisson sampler: one uniform point (conversion, rounded add, compare)
COUNT_OPS = 20            # Poisson sampler: guided inversion of the point count
INT32_LANES_PER_SM = 128  # Blackwell: 128 INT32-capable lanes per SM per clock
SM_MAX_MHZ = 2032.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="all", choices=["all", "config2", "config3", "implicit", "batch", "served"])
    ap.add_argument("--sampler", default="exp", choices=sorted(SAMPLER),
                    help="event-time sampler of the headline (the other is reported beside it)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU-baseline sample length")
    ap.add_argument("--batch-steps", type=int, default=2, help="config 4: timed batches")
    ap.add_argument("--plain-subset", type=int, default=32, help="config 4: simulations timed one by one")
    ap.add_argument("--served-rate", type=float, default=10.0,
                    help="config 5: offered requests per second (10: about the most the server sustains)")
    ap.add_argument("--served-window", type=float, default=20.0, help="config 5: arrival window in seconds")
    ap.add_argument("--served-plain", type=int, default=8,
                    help="config 5: requests re-run one by one on the plain path (0: none)")
    ap.add_argument("--served-tuning", default="",
                    help="config 5: server tuning overrides, name=value,... (ind_tuning fields)")
    ap.add_argument("--served-spec-window", type=float, default=4.0,
                    help="config 5 at its specified 50 requests/s: arrival window in seconds (0: skip)")
    ap.add_argument("--replicas", type=int, default=16,
                    help="single workloads: replicas in the batched-vs-plain comparison")
    ap.add_argument("--events", action="store_true",
                    help="single workloads: every step also produces the full event stream on the device")
    ap.add_argument("--no-floor", action="store_true", help="skip the hardware latency microbenchmark")
    ap.add_argument("--case", choices=["config2", "config3", "busy", "tail", "alias", "implicit"],
                    help="a named run for profilers instead of the benchmark")
    ap.add_argument("--rounds", type=int, default=6, help="case busy: rounds")
    ap.add_argument("--only", choices=["nonspatial", "torus", "map"], help="case tail: one landscape")
    ap.add_argument("--reps", type=int, default=3, help="cases tail and alias: repetitions")
    ap.add_argument("--block-threads", type=int)
    ap.add_argument("--blocks-per-sm", type=int)
    ap.add_argument("--tail-events", type=float, help="case tail: events per lineage per round")
    ap.add_argument("--map-side", type=int, default=1024, help="case config3: side of the habitat map")
    return ap.parse_args()


def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def allreduce(pg, x, op="max"):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX if op == "max" else pg.ReduceOp.SUM)
    return float(t.item())


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = (len(xs) - 1) * q / 100.0
    f = int(k)
    c = min(f + 1, len(xs) - 1)
    return xs[f] + (xs[c] - xs[f]) * (k - f)


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
        return self

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
# the spec's integer work per event, and the derived ALU peak
# --------------------------------------------------------------------------
def ops_per_event(sampler, kind):
    """integer operations per executed event (spec-derived): the event's
    own Philox blocks (two for Gaussian and map dispersal) and bookkeeping,
    plus the next-event search at lambda dt = 1: sums of exponentials draw
    on average 2.7 exponentials from 1.35 blocks; the Poisson sampler visits
    1.6 intervals of one block, one count and on average one point each"""
    blocks = 1 if kind == "nonspatial" else 2
    event = blocks * PHILOX_OPS + EVENT_FIXED_OPS + (ALIAS_OPS if kind == "map" else 0)
    if sampler == "poisson":
        return event + 1.6 * (PHILOX_OPS + COUNT_OPS + 1.0 * POINT_OPS)
    return event + 1.35 * PHILOX_OPS + 2.7 * EXP_DRAW_OPS


def int32_peak_tops(torch, dev):
    """(SMs, peak in Tops/s, its source): measured on this GPU where the
    microbenchmark runs (independent Philox4x32-10 blocks on every SM, 100
    integer ops per block, as ops_per_event counts them), else derived from
    the lane count and the maximum clock.  A block counts 100 ops for about 45
    instructions (a wide product is a high and a low product, a three-input
    xor two xors), so the measured figure can exceed the lane count"""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    derived = sms * INT32_LANES_PER_SM * SM_MAX_MHZ * 1e6 / 1e12
    if _floor_cache.get("use", False):
        _, lat = hw_latencies()
        return sms, lat["philox_tput_tops"], (
            "measured on this GPU: independent Philox4x32-10 blocks on all %d SMs (tests/hw_latency), 100 integer "
            "ops per block as ops_per_event counts them (the lane count x the maximum clock would give %.1f)"
            % (sms, derived))
    return sms, derived, ("derived, not measured: %d SMs x %d INT32 lanes x %.0f MHz maximum SM clock"
                          % (sms, INT32_LANES_PER_SM, SM_MAX_MHZ))


def busiest(st, ops, peak):
    ms, ev = st.get("busiest_launch_ms", 0.0), st.get("busiest_launch_events", 0)
    if not ms:
        return None
    a = ev * ops / (ms * 1e-3) / 1e12
    return {"events": ev, "ms": ms, "achieved": a, "frac": a / peak,
            "what": "the advance launch with the highest raw-event rate (throughput-bound phase)"}


# --------------------------------------------------------------------------
# fixtures written from the oracle: the longest line of descent
# --------------------------------------------------------------------------
def longest_descent(workload, sampler):
    """the most events one sampled lineage of the workload (seed 42, all
    sampled) runs before it speciates, from the oracle (mode P traces for
    configs 1 and 2, mode M's count for config 3), stored with the scripts
    that wrote them; None if not stored"""
    gold = os.path.join(ROOT, "tests", "golden")
    p = os.path.join(gold, "longest_chains.txt")
    if os.path.exists(p):
        for line in open(p):
            f = line.split()
            if len(f) == 5 and f[0] == workload and f[1] == sampler and f[2] == "42":
                return int(f[4])
    p = os.path.join(gold, "config3_digest.txt")
    if os.path.exists(p):
        for line in open(p):
            f = line.split()
            if len(f) == 8 and f[0] == workload and f[1] == sampler and f[2] == "42":
                return int(f[6])
    return None


def config4_longest(sampler):
    """the longest line of descent of any simulation of config 4 (the oracle's
    mode M, tests/golden/config4_digest.txt) and that simulation's index and
    landscape kind; None if not stored"""
    p = os.path.join(ROOT, "tests", "golden", "config4_digest.txt")
    if not os.path.exists(p):
        return None
    best = None
    for line in open(p):
        f = line.split()
        if len(f) == 9 and f[0] == "config4" and f[1] == sampler:
            if best is None or int(f[7]) > best[0]:
                best = (int(f[7]), int(f[2]), f[3])
    return best


# DRAM bytes (read + write) of one step's advance launches, from an ncu
# capture of this build (profiles/k_advance_coop_config3_dram.md): the
# roofline's traffic, per round like its achieved figure
DRAM_BYTES_PER_STEP = {("config3", "exp"): 117.74e9}

_floor_cache = {}


def hw_latencies():
    """dependent latencies of the event chain's operation classes on this GPU
    (the microbenchmark of tests/hw_latency), measured once per process"""
    if "lat" not in _floor_cache:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        import hw_latency
        _floor_cache["mod"] = hw_latency
        _floor_cache["lat"] = hw_latency.measure()
    return _floor_cache["mod"], _floor_cache["lat"]


def hw_floor(sampler, kind, crit, longest, ms_step):
    H, lat = hw_latencies()
    cyc = H.event_floor(lat, sampler, kind)
    cyc_compute = H.event_floor(lat, sampler, kind, memory=False)
    ns = cyc / lat["clock_mhz"] * 1e3
    out = {"cycles_per_event": cyc, "ns_per_event": ns, "clock_mhz": lat["clock_mhz"],
           "compute_cycles_per_event": cyc_compute,
           "critical_events_x_floor_ms": crit * ns * 1e-6, "step_over_critical_floor": ms_step / (crit * ns * 1e-6),
           "latencies_cycles": {k: round(v, 2) for k, v in lat.items()
                                if k not in ("clock_mhz", "steps_per_chain", "philox_tput_tops")},
           "path": {k: round(v, 1) for k, v in H.derived(lat).items()},
           "what": "cycles of one event on the method's critical path (two Philox blocks, the dispersal's lookups, "
                   "one logarithm or point count, the running sum's dependent adds; on a habitat map also the alias "
                   "row's fetch latency that the next search and event cannot cover), each operation costed at its "
                   "dependent latency measured on this GPU by tests/hw_latency; compute_*: without the row's "
                   "fetch; SM clock from a timed spin"}
    if longest:
        ns_c = cyc_compute / lat["clock_mhz"] * 1e3
        out.update({"longest_descent_events": longest, "longest_x_floor_ms": longest * ns * 1e-6,
                    "frac_of_longest_floor": longest * ns * 1e-6 / ms_step,
                    "frac_of_longest_compute_floor": longest * ns_c * 1e-6 / ms_step})
    return out


# --------------------------------------------------------------------------
# single-simulation workloads
# --------------------------------------------------------------------------
WORKLOADS = {
    "config3": ("config3: habitat map 1024x1024 (seeded site percolation, map seed 7, 60% habitable, deme uniform "
                "1..8: 2829667 sampled lineages), per-cell alias dispersal over radius 16 from Gaussian sigma=4 "
                "renormalised over habitat, nu=1e-5, lambda=1, delta_t=1, seed=42"),
    "config2": ("config2: torus 256x256, 1 individual per cell (65536 sampled lineages), Gaussian dispersal "
                "sigma=2 (discretised per axis), nu=1e-4, lambda=1, delta_t=1, seed=42"),
    "implicit": ("implicit: spatially implicit local community of 100000 individuals (all sampled), migration "
                 "0.01 per event, static metacommunity of 1e9 individuals with nu_meta=1e-4, local nu=0, "
                 "lambda=1, delta_t=1, seed=42"),
}
KIND_NAME = {"config3": "map", "config2": "torus", "implicit": "nonspatial"}


class Single:
    """one single-simulation workload: parameters, its map (config 3) and the
    simulations made from them"""

    def __init__(self, ind, name, map_side=1024):
        from paper_2108_05815_b300 import workloads as W
        self.ind, self.name = ind, name
        self.params = getattr(W, name)
        if name == "config3" and map_side != 1024:  # a smaller map of the same recipe (profiling only)
            self.params = lambda seed=42: W.config3(seed, side=map_side)
        self.desc = WORKLOADS[name]
        self.kind = KIND_NAME[name]
        c = self.params(42)
        self.dm_host = None
        if name == "config3":
            import numpy as np
            self.dm_host = np.zeros(c["width"] * c["height"], dtype=np.uint8)
            ind.habitat(c["map_seed"], c["width"], c["height"], c["p_habitable"], c["max_deme"], out=self.dm_host)
            self.n = int(self.dm_host.astype(np.int64).sum())
            self.h2d = int(self.dm_host.nbytes) + 400  # the habitat map + parameters
        elif name == "config2":
            self.n = c["width"] * c["height"] * c["deme"]
            self.h2d = 8 * 2 * 20 + 400                # discretised-normal table + parameters
        else:
            self.n = c["deme"]
            self.h2d = 400

    def make(self, seed=42, tuning=None, sampler=0):
        c = self.params(seed)
        return self.ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"],
                                   deme=c.get("deme", 1), sigma=c.get("sigma", 0.0), radius=c.get("radius", 0),
                                   deme_map=self.dm_host, migration=c.get("migration", 0.0),
                                   meta_size=c.get("meta_size", 0), meta_nu=c.get("meta_nu", 0.0), tuning=tuning,
                                   sampler=sampler)

    def count(self, seed=42, sampler=0, stats=False):
        s = self.make(seed, dict(count_unique=1), sampler)
        s.sample()
        assert s.run()
        st = s.stats()
        s.close()
        if stats:
            return st
        return st["unique_events"], st["raw_events"]


def time_steps(torch, sim, stream, steps, warmup, out, flush, log_cap=0):
    """warm-up, then `steps` timed steps (sample + run + species into the
    device tensor `out`), CUDA events on the simulation's stream, L2 flushed
    between steps; returns per-step device ms, host ms and summed stats"""
    for _ in range(warmup):
        sim.sample()
        assert sim.run()
        sim.species(out=out)
    torch.cuda.synchronize()
    dev_ms, host_ms = [], []
    acc = {"advance_ms": 0.0, "advance_launches": 0, "raw_events": 0, "best": None, "critical_events": 0}
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        e0.record(stream)
        sim.sample()
        ok = sim.run()
        _, K = sim.species(out=out)
        e1.record(stream)
        e1.synchronize()
        host_ms.append((time.perf_counter() - h0) * 1e3)
        assert ok
        dev_ms.append(e0.elapsed_time(e1))
        st = sim.stats()
        acc["advance_ms"] += st["advance_ms"]
        acc["advance_launches"] += st["advance_launches"]
        acc["raw_events"] += st["raw_events"]
        acc["critical_events"] = st["critical_events"]
        acc["K"] = K
        b = acc["best"]
        if st["busiest_launch_ms"] and (b is None or st["busiest_launch_events"] / st["busiest_launch_ms"] >
                                        b["busiest_launch_events"] / b["busiest_launch_ms"]):
            acc["best"] = st
    return dev_ms, host_ms, acc


def run_single(args, name, rank, world, local, pg):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = Single(ind, name)
    sampler = SAMPLER[args.sampler]
    cst = wl.count(42, sampler, stats=True)
    U, R = cst["unique_events"], cst["raw_events"]

    sim = wl.make(42, dict(profile=1), sampler)
    log_cap = int(R) + wl.n + 4096 if args.events else 0
    if log_cap:
        sim.set_event_log(log_cap)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ids = torch.empty(max(wl.n, 1), dtype=torch.int64, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ind.kernel_launches()
    barrier(pg)
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    dev_ms, host_ms, acc = time_steps(torch, sim, stream, args.steps, args.warmup, ids, flush)
    torch.cuda.synchronize()
    barrier(pg)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = ind.kernel_launches() - launches0
    ms_step = sum(dev_ms) / len(dev_ms)
    ms_step_max = allreduce(pg, ms_step)
    value = U * world / (ms_step_max * 1e-3)
    crit = acc["critical_events"]
    sim.close()

    # end to end through the public API with host buffers: the habitat map
    # from host memory, species identities into pinned host memory
    host_ids = torch.empty(max(wl.n, 1), dtype=torch.int64, pin_memory=True)
    e2e_ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        s2 = wl.make(42, None, sampler)
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
    e2e_ms_max = allreduce(pg, statistics.median(e2e_ms))
    d2h = wl.n * 8 + 64
    stream_line = None
    if log_cap:
        d2h += ev_host.nbytes + co_host.nbytes
        stream_line = {"distinct_events": int(len(ev_host)), "coalescences": int(len(co_host)),
                       "bytes_to_host": int(ev_host.nbytes + co_host.nbytes)}
        assert len(ev_host) == U

    # the other event-time sampler on the same workload (same protocol, fewer steps)
    other = "poisson" if args.sampler == "exp" else "exp"
    U_o, _ = wl.count(42, SAMPLER[other])
    so = wl.make(42, None, SAMPLER[other])
    o_ms, _, _ = time_steps(torch, so, stream, max(3, args.steps // 4), 2, ids, flush)
    so.close()
    other_line = {"sampler": other, "unique_events_per_step": U_o, "ms_per_step": sum(o_ms) / len(o_ms),
                  "value": U_o / (sum(o_ms) / len(o_ms) * 1e-3)}

    # The dependent chain: a round lasts as long as its busiest lineage, so a
    # step takes at least (critical events) x (the time of one event).  A few
    # lineages alone on the same landscape give this library's time per event
    # (t1); the hardware floor per event comes from measured latencies.
    lone = wl.make(42, dict(profile=1), sampler)
    lone.sample(8.0 / wl.n, 1)
    assert lone.run()
    ls = lone.stats()
    lone.close()
    lone_ns = ls["advance_ms"] * 1e6 / max(ls["critical_events"], 1)
    crit_ns = ms_step * 1e6 / max(crit, 1)
    longest = longest_descent(name, args.sampler)
    latency = {"critical_events_per_step": crit, "ns_per_critical_event": crit_ns,
               "lone_lineage_ns_per_event": lone_ns, "lone_lineages": ls["n_sampled"],
               "lone_over_critical": lone_ns / crit_ns,
               "what": "critical events = the sum over rounds of the most events one lineage ran in the round; "
                       "lone = this library's advance-kernel time per event of a few lineages alone on the same "
                       "landscape (a property of these kernels, not a roofline); hw_floor = the hardware floor"}
    if longest:
        latency.update({"longest_descent_events": longest, "longest_x_lone_ms": longest * lone_ns * 1e-6})
    if not args.no_floor:
        latency["hw_floor"] = hw_floor(args.sampler, wl.kind, crit, longest, ms_step)

    # ALU roofline of the advance launches, in unique events
    ops = ops_per_event(args.sampler, wl.kind)
    adv_n = max(acc["advance_launches"], 1)
    avg_launch_ms = acc["advance_ms"] / adv_n
    unique_per_launch = U * args.steps / adv_n
    achieved = unique_per_launch * ops / (avg_launch_ms * 1e-3) / 1e12
    sms, peak, peak_src = int32_peak_tops(torch, dev)
    step_bytes = None if log_cap else DRAM_BYTES_PER_STEP.get((name, args.sampler))
    traffic = step_bytes * args.steps / adv_n if step_bytes else None
    cpu = cpu_baseline(name, args.sampler, args.cpu_seconds) if rank == 0 else None

    # batched vs plain on replicas of the workload (different seeds)
    replicas = None
    if args.replicas > 0 and name != "config3":
        replicas = replicas_leg(torch, ind, wl, args.replicas, sampler, ids)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": wl.desc + (" + full event stream" if log_cap else ""),
                   "event_sampler": args.sampler, "units": "unique events (distinct (location, time) events of "
                   "the coalescence tree, counted exactly)",
                   "parallelism": "replicas (one independent simulation per GPU)",
                   "l2": "flushed by a 256 MiB write between timed steps",
                   "unique_events_per_step": U, "raw_events_per_step": acc["raw_events"] / args.steps,
                   "species": acc.get("K"), "lineages": wl.n, "tuning": ind.default_tuning(),
                   "dedup": dedup_counts(cst)},
        "latency_ms": {"p50": pct(host_ms, 50), "p99": pct(host_ms, 99),
                       "what": "step start to the species count on the host, one simulation at a time"},
        "raw_events_per_s": acc["raw_events"] / args.steps * world / (ms_step_max * 1e-3),
        "roofline": {"bound": "alu", "kernel": "k_advance_coop + k_advance + k_filter (one round's launches)",
                     "achieved": achieved, "peak": peak, "unit": "Tops/s (32-bit integer)", "frac": achieved / peak,
                     "traffic": traffic,
                     "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one step's advance "
                                        "launches on B300 (profiles/k_advance_coop_config3_dram.md), per round"
                                        if traffic else None),
                     "ops_per_event": ops, "unique_events_per_launch": unique_per_launch,
                     "avg_launch_ms": avg_launch_ms, "launches_timed": acc["advance_launches"],
                     "busiest_launch": busiest(acc["best"] or {}, ops, peak),
                     "peak_source": peak_src,
                     "binding": "the dependent chain of the longest lineage (latency_bound), not a pipe",
                     "chain_floor_frac": chain_floor_frac(latency),
                     "chain_floor_what": "the binding roofline: (longest line of descent x the hardware floor of "
                                         "one event, from measured latencies) / step time; see latency_bound"},
        "latency_bound": latency,
        "event_stream": stream_line,
        "cpu_baseline": cpu,
        "e2e": {"value": U * world / (e2e_ms_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": wl.h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max,
                "what": "sim_create (habitat map from host memory, alias tables built) + sim_sample + sim_run + "
                        "sim_species into pinned host memory"},
        "other_sampler": other_line,
        "replicas": replicas,
        "gpu_launches": launches, "clocks": clk, "wall_s_timed": t_wall,
    }
    return line


def dedup_counts(st):
    """the horizon dedup's inserts in the counting pass: a warp pre-collapse
    of equal slot keys before the table insert could save at most the
    warp-shadowed ones"""
    return {"inserts": st["dedup_inserts"], "slot_already_entered": st["dedup_repeats"],
            "same_slot_same_warp_instruction": st["dedup_warp_repeats"], "rounds": st["rounds"],
            "what": "counting pass: dedup inserts; inserts whose slot another lineage had entered; inserts "
                    "shadowed by a lower lane of the same warp inserting the same slot in the same instruction"}


def chain_floor_frac(latency):
    """the step against its hardware chain floor: longest line of descent x
    floor per event / step when the line is known, else critical events x
    floor per event / step"""
    hw = latency.get("hw_floor")
    if not hw:
        return None
    if "frac_of_longest_floor" in hw:
        return hw["frac_of_longest_floor"]
    return 1.0 / hw["step_over_critical_floor"]


def replicas_leg(torch, ind, wl, n, sampler, ids):
    """batched vs plain on n independent replicas (seeds 42..) of a workload"""
    seeds = [42 + k for k in range(n)]
    Us = [wl.count(s, sampler)[0] for s in seeds]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in seeds:
        x = wl.make(s, None, sampler)
        x.sample()
        x.run()
        x.species(out=ids)
        x.close()
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t0
    sims = [wl.make(s, None, sampler) for s in seeds]
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
    return {"sims": n, "workload": "%s replicas, seeds 42..%d" % (wl.name, 41 + n), "unique_events": sum(Us),
            "batched_events_per_s": sum(Us) / batch_s, "plain_events_per_s": sum(Us) / plain_s,
            "speedup": plain_s / batch_s}


# --------------------------------------------------------------------------
# config 4: 256 uneven simulations in one batch
# --------------------------------------------------------------------------
def _make_from(ind, c, tuning=None, sampler=0):
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c["deme"],
                          sigma=c.get("sigma", 0.0), tuning=tuning, sampler=sampler)


def batched_leg(args, local, sampler_name="exp"):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import autotune, build, workloads as W
    build.build()
    torch.cuda.set_device(local)
    sampler = SAMPLER[sampler_name]
    specs = W.config4()

    def make_all(specs_, tuning=None):
        sims = [_make_from(ind, c, tuning, sampler) for c in specs_]
        for x in sims:
            x.sample()
        return sims

    # exact unique events of every simulation (untimed counting pass)
    sims = make_all(specs)
    st = ind.batch_run(sims, count_unique=1)
    U_each = [x["unique_events"] for x in st]
    U = sum(U_each)
    dedup = dedup_counts(st[0])
    for x in sims:
        x.close()
    # autotuning on a probe of the same batch with short speciation times
    probe = [dict(c, nu=max(c["nu"], 2e-3)) for c in specs]
    tuned, probe_s, n_trials = autotune.tune(lambda: make_all(probe), passes=1, log=[])
    stream = torch.cuda.current_stream()
    sims = make_all(specs)
    ind.batch_run(sims, **tuned)  # warm-up batch
    for x in sims:
        x.close()
    clocks = ClockSampler(local).start()
    launches0 = ind.kernel_launches()
    step_ms, adv_ms, adv_n, raw, best, crit = [], 0.0, 0, 0, None, 0
    for _ in range(max(1, args.batch_steps)):
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
        crit = st[0]["critical_events"]
        if st[0]["busiest_launch_ms"] and (best is None or st[0]["busiest_launch_events"] / st[0]["busiest_launch_ms"]
                                           > best["busiest_launch_events"] / best["busiest_launch_ms"]):
            best = st[0]
        for x in sims:
            x.close()
    clk = clocks.stop()
    launches = ind.kernel_launches() - launches0
    ms = sum(step_ms) / len(step_ms)
    # the plain path (one simulation per sim_run) on a subset stratified by nu
    order = sorted(range(len(specs)), key=lambda k: specs[k]["nu"])
    stride = max(1, len(specs) // args.plain_subset)
    subset = order[::stride][: args.plain_subset]
    plain_s, plain_lat = 0.0, []
    for k in subset:
        x = _make_from(ind, specs[k], tuned, sampler)
        x.sample()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.run()
        x.species()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        plain_s += dt
        plain_lat.append(dt * 1e3)
        x.close()
    # every simulation of the subset at once stands for its share of the 256
    plain_est_s = plain_s * len(specs) / len(subset)
    ops = ops_per_event(sampler_name, "torus")
    avg_launch_ms = adv_ms / max(adv_n, 1)
    latency = {"critical_events_per_batch": crit, "ns_per_critical_event": ms * 1e6 / max(crit, 1),
               "what": "the batch lasts as long as its longest dependent chain of events"}
    longest = config4_longest(sampler_name)
    if longest and not args.no_floor:
        # the binding roofline: no schedule ends the batch before the longest
        # line of descent of its simulations has run, one hardware-floor event
        # after another
        L, k_long, kind = longest
        H, lat = hw_latencies()
        ns = H.event_floor(lat, sampler_name, kind) / lat["clock_mhz"] * 1e3
        latency["hw_floor"] = {"longest_descent_events": L, "simulation": k_long, "kind": kind,
                               "ns_per_event": ns, "clock_mhz": lat["clock_mhz"],
                               "longest_x_floor_ms": L * ns * 1e-6, "frac_of_longest_floor": L * ns * 1e-6 / ms,
                               "what": "the longest line of descent of any simulation of the batch (oracle, mode M) "
                                       "x the hardware floor of one event of its landscape kind, from latencies "
                                       "measured on this GPU (tests/hw_latency) / the batch's time"}
    achieved = U * len(step_ms) / max(adv_n, 1) * ops / (avg_launch_ms * 1e-3) / 1e12
    sms, peak, peak_src = int32_peak_tops(torch, torch.device("cuda", local))
    return {
        "workload": "config4: 256 simulations in one batch (sizes log-uniform 1e3..1e6, nu log-uniform 1e-6..1e-2, "
                    "half non-spatial, half torus with sigma uniform 1..8; master seed 42)",
        "event_sampler": sampler_name, "value": U / (ms * 1e-3), "unit": "unique events/s", "ms_per_batch": ms,
        "batches_timed": len(step_ms), "unique_events_per_batch": U, "raw_events_per_batch": raw / len(step_ms),
        "plain_events_per_s_estimated": U / plain_est_s, "speedup_vs_plain": plain_est_s / (ms * 1e-3),
        "plain": "sim_run one simulation at a time on %d of the 256 (stratified by nu), summed and scaled by 256/%d"
                 % (len(subset), len(subset)),
        "latency_ms": {"batch": ms, "plain_alone_p50": pct(plain_lat, 50), "plain_alone_p99": pct(plain_lat, 99),
                       "what": "every species count of the batch is ready when the batch ends; plain: one "
                               "simulation's sim_run + sim_species alone"},
        "tuning": tuned, "autotune": {"trials": n_trials, "probe_seconds": probe_s}, "dedup": dedup,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s (32-bit integer)",
                     "frac": achieved / peak, "peak_source": peak_src,
                     "ops_per_event": ops, "busiest_launch": busiest(best or {}, ops, peak)},
        "latency_bound": latency,
        "chain_floor_frac": latency.get("hw_floor", {}).get("frac_of_longest_floor"),
        "gpu_launches": launches, "clocks": clk,
    }


# --------------------------------------------------------------------------
# config 5: served Poisson arrivals with continuous batching
# --------------------------------------------------------------------------
def served_leg(args, local, rate, window, plain_n, sampler_name="exp"):
    import torch
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build, workloads as W
    build.build()
    torch.cuda.set_device(local)
    sampler = SAMPLER[sampler_name]
    reqs = W.config5(rate=rate, window_s=window)
    srv_stream = torch.cuda.Stream()
    prep_stream = torch.cuda.Stream()
    srv = ind.Server(150 * 10 ** 9, max_sims=4096, stream=srv_stream, **served_tuning(args))
    clocks = ClockSampler(local).start()
    launches0 = ind.kernel_launches()
    sims, lat, arrival, index, lat_of = {}, [], {}, {}, {}
    nxt, done, raw = 0, 0, 0
    q_max, res_max, lin_max, samples = 0, 0, 0, []
    t0 = time.perf_counter()
    t_last_arrival = reqs[-1]["arrival"] if reqs else 0.0
    while done < len(reqs):
        now = time.perf_counter() - t0
        while nxt < len(reqs) and reqs[nxt]["arrival"] <= now:
            r = reqs[nxt]
            with torch.cuda.stream(prep_stream):
                x = _make_from(ind, r, None, sampler)
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
        st = srv.stats()
        in_system = nxt - done
        q_max, res_max = max(q_max, in_system), max(res_max, st["resident"])
        lin_max = max(lin_max, st["resident_lineages"])
        if not samples or t_now - samples[-1][0] >= 1.0:
            samples.append((round(t_now, 2), in_system))
        if not fin and st["resident"] == 0 and nxt < len(reqs):
            time.sleep(max(0.0, min(0.01, reqs[nxt]["arrival"] - t_now)))
    total = time.perf_counter() - t0
    clk = clocks.stop()
    sst = srv.stats()
    srv.close()
    plain = served_plain(ind, torch, reqs, lat_of, total, plain_n, sampler) if plain_n > 0 else None
    out = {
        "workload": "config5: Poisson arrivals %.0f/s over %.0f s, torus side log-uniform 128..4096, deme 1..4, "
                    "sample fraction 0.01..1, nu log-uniform 1e-7..1e-3, sigma 1..8, HBM budget 150 GB"
                    % (rate, window),
        "event_sampler": sampler_name, "requests": len(reqs), "offered_rate_per_s": rate, "window_s": window,
        "server_tuning": dict(ind.server_default_tuning(), **served_tuning(args)),
        "wall_s": total, "achieved_rate_per_s": len(reqs) / total,
        "drain_s": total - t_last_arrival,
        "latency_s": {"p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat) if lat else None,
                      "what": "arrival to species identities on the device"},
        "raw_events_per_s": raw / total,
        "in_system": {"max": q_max, "max_resident": res_max, "max_resident_lineages": lin_max,
                      "per_second": samples, "what": "requests submitted and not finished, sampled about once a "
                                                     "second: (seconds since the first arrival, count)"},
        "server": sst, "clocks": clk, "gpu_launches": ind.kernel_launches() - launches0,
        "plain": plain,
    }
    if plain and plain.get("unique_over_raw_alone"):
        out["unique_events_per_s_estimated"] = out["raw_events_per_s"] * plain["unique_over_raw_alone"]
    return out


def served_tuning(args):
    """--served-tuning name=value,... as a dict of ind_tuning overrides"""
    out = {}
    for kv in filter(None, getattr(args, "served_tuning", "").split(",")):
        k, v = kv.split("=")
        out[k.strip()] = float(v) if "." in v or "e" in v else int(v)
    return out


def served_plain(ind, torch, reqs, lat_of, total_s, n, sampler):
    """the plain path on a subset of the served requests, stratified by nu:
    each request alone (sim_create + sim_sample + sim_run + sim_species) on
    an idle GPU, its unique events counted exactly in a separate untimed run.
    Scaled to all requests, the summed time is how long a server running one
    simulation at a time would take; per request, the served latency over
    its time alone is what sharing the GPU cost it"""
    order = sorted(range(len(reqs)), key=lambda k: reqs[k]["nu"])
    stride = max(1, len(reqs) // n)
    subset = order[stride // 2::stride][:n]
    alone, ratio, u_sum, r_sum = 0.0, [], 0, 0
    for k in subset:
        r = reqs[k]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = _make_from(ind, r, None, sampler)
        x.sample(r["fraction"], r["sample_seed"])
        x.run()
        x.species()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        x.close()
        alone += dt
        ratio.append(lat_of[k] / dt)
        c = _make_from(ind, r, dict(count_unique=1), sampler)
        c.sample(r["fraction"], r["sample_seed"])
        c.run()
        st = c.stats()
        c.close()
        u_sum += st["unique_events"]
        r_sum += st["raw_events"]
    est = alone * len(reqs) / len(subset)
    return {"requests_timed": len(subset), "seconds_alone": alone, "seconds_all_estimated": est,
            "speedup": est / total_s, "served_over_alone": {"p50": pct(ratio, 50), "max": max(ratio)},
            "unique_over_raw_alone": u_sum / max(r_sum, 1),
            "what": "each request alone on the plain path, %d of %d stratified by nu; speedup = their summed time "
                    "scaled to all requests / the served run's wall time; unique_over_raw_alone = the subset's "
                    "exact unique events over its raw events alone (the served rate in unique events is that "
                    "fraction of the served raw rate: an estimate)" % (len(subset), len(reqs))}


# --------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------
_oracle_models = {}


def _oracle_model(name, sampler_name):
    if (name, sampler_name) not in _oracle_models:
        _oracle_models[(name, sampler_name)] = _make_oracle_model(name, sampler_name)
    return _oracle_models[(name, sampler_name)]


def _make_oracle_model(name, sampler_name):
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = getattr(W, name)(42)
    s = SAMPLER[sampler_name]
    if name == "config3":
        dm = O.habitat(c["map_seed"], c["width"], c["height"], c["p_habitable"], c["max_deme"])
        return O, O.Model(c["kind"], c["width"], c["height"], 0, c["nu"], c["seed"], sigma=c["sigma"],
                          radius=c["radius"], deme_map=dm, sampler=s)
    if name == "implicit":
        return O, O.Model(c["kind"], 1, 1, c["deme"], c["nu"], c["seed"], sampler=s, migration=c["migration"],
                          meta_size=c["meta_size"], meta_nu=c["meta_nu"])
    return O, O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], c["seed"], sigma=c["sigma"], sampler=s)


TRACE_CAP = 20000  # events per traced lineage in a CPU-baseline chunk


def oracle_traces(name, sampler_name, seconds, start=0):
    """the oracle's per-lineage traces (mode P, the plain definition of the
    Independent algorithm) of the workload's sampled lineages in a seeded
    random order, chunks of four lineages per thread of OpenMP's team (the
    host's cores), each lineage traced for at most TRACE_CAP events (so that
    a chunk's threads finish together), until `seconds` of wall time are
    used.  Each traced event is one event of the method's work (a unique
    event of the event-ordered mode costs the same); returns (events,
    seconds, lineages, threads, lineages in all)"""
    import numpy as np
    O, m = _oracle_model(name, sampler_name)
    if not hasattr(m, "_bench_locs"):
        m._bench_locs = m.sample()
    locs = m._bench_locs
    order = np.random.default_rng(1234 + start).permutation(len(locs))
    threads = max(O.max_threads(), 1)
    chunk = 4 * threads
    events, t, k = 0, 0.0, 0
    while (t < seconds or k == 0) and k < len(locs):
        pick = locs[order[k:k + chunk]]
        t0 = time.perf_counter()
        _, _, ne = m.trace(pick, max_events=TRACE_CAP, partial=True)
        t += time.perf_counter() - t0
        events += int(ne.sum())
        k += len(pick)
    return events, t, k, threads, len(locs)


def cpu_baseline(name, sampler_name, seconds):
    events, t, k, threads, n = oracle_traces(name, sampler_name, seconds)
    return {"value": events / t, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": "%d of the %d lineages of %s traced alone (mode P, at most %d events each, %d events in "
                      "all) in a seeded random order, %d at a time on %d threads (all the host's cores); each "
                      "traced event is one event of the method's work"
                      % (k, n, name, TRACE_CAP, events, 4 * threads, threads)}


def run_reference(args):
    """--impl reference: the oracle as it stands, timed on the host cores on
    the headline's workload; each step traces a bounded sample of lineages"""
    name = "config3" if args.workload in ("all", "config3", "batch", "served") else args.workload
    per_step = 2.0
    for k in range(args.warmup):
        oracle_traces(name, args.sampler, per_step / 4, start=k)
    ev, tt, lin, thr, n = 0, 0.0, 0, 1, 0
    for k in range(args.steps):
        e, t, l, thr, n = oracle_traces(name, args.sampler, per_step, start=1000 + k)
        ev, tt, lin = ev + e, tt + t, lin + l
    value = ev / tt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[name], "event_sampler": args.sampler,
                                            "parallelism": "OpenMP over lineages on the host's %d cores" % thr},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": "per step about %.0f s of lineages of %s traced alone (mode P, at most %d "
                                       "events each), %d lineages of %d, %d events in all"
                                       % (per_step, name, TRACE_CAP, lin, n, ev)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# named runs for profilers
# --------------------------------------------------------------------------
def run_case(args):
    """named runs for profilers (ncu) and latency checks; each prints one
    JSON line.  Device memory held: well under 1 GB except config3 (about
    5 GB: the alias tables)
      config2   the 256 x 256 torus once without CUDA graphs, so that every
                advance launch is a separate kernel launch (--events: with the
                event stream)
      config3   the 1024 x 1024 habitat map once without CUDA graphs
                (--map-side: a smaller map of the same recipe)
      busy      a 1024 x 1024 torus (1,048,576 lineages, sigma 2, nu 1e-3) for
                --rounds rounds: the throughput-bound phase
      tail      one lineage, nu 1e-4 (about 10^4 events) on a non-spatial deme
                of one, on a 1 x 1 torus with sigma 2 and on a one-cell map:
                the latency-bound phase; prints the device time per event
                (fastest of --reps).  --block-threads 64 --blocks-per-sm 1
                leaves few idle warps beside the working one
      implicit  the spatially implicit workload once without CUDA graphs
      alias     config 3's map and its dispersal tables: the wall time of
                each sim_create (one alias row per habitable cell)"""
    import numpy as np
    import torch  # noqa: F401  (device memory comes from torch's allocator)
    import paper_2108_05815_b300 as ind
    from paper_2108_05815_b300 import build, workloads as W
    build.build()
    sampler = SAMPLER[args.sampler]
    launch = {}
    if args.block_threads:
        launch["block_threads"] = args.block_threads
    if args.blocks_per_sm:
        launch["blocks_per_sm"] = args.blocks_per_sm
    if args.tail_events:
        launch["tail_events"] = args.tail_events
    if args.case in ("config2", "config3", "implicit"):
        wl = Single(ind, args.case, map_side=args.map_side)
        s = wl.make(42, dict(use_graph=0, profile=1, **launch), sampler)
        if args.events:
            s.set_event_log(8 << 20)
        s.sample()
        assert s.run()
        _, K = s.species()
        st = s.stats()
        out = dict(case=args.case, species=K, **{k: st[k] for k in ("rounds", "raw_events", "advance_launches",
                                                                    "critical_events")})
        if args.events:
            ev, co = s.events()
            out.update(distinct_events=len(ev), coalescences=len(co))
        s.close()
    elif args.case == "busy":
        s = ind.Simulation(W.TORUS, 1e-3, 42, width=1024, height=1024, deme=1, sigma=2.0,
                           tuning=dict(use_graph=0, **launch), sampler=sampler)
        s.sample()
        done = s.run(round_budget=args.rounds)
        st = s.stats()
        s.close()
        out = dict(case="busy", finished=bool(done), rounds=st["rounds"], raw_events=st["raw_events"])
    elif args.case == "tail":
        out = dict(case="tail")
        one_cell = np.array([1], dtype=np.uint8)
        for nm, kw in (("nonspatial_deme1", dict(kind=W.NONSPATIAL, deme=1)),
                       ("torus_1x1_sigma2", dict(kind=W.TORUS, width=1, height=1, deme=1, sigma=2.0)),
                       ("map_1x1_radius16", dict(kind=W.MAP, width=1, height=1, sigma=4.0, radius=16,
                                                 deme_map=one_cell))):
            if args.only and not nm.startswith(args.only):
                continue
            best = None
            for _ in range(args.reps):
                kw2 = {k: v for k, v in kw.items() if k != "kind"}
                s = ind.Simulation(kw["kind"], 1e-4, 1, sampler=sampler, tuning=dict(profile=1, **launch), **kw2)
                s.sample()
                t0 = time.perf_counter()
                assert s.run()
                t1 = time.perf_counter()
                st = s.stats()
                s.close()
                per = dict(events=st["raw_events"], rounds=st["rounds"],
                           us_per_event_wall=(t1 - t0) * 1e6 / st["raw_events"],
                           us_per_event_device=st["advance_ms"] * 1e3 / st["raw_events"])
                if best is None or per["us_per_event_device"] < best["us_per_event_device"]:
                    best = per
            out[nm] = best
    else:  # alias
        c = W.config3()
        dm = ind.habitat(c["map_seed"], c["width"], c["height"], c["p_habitable"], c["max_deme"])
        times = []
        for _ in range(args.reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s = ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"],
                               sigma=c["sigma"], radius=c["radius"], deme_map=dm)
            torch.cuda.synchronize()
            times.append(round((time.perf_counter() - t0) * 1e3, 2))
            s.close()
        out = dict(case="alias", habitable_cells=int((dm > 0).sum()), sim_create_ms=times)
    out["sampler"] = args.sampler
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------------------
def main():
    args = parse()
    _floor_cache["use"] = not args.no_floor  # the microbenchmark also gives the measured integer peak
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only; other ranks exit
        if int(os.environ.get("RANK", "0")) == 0:
            run_reference(args)
        return
    rank, world, local, pg = dist_setup()
    if args.workload in ("all", "config3", "config2", "implicit"):
        name = "config3" if args.workload == "all" else args.workload
        line = run_single(args, name, rank, world, local, pg)
        if args.workload == "all":
            line["batched"] = batched_leg(args, local, args.sampler)
            line["served"] = served_leg(args, local, args.served_rate, args.served_window, args.served_plain,
                                        args.sampler)
            if args.served_spec_window > 0:
                line["served_at_50_per_s"] = served_leg(args, local, 50.0, args.served_spec_window, 0, args.sampler)
    elif args.workload == "batch":
        b = batched_leg(args, local, args.sampler)
        line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": world, "steps": b["batches_timed"],
                "warmup": 1, "ms_per_step": b["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
                "config": {"workload": b["workload"], "event_sampler": args.sampler}, "batched": b,
                "roofline": b["roofline"], "gpu_launches": b["gpu_launches"], "clocks": b["clocks"]}
    else:
        s = served_leg(args, local, args.served_rate, args.served_window, args.served_plain, args.sampler)
        line = {"metric": METRIC, "value": s["raw_events_per_s"], "unit": "raw events/s", "n_gpus": world,
                "steps": 1, "warmup": 0, "ms_per_step": s["wall_s"] * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
                "config": {"workload": s["workload"], "event_sampler": args.sampler}, "served": s,
                "gpu_launches": s["gpu_launches"], "clocks": s["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
