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
# Algorithmic 32-bit integer operations of the spec ("Roofline"):
PHILOX_OPS = 100          # 10 rounds x (2 mul.lo + 2 mul.hi + 4 xor + 2 key adds)
EXP_DRAW_OPS = 110        # fixed-point -ln U of one draw, incl. conversion to binary64
EVENT_FIXED_OPS = 40      # speciation compare, dispersal index arithmetic, wrap, bookkeeping
INT32_LANES_PER_SM = 128  # Blackwell: 128 INT32-capable lanes per SM per clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="simulations in the batched-vs-plain comparison")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="CPU-baseline sample length")
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
def make_sim(ind, seed=42, tuning=None):
    from paper_2108_05815_b300 import workloads as W
    c = W.config2(seed)
    return ind.Simulation(c["kind"], c["nu"], c["seed"], width=c["width"], height=c["height"], deme=c["deme"],
                          sigma=c["sigma"], tuning=tuning)


def unique_events(ind, seed):
    s = make_sim(ind, seed, tuning=dict(count_unique=1))
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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ids = torch.empty(65536, dtype=torch.int64, device=dev)

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
    torch.cuda.synchronize()
    barrier(pg)
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    launches = ind.kernel_launches() - launches0
    ms_step = sum(step_ms) / len(step_ms)
    ms_step_max = allreduce_max(pg, ms_step)
    value = U * world / (ms_step_max * 1e-3)

    # end to end through the public API with host buffers
    host_ids = torch.empty(65536, dtype=torch.int64, pin_memory=True)
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        s2 = make_sim(ind, 42)
        s2.sample()
        s2.run()
        s2.species(out=host_ids)
        h1 = time.perf_counter()
        s2.close()
        e2e_ms.append((h1 - h0) * 1e3)
    e2e_ms_max = allreduce_max(pg, statistics.median(e2e_ms))
    h2d = 8 * 2 * 20 + 400  # discretised-normal table (2 x 20 x 8 B) + simulation parameters
    d2h = 65536 * 8 + 64    # species identities + completion flags

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

    # roofline of the advance kernel (events per launch / its CUDA-event time)
    raw_per_step = raw / args.steps
    events_per_launch = raw / max(adv_n, 1)
    ops_per_event = ops_per_raw_event()
    avg_launch_ms = adv_ms / max(adv_n, 1)
    achieved = events_per_launch * ops_per_event / (avg_launch_ms * 1e-3) / 1e12
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = sm_count * INT32_LANES_PER_SM * 2032e6 / 1e12
    cpu = cpu_baseline(args.cpu_seconds) if rank == 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "replicas (one independent simulation per GPU)",
                   "l2": "flushed by a 256 MiB write between timed steps",
                   "unique_events_per_step": U, "raw_events_per_step": raw_per_step,
                   "species": K, "tuning": ind.default_tuning()},
        "latency_ms": {"p50": pct(lat_ms, 50), "p99": pct(lat_ms, 99), "what": "step start to species count on host"},
        "raw_events_per_s": raw_per_step * world / (ms_step_max * 1e-3),
        "roofline": {"bound": "alu", "kernel": "k_advance", "achieved": achieved, "peak": peak,
                     "unit": "Tops/s (32-bit integer)", "frac": achieved / peak, "traffic": None,
                     "ops_per_event": ops_per_event, "events_per_launch": events_per_launch,
                     "avg_launch_ms": avg_launch_ms, "launches_timed": adv_n,
                     "peak_source": "148 SMs x 128 INT32 lanes x 2032 MHz max SM clock (derived, see DESIGN.md)"},
        "cpu_baseline": cpu,
        "e2e": {"value": U * world / (e2e_ms_max * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms_max,
                "what": "sim_create + sim_sample + sim_run + sim_species into pinned host memory"},
        "batched": {"sims": args.batch, "workload": "config2 replicas, seeds 42..%d" % (41 + args.batch),
                    "unique_events": sum(Us), "batched_events_per_s": sum(Us) / batch_s,
                    "plain_events_per_s": sum(Us) / plain_s, "speedup": plain_s / batch_s},
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


def ops_per_raw_event():
    """integer operations per executed event of the workload (spec-derived; the
    per-event draw counts are those of the exponential and dispersal draws)"""
    # per event: one event block (two for Gaussian dispersal), plus the
    # re-prime interval walk: E[blocks] = 1.35, E[draws] = 2.7 at lambda dt = 1
    return 2 * PHILOX_OPS + 1.35 * PHILOX_OPS + 2.7 * EXP_DRAW_OPS + EVENT_FIXED_OPS


# --------------------------------------------------------------------------
# the oracle on the host cores
# --------------------------------------------------------------------------
def oracle_run(seed=42):
    import oracle as O
    from paper_2108_05815_b300 import workloads as W
    c = W.config2(seed)
    m = O.Model(c["kind"], c["width"], c["height"], c["deme"], c["nu"], c["seed"], sigma=c["sigma"])
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
    if args.impl == "reference":
        # the oracle runs on the host cores of rank 0 only; other ranks exit
        rank = int(os.environ.get("RANK", "0"))
        if rank == 0:
            run_reference(args, 0, int(os.environ.get("WORLD_SIZE", "1")), 0, None)
        return
    rank, world, local, pg = dist_setup(args)
    run_ours(args, rank, world, local, pg)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
