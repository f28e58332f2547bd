"""Hardware floor of one lineage's event chain, from measured latencies.

Measurement tool of the test side (not part of the library): it compiles
``chain_latency.cu`` with nvcc for sm_103a, measures the dependent latency
of each operation class on the event chain as a chain of that operation in
one warp (cycles from the SM clock counter), and the SM clock itself (a
spin of a known number of cycles timed with CUDA events).  ``event_floor``
adds those latencies along the critical path of one event as the method
defines it, so that a step's time can be set against the fewest cycles any
implementation on this GPU needs for its longest chain of dependent events.

The critical path of one event (lambda = 1, delta_t = 1; section "Summary of
the Independent Algorithm"; sums of exponentials per "Memoryless sums of
exponentials", Poisson points per "Homogeneous Poisson Point Process"):

  1. the event's stream at (location, event time): the two Philox blocks of
     draws 0-3 are independent, so one block (ten dependent rounds) is on
     the path;
  2. dispersal from those draws: non-spatial, one 64-bit high product; torus,
     one table lookup (shared memory) per axis, side by side, and the
     wrap-around add; habitat map, the column (a 32-bit high product), the
     alias entry (its cell is known one event before its column: the
     cheaper of the row copy's measured latency beyond what the next search
     and event's Philox block cover, and a dependent DRAM load), the
     take-or-alias choice, the offset-table read and the wrap-around add;
  3. the next event time at the new location after the event time: the
     interval's index is known before the move, so the interval block's
     first product is off the path; nine rounds and the key's xor remain.
     Sums of exponentials: the draws' logarithms run side by side (one
     logarithm on the path: normalise, table read, 32x64 product, two 64-bit
     high products, six 64-bit adds), then about three dependent add-and-
     compare steps (the running sum to the first point after the last
     event, at lambda dt = 1 on average 2.7 draws) and the final select.
     Poisson points: the count's table read and compare, then one add and a
     minimum over the interval's few points (two add-compare-select steps).

Every figure is a latency of this GPU measured here, so the floor is
hardware-derived: it does not move when the library's kernels change.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chain_latency.cu")
_LIB = os.path.join(_HERE, "_build", "libhwlat.so")

CLASSES = {"imad_hi": 0, "hi_xor": 1, "umul64hi": 2, "imad_wide": 3, "add64_sel": 4, "clz_norm": 5,
           "add_xor": 6, "ballot": 8, "redux_min": 9, "philox_round": 10, "lds": 11, "philox_round_split": 12,
           "philox_round_m1": 13, "shfl_add": 14}


def build(force=False):
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.run([nvcc if os.path.exists(nvcc) else "nvcc", "-std=c++17", "-O3", "-lineinfo",
                        "-gencode", "arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC", "-shared",
                        _SRC, "-o", tmp], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.hwlat_steps.restype = ctypes.c_int
        L.hwlat_run.restype = ctypes.c_longlong
        L.hwlat_run.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        L.hwlat_ring.restype = ctypes.c_longlong
        L.hwlat_ring.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        L.hwlat_bulk_row.restype = ctypes.c_longlong
        L.hwlat_bulk_row.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_int, ctypes.c_void_p]
        L.hwlat_clock_mhz.restype = ctypes.c_double
        L.hwlat_clock_mhz.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p]
        L.hwlat_philox_throughput.restype = ctypes.c_double
        L.hwlat_philox_throughput.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p]
        _lib = L
    return _lib


def _ring(torch, n, seed):
    """a random cyclic permutation of n entries (every hop stays below n)"""
    perm = np.random.default_rng(seed).permutation(n).astype(np.uint32)
    ring = np.empty(n, dtype=np.uint32)
    ring[perm] = np.roll(perm, -1)
    return torch.from_numpy(ring).cuda(), int(perm[0])


def measure(reps=3, dram_ring_mib=512, dram_steps=4000):
    """cycles per dependent step of every class (best of `reps`), dependent
    global-load latencies (L1 hit; L2 miss to DRAM over a ring larger than
    L2), the SM clock in MHz during the run, and the integer throughput of
    the Philox mix on all SMs in Tops/s (philox_tput_tops)"""
    import torch
    L = lib()
    steps = L.hwlat_steps()
    prm = torch.tensor([0x9E3779B97F4A7C15, 0xF39CC0605CEDC834, 0x1082276BF3A27251, 0xFFFFFFFF,
                        0x5BD1E995, 0x2545F4914F6CDD1D], dtype=torch.uint64, device="cuda")
    out = torch.zeros(2, dtype=torch.uint64, device="cuda")
    res = {}
    for name, cls in CLASSES.items():
        best = None
        for _ in range(reps):
            c = L.hwlat_run(cls, ctypes.c_void_p(prm.data_ptr()), ctypes.c_void_p(out.data_ptr()))
            if c < 0:
                raise RuntimeError("latency chain %s failed: CUDA error %d" % (name, -c))
            best = c if best is None else min(best, c)
        res[name] = best / steps
    # dependent global loads: a 4 KB ring (L1-resident after one pass) and a
    # ring of dram_ring_mib MiB (random hops: L2 misses)
    small, s0 = _ring(torch, 1024, 1)
    L.hwlat_ring(ctypes.c_void_p(small.data_ptr()), s0, 2048, 1, ctypes.c_void_p(out.data_ptr()))
    c = L.hwlat_ring(ctypes.c_void_p(small.data_ptr()), s0, 2048, 1, ctypes.c_void_p(out.data_ptr()))
    res["ldg_l1"] = c / 2048
    n = (dram_ring_mib << 20) // 4
    big, b0 = _ring(torch, n, 2)
    c = L.hwlat_ring(ctypes.c_void_p(big.data_ptr()), b0, dram_steps, 0, ctypes.c_void_p(out.data_ptr()))
    res["ldg_dram"] = c / dram_steps
    del big
    # the map row's bulk copy: 6,384 bytes (a 797-entry row from its 16-byte
    # boundary) from random rows of a buffer larger than L2, whole or in
    # 4, 8 or 31 pieces issued side by side; the fastest is the row's latency
    stride = ROW_BYTES
    rows = (dram_ring_mib << 20) // stride
    buf = torch.zeros(rows * stride, dtype=torch.uint8, device="cuda")
    for pieces, piece in ((1, 6384), (4, 1600), (8, 800), (31, 208)):
        c = L.hwlat_bulk_row(ctypes.c_void_p(buf.data_ptr()), rows, stride, ROW_BYTES, piece, 1000,
                             ctypes.c_void_p(out.data_ptr()))
        if c < 0:
            raise RuntimeError("bulk row copy probe failed (%d)" % c)
        res["bulk_row_%d" % pieces] = c / 1000
    res["bulk_row"] = min(res["bulk_row_%d" % k] for k in (1, 4, 8, 31))
    del buf
    res["clock_mhz"] = L.hwlat_clock_mhz(200_000_000, ctypes.c_void_p(out.data_ptr()))
    # integer throughput of the library's op mix on every SM: independent
    # Philox4x32-10 blocks, 100 integer ops each (best of `reps`)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    best = 0.0
    for _ in range(reps):
        v = L.hwlat_philox_throughput(sms, 8, 256, ctypes.c_void_p(out.data_ptr()))
        if v < 0:
            raise RuntimeError("Philox throughput kernel failed: CUDA error %d" % int(-v))
        best = max(best, v)
    res["philox_tput_tops"] = best / 1e12
    res["steps_per_chain"] = steps
    return res


ROW_BYTES = 6384  # an alias row of 797 entries, copied from its 16-byte boundary


def derived(lat):
    """latencies of the path's compound steps, in cycles"""
    philox = 10.0 * min(lat["philox_round"], lat["philox_round_split"], lat["philox_round_m1"])
    add64 = lat["add_xor"]           # two dependent 32-bit adds (the carry), costed as add + xor
    log = lat["clz_norm"] + lat["lds"] + lat["imad_wide"] + 2.0 * lat["umul64hi"] + 6.0 * add64
    return dict(philox_block=philox, add64=add64, logarithm=log, add_cmp_sel=lat["add64_sel"],
                interval_block=philox - lat["imad_hi"])


def event_floor(lat, sampler="exp", kind="torus", memory=True):
    """cycles of one event on the critical path (see the module docstring);
    memory=False leaves out the map row's fetch latency (the compute-only
    floor)"""
    d = derived(lat)
    event = d["philox_block"]
    if kind == "nonspatial":
        move = lat["umul64hi"]
    elif kind == "torus":
        move = lat["lds"] + d["add_cmp_sel"]
    elif kind == "map":
        move = lat["imad_hi"] + lat["lds"] + d["add_cmp_sel"] + lat["lds"] + d["add_cmp_sel"]
    else:
        raise ValueError(kind)
    if sampler == "exp":
        search = d["interval_block"] + d["logarithm"] + 3.0 * d["add_cmp_sel"] + d["add_cmp_sel"]
    else:
        search = d["interval_block"] + lat["lds"] + d["add_cmp_sel"] + 2.0 * d["add_cmp_sel"]
    wait = 0.0
    if kind == "map" and memory and "bulk_row" in lat:
        # The entry's cell is known after a move, its column only after the
        # next event's draws.  Either the row is fetched whole when the cell
        # is known (read after the next search and event's Philox block:
        # whatever of the copy's latency those do not cover is on the path),
        # or the entry alone once the column is known (a dependent DRAM load,
        # all of it on the path); the cheaper of the two.
        wait = min(lat["ldg_dram"], max(0.0, lat["bulk_row"] - (search + event)))
    return event + move + search + wait
