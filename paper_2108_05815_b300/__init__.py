"""Python binding of libindep.so -- argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels (sm_103a);
this module converts arguments, passes torch's current CUDA stream, and
routes the library's device allocations to torch's caching allocator.  If the
native library is missing it raises; there is no fallback.

Names follow the C ABI in include/indep.h: ``Simulation`` wraps
sim_create / sim_sample / sim_run / sim_species / sim_species_keys /
sim_destroy, ``batch_run`` wraps sim_batch_run, ``habitat`` wraps
ind_habitat and ``mem_estimate`` wraps sim_mem_estimate.
"""
import ctypes
import os
import threading

import numpy as np

NONSPATIAL, TORUS, MAP, IMPLICIT = 0, 1, 2, 3
SAMPLER_EXP, SAMPLER_POISSON = 0, 1
PARTITION_LANDSCAPE, PARTITION_INDIVIDUALS = 0, 1
DISPERSAL_UNIFORM, DISPERSAL_GAUSSIAN, DISPERSAL_ALIAS_GAUSSIAN = 0, 1, 2

STATUS = {0: "IND_OK", -1: "IND_ERR_ARG", -2: "IND_ERR_OOM", -3: "IND_ERR_CUDA", -4: "IND_ERR_BUDGET",
          -5: "IND_ERR_STATE", -6: "IND_ERR_DEVICE"}
IND_OK, IND_ERR_BUDGET = 0, -4

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libindep.so")


class IndError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (cuda error %d)" % (what, STATUS.get(status, status),
                                                            lib().ind_last_cuda_error()))


class Landscape(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("deme", ctypes.c_uint32), ("deme_map", ctypes.c_void_p), ("lambda_", ctypes.c_double),
                ("delta_t", ctypes.c_double), ("event_sampler", ctypes.c_int32),
                ("migration", ctypes.c_double), ("meta_size", ctypes.c_uint64), ("meta_nu", ctypes.c_double)]


class Dispersal(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sigma", ctypes.c_double), ("radius", ctypes.c_uint32)]


class RunStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("rounds", "raw_events", "unique_events", "culled", "n_sampled",
                                               "n_species", "n_roots")] + \
               [("ms_total", ctypes.c_double), ("advance_ms", ctypes.c_double),
                ("advance_launches", ctypes.c_uint64), ("busiest_launch_ms", ctypes.c_double),
                ("busiest_launch_events", ctypes.c_uint64), ("critical_events", ctypes.c_uint64),
                ("dedup_inserts", ctypes.c_uint64), ("dedup_repeats", ctypes.c_uint64),
                ("dedup_warp_repeats", ctypes.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("block_threads", "blocks_per_sm", "lineages_per_lane",
                                               "rounds_per_check", "use_graph", "dedup", "count_unique",
                                               "profile", "events_per_visit", "coop_lineages",
                                               "advance_variant", "reserved")] + \
               [("events_per_round", ctypes.c_double), ("min_events_per_lineage", ctypes.c_double),
                ("occupancy_step", ctypes.c_double), ("tail_events", ctypes.c_double),
                ("busy_lineages", ctypes.c_double), ("max_step_events", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_RELEASE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC), ("release", _RELEASE), ("ctx", ctypes.c_void_p)]


# ind_event / ind_coalescence
EVENT_DTYPE = np.dtype([("time_bits", "<u8"), ("prior_bits", "<u8"), ("loc", "<u8"), ("target", "<u8"),
                        ("lineage", "<u4"), ("reserved", "<u4")])
COALESCENCE_DTYPE = np.dtype([("loc", "<u8"), ("time_bits", "<u8"), ("parent", "<u4"), ("child", "<u4")])
SPECIATION = 0xFFFFFFFFFFFFFFFF

EXPORTS = {
    "ind_set_allocator": (ctypes.c_int, [ctypes.c_void_p]),
    "ind_default_tuning": (None, [ctypes.c_void_p]),
    "sim_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_void_p]),
    "sim_sample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p]),
    "sim_sample_partition": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint32,
                                            ctypes.c_uint32, ctypes.c_int32, ctypes.c_void_p]),
    "ind_keys_unique": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ind_keys_rank": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "sim_species": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_species_keys": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sim_mem_estimate": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "sim_destroy": (None, [ctypes.c_void_p]),
    "sim_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "sim_set_event_log": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "sim_events": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "ind_habitat": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double,
                                   ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
    "ind_selftest": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "sim_selftest_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_uint64, ctypes.c_void_p]),
    "sim_alias_row": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                     ctypes.c_uint32, ctypes.c_void_p]),
    "ind_species_rank_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
    "srv_create": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
    "srv_default_tuning": (None, [ctypes.c_void_p]),
    "srv_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "srv_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
                                ctypes.c_void_p]),
    "srv_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "srv_destroy": (None, [ctypes.c_void_p]),
    "ind_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ind_last_cuda_error": (ctypes.c_int, []),
    "ind_kernel_launches": (ctypes.c_uint64, []),
}

_lock = threading.Lock()
_lib = None
_torch_alloc = None


def lib():
    """the loaded native library (raises if it has not been built)"""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("native library %s is missing; build it with "
                                   "`python -m paper_2108_05815_b300.build`" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in EXPORTS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(status, what):
    if status != IND_OK:
        raise IndError(status, what)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the simulation runs only on the GPU")
    return torch


def use_torch_allocator():
    """route the library's device allocations to torch's caching allocator"""
    global _torch_alloc
    torch = _torch()
    if _torch_alloc is not None:
        return

    def _a(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _r(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a = Allocator(_ALLOC(_a), _RELEASE(_r), None)
    _check(lib().ind_set_allocator(ctypes.byref(a)), "ind_set_allocator")
    _torch_alloc = a


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def default_tuning():
    t = Tuning()
    lib().ind_default_tuning(ctypes.byref(t))
    return t.as_dict()


def _tuning(kw, server=False):
    t = Tuning()
    (lib().srv_default_tuning if server else lib().ind_default_tuning)(ctypes.byref(t))
    for k, v in (kw or {}).items():
        setattr(t, k, v)
    return t


def server_default_tuning():
    """srv_default_tuning as a dict"""
    return _tuning(None, server=True).as_dict()


_DISPERSAL_OF = {NONSPATIAL: DISPERSAL_UNIFORM, TORUS: DISPERSAL_GAUSSIAN, MAP: DISPERSAL_ALIAS_GAUSSIAN,
                 IMPLICIT: DISPERSAL_UNIFORM}


def landscape(kind, width=1, height=1, deme=1, deme_map=None, lam=1.0, delta_t=1.0, sampler=0,
              migration=0.0, meta_size=0, meta_nu=0.0):
    L = Landscape()
    L.kind, L.width, L.height, L.deme, L.lambda_, L.delta_t = kind, width, height, deme, lam, delta_t
    L.event_sampler = sampler
    L.migration, L.meta_size, L.meta_nu = float(migration), int(meta_size), float(meta_nu)
    keep = None
    if deme_map is not None:
        if hasattr(deme_map, "data_ptr"):
            keep = deme_map.contiguous()
            L.deme_map = keep.data_ptr()
        else:
            keep = np.ascontiguousarray(deme_map, dtype=np.uint8)
            L.deme_map = keep.ctypes.data
    return L, keep


def dispersal(kind, sigma=0.0, radius=0):
    D = Dispersal()
    D.kind, D.sigma, D.radius = kind, sigma, radius
    return D


class Simulation:
    """One simulation (sim_create ... sim_destroy)."""

    def __init__(self, kind, nu, seed, width=1, height=1, deme=1, sigma=0.0, radius=0, deme_map=None,
                 lam=1.0, delta_t=1.0, stream=None, tuning=None, sampler=0, migration=0.0, meta_size=0,
                 meta_nu=0.0):
        use_torch_allocator()
        L, keep = landscape(kind, width, height, deme, deme_map, lam, delta_t, sampler, migration, meta_size,
                            meta_nu)
        dk = _DISPERSAL_OF[kind]
        D = dispersal(dk, sigma, radius)
        self._h = ctypes.c_void_p()
        self._stream = _stream(stream)
        _check(lib().sim_create(ctypes.byref(L), ctypes.byref(D), float(nu), int(seed), self._stream,
                                ctypes.byref(self._h)), "sim_create")
        del keep
        self.kind, self.nu, self.seed = kind, nu, seed
        self.n_sampled = 0
        if tuning:
            self.set_tuning(**tuning)

    def close(self):
        if self._h:
            lib().sim_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, **kw):
        t = _tuning(kw)
        _check(lib().sim_set_tuning(self._h, ctypes.byref(t)), "sim_set_tuning")

    def sample(self, fraction=1.0, sample_seed=0):
        n = ctypes.c_uint64(0)
        _check(lib().sim_sample(self._h, float(fraction), int(sample_seed), ctypes.byref(n)), "sim_sample")
        self.n_sampled = int(n.value)
        return self.n_sampled

    def sample_partition(self, part, n_parts, scheme=PARTITION_LANDSCAPE, fraction=1.0, sample_seed=0):
        """sim_sample_partition: only part `part` of n_parts of the sample"""
        n = ctypes.c_uint64(0)
        _check(lib().sim_sample_partition(self._h, float(fraction), int(sample_seed), int(part), int(n_parts),
                                          int(scheme), ctypes.byref(n)), "sim_sample_partition")
        self.n_sampled = int(n.value)
        return self.n_sampled

    def run(self, round_budget=0):
        """run until finished (True) or the round budget is used (False)"""
        st = RunStats()
        s = lib().sim_run(self._h, int(round_budget), ctypes.byref(st))
        if s == IND_ERR_BUDGET:
            return False
        _check(s, "sim_run")
        return True

    def stats(self):
        st = RunStats()
        _check(lib().sim_stats(self._h, ctypes.byref(st)), "sim_stats")
        return st.as_dict()

    def species(self, out=None):
        """(species ids as a uint64 numpy array or into `out` (tensor/array), n_species)"""
        n = ctypes.c_uint64(0)
        if out is None:
            out = np.zeros(self.n_sampled, dtype=np.uint64)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        _check(lib().sim_species(self._h, ctypes.c_void_p(ptr), ctypes.byref(n)), "sim_species")
        return out, int(n.value)

    def set_event_log(self, capacity):
        """log the events of the next run (capacity in raw events; 0: off)"""
        _check(lib().sim_set_event_log(self._h, int(capacity)), "sim_set_event_log")

    def events(self):
        """after a logged run: (events, coalescences) as numpy structured arrays
        (EVENT_DTYPE in (time, location) order, COALESCENCE_DTYPE)"""
        ne, nc = ctypes.c_uint64(0), ctypes.c_uint64(0)
        _check(lib().sim_events(self._h, None, 0, ctypes.byref(ne), None, 0, ctypes.byref(nc)), "sim_events")
        ev = np.zeros(ne.value, dtype=EVENT_DTYPE)
        co = np.zeros(nc.value, dtype=COALESCENCE_DTYPE)
        _check(lib().sim_events(self._h, ctypes.c_void_p(ev.ctypes.data), ne.value, None,
                                ctypes.c_void_p(co.ctypes.data), nc.value, None), "sim_events")
        return ev, co

    def selftest_search(self, form, locs, taus):
        """device probe (sim_selftest_search): the first event time after each
        taus[i] at locs[i] by search form 0..5, float64 numpy array"""
        lv = np.ascontiguousarray(locs, dtype=np.uint64)
        tv = np.ascontiguousarray(taus, dtype=np.float64)
        assert lv.shape == tv.shape
        out = np.zeros(lv.size, dtype=np.float64)
        _check(lib().sim_selftest_search(self._h, int(form), ctypes.c_void_p(lv.ctypes.data),
                                         ctypes.c_void_p(tv.ctypes.data), lv.size, ctypes.c_void_p(out.ctypes.data)),
               "sim_selftest_search")
        return out

    def alias_row(self, x, y):
        """the device's alias row of habitable cell (x, y) of a map simulation
        (sim_alias_row): packed uint64 entries, one per dispersal offset"""
        n = ctypes.c_uint32(0)
        _check(lib().sim_alias_row(self._h, int(x), int(y), None, 0, ctypes.byref(n)), "sim_alias_row")
        out = np.zeros(n.value, dtype=np.uint64)
        _check(lib().sim_alias_row(self._h, int(x), int(y), ctypes.c_void_p(out.ctypes.data), n.value,
                                   ctypes.byref(n)), "sim_alias_row")
        return out

    def species_keys(self, device=False):
        """(speciation location, time bits) per sampled individual, uint64
        numpy arrays (device=True: device tensors)"""
        if device:
            torch = _torch()
            kl = torch.empty(max(self.n_sampled, 1), dtype=torch.uint64, device="cuda")
            kt = torch.empty(max(self.n_sampled, 1), dtype=torch.uint64, device="cuda")
            _check(lib().sim_species_keys(self._h, ctypes.c_void_p(kl.data_ptr()), ctypes.c_void_p(kt.data_ptr())),
                   "sim_species_keys")
            return kl[:self.n_sampled], kt[:self.n_sampled]
        kl = np.zeros(self.n_sampled, dtype=np.uint64)
        kt = np.zeros(self.n_sampled, dtype=np.uint64)
        _check(lib().sim_species_keys(self._h, ctypes.c_void_p(kl.ctypes.data), ctypes.c_void_p(kt.ctypes.data)),
               "sim_species_keys")
        return kl, kt


def batch_run(sims, **tuning):
    """sim_batch_run over sampled Simulations; returns per-simulation stats"""
    arr = (ctypes.c_void_p * len(sims))(*[s._h.value for s in sims])
    stats = (RunStats * len(sims))()
    t = _tuning(tuning) if tuning else None
    _check(lib().sim_batch_run(arr, len(sims), ctypes.byref(t) if t else None, stats), "sim_batch_run")
    return [s.as_dict() for s in stats]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "finished", "queued", "resident",
                                               "resident_lineages", "bytes_admitted", "rounds", "raw_events",
                                               "lineage_capacity")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Server:
    """Continuous-batching server (srv_create / srv_submit / srv_step / srv_destroy)."""

    def __init__(self, hbm_budget, max_sims=1024, stream=None, **tuning):
        use_torch_allocator()
        self._h = ctypes.c_void_p()
        t = _tuning(tuning, server=True) if tuning else None
        _check(lib().srv_create(int(hbm_budget), int(max_sims), ctypes.byref(t) if t else None, _stream(stream),
                                ctypes.byref(self._h)), "srv_create")
        self._fin = (ctypes.c_uint64 * 4096)()

    def submit(self, sim):
        t = ctypes.c_uint64(0)
        _check(lib().srv_submit(self._h, sim._h, ctypes.byref(t)), "srv_submit")
        return int(t.value)

    def step(self, rounds=8):
        """admit, run `rounds` horizon rounds, retire; returns finished tickets"""
        n = ctypes.c_uint32(0)
        _check(lib().srv_step(self._h, int(rounds), self._fin, len(self._fin), ctypes.byref(n)), "srv_step")
        return [int(self._fin[i]) for i in range(n.value)]

    def stats(self):
        st = ServerStats()
        _check(lib().srv_stats(self._h, ctypes.byref(st)), "srv_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            lib().srv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def habitat(map_seed, width, height, p_habitable=0.6, max_deme=8, out=None, stream=None):
    """synthetic percolation habitat (ind_habitat) into a uint8 numpy array or tensor"""
    if out is None:
        out = np.zeros(width * height, dtype=np.uint8)
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check(lib().ind_habitat(int(map_seed), width, height, float(p_habitable), max_deme, ctypes.c_void_p(ptr),
                             _stream(stream)), "ind_habitat")
    return out


def mem_estimate(kind, width=1, height=1, deme=1, sigma=0.0, radius=0, fraction=1.0, lam=1.0, delta_t=1.0,
                 migration=0.0, meta_size=1, meta_nu=1.0):
    dk = _DISPERSAL_OF[kind]
    L, _ = landscape(kind, width, height, deme, np.ones(1, np.uint8) if kind == MAP else None, lam, delta_t, 0,
                     migration, meta_size, meta_nu)
    D = dispersal(dk, sigma, radius)
    return int(lib().sim_mem_estimate(ctypes.byref(L), ctypes.byref(D), float(fraction)))


def selftest(values, want_exp=True, want_philox=True, stream=None):
    """device probe (ind_selftest): (exp_q58 uint64[n] or None, philox uint32[n, 4] or None)"""
    v = np.ascontiguousarray(values, dtype=np.uint64)
    n = v.size
    e = np.zeros(n, dtype=np.uint64) if want_exp else None
    p = np.zeros((n, 4), dtype=np.uint32) if want_philox else None
    _check(lib().ind_selftest(ctypes.c_void_p(v.ctypes.data), n,
                              ctypes.c_void_p(e.ctypes.data) if e is not None else None,
                              ctypes.c_void_p(p.ctypes.data) if p is not None else None, _stream(stream)),
           "ind_selftest")
    return e, p


def species_rank_static(key_loc, key_time, out, stream=None):
    """ind_species_rank_static: dense species ids of device key tensors into the
    device tensor `out` (nothing is allocated); returns the species count"""
    n = ctypes.c_uint64(0)
    _check(lib().ind_species_rank_static(ctypes.c_void_p(key_loc.data_ptr()), ctypes.c_void_p(key_time.data_ptr()),
                                         int(key_loc.numel()), ctypes.c_void_p(out.data_ptr()), ctypes.byref(n),
                                         _stream(stream)), "ind_species_rank_static")
    return int(n.value)


def keys_unique(key_loc, key_time, stream=None):
    """ind_keys_unique: the sorted distinct (location, time bits) keys of two
    device uint64 tensors, as two new device tensors"""
    torch = _torch()
    n = int(key_loc.numel())
    ol = torch.empty(max(n, 1), dtype=torch.uint64, device=key_loc.device)
    ot = torch.empty(max(n, 1), dtype=torch.uint64, device=key_loc.device)
    k = ctypes.c_uint64(0)
    _check(lib().ind_keys_unique(ctypes.c_void_p(key_loc.data_ptr()), ctypes.c_void_p(key_time.data_ptr()), n,
                                 ctypes.c_void_p(ol.data_ptr()), ctypes.c_void_p(ot.data_ptr()), ctypes.byref(k),
                                 _stream(stream)), "ind_keys_unique")
    return ol[:k.value], ot[:k.value]


def keys_rank(key_loc, key_time, ref_loc, ref_time, stream=None):
    """ind_keys_rank: each key's index among the sorted distinct reference
    keys (device tensors), as a device uint64 tensor"""
    torch = _torch()
    n = int(key_loc.numel())
    out = torch.empty(max(n, 1), dtype=torch.uint64, device=key_loc.device)
    _check(lib().ind_keys_rank(ctypes.c_void_p(key_loc.data_ptr()), ctypes.c_void_p(key_time.data_ptr()), n,
                               ctypes.c_void_p(ref_loc.data_ptr()), ctypes.c_void_p(ref_time.data_ptr()),
                               int(ref_loc.numel()), ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "ind_keys_rank")
    return out[:n]


def kernel_launches():
    return int(lib().ind_kernel_launches())
