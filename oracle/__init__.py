"""Plain CPU oracle of the Independent algorithm -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code, header, table or
helper with the CUDA library in ``paper_2108_05815_b300``; the library never
imports it, and it never imports the library.

The arithmetic lives in ``oracle.c`` (plain C, binary64, built with
``-ffp-contract=off``); the integer tables come from ``tables.py``
(arbitrary precision).  This module only marshals arguments and resolves the
per-individual speciation keys into dense species identities (species =
distinct speciation event, ranked by ascending (location, time bits); the
paper counts species as distinct speciation events, section "A Neutral
Coalescence-based Simulation").

Parity status of each function is recorded in its docstring.  The spatial
models (torus, habitat map) have no closed form in the paper; they are
pinned by mode P == mode M, by the per-step distribution tests and by the
special cases, not against a printed value.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

from . import tables

NONSPATIAL, TORUS, MAP, IMPLICIT = 0, 1, 2, 3
TAG_INTERVAL, TAG_EVENT, TAG_MAP, TAG_SAMPLE = 1, 2, 3, 4

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """compile oracle.c into oracle/_build/liboracle.so (gcc, binary64, no FMA contraction)"""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _LnTables(ctypes.Structure):
    _fields_ = [("ln_tab", ctypes.c_uint64 * (1 << tables.LN_TABLE_BITS)), ("ln2_q64", ctypes.c_uint64),
                ("c3", ctypes.c_int64)]


class _EventLog(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_uint64), ("n", ctypes.c_uint64), ("time_bits", ctypes.c_void_p),
                ("prior_bits", ctypes.c_void_p), ("loc", ctypes.c_void_p), ("target", ctypes.c_void_p),
                ("lineage", ctypes.c_void_p), ("co_cap", ctypes.c_uint64), ("n_co", ctypes.c_uint64),
                ("co_loc", ctypes.c_void_p), ("co_time_bits", ctypes.c_void_p), ("co_parent", ctypes.c_void_p),
                ("co_child", ctypes.c_void_p)]


class _Model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("deme", ctypes.c_uint32), ("deme_map", ctypes.c_void_p),
                ("lambda_", ctypes.c_double), ("delta_t", ctypes.c_double), ("nu", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("gauss_half", ctypes.c_int32),
                ("gauss_cdf", ctypes.c_void_p), ("radius", ctypes.c_int32),
                ("kw", ctypes.c_void_p), ("ln", ctypes.c_void_p), ("sampler", ctypes.c_int32),
                ("pois_n", ctypes.c_int32), ("pois_cdf", ctypes.c_void_p),
                ("migration", ctypes.c_double), ("meta_size", ctypes.c_uint64), ("meta_nu", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_void_p)
            sig = {
                "or_philox4x32_10": (None, [vp, vp, vp]),
                "or_seed_key": (None, [u64, vp]),
                "or_draw_pair": (None, [vp, u64, u64, u32, u32, vp]),
                "or_draw": (u64, [vp, u64, u64, u32, u32]),
                "or_ln_recip": (u32, [u32]),
                "or_exp1_q58": (u64, [u64, vp]),
                "or_exp1": (dbl, [u64, vp]),
                "or_trace": (ctypes.c_int, [vp, u64, u64, vp, vp, vp]),
                "or_trace_many": (ctypes.c_int, [vp, vp, u64, u64, vp, vp, vp]),
                "or_max_threads": (ctypes.c_int, []),
                "or_run_merge": (ctypes.c_int, [vp, vp, u64, u64, vp, vp, vp]),
                "or_run_merge_events": (ctypes.c_int, [vp, vp, u64, u64, vp, vp, vp, vp]),
                "or_run_merge_longest": (ctypes.c_int, [vp, vp, u64, u64, vp, vp, vp, vp]),
                "or_habitat": (None, [u64, u32, u32, dbl, u32, vp]),
                "or_sample": (u64, [vp, dbl, u64, vp]),
                "or_gauss_offset": (u64, [vp, u64]),
                "or_next_event_time": (dbl, [vp, u64, dbl]),
                "or_disperse": (u64, [vp, u64, dbl]),
                "or_speciates": (ctypes.c_int, [vp, u64, dbl]),
                "or_alias_row_dump": (u32, [vp, u32, u32, vp, vp, vp, vp, vp]),
                "or_trace_log": (ctypes.c_int64, [vp, u64, u64, vp, vp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def max_threads():
    """threads a mode-P trace over many lineages may use (OpenMP's default)"""
    return int(lib().or_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


_ln_struct = None


def _ln():
    global _ln_struct
    if _ln_struct is None:
        tab, ln2, c3, _ = tables.ln_tables()
        s = _LnTables()
        for j, v in enumerate(tab):
            s.ln_tab[j] = v
        s.ln2_q64 = ln2
        s.c3 = c3
        _ln_struct = s
    return _ln_struct


# --------------------------------------------------------------------------
# RNG and per-step building blocks
# --------------------------------------------------------------------------
def philox4x32_10(key, ctr):
    """Philox4x32-10 block (Salmon et al. 2011); key: 2 x u32, ctr: 4 x u32.
    Pinned by the published known-answer vectors (tests/golden/philox_kat.txt)."""
    k = np.array(key, dtype=np.uint32)
    c = np.array(ctr, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(k), _ptr(c), _ptr(out))
    return [int(x) for x in out]


def seed_key(seed):
    sk = np.zeros(2, dtype=np.uint32)
    lib().or_seed_key(seed, _ptr(sk))
    return sk


def draw(seed, loc, tkey, tag, idx):
    """the idx-th 64-bit draw of the stream primed at (seed, loc, tkey, tag)"""
    return int(lib().or_draw(_ptr(seed_key(seed)), loc, tkey, tag, idx))


def exp1(draw_u64):
    """Exp(1) = -ln U of the top 53 bits of a 64-bit draw, U = (r + 1) 2^-53.
    Pinned against the exact logarithm (mpmath) within 2^-57 plus half an ulp."""
    return lib().or_exp1(int(draw_u64), ctypes.byref(_ln()))


def exp1_q58(r53):
    """X58(r53): the frozen fixed-point definition of -ln((r53 + 1) 2^-53) in
    units of 2^-58 (stated plainly in ln_definition.py, equal to it on every
    bucket edge of every binade)"""
    return int(lib().or_exp1_q58(int(r53), ctypes.byref(_ln())))


def pack_loc(x, y, i):
    return int(x) | (int(y) << 20) | (int(i) << 40)


def unpack_loc(loc):
    loc = int(loc)
    return loc & 0xFFFFF, (loc >> 20) & 0xFFFFF, loc >> 40


def habitat(map_seed, width, height, p_habitable=0.6, max_deme=8):
    """seeded site-percolation map of demes (0 = not habitable), row-major"""
    out = np.zeros(width * height, dtype=np.uint8)
    lib().or_habitat(map_seed, width, height, p_habitable, max_deme, _ptr(out))
    return out


class Model:
    """One simulation of the Independent algorithm.

    sampler: 0 = inter-event times as sums of exponentials inside re-prime
    intervals (section "Memoryless sums of exponentials"), 1 = Poisson point
    counts with uniform points per interval (section "Homogeneous Poisson
    Point Process").
    kind: NONSPATIAL (width = height = 1, deme = J), TORUS (width x height
    cells of ``deme`` individuals, discretised N(0, sigma^2) dispersal per
    axis) or MAP (deme_map of demes, dispersal by a per-cell alias table over
    the disk of ``radius`` with Gaussian weights of ``sigma`` times the target
    deme, torus-wrapped) or IMPLICIT (the spatially implicit scenario: a
    local community of J = deme individuals, non-spatial, whose parent lives
    with probability ``migration`` per event in a static non-spatial
    metacommunity of ``meta_size`` individuals with speciation probability
    ``meta_nu``; nu is the local speciation probability and may be 0)."""

    def __init__(self, kind, width, height, deme, nu, seed, lam=1.0, delta_t=1.0,
                 sigma=None, radius=None, deme_map=None, sampler=0, migration=0.0, meta_size=0, meta_nu=0.0):
        self.kind, self.width, self.height = kind, int(width), int(height)
        self.nu, self.seed, self.lam, self.delta_t = float(nu), int(seed), float(lam), float(delta_t)
        self._keep = []
        m = _Model()
        m.kind, m.width, m.height = kind, self.width, self.height
        m.lambda_, m.delta_t, m.nu, m.seed = self.lam, self.delta_t, self.nu, self.seed
        m.ln = ctypes.cast(ctypes.pointer(_ln()), ctypes.c_void_p)
        if kind == MAP:
            dm = np.ascontiguousarray(deme_map, dtype=np.uint8)
            assert dm.size == self.width * self.height
            self._keep.append(dm)
            m.deme_map = dm.ctypes.data
            m.deme = int(dm.max())
            kw, _ = tables.kernel_weights(sigma, radius)
            kwa = np.array(kw, dtype=np.uint64)
            self._keep.append(kwa)
            m.kw = kwa.ctypes.data
            m.radius = int(radius)
        else:
            m.deme = int(deme)
        if kind == TORUS:
            cdf, half, _ = tables.gauss_cdf(sigma)
            ca = np.array(cdf, dtype=np.uint64)
            self._keep.append(ca)
            m.gauss_cdf = ca.ctypes.data
            m.gauss_half = half
        if kind == IMPLICIT:
            assert self.width == 1 and self.height == 1 and 1 <= int(meta_size) <= (1 << 31)
            m.migration, m.meta_size, m.meta_nu = float(migration), int(meta_size), float(meta_nu)
        m.sampler = int(sampler)
        if sampler == 1:
            cdf, _ = tables.poisson_cdf(self.lam * self.delta_t)
            pa = np.array(cdf, dtype=np.uint64)
            self._keep.append(pa)
            m.pois_cdf = pa.ctypes.data
            m.pois_n = len(cdf)
        self.deme = m.deme
        self._m = m

    @property
    def _mp(self):
        return ctypes.byref(self._m)

    def sample(self, fraction=1.0, sample_seed=0):
        """locations of the sampled individuals in (cell row-major, deme index) order"""
        n = lib().or_sample(self._mp, fraction, sample_seed, None)
        out = np.zeros(n, dtype=np.uint64)
        lib().or_sample(self._mp, fraction, sample_seed, _ptr(out))
        return out

    def trace(self, locs, max_events=1 << 40, partial=False):
        """Mode P: (key_loc, key_time_bits, n_events) per starting location.
        partial: a lineage may stop after max_events events without having
        speciated (its key is then undefined and its count is max_events)."""
        locs = np.ascontiguousarray(locs, dtype=np.uint64)
        n = locs.size
        kl = np.zeros(n, dtype=np.uint64)
        kt = np.zeros(n, dtype=np.uint64)
        ne = np.zeros(n, dtype=np.uint64)
        st = lib().or_trace_many(self._mp, _ptr(locs), n, max_events, _ptr(kl), _ptr(kt), _ptr(ne))
        if st != 0 and not (partial and st == -1):
            raise RuntimeError("oracle trace failed with status %d" % st)
        return kl, kt, ne

    def run_merge(self, locs, max_events=1 << 40):
        """Mode M: (key_loc, key_time_bits, n_unique_events)."""
        locs = np.ascontiguousarray(locs, dtype=np.uint64)
        n = locs.size
        kl = np.zeros(n, dtype=np.uint64)
        kt = np.zeros(n, dtype=np.uint64)
        nu = ctypes.c_uint64(0)
        st = lib().or_run_merge(self._mp, _ptr(locs), n, max_events, _ptr(kl), _ptr(kt),
                                ctypes.byref(nu))
        if st != 0:
            raise RuntimeError("oracle merge run failed with status %d" % st)
        return kl, kt, int(nu.value)

    def run_merge_longest(self, locs, max_events=1 << 40):
        """Mode M plus the longest line of descent: (key_loc, key_time_bits,
        n_unique_events, longest), longest = the most events any one sampled
        individual's lineage runs before it speciates (the longest mode-P
        trace, found without tracing every lineage alone)."""
        locs = np.ascontiguousarray(locs, dtype=np.uint64)
        n = locs.size
        kl = np.zeros(n, dtype=np.uint64)
        kt = np.zeros(n, dtype=np.uint64)
        nu = ctypes.c_uint64(0)
        lg = ctypes.c_uint64(0)
        st = lib().or_run_merge_longest(self._mp, _ptr(locs), n, max_events, _ptr(kl), _ptr(kt),
                                        ctypes.byref(nu), ctypes.byref(lg))
        if st != 0:
            raise RuntimeError("oracle merge run failed with status %d" % st)
        return kl, kt, int(nu.value), int(lg.value)

    def run_merge_events(self, locs, max_events=1 << 40):
        """Mode M with its event stream: (key_loc, key_time_bits, n_unique,
        events, coalescences).  events: dict of arrays time_bits, prior_bits,
        loc, target (~0 for a speciation) and lineage, one entry per executed
        event in time order; coalescences: dict of arrays loc, time_bits,
        parent, child (the child dispersed at time into the parent's
        location)."""
        locs = np.ascontiguousarray(locs, dtype=np.uint64)
        n = locs.size
        _, _, U = self.run_merge(locs, max_events)
        ev = {k: np.zeros(max(U, 1), dtype=np.uint64) for k in ("time_bits", "prior_bits", "loc", "target")}
        ev["lineage"] = np.zeros(max(U, 1), dtype=np.int64)
        co = {k: np.zeros(max(n, 1), dtype=np.uint64) for k in ("loc", "time_bits")}
        co["parent"] = np.zeros(max(n, 1), dtype=np.int64)
        co["child"] = np.zeros(max(n, 1), dtype=np.int64)
        lg = _EventLog()
        lg.cap, lg.co_cap = U, n
        lg.time_bits, lg.prior_bits, lg.loc = _ptr(ev["time_bits"]), _ptr(ev["prior_bits"]), _ptr(ev["loc"])
        lg.target, lg.lineage = _ptr(ev["target"]), _ptr(ev["lineage"])
        lg.co_loc, lg.co_time_bits = _ptr(co["loc"]), _ptr(co["time_bits"])
        lg.co_parent, lg.co_child = _ptr(co["parent"]), _ptr(co["child"])
        kl = np.zeros(n, dtype=np.uint64)
        kt = np.zeros(n, dtype=np.uint64)
        nu = ctypes.c_uint64(0)
        st = lib().or_run_merge_events(self._mp, _ptr(locs), n, max_events, _ptr(kl), _ptr(kt),
                                       ctypes.byref(nu), ctypes.byref(lg))
        if st != 0:
            raise RuntimeError("oracle merge run failed with status %d" % st)
        ev = {k: v[:lg.n] for k, v in ev.items()}
        co = {k: v[:lg.n_co] for k, v in co.items()}
        return kl, kt, int(nu.value), ev, co

    def trace_log(self, loc, cap=1 << 24):
        """Mode P event log of one lineage: arrays of (location, time bits)."""
        el = np.zeros(cap, dtype=np.uint64)
        et = np.zeros(cap, dtype=np.uint64)
        n = lib().or_trace_log(self._mp, int(loc), cap, _ptr(el), _ptr(et))
        if n < 0:
            raise RuntimeError("oracle trace log overflow")
        return el[:n], et[:n]

    # building blocks, for the oracle's own tests
    def next_event_time(self, loc, tau):
        return lib().or_next_event_time(self._mp, int(loc), float(tau))

    def disperse(self, loc, tau):
        return int(lib().or_disperse(self._mp, int(loc), float(tau)))

    def speciates(self, loc, tau):
        return bool(lib().or_speciates(self._mp, int(loc), float(tau)))

    def gauss_offset(self, r):
        v = int(lib().or_gauss_offset(self._mp, int(r)))
        return v - (1 << 64) if v >= (1 << 63) else v

    def alias_row(self, cx, cy):
        q = np.zeros(4096, dtype=np.uint32)
        al = np.zeros(4096, dtype=np.uint16)
        full = np.zeros(4096, dtype=np.uint8)
        dx = np.zeros(4096, dtype=np.int8)
        dy = np.zeros(4096, dtype=np.int8)
        n = lib().or_alias_row_dump(self._mp, cx, cy, _ptr(q), _ptr(al), _ptr(full), _ptr(dx), _ptr(dy))
        return q[:n], al[:n], full[:n], dx[:n], dy[:n]


def species_ids(key_loc, key_time):
    """dense species identity per individual: the rank of its speciation key
    among the distinct keys in ascending (location, time bits) order; and the
    species count"""
    key_loc = np.asarray(key_loc, dtype=np.uint64)
    key_time = np.asarray(key_time, dtype=np.uint64)
    keys = sorted(set(zip(key_loc.tolist(), key_time.tolist())))
    rank = {k: r for r, k in enumerate(keys)}
    ids = np.array([rank[k] for k in zip(key_loc.tolist(), key_time.tolist())], dtype=np.uint64)
    return ids, len(keys)
