"""The event search's one-step rounding of a draw to the interval's grid,
against the oracle (CPU; the device's own form is compared bit for bit by
the GPU search tests).

Method reading: each exponential inter-event time is -ln U rounded to
binary64 and added to the running event time in binary64 (summary of the
Independent algorithm; appendix "Inverse Transform: Uniform and
Exponential").  Within one interval's binade the binary64 values are the
multiples of a grid step of 2^sft units of 2^-58, so the draw enters the
sum rounded twice: to 53 significant bits, then to the grid (half up or
down by the sum's parity at an exact tie).  The library's exp1_grid rounds
X58 to the grid once and flags the draws near a grid midpoint, where it
takes the two roundings in turn.  Here the expected values come from the
oracle: X58 from its fixed-point logarithm, the binary64 value from its
exp1, the grid rounding written out with exact integers.
"""
import math

import numpy as np

import oracle as O
from oracle import ln_definition as LD
from host_grid import grid_draws


def _expected(r, sft):
    """(x58, grid rounding half down, exact midpoint) from the oracle"""
    x58 = O.exp1_q58(r)
    R = int(math.ldexp(O.exp1(r << 11), 58))  # the binary64 draw in units of 2^-58 (exact)
    half = 1 << (sft - 1)
    return x58, (R + half - 1) >> sft, (R & ((1 << sft) - 1)) == half


def _check(rs, sfts):
    x58, a, near = grid_draws(rs, sfts)
    n_near = 0
    for k in range(len(rs)):
        r, s = int(rs[k]), int(sfts[k])
        want_x, want_a, tie = _expected(r, s)
        assert int(x58[k]) == want_x, (r, s)
        if near[k]:
            n_near += 1
            continue
        # away from a midpoint: one rounding equals the two, and no tie
        assert not tie, (r, s)
        assert int(a[k]) == want_a, (r, s, int(a[k]), want_a)
    return n_near


def test_grid_rounding_on_bucket_edges():
    # every bucket edge of binades at the ends and the word boundaries, at
    # grid shifts from a single unit of the draw to far coarser grids
    rs = []
    for e in (0, 11, 12, 31, 32, 51, 52):
        rs += LD.bucket_edges(e)
    rs = np.array(rs, dtype=np.uint64)
    for s in (1, 6, 7, 12, 20, 33, 52, 63):
        _check(rs, np.full(len(rs), s, dtype=np.int32))


def test_grid_rounding_near_midpoints_and_random():
    rng = np.random.default_rng(2108)
    r = rng.integers(0, 1 << 53, size=20000, dtype=np.uint64)
    # random grids
    n_near = _check(r, rng.integers(1, 41, size=len(r)).astype(np.int32))
    assert n_near < len(r) // 2
    # draws placed beside a grid midpoint: for each draw the grid shifts at
    # which X58 lies within 2^12 units of a midpoint
    rs, ss = [], []
    for v in r[:6000]:
        x = O.exp1_q58(int(v))
        for s in range(6, 41):
            d = (x & ((1 << s) - 1)) - (1 << (s - 1))
            if abs(d) < 4096:
                rs.append(int(v))
                ss.append(s)
    assert len(rs) > 1000
    n_near = _check(np.array(rs, dtype=np.uint64), np.array(ss, dtype=np.int32))
    assert n_near > 0


def test_grid_rounding_flags_every_tie():
    # exact ties of the second rounding exist (a binary64 draw on a grid
    # midpoint); each must be flagged, never rounded in one step
    rng = np.random.default_rng(7)
    found = 0
    for v in rng.integers(0, 1 << 53, size=4000, dtype=np.uint64):
        v = int(v)
        R = int(math.ldexp(O.exp1(v << 11), 58))
        tz = (R & -R).bit_length() - 1  # trailing zeros: R is a midpoint of the grid 2^(tz + 1)
        if 1 <= tz + 1 <= 63:
            x58, a, near = grid_draws(np.array([v], dtype=np.uint64), np.array([tz + 1], dtype=np.int32))
            assert near[0], v
            found += 1
    assert found > 3000
