"""The FP32 screen of the pair form's failure check before a read (the break test s >= s0 of
Eqs 1.17 / 1.30 in its sqrt-free form xi.(u_j - u_i) >= s0 |xi|^2).

The kernel first evaluates each bond in FP32 from FP32 copies of xi and u and keeps it intact only
when value + 2^-19 (M + |value|) (plus two tiny absolute terms) is below the threshold rounded down
to FP32, M = sum_c |xi_c| (|u_jc| + |u_ic|); every other bond is evaluated in FP64.  The screen is
sound if every bond it keeps intact is below the threshold by more than the FP64 evaluation error
(under 3 * 2^-53 M), in exact arithmetic.  Here its FP32 operations are replayed with numpy float32
(fmaf: the exact product and sum, rounded once) on adversarial inputs: bonds from 1e-9 to 0.5 of
their threshold away from it, displacements up to 1e6 times their differences, and scales down to
FP32 underflow and up to overflow.  Random samples stay inside the worst case of the error
analysis (6.01 * 2^-24 M): a margin of 2^-25 M already fails here, one of 2^-23 M does not.
Host-only.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

F = np.float32


def fmaf(a, b, c):
    a, b, c = float(a), float(b), float(c)
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        return F(a * b + c)
    return F(float(Fr(a) * Fr(b) + Fr(c)))


def round_down_f32(x):
    r = F(x)
    if float(r) > x:
        r = np.nextafter(r, F(-np.inf))
    return r


def screen_keeps_intact(xi, ui, uj, thr):
    """The kernel's FP32 screen, operation by operation."""
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        s = [F(v) for v in xi]
        a = [F(v) for v in ui]
        b = [F(v) for v in uj]
        w = round_down_f32(thr)
        dx, dy = b[0] - a[0], b[1] - a[1]
        d = fmaf(s[0], dx, s[1] * dy)
        m = fmaf(abs(s[0]), abs(b[0]) + abs(a[0]), abs(s[1]) * (abs(b[1]) + abs(a[1])))
        l1 = abs(s[0]) + abs(s[1])
        d = fmaf(s[2], b[2] - a[2], d)
        m = fmaf(abs(s[2]), abs(b[2]) + abs(a[2]), m)
        l1 = l1 + abs(s[2])
        bound = fmaf(F(2.0 ** -19), m + abs(d), fmaf(F(2.0 ** -120), l1, F(2.0 ** -140)))
        return bool(d + bound < w)


def exact_gap(xi, ui, uj, thr):
    """thr - xi.(u_j - u_i) - 2^-50 M in exact arithmetic (> 0: any FP64 evaluation is below thr)."""
    d = sum(Fr(float(x)) * (Fr(float(q)) - Fr(float(p))) for x, p, q in zip(xi, ui, uj))
    m = sum(abs(Fr(float(x))) * (abs(Fr(float(p))) + abs(Fr(float(q)))) for x, p, q in zip(xi, ui, uj))
    return Fr(float(thr)) - d - m / 2 ** 50


def near_threshold_bonds(rng, count, xi_scale, u_scale, s0_range, rel=None):
    """Bonds whose extension xi.(u_j - u_i) is s0 |xi|^2 (1 + r), at displacement offsets u_scale
    and with random perpendicular components; r = rel, or +-10^U(-9, -0.3) so that the samples
    straddle the screen's own margin whatever its width."""
    out = []
    for _ in range(count):
        xi = rng.normal(size=3) * xi_scale
        s0 = 10.0 ** rng.uniform(*s0_range)
        thr = s0 * float(xi @ xi)
        ui = rng.normal(size=3) * u_scale
        r = rel if rel is not None else rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9.0, -0.3)
        t = thr * (1.0 + r) / float(xi @ xi)
        perp = rng.normal(size=3)
        perp -= (perp @ xi) / (xi @ xi) * xi
        uj = ui + t * xi + perp * (t * np.linalg.norm(xi))
        out.append((xi, ui, uj, thr))
    return out


@pytest.mark.parametrize("xi_scale,u_scale,s0_range", [
    (1e-3, 1e-4, (-5, -1)),    # lattice bonds of the benchmark block, displacements of its torsion
    (1e-3, 1e-1, (-5, -3)),    # a large rigid offset: differences ~1e-6 of the displacements
    (1.0, 1e3, (-6, -2)),      # unit bonds, huge offsets
    (1e-18, 1e-17, (-6, -2)),  # thresholds near and below FP32 underflow
    (1e18, 1e19, (-3, -1)),    # products near FP32 overflow
])
def test_screened_intact_bonds_are_below_threshold_in_fp64(xi_scale, u_scale, s0_range):
    rng = np.random.default_rng(11)
    kept = deferred_below = 0
    for xi, ui, uj, thr in near_threshold_bonds(rng, 2000, xi_scale, u_scale, s0_range):
        below = exact_gap(xi, ui, uj, thr) > 0
        if screen_keeps_intact(xi, ui, uj, thr):
            kept += 1
            assert below
        else:
            deferred_below += below
    # both branches are exercised: bonds kept intact by the screen, and bonds below the threshold
    # that it still passes on to FP64 (those inside its margin)
    assert kept > 0 and deferred_below > 0


def test_screen_settles_bonds_clear_of_the_threshold():
    """Bonds at half their threshold and typical displacement offsets never reach FP64."""
    rng = np.random.default_rng(12)
    for xi, ui, uj, thr in near_threshold_bonds(rng, 500, 1e-3, 1e-4, (-4, -2), rel=0.0):
        uj_half = ui + 0.5 * (uj - ui)
        assert screen_keeps_intact(xi, ui, uj_half, thr)


def test_screen_defers_nonfinite_and_underflowing_bonds():
    xi = np.array([1e-3, 0.0, 0.0])
    ui = np.zeros(3)
    for bad in (np.nan, np.inf, -np.inf):
        assert not screen_keeps_intact(xi, ui, np.array([bad, 0.0, 0.0]), 1e-9)
    # a threshold that rounds down to zero in FP32 keeps nothing intact unless clearly negative
    tiny = np.array([1e-30, 0.0, 0.0])
    assert not screen_keeps_intact(tiny, ui, np.array([1e-40, 0.0, 0.0]), 1e-63)
    assert not screen_keeps_intact(tiny, ui, np.zeros(3), 1e-63)
