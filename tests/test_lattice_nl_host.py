"""Host test of the FP32 break decision of the lattice kernels for geometrically nonlinear bonds
(csrc/pd_lattice.h: lat_p_nl, lat_g_nl, lat_screen_nl, lat_code_nl, lattice_band_nl), compiled with
the host compiler.

Eq 1.30 with the nonlinear extension (Eq 1.10) as |Y|^2 - |xi|^2 >= s0 (2 + s0) |xi|^2.  Bonds are
placed within 1e-9 .. 0.5 of their threshold (relative), on lattice positions rounded in FP64, with
displacements from 1e-6 to 1e3 lattice spacings, rigid offsets and a perpendicular part; the header's
FP32 operations decide them from FP32 copies of u / h, one word per component or two (hi + lo, the
two-word shadow).  Every bond the screen (at its tightest
per-body bound, max(U_i, U_j)) or the full band decides in FP32 must be decided the same way by any
FP64 evaluation: its exact margin eta.(2 xi + eta) - c |xi|^2 (rational arithmetic on the FP64
inputs) has that sign and exceeds 2^-50 times the sum of the magnitudes of its terms.  At a safety
factor of 0.02 (a band 50 times too narrow) such samples violate this.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile
from fractions import Fraction as Fr

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2309_11273_gb300", "csrc")

SRC = r"""
#include "pd_lattice.h"
#include <math.h>
using namespace pd;
// per bond: n (3), ui (3), uj (3) in metres, h, s0; band safety k, the family's N1, Ninf, qmax
// out: screen (1 = settled intact), code (0, 1, 2)
extern "C" void decide_nl(long m, const int* n, const double* ui, const double* uj, const double* h,
                          const double* s0, double k, int n1, int ninf, int qmax, int lo, int* screen, int* code) {
  for (long e = 0; e < m; ++e) {
    const double ih = 1.0 / h[e];
    float a[3], b[3], al[3], bl[3];
    for (int c = 0; c < 3; ++c) {
      const double va = ui[3 * e + c] * ih, vb = uj[3 * e + c] * ih;
      a[c] = (float)va;
      b[c] = (float)vb;
      al[c] = (float)(va - (double)a[c]);  // the two-word shadow's lo words
      bl[c] = (float)(vb - (double)b[c]);
    }
    const float Ui = fmaxf(fabsf(a[0]), fmaxf(fabsf(a[1]), fabsf(a[2])));
    const float Uj = fmaxf(fabsf(b[0]), fmaxf(fabsf(b[1]), fabsf(b[2])));
    const float nx = (float)n[3 * e], ny = (float)n[3 * e + 1], nz = (float)n[3 * e + 2];
    const float q = nx * nx + ny * ny + nz * nz;
    const float ex = lo ? lat_delta_lo(b[0], bl[0], a[0], al[0]) : b[0] - a[0];
    const float ey = lo ? lat_delta_lo(b[1], bl[1], a[1], al[1]) : b[1] - a[1];
    const float ez = lo ? lat_delta_lo(b[2], bl[2], a[2], al[2]) : b[2] - a[2];
    const float p = lat_p_nl<3>(nx, ny, nz, ex, ey, ez);
    const double c = s0[e] * (2.0 + s0[e]);
    const float g = lat_g_nl(p, (float)c, q);
    const float D = fabsf(ex) + fabsf(ey) + fabsf(ez);
    const LatBandNL B = lattice_band_nl(k, s0[e], n1, ninf, qmax);
    code[e] = lat_code_nl(g, D, Ui + Uj, B);
    // the kernels' screen at its tightest: the body's largest |u'| is max(U_i, U_j)
    const float S = Ui + lat_umax_bound(fmaxf(Ui, Uj));
    const float f0 = fmaf(B.F0s, S, B.F0), f1 = fmaf(B.F1s, S, B.F1);
    screen[e] = lat_max_nan(-INFINITY, g) + lat_screen_nl(D, f0, f1, B.F2) < 0.0f ? 1 : 0;
  }
}
"""


@pytest.fixture(scope="module")
def so():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    tmp = tempfile.mkdtemp(prefix="pd_latnl_")
    src, lib = os.path.join(tmp, "l.cc"), os.path.join(tmp, "l.so")
    with open(src, "w") as f:
        f.write(SRC)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + HDR, src, "-o", lib],
                   check=True)
    L = ctypes.CDLL(lib)
    L.decide_nl.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 5 + [ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                                                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                                      ctypes.c_void_p]
    yield L
    shutil.rmtree(tmp, ignore_errors=True)


def family(q=9):
    r = range(-3, 4)
    return np.array([(x, y, z) for z in r for y in r for x in r if 0 < x * x + y * y + z * z <= q], dtype=np.int32)


def near_threshold_nl(rng, m, h, umag, s0_lo, s0_hi, dirs, rel=None):
    """Bonds with |Y|^2 - |xi|^2 = c (1 + r) |xi|^2 (c = s0 (2 + s0)): a stretch along xi, a
    perpendicular part up to 5 % of |xi| and a rigid offset of size umag h."""
    n = dirs[rng.integers(0, len(dirs), m)]
    i0 = rng.integers(0, 100000, size=(m, 3)).astype(np.float64)
    xi = (i0 + n + 0.5) * h - (i0 + 0.5) * h
    s0 = 10.0 ** rng.uniform(np.log10(s0_lo), np.log10(s0_hi), m)
    c = s0 * (2.0 + s0)
    r = rel if rel is not None else rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-9.0, -0.3, m)
    q = (xi * xi).sum(1)
    perp = rng.normal(size=(m, 3))
    perp -= ((perp * xi).sum(1) / q)[:, None] * xi
    f = rng.uniform(0, 0.05, m)
    perp *= (f * np.sqrt(q) / np.maximum(np.linalg.norm(perp, axis=1), 1e-300))[:, None]
    t = np.sqrt(1.0 + c * (1.0 + r) - f * f) - 1.0
    ui = rng.normal(size=(m, 3)) * umag * h
    uj = ui + t[:, None] * xi + perp
    return xi, n.astype(np.int32), ui, uj, np.full(m, h), s0


def exact_margin_nl(xi, ui, uj, s0):
    """(eta.(2 xi + eta) - c |xi|^2, 2^-50 (sum |2 xi_c eta_c| + |eta|^2 + c |xi|^2)), exactly."""
    out = []
    for k in range(len(s0)):
        X = [Fr(float(v)) for v in xi[k]]
        E = [Fr(float(b)) - Fr(float(a)) for a, b in zip(ui[k], uj[k])]
        S = Fr(float(s0[k]))
        c = S * (2 + S)
        q = sum(x * x for x in X)
        G = sum(e * (2 * x + e) for x, e in zip(X, E)) - c * q
        M = (sum(abs(2 * x * e) for x, e in zip(X, E)) + sum(e * e for e in E) + c * q) / 2 ** 50
        out.append((G, M))
    return out


def run_nl(so, xi, n, ui, uj, h, s0, k, n1=5, ninf=3, qmax=9, lo=0):
    m = len(s0)
    screen = np.zeros(m, dtype=np.int32)
    code = np.zeros(m, dtype=np.int32)
    arrs = [np.ascontiguousarray(a) for a in (n, ui, uj, h, s0)]
    so.decide_nl(m, *[a.ctypes.data for a in arrs], k, n1, ninf, qmax, lo, screen.ctypes.data, code.ctypes.data)
    return screen, code


def violations_nl(so, sample, k, lo=0):
    screen, code = run_nl(so, *sample, k, lo=lo)
    xi, n, ui, uj, h, s0 = sample
    bad = 0
    counts = dict(screened=0, fp32_broken=0, fp32_intact=0, fp64=0)
    for e, (G, M) in enumerate(exact_margin_nl(xi, ui, uj, s0)):
        if screen[e]:
            counts["screened"] += 1
            bad += not (G < -M)
            bad += code[e] != 0  # the screen implies the band's intact decision
        if code[e] == 1:
            counts["fp32_broken"] += 1
            bad += not (G > M)
        elif code[e] == 0:
            counts["fp32_intact"] += 1
            bad += not (G < -M)
        else:
            counts["fp64"] += 1
    return bad, counts


CASES = [
    (1e-3, 1e-3, 1e-4, 1e-2),    # the benchmark block: mm spacing, small displacements
    (1e-3, 1.0, 1e-4, 1e-2),     # displacements of a whole spacing (the torsion's far end)
    (2.5e-4, 30.0, 1e-5, 1e-3),  # large rigid offsets
    (1.0, 1e3, 1e-3, 1e-1),      # unit spacing, huge offsets
    (1e-9, 1e-6, 1e-4, 1e-2),    # tiny spacing, displacements far below it
]


@pytest.mark.parametrize("h,umag,s0lo,s0hi", CASES)
@pytest.mark.parametrize("k", [1.05, 4.0])
@pytest.mark.parametrize("lo", [0, 1])
def test_fp32_nonlinear_decisions_match_every_fp64_evaluation(so, h, umag, s0lo, s0hi, k, lo):
    rng = np.random.default_rng(int(h * 1e9) % 1000 + int(umag * 10) + int(k * 7) + lo)
    sample = near_threshold_nl(rng, 1500, h, umag, s0lo, s0hi, family())
    bad, counts = violations_nl(so, sample, k, lo)
    assert bad == 0, counts
    assert counts["fp32_intact"] > 0 and counts["fp32_broken"] > 0 and counts["fp64"] > 0, counts


def test_nonlinear_screen_settles_bonds_clear_of_the_threshold(so):
    """Bonds at half their threshold never leave the screen (benchmark scales)."""
    rng = np.random.default_rng(5)
    xi, n, ui, uj, h, s0 = near_threshold_nl(rng, 500, 1e-3, 0.9, 6.7e-4, 6.8e-4, family(), rel=-0.5)
    screen, code = run_nl(so, xi, n, ui, uj, h, s0, 4.0)
    assert screen.all() and (code == 0).all()


def test_undersized_nonlinear_band_is_caught(so):
    """At a safety factor of 0.02 the same check finds FP32 decisions that some FP64 evaluation
    contradicts (in the band and in the screen), so the test above has teeth."""
    rng = np.random.default_rng(9)
    sample = near_threshold_nl(rng, 3000, 1e-3, 1.0, 1e-4, 1e-2, family())
    for lo in (0, 1):
        bad, counts = violations_nl(so, sample, 0.02, lo)
        assert bad > 0, (lo, counts)


def test_nonfinite_nonlinear_extension_goes_to_fp64(so):
    xi = np.array([[1e-3, 0.0, 0.0]])
    n = np.array([[1, 0, 0]], dtype=np.int32)
    for bad in (np.nan, np.inf, -np.inf):
        screen, code = run_nl(so, xi, n, np.zeros((1, 3)), np.array([[bad, 0.0, 0.0]]), np.array([1e-3]),
                              np.array([1e-3]), 4.0)
        assert screen[0] == 0 and code[0] == 2
