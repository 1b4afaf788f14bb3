"""Host tests of the lattice layout's shared code (csrc/pd_lattice.h), compiled with the host compiler.

1. The direction table: every non-zero integer vector with |n|^2 up to the table's bound appears once,
   in groups (|n|^2 <= 9, then rings up to each next square) so that every family (the closed ball
   of Section 2.1, |n|^2 <= (delta/h)^2) of radius 3, 4, ... lattice spacings is a prefix, ordered
   by row (n_z, n_y) then n_x inside a group, with entry k ^ 1 = -entry k (the two directed entries of
   one bond); the family sizes of the workloads' horizons (28 and 48 in 2D for delta = 3.015 h and
   4.015 h, 122 in 3D) are prefixes, and balls ending inside a group are not.
2. The FP32 break decision of the lattice kernels (Eq 1.30 as n.(u'_j - u'_i) >= s0 |n|^2 in lattice
   units): its FP32 operations (lat_dprime, lat_g, both forms of the screen -- per neighbour, and
   per body with the body's largest |u'| at its tightest, max(U_i, U_j) -- and the full band) are run by the
   header's own code on bonds placed within 1e-9 .. 0.5 of their threshold, with lattice positions
   rounded in FP64, displacements from 1e-6 to 1e3 lattice spacings and rigid rotations on top.  Every
   bond the screen or the band decides in FP32 must be decided the same way by any FP64 evaluation:
   its exact margin xi.(u_j - u_i) - s0 |xi|^2 (rational arithmetic on the FP64 inputs) has that sign
   and exceeds 2^-50 times the sum of the magnitudes of its terms.  With the safety factor at 0.02
   (a band 50 times too narrow) such samples violate this, so the test has teeth.
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
extern "C" int table(int dim, int* out, int cap) {
  const std::vector<LatDir> t = lattice_directions(dim);
  if ((int)t.size() * 4 > cap) return -1;
  for (size_t k = 0; k < t.size(); ++k) {
    out[4 * k] = t[k].n[0]; out[4 * k + 1] = t[k].n[1]; out[4 * k + 2] = t[k].n[2]; out[4 * k + 3] = t[k].q;
  }
  return (int)t.size();
}
extern "C" int prefix(int dim, int q) { return lattice_prefix(dim, q); }
// d' = n.(u_j - u_i) / h in FP32 from one-word (lo = 0) or two-word (lo = 1) shadows of u / h
extern "C" void dprime(long m, const int* n, const double* ui, const double* uj, double h, int lo, float* out) {
  for (long k = 0; k < m; ++k) {
    float a[3], b[3], al[3], bl[3];
    for (int c = 0; c < 3; ++c) {
      const double va = ui[3 * k + c] / h, vb = uj[3 * k + c] / h;
      a[c] = (float)va; b[c] = (float)vb;
      al[c] = (float)(va - (double)a[c]); bl[c] = (float)(vb - (double)b[c]);
    }
    const float nx = (float)n[3 * k], ny = (float)n[3 * k + 1], nz = (float)n[3 * k + 2];
    out[k] = lo ? lat_dprime_d<3>(nx, ny, nz, lat_delta_lo(b[0], bl[0], a[0], al[0]),
                                  lat_delta_lo(b[1], bl[1], a[1], al[1]), lat_delta_lo(b[2], bl[2], a[2], al[2]))
                : lat_dprime<3>(nx, ny, nz, b[0], b[1], b[2], a[0], a[1], a[2]);
  }
}
// both forms of the screen on the same FP32 operands: 1 = settled as intact
extern "C" void screens(long m, const float* g, const float* kf, const float* uj, const float* scr, int* a, int* b) {
  for (long k = 0; k < m; ++k) {
    a[k] = lat_screen_intact(g[k], kf[k], uj[k], scr[k]) ? 1 : 0;
    b[k] = lat_screen_value(g[k], kf[k], uj[k], scr[k]) < 0.0f ? 1 : 0;
  }
}
// the compile-time table and prefix (the specialized kernels' directions)
extern "C" int table_c(int dim, int k, int c) {
  constexpr LatTable<3> t3 = lattice_table<3>();
  constexpr LatTable<2> t2 = lattice_table<2>();
  const LatDir& e = dim == 3 ? t3.d[k] : t2.d[k];
  return c < 3 ? e.n[c] : e.q;
}
extern "C" int prefix_c(int dim, int q) { return dim == 3 ? lattice_prefix_c<3>(q) : lattice_prefix_c<2>(q); }
// per bond: xi (3, FP64 positions' difference), n (3), ui (3), uj (3) in metres, h, s0;
// band_safety, n1, qmax, lo (1: two-word shadow hi + lo); out: screen (1 = settled intact), code (0, 1, 2)
extern "C" void decide(long m, const double* xi, const int* n, const double* ui, const double* uj, const double* h,
                       const double* s0, double bc, int n1, int qmax, int lo, int* screen, int* code,
                       int* screen_c) {
  for (long k = 0; k < m; ++k) {
    const double ih = 1.0 / h[k];
    float a[3], b[3], al[3], bl[3];
    for (int c = 0; c < 3; ++c) {
      const double va = ui[3 * k + c] * ih, vb = uj[3 * k + c] * ih;
      a[c] = (float)va;
      b[c] = (float)vb;
      al[c] = (float)(va - (double)a[c]);
      bl[c] = (float)(vb - (double)b[c]);
    }
    const float Ui = fmaxf(fabsf(a[0]), fmaxf(fabsf(a[1]), fabsf(a[2])));
    const float Uj = fmaxf(fabsf(b[0]), fmaxf(fabsf(b[1]), fabsf(b[2])));
    const float nx = (float)n[3 * k], ny = (float)n[3 * k + 1], nz = (float)n[3 * k + 2];
    const float q = nx * nx + ny * ny + nz * nz;
    const float d = lo ? lat_dprime_d<3>(nx, ny, nz, lat_delta_lo(b[0], bl[0], a[0], al[0]),
                                         lat_delta_lo(b[1], bl[1], a[1], al[1]), lat_delta_lo(b[2], bl[2], a[2], al[2]))
                       : lat_dprime<3>(nx, ny, nz, b[0], b[1], b[2], a[0], a[1], a[2]);
    const float s0f = (float)s0[k];
    const float g = lat_g(d, s0f, q);
    const LatBand L = lattice_band(bc, s0[k], n1, qmax);
    const float scr = fmaf(L.Kfast, Ui, L.Kcfast);
    screen[k] = lat_screen_value(g, L.Kfast, Uj, scr) < 0.0f ? 1 : 0;  // the per-neighbour screen
    // the kernels' per-body screen at its tightest: the body's largest |u'| is max(U_i, U_j)
    const float scr_c = lat_screen_part(L.Kfast, Ui, lat_umax_bound(fmaxf(Ui, Uj)), L.Kcfast);
    screen_c[k] = lat_max_nan(-INFINITY, g) + scr_c < 0.0f ? 1 : 0;
    code[k] = lat_code(g, Ui, Uj, s0f, q, L.Kf, L.sq, L.eps_c, L.s0n1);
  }
}
"""


@pytest.fixture(scope="module")
def so():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    tmp = tempfile.mkdtemp(prefix="pd_lat_")
    src, lib = os.path.join(tmp, "lat.cc"), os.path.join(tmp, "lat.so")
    with open(src, "w") as f:
        f.write(SRC)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I" + HDR, src, "-o", lib],
                   check=True)
    L = ctypes.CDLL(lib)
    L.table.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int]
    L.prefix.argtypes = [ctypes.c_int, ctypes.c_int]
    L.screens.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 6
    L.dprime.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 3 + [ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
    L.prefix_c.argtypes = [ctypes.c_int, ctypes.c_int]
    L.table_c.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.decide.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 6 + [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    yield L
    shutil.rmtree(tmp, ignore_errors=True)


def get_table(L, dim):
    buf = np.zeros(4 * 4096, dtype=np.int32)
    m = L.table(dim, buf.ctypes.data, buf.size)
    assert m > 0
    return buf[:4 * m].reshape(m, 4)


@pytest.mark.parametrize("dim,qmax,count", [(2, 64, 196), (3, 25, 514)])
def test_direction_table(so, dim, qmax, count):
    t = get_table(so, dim)
    assert len(t) == count
    R = int(np.floor(np.sqrt(qmax)))
    rng = range(-R, R + 1)
    brute = {(x, y, z) for x in rng for y in rng for z in (rng if dim == 3 else [0])
             if 0 < x * x + y * y + z * z <= qmax}
    got = [tuple(r[:3]) for r in t]
    assert len(set(got)) == len(got) and set(got) == brute
    assert np.array_equal(t[:, 3], (t[:, :3] ** 2).sum(1))
    grp = np.maximum(3, np.ceil(np.sqrt(t[:, 3]) - 1e-9)).astype(int)
    assert np.all(np.diff(grp) >= 0)  # groups |n|^2 <= 9, then rings up to each next square
    for m in range(3, int(np.sqrt(qmax)) + 1):  # every ball |n|^2 <= m^2, m >= 3, is a prefix
        k = int((t[:, 3] <= m * m).sum())
        assert np.all(t[:k, 3] <= m * m)
    rep = t[0::2, :3]
    for g in np.unique(grp):  # inside a group: positive representatives by (z, y, x)
        r = rep[grp[0::2] == g]
        assert r.tolist() == sorted(r.tolist(), key=lambda n: (n[2], n[1], n[0]))
    assert np.array_equal(t[1::2, :3], -t[0::2, :3])  # k ^ 1 is the opposite direction


def test_family_prefixes(so):
    # the closed balls of the workloads' horizons (lattice counts, Section 2.1)
    assert so.prefix(2, 9) == 28 and so.prefix(2, 16) == 48 and so.prefix(3, 9) == 122
    # balls that end inside a group are not prefixes (such bodies keep the general layout)
    assert so.prefix(3, 4) == -1 and so.prefix(2, 5) == -1 and so.prefix(3, 12) == -1
    for dim, q in ((2, 9), (2, 16), (3, 9), (3, 16)):
        t = get_table(so, dim)
        assert so.prefix(dim, q) == int((t[:, 3] <= q).sum())


@pytest.mark.parametrize("dim", [2, 3])
def test_compile_time_table_is_the_runtime_table(so, dim):
    """The kernels compiled for one family take their directions from the compile-time table: it is
    the table the layout is built with, entry by entry, and so are its prefixes."""
    t = get_table(so, dim)
    for k in range(len(t)):
        assert [so.table_c(dim, k, c) for c in range(4)] == list(t[k]), k
    for q in range(1, 26 if dim == 3 else 65):
        assert so.prefix_c(dim, q) == so.prefix(dim, q), q


def near_threshold(rng, m, h, umag, s0_lo, s0_hi, dirs, rel=None):
    """Lattice bonds (positions (i + 1/2) h rounded in FP64, i up to 1e5) whose extension is
    s0 |xi|^2 (1 + r), with displacement offsets of size umag h and a rotation part."""
    n = dirs[rng.integers(0, len(dirs), m)]
    i0 = rng.integers(0, 100000, size=(m, 3)).astype(np.float64)
    xi_pos = (i0 + 0.5) * h
    xj_pos = (i0 + n + 0.5) * h
    xi = xj_pos - xi_pos  # the FP64 bond vector of the positions
    s0 = 10.0 ** rng.uniform(np.log10(s0_lo), np.log10(s0_hi), m)
    q = (xi * xi).sum(1)
    r = rel if rel is not None else rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-9.0, -0.3, m)
    t = s0 * (1.0 + r)
    perp = rng.normal(size=(m, 3))
    perp -= ((perp * xi).sum(1) / q)[:, None] * xi
    perp *= (rng.uniform(0, 0.05, m) * np.sqrt(q) / np.maximum(np.linalg.norm(perp, axis=1), 1e-300))[:, None]
    ui = rng.normal(size=(m, 3)) * umag * h
    uj = ui + t[:, None] * xi + perp
    return xi, n.astype(np.int32), ui, uj, np.full(m, h), s0


def exact_margin(xi, ui, uj, s0):
    """(xi.(u_j - u_i) - s0 |xi|^2, 2^-50 (sum |xi_c||du_c| + s0 |xi|^2)) in exact arithmetic."""
    out = []
    for k in range(len(s0)):
        X = [Fr(float(v)) for v in xi[k]]
        D = [Fr(float(b)) - Fr(float(a)) for a, b in zip(ui[k], uj[k])]
        S0 = Fr(float(s0[k]))
        q = sum(x * x for x in X)
        G = sum(x * d for x, d in zip(X, D)) - S0 * q
        M = (sum(abs(x * d) for x, d in zip(X, D)) + S0 * q) / 2 ** 50
        out.append((G, M))
    return out


def run_case(so, xi, n, ui, uj, h, s0, bc, n1, qmax, lo=0, with_body_screen=False):
    m = len(s0)
    screen = np.zeros(m, dtype=np.int32)
    code = np.zeros(m, dtype=np.int32)
    screen_c = np.zeros(m, dtype=np.int32)
    arrs = [np.ascontiguousarray(a) for a in (xi, n, ui, uj, h, s0)]
    so.decide(m, *[a.ctypes.data for a in arrs], bc, n1, qmax, lo, screen.ctypes.data, code.ctypes.data,
              screen_c.ctypes.data)
    if with_body_screen:
        return screen, code, screen_c
    return screen, code


def violations(so, sample, bc, n1, qmax, lo=0):
    screen, code, screen_c = run_case(so, *sample, bc, n1, qmax, lo, with_body_screen=True)
    xi, n, ui, uj, h, s0 = sample
    bad = 0
    counts = dict(screened=0, body_screened=0, fp32_broken=0, fp32_intact=0, fp64=0)
    for k, (G, M) in enumerate(exact_margin(xi, ui, uj, s0)):
        if screen_c[k]:
            counts["body_screened"] += 1
            bad += not (G < -M)
            bad += code[k] != 0  # the per-body screen implies the band's intact decision
        if screen[k]:
            counts["screened"] += 1
            bad += not (G < -M)
        if code[k] == 1:
            counts["fp32_broken"] += 1
            bad += not (G > M)
        elif code[k] == 0:
            counts["fp32_intact"] += 1
            bad += not (G < -M)
        else:
            counts["fp64"] += 1
        if screen[k] and code[k] != 0:
            bad += 1  # the screen implies the band's intact decision
    return bad, counts


CASES = [
    (1e-3, 1e-3, 1e-4, 1e-2),   # the benchmark block: mm spacing, small displacements
    (1e-3, 1.0, 1e-4, 1e-2),    # displacements of a whole spacing (the torsion's far end)
    (2.5e-4, 30.0, 1e-5, 1e-3),  # large rigid offsets: differences ~1e-6 of the displacements
    (1.0, 1e3, 1e-3, 1e-1),     # unit spacing, huge offsets
    (1e-9, 1e-6, 1e-4, 1e-2),   # tiny spacing, displacements far below it
]


@pytest.mark.parametrize("h,umag,s0lo,s0hi", CASES)
@pytest.mark.parametrize("bc", [1.05, 4.0])
@pytest.mark.parametrize("lo", [0, 1])
def test_fp32_decisions_match_every_fp64_evaluation(so, h, umag, s0lo, s0hi, bc, lo):
    t = get_table(so, 3)
    fam = t[t[:, 3] <= 9]  # delta = 3.015 h
    rng = np.random.default_rng(int(h * 1e9) % 1000 + int(umag * 10) + int(bc * 7))
    sample = near_threshold(rng, 1500, h, umag, s0lo, s0hi, fam[:, :3])
    n1 = int(np.abs(fam[:, :3]).sum(1).max())
    bad, counts = violations(so, sample, bc, n1, 9, lo)
    assert bad == 0, counts
    # the FP32 path decides bonds on both sides and passes the closest to FP64
    assert counts["fp32_intact"] > 0 and counts["fp32_broken"] > 0 and counts["fp64"] > 0, counts


def test_screen_settles_bonds_clear_of_the_threshold(so):
    """Bonds at half their threshold never leave the two-instruction screen (benchmark scales)."""
    t = get_table(so, 3)
    fam = t[t[:, 3] <= 9]
    rng = np.random.default_rng(5)
    xi, n, ui, uj, h, s0 = near_threshold(rng, 500, 1e-3, 0.9, 6.7e-4, 6.8e-4, fam[:, :3], rel=-0.5)
    screen, code, screen_c = run_case(so, xi, n, ui, uj, h, s0, 4.0, 5, 9, with_body_screen=True)
    assert screen.all() and screen_c.all() and (code == 0).all()


def test_an_undersized_band_is_caught(so):
    """The same check with the safety factor at 0.02 (a band 50 times too narrow) finds bonds that
    FP32 decides against some FP64 evaluation: the test above would catch a band that is too small
    (the worst case of the analysis is several times the typical rounding, so a band at 0.1 of it
    can still pass random samples)."""
    t = get_table(so, 3)
    fam = t[t[:, 3] <= 9]
    rng = np.random.default_rng(9)
    sample = near_threshold(rng, 3000, 1e-3, 1.0, 1e-4, 1e-2, fam[:, :3],
                            rel=None)
    bad, counts = violations(so, sample, 0.02, 5, 9)
    assert bad > 0, counts
    # the per-body screen alone, too
    screen, code, screen_c = run_case(so, *sample, 0.02, 5, 9, with_body_screen=True)
    xi, n, ui, uj, h, s0 = sample
    margins = exact_margin(xi, ui, uj, s0)
    assert sum(1 for k in np.flatnonzero(screen_c) if not (margins[k][0] < -margins[k][1])) > 0


def test_nonfinite_extension_goes_to_fp64(so):
    xi = np.array([[1e-3, 0.0, 0.0]])
    n = np.array([[1, 0, 0]], dtype=np.int32)
    for bad in (np.nan, np.inf, -np.inf):
        screen, code, screen_c = run_case(so, xi, n, np.zeros((1, 3)), np.array([[bad, 0.0, 0.0]]), np.array([1e-3]),
                                          np.array([1e-3]), 4.0, 5, 9, with_body_screen=True)
        assert screen[0] == 0 and screen_c[0] == 0 and code[0] == 2


def test_screen_value_form_is_the_screen(so):
    """The kernels test the screen as lat_screen_value < 0 (one addition, the body's 'cannot break'
    folded in as scr_i = -inf); it must settle exactly the bonds lat_screen_intact settles:
    operands over many magnitudes, sums that cancel to the last bit, subnormals, infinities, NaN."""
    rng = np.random.default_rng(17)
    m = 400000
    kf = (10.0 ** rng.uniform(-8, 0, m)).astype(np.float32)
    uj = (10.0 ** rng.uniform(-10, 3, m)).astype(np.float32)
    g = (rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-12, 2, m)).astype(np.float32)
    # fmaf(Kfast, U_j, g) to within an ulp (the product is exact in FP64)
    a = (kf.astype(np.float64) * uj.astype(np.float64) + g.astype(np.float64)).astype(np.float32)
    scr = (rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-12, 2, m)).astype(np.float32)
    # a third of the samples put scr_i within a few ulps of -fmaf(Kfast, U_j, g)
    near = rng.random(m) < 0.35
    scr[near] = np.nextafter(-a[near], np.float32(np.inf) * rng.choice([-1, 1], near.sum()))
    exact = rng.random(m) < 0.05
    scr[exact] = -a[exact]
    tiny = np.array([1e-45, -1e-45, 1e-40, -1e-40, 0.0, -0.0], dtype=np.float32)
    spec = np.array([np.inf, -np.inf, np.nan, 3.4e38, -3.4e38], dtype=np.float32)
    extra = np.array(np.meshgrid(np.concatenate([tiny, spec]), np.concatenate([tiny, spec]))).reshape(2, -1)
    g = np.concatenate([g, extra[0], extra[0]]).astype(np.float32)
    scr = np.concatenate([scr, extra[1], np.full(extra.shape[1], -np.inf, np.float32)]).astype(np.float32)
    kf = np.concatenate([kf, np.full(2 * extra.shape[1], 1e-6, np.float32)]).astype(np.float32)
    uj = np.concatenate([uj, np.full(2 * extra.shape[1], 0.5, np.float32)]).astype(np.float32)
    n = g.size
    r1, r2 = np.zeros(n, np.int32), np.zeros(n, np.int32)
    so.screens(n, g.ctypes.data, kf.ctypes.data, uj.ctypes.data, scr.ctypes.data, r1.ctypes.data, r2.ctypes.data)
    assert np.array_equal(r1, r2), np.flatnonzero(r1 != r2)[:10]
    assert 0 < r1.sum() < n


def test_two_word_shadow_rounds_relative_to_the_difference(so):
    """A displacement of 0.2 h carried by bonds whose extension is ~1e-3 h (a twisted body far from
    its axis): one FP32 word per component rounds n.(u'_j - u'_i) to ~eps |n|_1 |u'| (about 1e-5
    of the extension), the two-word shadow to ~eps of the extension itself.  Exact values from
    rational arithmetic on the FP64 inputs."""
    rng = np.random.default_rng(31)
    m, h = 4000, 1e-3
    t = get_table(so, 3)
    n = np.ascontiguousarray(t[rng.integers(0, 122, m), :3]).astype(np.int32)
    base = rng.uniform(-0.2, 0.2, (m, 3)) * h
    ui = np.ascontiguousarray(base)
    uj = np.ascontiguousarray(base + rng.normal(0, 1e-3, (m, 3)) * h)
    exact = np.array([float(sum(Fr(int(n[k, c])) * (Fr(uj[k, c]) - Fr(ui[k, c])) for c in range(3)) / Fr(h))
                      for k in range(m)])
    err = {}
    for lo in (0, 1):
        out = np.zeros(m, dtype=np.float32)
        so.dprime(m, n.ctypes.data, ui.ctypes.data, uj.ctypes.data, h, lo, out.ctypes.data)
        err[lo] = np.abs(out.astype(np.float64) - exact) / np.abs(exact).clip(1e-30)
    assert np.median(err[1]) < 1e-6 and np.median(err[0]) > 100 * np.median(err[1]), (np.median(err[0]),
                                                                                        np.median(err[1]))

