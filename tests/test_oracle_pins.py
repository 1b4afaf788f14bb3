"""Pins of the CPU oracle against values fixed by the paper, closed forms and brute force.

Each test checks the oracle (``oracle/``) against something other than itself: a number printed in
the paper, a lattice sum done in integers here, a continuum integral evaluated by quadrature here,
a classical elasticity formula, or an exact rational computation.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import oracle as O
from paper_2309_11273_gb300 import workloads as W


def lattice_offsets(dim, ratio):
    """Integer offsets k != 0 with |k| <= ratio (exact integer test |k|^2 <= floor(ratio^2))."""
    r = int(math.floor(ratio))
    lim = ratio * ratio
    out = []
    for k in itertools.product(range(-r, r + 1), repeat=dim):
        s = sum(c * c for c in k)
        if 0 < s <= lim:
            out.append(k)
    return out


# --------------------------------------------------------------------------- family / Section 3.3
def _golden(name):
    """Rows of a fixture under tests/golden/ (comments and blank lines skipped)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


def test_paper_bond_count_10x10():
    """Section 3: a 10 x 10 grid with m-ratio 3 has 1058 PD bonds (undirected); the printed value
    is the fixture tests/golden/paper_bond_count.txt."""
    rows = {r[0]: r[1:] for r in _golden("paper_bond_count.txt")}
    nx, ny, ratio, bonds = rows["bonds_10x10_m3"]
    x, y = W.grid_2d(int(nx), int(ny), 1.0)
    for method in ("bruteforce", "binned"):
        rp, col = O.family(x, y, None, float(ratio), method=method)
        assert col.size == 2 * int(bonds)


@pytest.mark.parametrize("dim,ratio,expected", [(2, 3.015, 28), (3, 3.015, 122), (2, 4.015, 48)])
def test_interior_family_size(dim, ratio, expected):
    assert len(lattice_offsets(dim, ratio)) == expected
    n = 13
    if dim == 2:
        x, y = W.grid_2d(n, n, 1e-3); z = None
        centre = (n // 2) + n * (n // 2)
    else:
        x, y, z = W.grid_3d(n, n, n, 1e-3)
        centre = (n // 2) * (1 + n + n * n)
    rp, col = O.family(x, y, z, ratio * 1e-3)
    assert rp[centre + 1] - rp[centre] == expected


def _jittered(dim, n, seed):
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 1.0, size=(dim, n))
    return [pts[k] for k in range(dim)]


@pytest.mark.parametrize("dim", [2, 3])
def test_family_binned_equals_bruteforce(dim):
    pts = _jittered(dim, 700, seed=dim)
    x, y = pts[0], pts[1]
    z = pts[2] if dim == 3 else None
    if dim == 2:
        cracks = [(0.1, 0.52, 0, 0.63, 0.41, 0, 0, 0, 0)]
    else:
        cracks = [(0.2, 0.1, 0.3, 0.8, 0.2, 0.35, 0.25, 0.9, 0.4)]
    for cr in ([], cracks):
        a = O.family(x, y, z, 0.11, cr, method="bruteforce")
        b = O.family(x, y, z, 0.11, cr, method="binned")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # brute force itself against a direct numpy distance test (no crack)
    P = np.stack(pts, 1)
    d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    ref = [np.nonzero((d2[i] <= 0.11 ** 2) & (np.arange(P.shape[0]) != i))[0] for i in range(P.shape[0])]
    rp, col = O.family(x, y, z, 0.11, [], method="bruteforce")
    for i in range(P.shape[0]):
        assert np.array_equal(col[rp[i]:rp[i + 1]], ref[i])


def _cut_exact_2d(a, b, p0, p1):
    """Exact rational segment test with the same tie semantics (strict sides, closed crack)."""
    F = Fraction
    a = [F(v) for v in a]; b = [F(v) for v in b]; p0 = [F(v) for v in p0]; p1 = [F(v) for v in p1]
    dx, dy = p1[0] - p0[0], p1[1] - p0[1]
    sa = dx * (a[1] - p0[1]) - dy * (a[0] - p0[0])
    sb = dx * (b[1] - p0[1]) - dy * (b[0] - p0[0])
    if not ((sa > 0 and sb < 0) or (sa < 0 and sb > 0)):
        return False
    t = sa / (sa - sb)
    px, py = a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])
    lam = ((px - p0[0]) * dx + (py - p0[1]) * dy) / (dx * dx + dy * dy)
    return 0 <= lam <= 1


def test_precrack_filter_exact_2d():
    """Bond removal by the pre-crack of configuration 2 (scaled down) vs exact rational arithmetic."""
    w = W.cracked_plate(nx=40, ny=16, dx=1.0, crack_cells=20.125)
    full = O.family(w.x, w.y, None, w.delta, [])
    cut = O.family(w.x, w.y, None, w.delta, w.cracks)
    c = w.cracks[0]
    removed = 0
    for i in range(w.n):
        nb_full = set(full[1][full[0][i]:full[0][i + 1]].tolist())
        nb_cut = set(cut[1][cut[0][i]:cut[0][i + 1]].tolist())
        for j in nb_full:
            exp_cut = _cut_exact_2d((w.x[i], w.y[i]), (w.x[j], w.y[j]), c[0:2], c[3:5])
            assert (j not in nb_cut) == exp_cut
            removed += exp_cut
    assert removed > 0


def test_notch_filter_exact_3d():
    """The 45-degree notch of configuration 3 (scaled down) vs an exact integer-lattice test."""
    nx, ny, nz = 24, 12, 6
    w = W.notched_block(nx=nx, ny=ny, nz=nz, dx=1.0, notch_cells=9.5)
    full = O.family(w.x, w.y, w.z, w.delta, [])
    cut = O.family(w.x, w.y, w.z, w.delta, w.cracks)
    ylo = Fraction(7537, 10000) * ny
    removed = 0
    for i in range(w.n):
        ii, jj, kk = i % nx, (i // nx) % ny, i // (nx * ny)
        nb_cut = set(cut[1][cut[0][i]:cut[0][i + 1]].tolist())
        for j in full[1][full[0][i]:full[0][i + 1]]:
            i2, j2, k2 = j % nx, (j // nx) % ny, j // (nx * ny)
            sa, sb = Fraction(2 * (ii - kk) - 19, 2), Fraction(2 * (i2 - k2) - 19, 2)
            exp_cut = False
            if (sa > 0) != (sb > 0):
                t = sa / (sa - sb)
                py = Fraction(2 * jj + 1, 2) + t * (j2 - jj)
                exp_cut = ylo <= py <= ny + 1
            assert (int(j) not in nb_cut) == exp_cut
            removed += exp_cut
    assert removed > 0


# --------------------------------------------------------------------------- Eq 1.9 weighted volume
@pytest.mark.parametrize("dim,ratio,expected", [(2, 3.015, 136), (2, 4.015, 384), (3, 3.015, 708)])
def test_interior_weighted_volume_lattice_sum(dim, ratio, expected):
    offs = lattice_offsets(dim, ratio)
    assert sum(sum(c * c for c in k) for k in offs) == expected
    dx, n = 1e-3, 13
    if dim == 2:
        x, y = W.grid_2d(n, n, dx); z = None
        centre = (n // 2) + n * (n // 2)
    else:
        x, y, z = W.grid_3d(n, n, n, dx)
        centre = (n // 2) * (1 + n + n * n)
    vol = np.full(x.size, dx ** dim)
    rp, col = O.family(x, y, z, ratio * dx)
    m = O.weighted_volume(x, y, z, vol, rp, col)
    assert m[centre] == pytest.approx(expected * dx ** (dim + 2), rel=1e-12)


def test_weighted_volume_approaches_continuum():
    """Eq 1.9 with w = 1 integrates to pi delta^4 / 2 (2D) and 4 pi delta^5 / 5 (3D); the lattice sums
    the oracle reproduces (checked at ratios 6.015 and 12.015 here) converge to them, oscillating."""
    def lattice_m(dim, ratio):
        R = int(ratio)
        k = np.arange(-R, R + 1)
        g = np.meshgrid(*([k] * dim), indexing="ij")
        s = sum(c ** 2 for c in g)
        return int(s[(s > 0) & (s <= ratio * ratio)].sum())
    assert abs(lattice_m(2, 48.015) / (math.pi * 48.015 ** 4 / 2) - 1) < 0.005
    assert abs(lattice_m(3, 24.015) / (4 * math.pi * 24.015 ** 5 / 5) - 1) < 0.01
    for ratio in (6.015, 12.015):
        n = 2 * int(ratio) + 3
        x, y = W.grid_2d(n, n, 1.0)
        rp, col = O.family(x, y, None, ratio)
        m = O.weighted_volume(x, y, None, np.ones(x.size), rp, col)
        assert m[(n // 2) * (n + 1)] == lattice_m(2, ratio)


# --------------------------------------------------------------------------- Eqs 1.8, 1.15, 1.16
@pytest.mark.parametrize("model", [O.MODEL_3D, O.MODEL_PLANE_STRESS, O.MODEL_PLANE_STRAIN])
def test_constants_reproduce_classical_energy(model):
    """Continuum PD energy density under uniform strain equals 1/2 eps : C : eps.

    PD side (w = 1, Eq 1.20 form): W = (K - G/3)/(2A) theta^2 + G/2 <(n.eps.n)^2>, theta = (A/d) tr eps,
    with the angular mean taken by quadrature here.  Classical side: Lame form for 3D / plane strain,
    plane-stress reduced lambda* = 2 lambda mu / (lambda + 2 mu).
    """
    E, nu = 72e9, 0.22
    c = O.constants(model, E, nu)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    rng = np.random.default_rng(3)
    d = 3 if model == O.MODEL_3D else 2
    for _ in range(3):
        a = rng.normal(size=(d, d)); eps = 1e-4 * (a + a.T)
        tr = np.trace(eps)
        if d == 2:
            f = lambda ph: (np.array([np.cos(ph), np.sin(ph)]) @ eps @ np.array([np.cos(ph), np.sin(ph)])) ** 2
            mean = integrate.quad(f, 0, 2 * math.pi, epsabs=0, epsrel=1e-13)[0] / (2 * math.pi)
            lstar = 2 * lam * mu / (lam + 2 * mu) if model == O.MODEL_PLANE_STRESS else lam
        else:
            def f(ph, th):
                n = np.array([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)])
                return (n @ eps @ n) ** 2 * np.sin(th)
            mean = integrate.dblquad(f, 0, math.pi, 0, 2 * math.pi, epsabs=0, epsrel=1e-12)[0] / (4 * math.pi)
            lstar = lam
        theta = c["A"] / d * tr
        w_pd = (c["K"] - c["G"] / 3) / (2 * c["A"]) * theta ** 2 + c["G"] / 2 * mean
        w_cl = 0.5 * lstar * tr ** 2 + mu * np.sum(eps * eps)
        assert w_pd == pytest.approx(w_cl, rel=1e-10)


# --------------------------------------------------------------------------- Eqs 1.24-1.29
def _varpi_3d(z, delta):
    # m_l / m for the spherical cap beyond a plane at distance z (w = 1), by quadrature of |x|^2.
    g = lambda x3: 2 * math.pi * ((delta ** 2 - x3 ** 2) ** 2 / 4 + x3 ** 2 * (delta ** 2 - x3 ** 2) / 2)
    ml = integrate.quad(g, z, delta, epsabs=0, epsrel=1e-13)[0]
    return ml / (4 * math.pi * delta ** 5 / 5)


def _varpi_2d(z, delta):
    g = lambda x2: 2 * (delta ** 2 - x2 ** 2) ** 1.5 / 3 + 2 * x2 ** 2 * math.sqrt(delta ** 2 - x2 ** 2)
    ml = integrate.quad(g, z, delta, epsabs=0, epsrel=1e-13)[0]
    return ml / (math.pi * delta ** 4 / 2)


def test_beta_closed_forms_by_quadrature():
    """Eq 1.25 integrated numerically: 3D beta = 125 delta/1848 (Eq 1.27) and beta' = 5 delta/24 (the
    printed 5 delta/(24 pi) is off by pi); 2D beta = 1087 delta/(1250 pi^2), beta' = 4 delta/(5 pi)."""
    delta = 1.0
    b3 = integrate.quad(lambda z: _varpi_3d(z, delta) ** 2, 0, delta, epsrel=1e-12)[0]
    bp3 = integrate.quad(lambda z: _varpi_3d(z, delta), 0, delta, epsrel=1e-12)[0]
    assert b3 == pytest.approx(125 / 1848, rel=1e-9)
    assert bp3 == pytest.approx(5 / 24, rel=1e-9)
    assert abs(bp3 / (5 / (24 * math.pi)) - 1) > 1.0
    b2 = integrate.quad(lambda z: _varpi_2d(z, delta) ** 2, 0, delta, epsrel=1e-12)[0]
    bp2 = integrate.quad(lambda z: _varpi_2d(z, delta), 0, delta, epsrel=1e-12)[0]
    assert bp2 == pytest.approx(4 / (5 * math.pi), rel=1e-9)
    # Eq 1.29 prints a rounded coefficient: the integral is 1087.27 delta / (1250 pi^2).
    assert b2 == pytest.approx(1087 / (1250 * math.pi ** 2), rel=5e-4)


def test_critical_stretch_formulas():
    """The oracle's s_c against Eq 1.26 (3D, with the quadrature beta') / Eq 1.28 (2D) typed from the
    quadrature results above, and against the configuration values quoted with 5 digits."""
    E, nu, G0, delta = 30e9, 0.2, 50.0, 3.015e-3
    kappa, mu = E / (3 * (1 - 2 * nu)), E / (2 * (1 + nu))
    b = integrate.quad(lambda z: _varpi_3d(z, delta) ** 2, 0, delta, epsrel=1e-12)[0]
    bp = integrate.quad(lambda z: _varpi_3d(z, delta), 0, delta, epsrel=1e-12)[0]
    s3 = math.sqrt(G0 / ((9 * kappa - 15 * mu) * b + 15 * mu * bp))
    assert O.critical_stretch(O.MODEL_3D, E, nu, G0, delta) == pytest.approx(s3, rel=1e-9)
    assert O.critical_stretch(O.MODEL_3D, E, nu, G0, delta) == pytest.approx(6.7381e-4, rel=1e-4)
    assert O.critical_stretch(O.MODEL_3D, E, nu, G0, 3.015 * 5e-4) == pytest.approx(9.5292e-4, rel=1e-4)
    assert O.critical_stretch(O.MODEL_PLANE_STRESS, 72e9, 0.22, 3.8, 3.015 * 2.5e-4) == pytest.approx(
        2.7646e-4, rel=1e-4)


# --------------------------------------------------------------------------- stable time step
def _dt_crit(model, E, nu, rho, ratio, shape, dx=1e-3):
    from scipy.sparse.linalg import LinearOperator, eigsh
    if len(shape) == 2:
        x, y = W.grid_2d(*shape, dx); z = None; vol = np.full(x.size, dx * dx)
    else:
        x, y, z = W.grid_3d(*shape, dx); vol = np.full(x.size, dx ** 3)
    sim = O.OracleSim(model, E, nu, rho, ratio * dx, 0.0, 1.0, x, y, z, vol)
    mass = rho * vol

    def mv(v):
        _, f = sim.internal_force(v.reshape(sim.dim, sim.n))
        return (-f / mass).reshape(-1)

    op = LinearOperator((sim.dim * sim.n,) * 2, matvec=mv, dtype=np.float64)
    lam = eigsh(op, k=1, which="LA", tol=1e-10, return_eigenvectors=False)[0]
    return 2.0 / math.sqrt(lam)


def test_stable_dt_config1():
    """The explicit scheme of Eq 2.11 is stable for dt < 2/sqrt(lambda_max(M^-1 K)); configuration 1
    uses 0.8 x that bound.  (Eq 2.13 would allow delta/c' = 5.19e-7 s, above the true bound.)"""
    w = W.config1()
    dc = _dt_crit(w.model, w.E, w.nu, w.rho, 3.015, (40, 40))
    assert 0.8 * dc == pytest.approx(w.dt, rel=1e-4)
    lam_ = w.E * w.nu / ((1 + w.nu) * (1 - 2 * w.nu)); mu = w.E / (2 * (1 + w.nu))
    assert w.delta / math.sqrt((lam_ + 2 * mu) / w.rho) > dc


def test_stable_dt_3d_and_scaled_configs():
    dc = _dt_crit(O.MODEL_3D, 30e9, 0.2, 2400.0, 3.015, (32, 20, 16))
    assert 0.8 * dc == pytest.approx(W.config3().dt, rel=2e-4)
    assert 0.8 * dc * 0.5 == pytest.approx(W.config5().dt, rel=2e-4)
    c1 = W.config1()
    assert 0.25 * c1.dt == pytest.approx(W.config2().dt, rel=2e-4)


@pytest.mark.parametrize("ratio", [3.015, 4.015])
def test_batch_dt_coefficients(ratio):
    for nu in (0.1, 0.3, 0.45):
        C = _dt_crit(O.MODEL_PLANE_STRESS, 72e9, nu, 2440.0, ratio, (40, 40)) / (1e-3 * math.sqrt(2440 / 72e9))
        assert W.BATCH_DT_COEF[ratio] < C


# --------------------------------------------------------------------------- hand-worked cases
def test_two_particle_bond():
    """Two particles h apart along x, stretched by e.  With m = h^2 V: theta_i = A h e V / m = A e / h;
    Eq 2.2 with theta~ = 2 A e / (h^3 V), e~ = 2 e / (h^2 V) gives
    F_1 = [(K - G/3) theta~ h + G e~] V^2 = 2 [(K - G/3) A + G] e V / h^2 along +x (towards 2)."""
    h, V, e = 1e-3, 2e-9, 3e-9
    x = np.array([0.0, h]); y = np.zeros(2)
    sim = O.OracleSim(O.MODEL_PLANE_STRAIN, 1e9, 0.25, 1000.0, 1.5 * h, 0.0, 1e-9, x, y, None,
                      np.array([V, V]))
    assert sim.m == pytest.approx([h * h * V] * 2, rel=1e-15)
    th, f = sim.internal_force(np.array([[0.0, e], [0.0, 0.0]]))
    assert th == pytest.approx([sim.A * e / h] * 2, rel=1e-14)
    fx = 2 * ((sim.K - sim.G / 3) * sim.A + sim.G) * e * V / h ** 2
    assert f[0] == pytest.approx([fx, -fx], rel=1e-13)
    assert f[1] == pytest.approx([0.0, 0.0], abs=1e-30)


def test_three_particle_shear_is_zero_extension():
    """A transverse displacement of one end of a bond produces no linearized extension (Eq 2.7 keeps
    only the component along M), so no force and no dilatation."""
    h = 1.0
    x = np.array([0.0, h, 0.0]); y = np.array([0.0, 0.0, h])
    sim = O.OracleSim(O.MODEL_PLANE_STRESS, 1e9, 0.3, 1.0, 1.2 * h, 0.0, 1.0, x, y, None, np.ones(3))
    assert sim.nbonds == 4  # 0-1 and 0-2 in both directions; 1-2 is sqrt(2) h > delta
    u = np.array([[0.0, 0.0, 0.7], [0.0, 0.5, 0.0]])  # 1 moves along y, 2 along x: both transverse
    th, f = sim.internal_force(u)
    assert np.all(th == 0.0) and np.all(f == 0.0)


def test_damage_counts():
    """Eq 1.31 with unit weights: phi = broken share of the built family's volume."""
    x, y = W.grid_2d(6, 6, 1.0)
    vol = np.linspace(1.0, 2.0, 36)
    rp, col = O.family(x, y, None, 1.5)
    status = np.ones(col.size, dtype=np.uint8)
    status[::3] = 0
    phi = O.damage(vol, rp, col, status)
    for i in range(36):
        nb = col[rp[i]:rp[i + 1]]; st = status[rp[i]:rp[i + 1]]
        assert phi[i] == pytest.approx(1 - vol[nb][st == 1].sum() / vol[nb].sum(), rel=1e-14)
