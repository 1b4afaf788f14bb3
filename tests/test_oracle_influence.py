"""Pins of the oracle with the influence function w = delta / |xi| (infl = W_INV).

Eq 1.9 defines the weighted volume with a general influence function w and the paper refers there to
a published catalogue of forms; it uses w = 1 itself (Section 2.3, where the critical stretch is
derived).  w enters the dilatation (Eq 1.6), the force state (Eq 1.14, so the bond force of Eq 2.2)
and the damage (Eq 1.31).  These tests pin the oracle's w = delta / |xi| against values fixed without
it: integer lattice sums (m_i = delta V h sum_n |n| in the interior), its continuum limit, the
uniform-strain dilatation (A/d) tr(eps) (the family sum of w xi xi^T V_j is (m / d) I for any radial
w on a cubic lattice), zero force under rigid motions, Newton's third law, F = -grad U against an
energy written here, and the damage by direct count.  Dropping w from any one of m, theta or the
force fails the energy test (a planted mistake is checked below).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W


def lattice_sum_abs(dim, ratio):
    """sum of |n| over the integer vectors 0 < |n| <= ratio (the closed ball of Section 2.1)."""
    R = int(ratio)
    k = np.arange(-R, R + 1)
    g = np.meshgrid(*([k] * dim), indexing="ij")
    s = sum(c.astype(np.int64) ** 2 for c in g)
    sel = (s > 0) & (s <= ratio * ratio)
    return float(np.sqrt(s[sel]).sum())


@pytest.mark.parametrize("dim,ratio", [(2, 3.015), (2, 4.015), (3, 3.015)])
def test_interior_weighted_volume_lattice_sum(dim, ratio):
    dx, n = 1e-3, 13
    if dim == 2:
        x, y = W.grid_2d(n, n, dx); z = None
        centre = (n // 2) + n * (n // 2)
    else:
        x, y, z = W.grid_3d(n, n, n, dx)
        centre = (n // 2) * (1 + n + n * n)
    vol = np.full(x.size, dx ** dim)
    delta = ratio * dx
    rp, col = O.family(x, y, z, delta)
    m = O.weighted_volume(x, y, z, vol, rp, col, O.W_INV, delta)
    # m = sum_j (delta / |xi|) |xi|^2 V = delta V dx sum |n|
    assert m[centre] == pytest.approx(delta * dx ** dim * dx * lattice_sum_abs(dim, ratio), rel=1e-13)
    # and it is not the w = 1 value
    m1 = O.weighted_volume(x, y, z, vol, rp, col)
    assert abs(m[centre] / m1[centre] - 1) > 0.05


def test_weighted_volume_approaches_continuum():
    """int_ball (delta / r) r^2 dV = pi delta^5 (3D) and 2 pi delta^4 / 3 per unit thickness (2D)."""
    for dim, ratio, cont, tol in ((2, 60.015, 2 * math.pi / 3, 0.01), (3, 20.015, math.pi, 0.02)):
        lat = ratio * lattice_sum_abs(dim, ratio)  # m / (V h^(dim+2)) with delta = ratio h
        assert abs(lat / (cont * ratio ** (dim + 2)) - 1) < tol, (dim, lat / (cont * ratio ** (dim + 2)))


def _sim(dim, n=12, ratio=3.015, nonuniform=False, seed=0, infl=O.W_INV):
    dx = 1e-3
    if dim == 2:
        x, y = W.grid_2d(n, n, dx); z = None
        model = O.MODEL_PLANE_STRESS
    else:
        x, y, z = W.grid_3d(n, n - 2, n - 4, dx)
        model = O.MODEL_3D
    vol = np.full(x.size, dx ** dim)
    if nonuniform:
        vol = vol * np.random.default_rng(seed + 100).uniform(0.5, 1.5, x.size)
    return O.OracleSim(model, 72e9, 0.22, 2440.0, ratio * dx, 0.0, 1e-8, x, y, z, vol, infl=infl)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_strain_interior(dim):
    sim = _sim(dim, n=16 if dim == 2 else 18)
    rng = np.random.default_rng(1)
    a = rng.normal(size=(dim, dim)); eps = 1e-4 * (a + a.T)
    P = np.stack([sim.x, sim.y] + ([sim.z] if dim == 3 else []))
    th, f = sim.internal_force(eps @ P)
    dx, delta = 1e-3, 3.015e-3
    inner = np.all((P > 2 * delta) & (P < P.max(axis=1, keepdims=True) + 0.5 * dx - 2 * delta), axis=0)
    assert inner.sum() > 0
    assert np.allclose(th[inner], sim.A / dim * np.trace(eps), rtol=1e-12, atol=0)
    assert np.abs(f[:, inner]).max() <= 1e-11 * np.abs(f).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_motions_and_third_law(dim):
    sim = _sim(dim, nonuniform=True)
    P = np.stack([sim.x, sim.y] + ([sim.z] if dim == 3 else []))
    rng = np.random.default_rng(2)
    _, fr = sim.internal_force(1e-6 * rng.normal(size=P.shape))
    ref = np.abs(fr).max()
    assert np.abs(fr.sum(axis=1)).max() <= 1e-13 * np.abs(fr).sum()
    t = rng.normal(size=(dim, 1)) * 1e-3
    th, f = sim.internal_force(np.repeat(t, sim.n, axis=1))
    assert np.abs(th).max() < 1e-12 and np.abs(f).max() <= 1e-9 * ref
    a = rng.normal(size=(dim, dim)); Wm = 1e-4 * (a - a.T)
    th, f = sim.internal_force(Wm @ P)
    assert np.abs(th).max() < 1e-14 and np.abs(f).max() <= 1e-9 * ref


def _energy(sim, u, w_in_m=True, w_in_theta=True):
    """U = sum_i V_i [ (K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j w e_ij^2 V_j ] with
    theta_i = (A / m_i) sum_j w |xi| e_ij V_j and m_i = sum_j w |xi|^2 V_j, all written out here."""
    P = np.stack([sim.x, sim.y] + ([sim.z] if sim.dim == 3 else []))
    U = 0.0
    for i in range(sim.n):
        js = sim.col[sim.row_ptr[i]:sim.row_ptr[i + 1]]
        st = sim.status[sim.row_ptr[i]:sim.row_ptr[i + 1]].astype(bool)
        xi = P[:, js] - P[:, [i]]
        xl = np.sqrt((xi ** 2).sum(0))
        w = sim.delta / xl
        e = ((xi / xl) * (u[:, js] - u[:, [i]])).sum(0)
        V = sim.vol[js]
        m = ((w if w_in_m else 1.0) * xl ** 2 * V).sum()
        th = sim.A / m * ((w if w_in_theta else 1.0) * xl * e * V)[st].sum()
        U += sim.vol[i] * ((sim.K - sim.G / 3) / (2 * sim.A) * th ** 2 + sim.G / (2 * m) * (w * e ** 2 * V)[st].sum())
    return U


@pytest.mark.parametrize("dim", [2, 3])
def test_force_is_minus_energy_gradient(dim):
    sim = _sim(dim, n=8, nonuniform=True)
    sim.status[::7] = 0
    for i in range(sim.n):
        for b in range(sim.row_ptr[i], sim.row_ptr[i + 1]):
            j = sim.col[b]
            bb = sim.row_ptr[j] + np.searchsorted(sim.col[sim.row_ptr[j]:sim.row_ptr[j + 1]], i)
            if sim.status[b] == 0:
                sim.status[bb] = 0
    rng = np.random.default_rng(4)
    u = 1e-6 * rng.normal(size=(dim, sim.n))
    _, f = sim.internal_force(u)
    assert 0.5 * np.sum(-f * u) == pytest.approx(_energy(sim, u), rel=1e-12)
    d = rng.normal(size=u.shape) * 1e-6
    h = 1e-3
    dU = (_energy(sim, u + h * d) - _energy(sim, u - h * d)) / (2 * h)
    assert dU == pytest.approx(np.sum(-f * d), rel=1e-9)
    # a planted mistake (w left out of the dilatation) breaks the identity
    bad = 0.5 * np.sum(-f * u)
    assert abs(bad / _energy(sim, u, w_in_theta=False) - 1) > 1e-6


def test_damage_counts():
    """Eq 1.31: phi = 1 - sum_j w rho V_j / sum_j w V_j with w = delta / |xi|, by direct count."""
    x, y = W.grid_2d(6, 6, 1.0)
    vol = np.linspace(1.0, 2.0, 36)
    delta = 1.5
    rp, col = O.family(x, y, None, delta)
    status = np.ones(col.size, dtype=np.uint8)
    status[::3] = 0
    phi = O.damage(vol, rp, col, status, x, y, None, O.W_INV, delta)
    D = O.damage_denominator(vol, rp, col, x, y, None, O.W_INV, delta)
    for i in range(36):
        nb = col[rp[i]:rp[i + 1]]; st = status[rp[i]:rp[i + 1]]
        w = delta / np.hypot(x[nb] - x[i], y[nb] - y[i])
        assert D[i] == pytest.approx((w * vol[nb]).sum(), rel=1e-14)
        assert phi[i] == pytest.approx(1 - (w * vol[nb])[st == 1].sum() / (w * vol[nb]).sum(), rel=1e-14)


def test_dynamics_differ_from_w_one_and_conserve_shadow_energy():
    """A short free vibration with w = delta / |xi| differs from w = 1 and conserves the leapfrog
    shadow energy U(u^n) + 1/2 sum rho V v^n . v^{n+1} (Eq 2.11), with the energy above."""
    w = W.plate_vibration(nx=10, ny=10, nsteps=50, dt=2e-7)
    res = {}
    for infl in (O.W_ONE, O.W_INV):
        sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, None, w.vol, infl=infl)
        sim.set_state(w.initial_u())
        H = []
        for _ in range(5):
            u0, v0 = sim.u.copy(), sim.v.copy()
            sim.step(1)
            if infl == O.W_INV:
                H.append(_energy(sim, u0) + 0.5 * np.sum(w.rho * sim.vol * (v0 * sim.v)))
            sim.step(9)
        res[infl] = sim.u.copy()
    assert np.linalg.norm(res[O.W_INV] - res[O.W_ONE]) > 1e-3 * np.linalg.norm(res[O.W_ONE])
    assert np.abs(np.array(H) - H[0]).max() <= 1e-10 * abs(H[0])
