"""Pins of the oracle's geometrically nonlinear bond kinematics (kin=NONLINEAR): e = |xi + eta| - |xi|
(Eq 1.10) and the force along the deformed bond M = Y / |Y| (Eq 1.13), with the force state of
Eq 1.14.  Each test would fail for a plausible mistake: the reference direction xi/|xi| instead of
Y/|Y| (rotation and angular-momentum tests), a wrong extension formula (stretch, two-particle and
energy tests), a sign (energy test), or the linearized failure stretch (rotated two-particle bond)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W

NL, LIN = O.NONLINEAR, O.LINEARIZED


def _sim(dim, n, kin, ratio=3.015, nonuniform=False, s0=0.0, dt=1e-8, E=72e9, nu=0.22):
    dx = 1e-3
    if dim == 2:
        x, y = W.grid_2d(n, n - 1, dx); z = None
        model = O.MODEL_PLANE_STRESS
    else:
        x, y, z = W.grid_3d(n, n - 1, n - 2, dx)
        model = O.MODEL_3D
    vol = np.full(x.size, dx ** dim)
    if nonuniform:
        vol = vol * np.random.default_rng(7).uniform(0.5, 1.5, x.size)
    return O.OracleSim(model, E, nu, 2440.0, ratio * dx, s0, dt, x, y, z, vol, kin=kin)


def _coords(sim):
    return np.stack([sim.x, sim.y] + ([sim.z] if sim.dim == 3 else []))


def _rotation(dim, angle, axis=(0.3, -0.5, 0.8)):
    if dim == 2:
        c, s = np.cos(angle), np.sin(angle)
        return np.array([[c, -s], [s, c]])
    a = np.asarray(axis, dtype=float); a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K  # Rodrigues


def _energy(sim, u, kin):
    """U = sum_i V_i [(K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j e_ij^2 V_j] (the energy whose
    derivative with respect to e is the force state of Eq 1.14), theta_i from Eq 1.6 and e_ij from
    Eq 1.10 (nonlinear) or the linearized extension, all recomputed here from the coordinates."""
    P = _coords(sim)
    U = 0.0
    for i in range(sim.n):
        js = sim.col[sim.row_ptr[i]:sim.row_ptr[i + 1]]
        st = sim.status[sim.row_ptr[i]:sim.row_ptr[i + 1]].astype(bool)
        xi = P[:, js] - P[:, [i]]
        xl = np.sqrt((xi ** 2).sum(0))
        eta = u[:, js] - u[:, [i]]
        if kin == NL:
            e = np.sqrt(((xi + eta) ** 2).sum(0)) - xl
        else:
            e = ((xi / xl) * eta).sum(0)
        e, xl, vj = e[st], xl[st], sim.vol[js][st]
        th = sim.A / sim.m[i] * (xl * e * vj).sum() if sim.m[i] > 0 else 0.0
        U += sim.vol[i] * ((sim.K - sim.G / 3) / (2 * sim.A) * th ** 2 + sim.G / (2 * sim.m[i]) * (e ** 2 * vj).sum())
    return U


def _break_symmetric(sim, every):
    sim.status[::every] = 0
    for i in range(sim.n):
        for b in range(sim.row_ptr[i], sim.row_ptr[i + 1]):
            j = sim.col[b]
            bb = sim.row_ptr[j] + np.searchsorted(sim.col[sim.row_ptr[j]:sim.row_ptr[j + 1]], i)
            if sim.status[b] == 0:
                sim.status[bb] = 0


@pytest.mark.parametrize("dim", [2, 3])
def test_finite_rigid_rotation_gives_no_force(dim):
    """u = (R - I) x + c with a 35 degree rotation: every bond keeps its length, so theta = 0 and
    F = 0 up to rounding; the linearized kinematics gives forces of the order of a 20 % strain."""
    sim = _sim(dim, 9 if dim == 2 else 6, NL)
    P = _coords(sim)
    R = _rotation(dim, np.deg2rad(35.0))
    u = (R - np.eye(dim)) @ P + np.arange(1, dim + 1)[:, None] * 1e-3
    th, f = sim.internal_force(u)
    ref = np.abs(sim.internal_force(0.01 * P)[1]).max()  # a 1 % uniform stretch (boundary forces)
    assert np.abs(th).max() <= 1e-12 and np.abs(f).max() <= 1e-10 * ref
    lin = _sim(dim, 9 if dim == 2 else 6, LIN)
    assert np.abs(lin.internal_force(u)[1]).max() > 1.0 * ref


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kin", [NL, LIN])
def test_force_is_minus_energy_gradient(dim, kin):
    """F_i = -dU/du_i (the force of Eqs 1.11-1.14 summed over bond pairs), checked by central
    differences along random directions at a large random displacement (|u| ~ 5 % of dx), with
    non-uniform volumes and symmetric broken bonds."""
    sim = _sim(dim, 6 if dim == 2 else 4, kin, nonuniform=True)
    _break_symmetric(sim, 5)
    rng = np.random.default_rng(11 + dim)
    u = 5e-5 * rng.normal(size=(dim, sim.n))
    _, f = sim.internal_force(u)
    for _ in range(3):
        d = rng.normal(size=u.shape) * 1e-5
        h = 1e-3
        dU = (_energy(sim, u + h * d, kin) - _energy(sim, u - h * d, kin)) / (2 * h)
        assert dU == pytest.approx(np.sum(-f * d), rel=1e-7)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_stretch_dilatation_closed_form(dim):
    """u = (lambda - 1) x with lambda = 1.05: every bond has e = (lambda - 1) |xi|, so an interior
    particle has theta = A (lambda - 1) exactly (Eq 1.6 with Eq 1.9) and zero force."""
    n = 14 if dim == 2 else 16
    sim = _sim(dim, n, NL)
    P = _coords(sim)
    th, f = sim.internal_force(0.05 * P)
    delta, dx = 3.015e-3, 1e-3
    inner = np.all((P > 2 * delta) & (P < P.max(axis=1, keepdims=True) + 0.5 * dx - 2 * delta), axis=0)
    assert inner.sum() > 0
    assert np.allclose(th[inner], sim.A * 0.05, rtol=1e-12, atol=0)
    assert np.abs(f[:, inner]).max() <= 1e-11 * np.abs(f).max()


def test_two_particles_rotated_and_stretched():
    """Two particles h apart along x; particle 1 moves by (a, t).  Y = (h + a, t), e = |Y| - h,
    M = Y / |Y|, m = h^2 V, theta = A h e V / m on both, and
    F_0 = [(K - G/3) 2 theta h / m + 2 G e / m] V^2 M (Eq 1.14 summed over the pair)."""
    h, V = 1e-3, 1e-6
    x, y = np.array([0.0, h]), np.array([0.0, 0.0])
    sim = O.OracleSim(O.MODEL_PLANE_STRESS, 72e9, 0.22, 2440.0, 1.5 * h, 0.0, 1e-8, x, y, None,
                      np.full(2, V), kin=NL)
    a, t = 0.2 * h, 0.4 * h
    u = np.array([[0.0, a], [0.0, t]])
    th, f = sim.internal_force(u)
    Y = np.array([h + a, t]); yl = np.linalg.norm(Y)
    e = yl - h
    m = h * h * V
    theta = sim.A * h * e * V / m
    F0 = ((sim.K - sim.G / 3) * 2 * theta * h / m + 2 * sim.G * e / m) * V * V * Y / yl
    assert np.allclose(th, theta, rtol=1e-14)
    assert np.allclose(f[:, 0], F0, rtol=1e-13) and np.allclose(f[:, 1], -F0, rtol=1e-13)


def test_rotated_bond_breaks_only_with_nonlinear_kinematics():
    """A pure transverse motion t of one end stretches the bond by sqrt(1 + (t/h)^2) - 1 (Eq 1.10):
    with t/h = 0.05 that is 1.249e-3 > s0 = 1e-3, so the bond breaks (Eq 1.30); the linearized
    extension of the same motion is zero and the bond survives."""
    h, V = 1e-3, 1e-6
    x, y = np.array([0.0, h]), np.array([0.0, 0.0])
    u = np.array([[0.0, 0.0], [0.0, 0.05 * h]])
    res = {}
    for kin in (NL, LIN):
        st = np.ones(2, dtype=np.uint8)
        rp, col = O.family(x, y, None, 1.5 * h)
        nb, _ = O.failure(x, y, None, rp, col, st, 1e-3, u, kin=kin)
        res[kin] = (nb, st.copy())
    assert res[NL][0] == 2 and not res[NL][1].any()
    assert res[LIN][0] == 0 and res[LIN][1].all()


@pytest.mark.parametrize("dim", [2, 3])
def test_small_displacement_limit_is_the_linearized_force(dim):
    """F_nonlinear(eps u0) - F_linearized(eps u0) is second order in eps: the relative difference
    falls tenfold when eps does."""
    n = 8 if dim == 2 else 5
    snl, sl = _sim(dim, n, NL), _sim(dim, n, LIN)
    u0 = np.random.default_rng(5).normal(size=(dim, snl.n)) * 1e-3
    rel = []
    for eps in (1e-3, 1e-4):
        fn, fl = snl.internal_force(eps * u0)[1], sl.internal_force(eps * u0)[1]
        rel.append(np.linalg.norm(fn - fl) / np.linalg.norm(fl))
    assert rel[0] < 0.1 and 7.0 < rel[0] / rel[1] < 13.0


def _momenta(sim):
    q = _coords(sim) + sim.u
    mass = sim.rho * sim.vol
    p = (mass * sim.v).sum(axis=1)
    if sim.dim == 2:
        L = (mass * (q[0] * sim.v[1] - q[1] * sim.v[0])).sum()
    else:
        L = (mass * np.cross(q.T, sim.v.T).T).sum(axis=1)
    return p, np.atleast_1d(L)


@pytest.mark.parametrize("dim", [2, 3])
def test_spinning_body_conserves_angular_momentum(dim):
    """A free body turned rigidly by 35 degrees and spun at omega: the pair forces act along the
    current bond (M = Y/|Y|), so the integrator of Eq 2.11 conserves sum_i rho V_i (x_i + u_i^n) x v_i^n
    exactly in exact arithmetic (the drift term q_n x v_n cancels and the pair torques vanish).  With
    M = xi/|xi| (linearized) the turned body is under a spurious compression along the reference
    bond directions, those forces are not central in the turned body, and the angular momentum
    drifts."""
    res = {}
    for kin in (NL, LIN):
        sim = _sim(dim, 8 if dim == 2 else 5, kin, dt=2e-7)
        P = _coords(sim)
        c = P.mean(axis=1, keepdims=True)
        R = _rotation(dim, np.deg2rad(35.0))
        r = R @ (P - c)
        w = np.array([0.0, 0.0, 2e3]) if dim == 2 else np.array([300.0, -500.0, 800.0])
        r3 = np.vstack([r, np.zeros((1, sim.n))]) if dim == 2 else r
        v0 = np.cross(w, r3.T).T[:dim]
        sim.set_state(r + c - P, v0)
        sim.step(1)
        p1, L1 = _momenta(sim)
        sim.step(300)
        p2, L2 = _momenta(sim)
        res[kin] = (np.abs(p2 - p1).max() / (np.abs(p1).max() + np.linalg.norm(L1) / 1e-3),
                    np.linalg.norm(L2 - L1) / np.linalg.norm(L1))
    assert res[NL][0] <= 1e-12 and res[LIN][0] <= 1e-12  # linear momentum: both (Newton's third law)
    assert res[NL][1] <= 1e-12
    assert res[LIN][1] >= 1e-6
