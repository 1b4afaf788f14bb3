"""Invariants of the oracle that a dropped term, a wrong sign, index or volume would violate."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W


def _sim(dim, n=12, ratio=3.015, model=None, nonuniform=False, seed=0, s0=0.0, E=72e9, nu=0.22):
    dx = 1e-3
    if dim == 2:
        x, y = W.grid_2d(n, n, dx); z = None
        model = O.MODEL_PLANE_STRESS if model is None else model
    else:
        x, y, z = W.grid_3d(n, n - 2, n - 4, dx)
        model = O.MODEL_3D
    vol = np.full(x.size, dx ** dim)
    if nonuniform:
        vol = vol * np.random.default_rng(seed + 100).uniform(0.5, 1.5, x.size)
    return O.OracleSim(model, E, nu, 2440.0, ratio * dx, s0, 1e-8, x, y, z, vol)


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_strain_interior(dim):
    """u = eps x (symmetric eps): interior theta = (A/d) tr(eps) and interior force = 0 (Section 2.2:
    for a symmetric family sum_j xi xi^T V_j = (m/d) I)."""
    sim = _sim(dim, n=16 if dim == 2 else 18)
    rng = np.random.default_rng(1)
    a = rng.normal(size=(dim, dim)); eps = 1e-4 * (a + a.T)
    P = np.stack([sim.x, sim.y] + ([sim.z] if dim == 3 else []))
    th, f = sim.internal_force(eps @ P)
    dx, delta = 1e-3, 3.015e-3
    inner = np.all((P > 2 * delta) & (P < P.max(axis=1, keepdims=True) + 0.5 * dx - 2 * delta), axis=0)
    assert inner.sum() > 0
    expected = sim.A / dim * np.trace(eps)
    assert np.allclose(th[inner], expected, rtol=1e-12, atol=0)
    scale = np.abs(f).max()
    assert np.abs(f[:, inner]).max() <= 1e-11 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_motions_give_no_force(dim):
    sim = _sim(dim)
    P = np.stack([sim.x, sim.y] + ([sim.z] if dim == 3 else []))
    rng = np.random.default_rng(2)
    ref = np.abs(sim.internal_force(1e-6 * rng.normal(size=P.shape))[1]).max()
    t = rng.normal(size=(dim, 1)) * 1e-3
    th, f = sim.internal_force(np.repeat(t, sim.n, axis=1))
    assert np.abs(th).max() < 1e-12 and np.abs(f).max() <= 1e-9 * ref
    a = rng.normal(size=(dim, dim)); Wm = 1e-4 * (a - a.T)  # infinitesimal rotation
    th, f = sim.internal_force(Wm @ P)
    assert np.abs(th).max() < 1e-14 and np.abs(f).max() <= 1e-9 * ref


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_third_law(dim):
    """F_j^{xi_ij} = -F_i^{xi_ij} (Eq 2.2), so the internal forces sum to zero."""
    sim = _sim(dim, nonuniform=True)
    u = 1e-6 * np.random.default_rng(3).normal(size=(dim, sim.n))
    _, f = sim.internal_force(u)
    assert np.abs(f.sum(axis=1)).max() <= 1e-13 * np.abs(f).sum()


def _strain_energy(sim, u):
    """U = sum_i V_i [ (K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j e_ij^2 V_j ] (Eq 1.20 generalised to
    the two-constant 2D/3D form of Eq 1.14), with e_ij recomputed here from the coordinates."""
    th = O.dilatation(sim.x, sim.y, sim.z, sim.vol, sim.row_ptr, sim.col, sim.status, sim.m, sim.A, u)
    P = np.stack([sim.x, sim.y] + ([sim.z] if sim.dim == 3 else []))
    U = 0.0
    for i in range(sim.n):
        js = sim.col[sim.row_ptr[i]:sim.row_ptr[i + 1]]
        st = sim.status[sim.row_ptr[i]:sim.row_ptr[i + 1]].astype(bool)
        xi = P[:, js] - P[:, [i]]
        xl = np.sqrt((xi ** 2).sum(0))
        e = ((xi / xl) * (u[:, js] - u[:, [i]])).sum(0)
        U += sim.vol[i] * ((sim.K - sim.G / 3) / (2 * sim.A) * th[i] ** 2
                           + sim.G / (2 * sim.m[i]) * (e[st] ** 2 * sim.vol[js][st]).sum())
    return U


@pytest.mark.parametrize("dim", [2, 3])
def test_force_is_minus_energy_gradient(dim):
    """F = -dU/du: the work identity 1/2 u.(-F(u)) = U(u) for the quadratic energy, plus a directional
    finite difference, with non-uniform volumes and some broken bonds."""
    sim = _sim(dim, n=9, nonuniform=True)
    sim.status[::7] = 0
    # keep the status symmetric: a bond is broken in both directions
    for i in range(sim.n):
        for b in range(sim.row_ptr[i], sim.row_ptr[i + 1]):
            j = sim.col[b]
            bb = sim.row_ptr[j] + np.searchsorted(sim.col[sim.row_ptr[j]:sim.row_ptr[j + 1]], i)
            if sim.status[b] == 0:
                sim.status[bb] = 0
    rng = np.random.default_rng(4)
    u = 1e-6 * rng.normal(size=(dim, sim.n))
    _, f = sim.internal_force(u)
    U = _strain_energy(sim, u)
    assert 0.5 * np.sum(-f * u) == pytest.approx(U, rel=1e-12)
    d = rng.normal(size=u.shape) * 1e-6
    h = 1e-3
    dU = (_strain_energy(sim, u + h * d) - _strain_energy(sim, u - h * d)) / (2 * h)
    assert dU == pytest.approx(np.sum(-f * d), rel=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_stiffness_symmetric_psd_with_rigid_null_space(dim):
    """The stiffness K = -dF/du (Eq 2.14) built column by column is symmetric PSD and its null space
    is exactly the d(d+1)/2 rigid modes."""
    sim = _sim(dim, n=8 if dim == 2 else 7, nonuniform=True)
    N = dim * sim.n
    K = np.zeros((N, N))
    for c in range(N):
        e = np.zeros(N); e[c] = 1.0
        K[:, c] = -sim.internal_force(e.reshape(dim, sim.n))[1].reshape(-1)
    sc = np.abs(K).max()
    assert np.abs(K - K.T).max() <= 1e-12 * sc
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    assert ev.min() > -1e-10 * sc
    assert int((ev < 1e-9 * sc).sum()) == dim * (dim + 1) // 2


def test_shadow_energy_conserved_config1():
    """Eq 2.11 is the leapfrog / Stormer-Verlet scheme, which conserves H_n = 1/2 v^{n+1}.M v^n
    + 1/2 u^n.K u^n exactly (up to rounding) for the linear undamped system, while the plain energy
    oscillates."""
    w = W.config1()
    sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, None, w.vol)
    sim.set_state(w.initial_u())
    mass = w.rho * w.vol
    H, E = [], []
    for n in range(400):
        un, vn = sim.u.copy(), sim.v.copy()
        sim.step(1)
        H.append(0.5 * np.sum(mass * sim.v * vn) + 0.5 * np.sum(un * -sim.f))
        E.append(0.5 * np.sum(mass * vn * vn) + 0.5 * np.sum(un * -sim.f))
    H = np.array(H); E = np.array(E)
    assert np.abs(H / H[0] - 1).max() < 1e-12
    assert np.abs(E / E[0] - 1).max() > 1e-3


def test_prescribed_rotation_and_clamp():
    """Appendix B boundary handling: fixed particles stay at rest, prescribed ones follow
    u = rate t a x (p - c) exactly at the end of every step."""
    w = W.notched_block(nx=10, ny=6, nz=5, dx=1e-3)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    rate = 1e3
    sim.set_bc(w.flag, None, w.axis_point, w.axis_dir, rate)
    sim.step(5)
    t = 5 * w.dt
    P = np.stack([w.x, w.y, w.z]) - w.axis_point[:, None]
    g = np.cross(w.axis_dir, P.T).T
    pres = w.flag == O.PRESCRIBED
    assert np.array_equal(sim.u[:, pres], rate * t * g[:, pres])
    assert np.all(sim.u[:, w.flag == O.FIXED] == 0) and np.all(sim.v[:, w.flag == O.FIXED] == 0)
    assert np.abs(sim.u[:, w.flag == O.FREE]).max() > 0


def test_failure_irreversible_and_symmetric():
    """Eq 1.30: bonds break when s >= s0 and never heal; both directed copies decide alike."""
    sim = _sim(2, n=10, s0=1e-3)
    P = np.stack([sim.x, sim.y])
    u = np.zeros_like(P); u[0] = 2e-3 * (P[0] > P[0].mean()) * 1e-3  # a jump across the middle
    nb1, mm = O.failure(sim.x, sim.y, None, sim.row_ptr, sim.col, sim.status, sim.s0, u)
    assert nb1 > 0
    for i in range(sim.n):
        for b in range(sim.row_ptr[i], sim.row_ptr[i + 1]):
            j = sim.col[b]
            bb = sim.row_ptr[j] + np.searchsorted(sim.col[sim.row_ptr[j]:sim.row_ptr[j + 1]], i)
            assert sim.status[b] == sim.status[bb]
    before = sim.status.copy()
    nb2, _ = O.failure(sim.x, sim.y, None, sim.row_ptr, sim.col, sim.status, sim.s0, -u)
    assert nb2 == 0 and np.array_equal(before, sim.status)


def test_thickness_cancels():
    """2D: scaling every volume by a thickness h leaves u, v and damage unchanged (bitwise for a
    power-of-two h)."""
    w = W.cracked_plate(nx=30, ny=12, dx=2.5e-4, crack_cells=15.125, sigma=4e7)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    out = []
    for h in (1.0, 4.0):
        sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, None, w.vol * h,
                          w.cracks)
        sim.set_bc(None, w.b)
        sim.step(200)
        out.append((sim.u.copy(), sim.damage()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_thread_count_does_not_change_results():
    w = W.config1()
    res = []
    orig = O.get_threads()
    for t in (1, 3):
        O.set_threads(t)
        sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, None, w.vol)
        sim.set_state(w.initial_u())
        sim.step(20)
        res.append(sim.u.copy())
    O.set_threads(orig)
    assert np.array_equal(res[0], res[1])


def test_edge_traction_response_is_mirror_symmetric():
    """The edge traction of the plate workloads (body force +-sigma/dx on the top and bottom rows)
    loads the uncracked plate symmetrically about its mid-plane: u_x(x, y) = u_x(x, -y) and
    u_y(x, y) = -u_y(x, -y) to rounding (mirrored particles sum their bonds in mirrored order).  A
    traction applied to one row only, on the wrong row or with one sign flipped breaks it."""
    w = W.cracked_plate(nx=40, ny=16, dx=2.5e-4, crack_cells=20.125, sigma=5e6)
    sim = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, None, w.vol)
    sim.set_bc(None, w.b)
    sim.step(300)
    u = sim.u.reshape(2, 16, 40)  # [component, row j, column i], rows at y = (j + 1/2) dx
    scale = np.abs(u).max()
    assert scale > 0.0
    assert np.abs(u[0] - u[0, ::-1]).max() <= 1e-12 * scale
    assert np.abs(u[1] + u[1, ::-1]).max() <= 1e-12 * scale
    assert u[1, -1].mean() > 0.0 > u[1, 0].mean()  # the top row moves up, the bottom row down
