"""Pins of the oracle's adaptive dynamic relaxation (the quasi-static solver of Section 4.4): the
fictitious density bounds the stiffness as its Gerschgorin construction claims, and the iteration
converges to the static solution that a direct dense solve of the same linear problem gives."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W


def _sim(dim, shape, nonuniform=False, kin=O.LINEARIZED, model=None, nu=0.22):
    dx = 1e-3
    if dim == 2:
        x, y = W.grid_2d(*shape, dx); z = None
        model = O.MODEL_PLANE_STRESS if model is None else model
    else:
        x, y, z = W.grid_3d(*shape, dx)
        model = O.MODEL_3D
    vol = np.full(x.size, dx ** dim)
    if nonuniform:
        vol = vol * np.random.default_rng(3).uniform(0.6, 1.4, x.size)
    return O.OracleSim(model, 72e9, nu, 2440.0, 3.015 * dx, 0.0, 1.0, x, y, z, vol, kin=kin)


def _stiffness(sim):
    """S = -d f / d u (f = F / V, force density), dense (dim n x dim n), column by column: the
    linearized force is linear in u, so a unit displacement gives a column exactly."""
    n, d = sim.n, sim.dim
    S = np.zeros((d * n, d * n))
    for k in range(n):
        for b in range(d):
            u = np.zeros((d, n)); u[b, k] = 1.0
            f = sim.internal_force(u)[1] / sim.vol
            S[:, b * n + k] = -f.reshape(-1)
    return S  # rows / columns ordered component-major: index = comp * n + particle


@pytest.mark.parametrize("dim,shape,model,nu", [(2, (7, 6), O.MODEL_PLANE_STRESS, 0.22),
                                                (2, (6, 6), O.MODEL_PLANE_STRAIN, 0.45),
                                                (3, (5, 4, 4), O.MODEL_3D, 0.2), (3, (5, 4, 4), O.MODEL_3D, 0.45)])
def test_lambda_bounds_the_stiffness(dim, shape, model, nu):
    """4 lambda_i >= sum_k |S_(i,a),k| for every row (Gerschgorin bound, non-uniform volumes), within a
    factor 8 of the true row sum, and so every eigenvalue of L^-1 S lies in [0, 4]: the unit
    fictitious step is stable.  nu = 0.45 makes the dilatation term dominate (K - G/3 > G)."""
    sim = _sim(dim, shape, nonuniform=True, model=model, nu=nu)
    S = _stiffness(sim)
    lam = O.adr_lambda(sim.x, sim.y, sim.z, sim.vol, sim.row_ptr, sim.col, sim.m, sim.A, sim.K, sim.G)
    rows = np.abs(S).sum(axis=1).reshape(dim, sim.n).max(axis=0)
    assert np.all(4 * lam >= rows * (1 - 1e-12))
    assert np.all(4 * lam <= 8 * rows)
    L = np.tile(lam, dim)
    ev = np.linalg.eigvals(S / L[:, None]).real
    assert ev.max() <= 4.0 + 1e-9 and ev.min() >= -1e-9


def _clamped(dim, shape, kin=O.LINEARIZED):
    sim = _sim(dim, shape, kin=kin)
    flag = np.where(sim.x < 3e-3, O.FIXED, O.FREE).astype(np.uint8)
    b = np.zeros((dim, sim.n)); b[1] = -2e9  # downward body-force density [N/m^3]
    sim.set_bc(flag, b)
    sim.set_state(np.zeros((dim, sim.n)))
    return sim, flag, b


@pytest.mark.parametrize("dim,shape,iters", [(2, (12, 8), 3000), (3, (7, 5, 4), 3000)])
def test_adr_converges_to_the_direct_solution(dim, shape, iters):
    """Clamped block under a body force: ADR reaches the solution of S_ff u_f = b_f (direct dense
    solve of the same linearized problem) to 1e-7, with damping from the Rayleigh quotient."""
    sim, flag, b = _clamped(dim, shape)
    S = _stiffness(sim)
    free = np.tile(flag == O.FREE, dim)
    u_direct = np.zeros(dim * sim.n)
    u_direct[free] = np.linalg.solve(S[np.ix_(free, free)], b.reshape(-1)[free])
    damping, _, _ = sim.adr_step(iters)
    assert damping[0] == 0.0 and np.all(damping[1:] >= 0.0) and damping.max() > 0.0
    err = np.linalg.norm(sim.u.reshape(-1) - u_direct) / np.linalg.norm(u_direct)
    assert err <= 1e-7, err


def test_adr_calls_continue_the_same_iteration():
    """Two calls of k and m iterations equal one call of k + m (state v, previous force carried)."""
    s1, _, _ = _clamped(2, (10, 6))
    s1.adr_step(150)
    s1.adr_step(250)
    s2, _, _ = _clamped(2, (10, 6))
    s2.adr_step(400)
    assert np.array_equal(s1.u, s2.u)


def test_nonlinear_adr_reaches_equilibrium():
    """Nonlinear kinematics: the ADR state satisfies f(u) + b = 0 on the free particles to 1e-8 of
    |b| (the residual is evaluated with the oracle's force, independently of the iteration)."""
    sim, flag, b = _clamped(2, (12, 8), kin=O.NONLINEAR)
    sim.adr_step(4000)
    _, F = sim.internal_force()
    r = (F / sim.vol + b)[:, flag == O.FREE]
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(b[:, flag == O.FREE])
