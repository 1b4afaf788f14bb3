"""Configuration 5 at full size (400 x 200 x 100 = 8M particles, ~9.6e8 directed bonds) on the GPU,
every particle compared with the oracle after two steps from a random state (GPU only; the oracle
runs on all host cores and holds the ~5 GB family in host memory).  FP64 bars as in
tests/parity.py: u and v in rel-L2 and per particle, theta per particle, and the bond status exactly
while the oracle's smallest stretch margin stays above 1e-9."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, Simulation
from paper_2309_11273_gb300 import workloads as W

pytestmark = pytest.mark.gpu


from parity import assert_fp64_close, compare, elem, elem_v, rel


def test_config5_full_size_two_steps():
    w = W.notched_block(nx=400, ny=200, nz=100, dx=5e-4, nsteps=1000, dt=1.895e-7, seed=11, amp=5e-7)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
    ref.set_state(w.initial_u(), w.initial_v())
    assert ref.nbonds > 9.4e8
    margins, _ = ref.step(2)
    assert int((ref.status == 0).sum()) > 0  # stretches near 2 s0 from the random state: bonds break
    for precision, tol in ((PD_FP64, 1e-12), (PD_MIXED, 1e-4)):
        sim = Simulation(w, s0=s0, precision=precision)
        assert sim.nbonds == ref.nbonds
        sim.step(2)
        u, v, th = sim.state()
        if precision == PD_FP64:
            assert_fp64_close(compare(u, v, th, ref, with_global_theta=False), tol)
            if margins.min() > 1e-9:
                _, _, intact = sim.neighbors()
                assert np.array_equal(intact, ref.status)
        else:
            assert rel(u, ref.u) <= tol and rel(v, ref.v) <= tol, (precision, rel(u, ref.u), rel(v, ref.v))
        sim.close()


def _config5_small_amp():
    return W.notched_block(nx=400, ny=200, nz=100, dx=5e-4, nsteps=1000, dt=1.895e-7, seed=11, amp=5e-7)


def test_config5_full_size_nonlinear_two_steps():
    """Nonlinear bonds (Eqs 1.10, 1.13) at full size: FP64 against the oracle's kin=NONLINEAR."""
    from paper_2309_11273_gb300 import PD_NONLINEAR
    w = _config5_small_amp()
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks, kin=O.NONLINEAR)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
    ref.set_state(w.initial_u(), w.initial_v())
    ref.step(2)
    sim = Simulation(w, s0=s0, kinematics=PD_NONLINEAR)
    sim.step(2)
    u, v, _ = sim.state()
    sim.close()
    assert rel(u, ref.u) <= 1e-12 and rel(v, ref.v) <= 1e-12
    assert elem(u, ref.u) <= 1e-12 and elem_v(v, ref) <= 1e-12


def test_config5_full_size_adr_three_iterations():
    """Adaptive dynamic relaxation at full size (8M particles, one damping reduction over all of
    them): three iterations against the oracle's from rest under the twist, without bond failure.
    (A random start is not used: the local stiffness -(g^n - g^{n-1}) / (lambda v) divides by
    velocity components that are tiny but not zero, so the damping's Rayleigh quotient becomes a
    sum of huge terms of both signs whose rounding two correct evaluations do not share.)"""
    from paper_2309_11273_gb300 import _binding as B
    w = W.notched_block(nx=400, ny=200, nz=100, dx=5e-4, nsteps=1000, dt=1.895e-7)
    s0 = 0.0
    rate = w.rotation_rate(9.5292e-4)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, rate)
    ref.set_state(w.initial_u(), w.initial_v())
    ref.adr_step(3)
    sim = Simulation(w, s0=s0, rate=rate)
    sim.set_option(B.PD_OPT_SOLVER, B.PD_SOLVER_ADR)
    sim.step(3)
    u, v, _ = sim.state()
    sim.close()
    assert rel(u, ref.u) <= 1e-12 and np.linalg.norm(v - ref.v) <= 1e-12 * np.linalg.norm(ref.u)
    assert elem(u, ref.u) <= 1e-12 and np.abs(v - ref.v).max() <= 1e-12 * np.abs(ref.u).max()
