"""Kalthoff-Winkler-like plane-strain impact (prescribed velocity, two notches) on the GPU against
the oracle (GPU only): FP64 to 1e-12 with exact bond status through crack initiation at the notch
tips; the mixed form with zero decisions differing from FP64 on its own state."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W
from parity import elem, elem_v

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _oracle(w, s0):
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, None, w.vol, w.cracks)
    ref.set_bc(w.flag, None, w.axis_point, w.axis_dir, 0.0, vp=w.vp)
    return ref


def test_kalthoff_reduced_fp64_parity_through_crack_initiation():
    w = W.kalthoff(nx=120, ny=60, dx=5e-4 * 402 / 120, notch_cells=30.125, gap_cells=30, nsteps=1500)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0)
    ref = _oracle(w, s0)
    exact = True
    for _ in range(5):
        margins, _ = ref.step(300)
        sim.step(300)
        exact = exact and margins.min() > 1e-9
        u, v, _ = sim.state()
        assert rel(u, ref.u) <= 1e-12 and rel(v, ref.v) <= 1e-12
        assert elem(u, ref.u) <= 1e-12 and elem_v(v, ref) <= 1e-12
        if exact:
            assert np.array_equal(sim.neighbors()[2], ref.status)
    assert (ref.status == 0).sum() > 0 and exact
    hit = w.flag == W.PRESCRIBED
    assert np.array_equal(u[:, hit], ref.u[:, hit])
    sim.close()


def test_kalthoff_reduced_mixed_decisions():
    w = W.kalthoff(nx=120, ny=60, dx=5e-4 * 402 / 120, notch_cells=30.125, gap_cells=30, nsteps=1500)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0, precision=PD_MIXED)
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    sim.step(1500)
    st = sim.stats()
    u = sim.state()[0]
    sim.close()
    ref = _oracle(w, s0)
    ref.step(1500)
    assert st["broken_bonds"] > 0 and st["validate_mismatches"] == 0
    assert rel(u, ref.u) <= 1e-4


def test_kalthoff_full_size_first_steps():
    """80,802 particles (the paper's node count): FP64 against the oracle over the first 500 steps."""
    w = W.kalthoff()
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    sim = Simulation(w, s0=s0)
    ref = _oracle(w, s0)
    ref.step(500)
    sim.step(500)
    u, v, _ = sim.state()
    sim.close()
    assert rel(u, ref.u) <= 1e-12 and rel(v, ref.v) <= 1e-12
    assert elem(u, ref.u) <= 1e-12 and elem_v(v, ref) <= 1e-12
