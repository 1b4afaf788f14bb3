"""The oracle's pdref_* call sequence (the GPU library's C ABI shape) gives exactly what the oracle's
own OracleSim gives (CPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W

from harness import drive, oracle_api


@pytest.mark.parametrize("case", ["plate", "cracked", "notched"])
def test_pdref_sequence_equals_oraclesim(case):
    if case == "plate":
        w, rate = W.plate_vibration(nx=16, ny=12, nsteps=50), 0.0
    elif case == "cracked":
        w, rate = W.cracked_plate(nx=30, ny=14, dx=2.5e-4, crack_cells=15.125, sigma=3e6, nsteps=150), 0.0
    else:
        w = W.notched_block(nx=14, ny=8, nz=6, dx=1e-3, notch_cells=5.5, nsteps=80, seed=2, amp=1e-7)
        rate = None
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0
    rate = w.rotation_rate(s0) if rate is None else rate
    got = drive(oracle_api(), w, s0, rate, w.nsteps)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, rate)
    ref.set_state(w.initial_u(), w.initial_v())
    ref.step(w.nsteps)
    assert np.array_equal(got["u"], ref.u) and np.array_equal(got["v"], ref.v)
    assert np.array_equal(got["theta"], ref.theta) and np.array_equal(got["phi"], ref.damage())
    assert np.array_equal(got["col"], ref.col) and np.array_equal(got["intact"], ref.status)
