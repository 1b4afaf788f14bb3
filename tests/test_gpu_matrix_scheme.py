"""The matrix-based baseline (Eqs 2.4-2.10 through cuSPARSE) on the GPU reproduces the oracle (GPU)."""
import numpy as np

from parity import elem, elem_v
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W
from paper_2309_11273_gb300.matrix_scheme import MatrixScheme

pytestmark = pytest.mark.gpu


def test_matrix_scheme_on_gpu_matches_oracle():
    w = W.notched_block(nx=20, ny=12, nz=10, dx=1e-3, notch_cells=8.5, nsteps=60, seed=4, amp=1e-6)
    c = O.constants(w.model, w.E, w.nu)
    rp, col = O.family(w.x, w.y, w.z, w.delta, w.cracks)
    ms = MatrixScheme(w, rp, col, c["A"], c["K"], c["G"], rate=5e3, device="cuda")
    ms.set_state(w.initial_u(), w.initial_v())
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, 5e3)
    ref.set_state(w.initial_u(), w.initial_v())
    ms.step(60)
    ref.step(60)
    u, v = ms.state()
    assert np.linalg.norm(u - ref.u) <= 1e-12 * np.linalg.norm(ref.u)
    assert np.linalg.norm(v - ref.v) <= 1e-12 * np.linalg.norm(ref.v)
    assert elem(u, ref.u) <= 1e-12 and elem_v(v, ref) <= 1e-12
