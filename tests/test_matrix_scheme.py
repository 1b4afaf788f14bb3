"""The paper's matrix-based scheme (Eqs 2.4-2.10, Appendix B), the same-box baseline, against the
oracle: assembled matrices reproduce the gather-form dynamics to 1e-12 (CPU; the bench runs the same
code on the GPU)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W

torch = pytest.importorskip("torch")
from paper_2309_11273_gb300.matrix_scheme import MatrixScheme  # noqa: E402


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("case", ["plate", "block"])
def test_matrix_scheme_matches_oracle(case):
    if case == "plate":
        w = W.plate_vibration(nx=20, ny=16, nsteps=60)
        rate = 0.0
    else:
        w = W.notched_block(nx=16, ny=10, nz=8, dx=1e-3, notch_cells=6.5, nsteps=60, seed=3, amp=1e-6)
        rate = 5e3
    c = O.constants(w.model, w.E, w.nu)
    rp, col = O.family(w.x, w.y, w.z, w.delta, w.cracks)
    ms = MatrixScheme(w, rp, col, c["A"], c["K"], c["G"], rate=rate, device="cpu")
    ms.set_state(w.initial_u(), w.initial_v())
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, rate)
    ref.set_state(w.initial_u(), w.initial_v())
    for _ in range(3):
        ms.step(20)
        ref.step(20)
        u, v = ms.state()
        assert rel(u, ref.u) <= 1e-12 and rel(v, ref.v) <= 1e-12, (rel(u, ref.u), rel(v, ref.v))
    assert ms.nbonds_undirected * 2 == col.size
