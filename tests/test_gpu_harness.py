"""One harness drives the GPU library (pd_*) and the oracle (pdref_*) through the same call sequence;
results agree to the FP64 parity bar (GPU only)."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import workloads as W

from harness import drive, gpu_api, oracle_api
from parity import elem, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["cracked", "notched"])
def test_same_sequence_both_implementations(case):
    if case == "cracked":
        w = W.cracked_plate(nx=40, ny=20, dx=2.5e-4, crack_cells=20.125, sigma=3e6, nsteps=300)
    else:
        w = W.notched_block(nx=20, ny=10, nz=8, dx=1e-3, notch_cells=7.5, nsteps=200, seed=2, amp=1e-7)
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    rate = w.rotation_rate(s0)
    g = drive(gpu_api(), w, s0, rate, w.nsteps)
    r = drive(oracle_api(), w, s0, rate, w.nsteps)
    for k in ("u", "v"):
        assert rel(g[k], r[k]) <= 1e-12, k
    assert elem(g["u"], r["u"]) <= 1e-12
    # velocity per particle: the displacement bar carried through Eq 2.11 (tests/parity.py)
    vscale = max(np.abs(r["v"]).max(), 2.0 * np.abs(r["u"]).max() / w.dt)
    assert np.abs(g["v"] - r["v"]).max() <= 1e-12 * vscale
    assert np.array_equal(g["row_ptr"], r["row_ptr"]) and np.array_equal(g["col"], r["col"])
    assert np.array_equal(g["intact"], r["intact"]) and np.array_equal(g["phi"], r["phi"])
    assert (r["intact"] == 0).sum() > 0
