"""Checkpoint / resume through pd_save_state / pd_load_state (GPU only).  N steps equal k steps, a
save, a load into a fresh context and N - k steps, bit for bit -- u, v and the bond status -- through
bond breaking, in FP64 and in the mixed form.  A file written for a different problem, or damaged,
is rejected with PD_ERR_ARG and leaves the context as it was."""
import numpy as np
import pytest

from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _plate(**kw):
    # bonds break from step 40 to 180 of the 400
    return W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400, **kw)


def _final(sim):
    u, v, _ = sim.state()
    return u, v, sim.neighbors()[2], sim.stats()["steps"]


@pytest.mark.parametrize("precision", [PD_FP64, PD_MIXED])
def test_resume_is_bitwise(precision, tmp_path):
    w = _plate()
    ref = Simulation(w, precision=precision)
    ref.step(400)
    want = _final(ref)
    ref.close()
    a = Simulation(w, precision=precision)
    a.step(150)
    path = str(tmp_path / "state.ck")
    B.pd_save_state(a.h, path)
    a.close()
    b = Simulation(w, precision=precision)
    B.pd_load_state(b.h, path)
    b.step(250)
    got = _final(b)
    b.close()
    assert want[3] == got[3] == 400
    assert int((want[2] == 0).sum()) > 1000
    for x, y in zip(want[:3], got[:3]):
        assert np.array_equal(x, y)


def test_rejected_files_leave_the_context_unchanged(tmp_path):
    w = _plate()
    a = Simulation(w)
    a.step(60)
    path = str(tmp_path / "state.ck")
    B.pd_save_state(a.h, path)
    a.close()
    other = Simulation(_plate(ratio=4.015))  # another family and horizon
    u0 = other.state()[0]
    with pytest.raises(B.PDError) as e:
        B.pd_load_state(other.h, path)
    assert e.value.status == B.PD_ERR_ARG
    assert np.array_equal(other.state()[0], u0)
    other.close()
    raw = bytearray(open(path, "rb").read())
    raw[len(raw) // 2] ^= 0x40  # a bit of the payload
    bad = str(tmp_path / "damaged.ck")
    open(bad, "wb").write(bytes(raw))
    b = Simulation(w)
    u0 = b.state()[0]
    for p in (bad, str(tmp_path / "missing.ck")):
        with pytest.raises(B.PDError) as e:
            B.pd_load_state(b.h, p)
        assert e.value.status == B.PD_ERR_ARG
    assert np.array_equal(b.state()[0], u0) and b.stats()["steps"] == 0
    B.pd_load_state(b.h, path)
    assert b.stats()["steps"] == 60
    b.close()
