"""Error of the FP32-bond / FP64-integration form per configuration, at each configuration's full
length (GPU only; takes a few minutes).

Reported per configuration: rel-L2(u) against an FP64 reference and the number of directed bonds
whose status differs from it.  The reference is the oracle for configurations 1 and 2, and the FP64
GPU path -- itself held to 1e-12 of the oracle by test_gpu_parity / test_gpu_scale -- for the 3D and
batched configurations, whose full runs (thousands of steps over 1e8-1e9 bonds) are beyond the
oracle's reach.  Status differences are expected once bonds break: a different FP32 force history
moves the crack front by whole bonds; the decisions themselves are certified separately (zero
differences from FP64 on the mixed run's own state, test_mixed_decisions_equal_fp64_on_own_state).
"""
import json

import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation
from paper_2309_11273_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# stated bounds on rel-L2(u) at the end of the full run (configurations 1, 2, 4) and at the first
# tenth of the run (configurations 3, 5, whose torsion fractures millions of bonds; once the FP32 and
# FP64 runs break different bonds the two crack patterns diverge and the end-of-run difference is a
# property of the fracture, reported but not bounded).  Configuration 5 has already broken ~4e6
# bonds at its first tenth (step 100), so its bound there is looser than configuration 3's.
BOUNDS = {"config1": 1e-4, "config2": 1e-5, "config4": 1e-3, "config3": 1e-3, "config5": 1e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_mixed_error_per_configuration(capsys):
    out = {}
    for name, w in (("config1", W.config1()), ("config2", W.config2())):
        s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0
        ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
        ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
        ref.set_state(w.initial_u(), w.initial_v())
        margins, _ = ref.step(w.nsteps)
        sim = Simulation(w, s0=s0, precision=PD_MIXED)
        sim.step(w.nsteps)
        u = sim.state()[0]
        st = sim.neighbors()[2]
        stats = sim.stats()
        sim.close()
        out[name] = {"steps": w.nsteps, "reference": "oracle", "rel_l2_u": _rel(u, ref.u),
                     "status_mismatch": int((st != ref.status).sum()),
                     "broken_reference": int((ref.status == 0).sum()), "band_rechecks": stats["band_rechecks"]}
    for name, w in (("config3", W.config3()), ("config5", W.config5())):
        ref = Simulation(w, precision=PD_FP64)
        sim = Simulation(w, precision=PD_MIXED)
        traj = []
        for _ in range(10):
            ref.step(w.nsteps // 10)
            sim.step(w.nsteps // 10)
            u64, st64 = ref.state()[0], ref.neighbors()[2]
            u32, st32 = sim.state()[0], sim.neighbors()[2]
            traj.append({"step": ref.stats()["steps"], "rel_l2_u": _rel(u32, u64),
                         "status_mismatch": int((st32 != st64).sum()), "broken_reference": int((st64 == 0).sum())})
        out[name] = dict(traj[-1], reference="FP64 GPU path", band_rechecks=sim.stats()["band_rechecks"],
                         first_tenth=traj[0], trajectory=traj)
        ref.close()
        sim.close()
    bw = W.config4()
    res = {}
    for prec in (PD_FP64, PD_MIXED):
        bs = BatchSimulation(bw, precision=prec)
        bs.step(bw.bodies[0].nsteps)
        res[prec] = (bs.state()[0], bs.neighbors()[2], bs.stats())
        bs.close()
    out["config4"] = {"steps": bw.bodies[0].nsteps, "reference": "FP64 GPU path",
                      "rel_l2_u": _rel(res[PD_MIXED][0], res[PD_FP64][0]),
                      "status_mismatch": int((res[PD_MIXED][1] != res[PD_FP64][1]).sum()),
                      "broken_reference": int(res[PD_FP64][2]["broken_bonds"]),
                      "band_rechecks": res[PD_MIXED][2]["band_rechecks"]}
    with capsys.disabled():
        print("\nMIXED_ACCURACY " + json.dumps(out))
    for name, r in out.items():
        val = r["first_tenth"]["rel_l2_u"] if "first_tenth" in r else r["rel_l2_u"]
        assert val <= BOUNDS[name], (name, r)
