"""Error of the FP32-bond / FP64-integration form per configuration (GPU only; a few minutes).

Reported per configuration: rel-L2(u) against an FP64 reference and the number of directed bonds
whose status differs from it.  The reference is the oracle for configurations 1 and 2, and the FP64
GPU path -- itself held to 1e-12 of the oracle by test_gpu_parity / test_gpu_scale -- for the 3D and
batched configurations, whose full runs (thousands of steps over 1e8-1e9 bonds) are beyond the
oracle's reach.

On the torsion blocks (configurations 3 and 5) and the batched plates (configuration 4) bonds break
by the hundred thousand or million.  Eq 1.30 decides each bond by a threshold, so two runs whose
states differ eventually break different bonds once a bond comes closer to its threshold than that
difference, and the crack patterns then separate.  Beside the mixed runs (one-word FP32 shadow, the
default, and the two-word shadow of PD_OPT_SHADOW_LO) two FP64 trajectories measure the method's own
sensitivity:
  * another summation order (two warps per 32-particle slice, each summing every other slot, the
    halves then added: the same physics rounded differently; the particle order alone does not
    change any sum, rows being sorted by bond direction) -- a perturbation of ~1e-16;
  * the FP64 run with its displacements and velocities rounded to FP32 once, at step 20 (before the
    first bond breaks).
Both stay far below the one-word mixed error on the blocks (measured ~1e-15 and ~1e-10 on
configuration 3 over 2000 steps, with no status difference), so that error is the FP32 shadow's:
one FP32 word per component rounds n.(u_j - u_i) / h^2 to about 2^-24 |u| / h, and under the twist
|u| is tens of times a bond's relative displacement; the resulting force error shifts the step at
which near-threshold bonds break.  The two-word shadow rounds relative to the difference instead and
follows FP64 to ~1e-9 with identical bond status through step 600 of configuration 3.
Configuration 1 is a free plate: its one-word error is 99% rigid drift (the FP32 force sums are
rounded per particle, so the body's momentum takes a random walk), and the deformation part, the
error less its best-fit rigid motion, is held to 2e-5 beside the total.
Bounds: configurations 1, 2, 4 as BOUNDS (both shadows); the blocks at their first checkpoint
(FIRST_BOUND, one word); with two words configuration 3 within 1e-8 and no status difference through
step 600.  Configuration 5 with two words is reported, not bounded: it follows FP64 until a bond
closer to its threshold than the two-word rounding (~1e-9 of the state) is decided on the other side,
and when that happens depends on the rounding pattern: with the slots ordered by |n|^2 it was
2.3e-9 after 100 steps with the same broken bonds; with the slots ordered by row, 3.3e-3 with 3,444
more (both with every decision equal to FP64's on the run's own state).  Configuration 5's mixed
runs take every decision in validation mode here, and the test requires zero mismatches; the other
configurations' decisions are certified in tests/test_gpu_lattice.py.
"""
import json

import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W
from parity import rigid_split

pytestmark = pytest.mark.gpu

# stated bounds on rel-L2(u) at the end of the full run (configurations 1, 2, 4)
BOUNDS = {"config1": 1e-4, "config2": 1e-5, "config4": 1e-3}
# stated bounds at the first checkpoint of the torsion blocks (step 200 of configuration 3, step 100
# of configuration 5)
FIRST_BOUND = {"config3": 1e-6, "config5": 1e-2}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


ROUND_AT = 20  # step of the FP32 rounding of the perturbed FP64 run (before the first bond breaks)


def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _round_state(sim):
    u, v, _ = sim.state()
    sim.set_state(_f32(u), _f32(v))


def _block_trajectories(w, nsteps, nchk, with_status=True, validate=False):
    """Reference FP64 and, from the same state, FP64 with another summation order, FP64 rounded to
    FP32 once at step ROUND_AT, and mixed; at nchk checkpoints rel-L2(u) and status mismatches of the
    latter three against the reference.  Two contexts at a time (the reference is deterministic:
    each of its runs is bitwise the first)."""
    k = nsteps // nchk
    out = {"fp64_order": [], "fp64_rounded": [], "mixed": [], "mixed_lo": []}
    for tag, kw in (("fp64_order", dict(precision=PD_FP64)), ("fp64_rounded", dict(precision=PD_FP64)),
                    ("mixed", dict(precision=PD_MIXED)), ("mixed_lo", dict(precision=PD_MIXED, shadow_lo=1))):
        ref = Simulation(w, precision=PD_FP64)
        sim = Simulation(w, **kw)
        if tag == "fp64_order":
            sim.set_option(B.PD_OPT_SPLIT, 2)  # another summation order
        if validate and tag.startswith("mixed"):
            sim.set_option(B.PD_OPT_VALIDATE, 1)  # every decision also taken in FP64 and compared
        for c in range(nchk):
            if c == 0 and tag == "fp64_rounded":
                ref.step(ROUND_AT)
                sim.step(ROUND_AT)
                _round_state(sim)
                ref.step(k - ROUND_AT)
                sim.step(k - ROUND_AT)
            else:
                ref.step(k)
                sim.step(k)
            u64, u = ref.state()[0], sim.state()[0]
            row = {"step": ref.stats()["steps"], "rel_l2_u": _rel(u, u64)}
            if with_status:
                s64, s = ref.neighbors()[2], sim.neighbors()[2]
                row.update(status_mismatch=int((s != s64).sum()), broken_reference=int((s64 == 0).sum()))
            else:
                row.update(broken_reference=int(ref.stats()["broken_bonds"]), broken=int(sim.stats()["broken_bonds"]))
            out[tag].append(row)
        if tag.startswith("mixed"):
            out["band_rechecks" + tag[5:]] = sim.stats()["band_rechecks"]
            if validate:
                out["validate_mismatches" + tag[5:]] = sim.stats()["validate_mismatches"]
            out["lattice"] = sim.get_option(B.PD_OPT_LATTICE)
        ref.close()
        sim.close()
    return out


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
        P = np.stack([w.x, w.y])
        rig, dfm = rigid_split(u - ref.u, P)
        out[name] = {"steps": w.nsteps, "reference": "oracle", "rel_l2_u": _rel(u, ref.u),
                     "rigid": rig / np.linalg.norm(ref.u), "deformation": dfm / np.linalg.norm(ref.u),
                     "status_mismatch": int((st != ref.status).sum()),
                     "broken_reference": int((ref.status == 0).sum()), "band_rechecks": stats["band_rechecks"]}
    out["config3"] = dict(_block_trajectories(W.config3(), 2000, 10), steps=2000, reference="FP64 GPU path")
    # configuration 5 (8M particles, ~9.6e8 bonds): its first 200 steps (millions of bonds break by
    # step 100), broken counts instead of per-bond mismatches (a full status read-back takes ~30 s)
    out["config5"] = dict(_block_trajectories(W.config5(), 200, 2, with_status=False, validate=True), steps=200,
                          reference="FP64 GPU path")
    bw = W.config4()
    res = {}
    for tag, prec, split in (("fp64", PD_FP64, 1), ("fp64_order", PD_FP64, 2), ("fp64_rounded", PD_FP64, 1),
                             ("mixed", PD_MIXED, 1), ("mixed_lo", PD_MIXED, 1)):
        bs = BatchSimulation(bw, precision=prec)
        if split != 1:
            bs.set_option(B.PD_OPT_SPLIT, split)
        if tag == "mixed_lo":
            bs.set_option(B.PD_OPT_SHADOW_LO, 1)
        if tag == "fp64_rounded":
            bs.step(ROUND_AT)
            _round_state(bs)
            bs.step(bw.bodies[0].nsteps - ROUND_AT)
        else:
            bs.step(bw.bodies[0].nsteps)
        res[tag] = (bs.state()[0], bs.neighbors()[2], bs.stats())
        bs.close()

    def floor(tag):
        return {"rel_l2_u": _rel(res[tag][0], res["fp64"][0]),
                "status_mismatch": int((res[tag][1] != res["fp64"][1]).sum())}

    out["config4"] = {"steps": bw.bodies[0].nsteps, "reference": "FP64 GPU path",
                      "rel_l2_u": _rel(res["mixed"][0], res["fp64"][0]),
                      "status_mismatch": int((res["mixed"][1] != res["fp64"][1]).sum()),
                      "broken_reference": int(res["fp64"][2]["broken_bonds"]),
                      "band_rechecks": res["mixed"][2]["band_rechecks"],
                      "fp64_order": floor("fp64_order"), "fp64_rounded": floor("fp64_rounded"),
                      "mixed_lo": floor("mixed_lo")}
    with capsys.disabled():
        print("\nMIXED_ACCURACY " + json.dumps(out))
    for name in ("config1", "config2"):
        assert out[name]["rel_l2_u"] <= BOUNDS[name], (name, out[name])
    # the free plate's error less its rigid drift (FP32 sums move the body's momentum)
    assert out["config1"]["deformation"] <= 2e-5, out["config1"]
    c4 = out["config4"]
    assert c4["rel_l2_u"] <= BOUNDS["config4"] and c4["mixed_lo"]["rel_l2_u"] <= BOUNDS["config4"], c4
    # the torsion blocks: one word to the stated bound at the first checkpoint (fracture starting)
    for name in ("config3", "config5"):
        first = out[name]["mixed"][0]
        assert first["rel_l2_u"] <= FIRST_BOUND[name], (name, first)
    assert out["config3"]["mixed"][0]["status_mismatch"] == 0
    # two words: configuration 3 through step 600, configuration 5 over its 200 steps
    for row in out["config3"]["mixed_lo"]:
        if row["step"] <= 600:
            assert row["rel_l2_u"] <= 1e-8 and row["status_mismatch"] == 0, row
    # configuration 5 (reported): both forms decide every bond as FP64 does on their own state
    assert out["config5"]["validate_mismatches"] == 0 and out["config5"]["validate_mismatches_lo"] == 0
