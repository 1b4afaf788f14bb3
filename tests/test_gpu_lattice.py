"""The lattice layout of the mixed-precision form (PD_OPT_LATTICE, GPU only).

On bodies whose particles lie on a regular lattice, the family is laid out by lattice direction and
the step kernels take each slot's bond vector from a table (csrc/pd_lattice.h, k_pass1_lat /
k_pass2_lat).  Checked here: the family is still exactly the oracle's (Section 2.1 horizon, cracks);
bodies that are not lattices keep the general layout; the lattice kernels follow the FP64 oracle to
the mixed form's stated bounds and decide every bond as FP64 does on their own state (validation
mode, Eq 1.30), on 2D and 3D bodies with breaking, on a batch of uneven plates, and on the
benchmark's 1M-particle block through its first 400 steps; graph chunks equal eager launches and a
batch equals its bodies run one by one, bit for bit.  The same holds with the two-word shadow
(PD_OPT_SHADOW_LO), which in addition follows the FP64 oracle more closely than one word.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W
from parity import rel

pytestmark = pytest.mark.gpu


def s0_of(w):
    return O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0


def oracle_for(w, s0):
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0), vp=getattr(w, "vp", None))
    ref.set_state(w.initial_u(), w.initial_v())
    return ref


CASES = {
    "cracked_plate": lambda: W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400),
    "notched_block": lambda: W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3,
                                             amp=1e-7),
    "ratio_4": lambda: W.plate_vibration(nx=30, ny=17, ratio=4.015, nsteps=300),
    "plane_strain": lambda: W.kalthoff(nx=120, ny=60, dx=5e-4 * 402 / 120, notch_cells=30.125, gap_cells=30,
                                       nsteps=1500),  # the notch tips start to crack within these steps
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_lattice_family_is_the_oracles(case):
    w = CASES[case]()
    sim = Simulation(w, s0=0.0, precision=PD_MIXED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 1
    rp, col, intact = sim.neighbors()
    sim.close()
    orp, ocol = O.family(w.x, w.y, w.z, w.delta, w.cracks)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol) and intact.all()


def test_non_lattice_bodies_keep_the_general_layout():
    rng = np.random.default_rng(3)
    n = 2000
    pts = rng.uniform(0.0, 1e-2, size=(2, n))
    w = W.Workload("cloud", W.MODEL_PLANE_STRAIN, E=1e9, nu=0.25, rho=1000.0, dx=2.5e-4, delta=8e-4, dt=1e-9,
                   nsteps=20, x=pts[0], y=pts[1], z=None, vol=np.full(n, (2.5e-4) ** 2),
                   u0=1e-7 * rng.normal(size=(2, n)))
    sim = Simulation(w, s0=0.0, precision=PD_MIXED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 0
    sim.step(20)
    sim.close()
    # a lattice with one non-uniform volume does not qualify either
    w2 = W.plate_vibration(nx=20, ny=20, nsteps=10)
    w2.vol = w2.vol.copy()
    w2.vol[7] *= 1.5
    sim = Simulation(w2, s0=0.0, precision=PD_MIXED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 0
    sim.close()
    # and PD_OPT_LATTICE = 0 (set before the build) keeps it off on a lattice
    w3 = W.plate_vibration(nx=20, ny=20, nsteps=10)
    prm = B.make_params(w3.model, w3.E, w3.nu, w3.rho, w3.delta, 0.0, w3.dt, PD_MIXED, 0.0, 0, None,
                        B.PD_ORDER_BRICKS, B.PD_LINEARIZED)
    h = B.pd_create_particles(prm, w3.x, w3.y, None, w3.vol)
    B.pd_set_option(h, B.PD_OPT_LATTICE, 0)
    B.pd_build_neighbors(h, [])
    assert B.pd_get_option(h, B.PD_OPT_LATTICE) == 0
    B.pd_destroy(h)
    # a lattice whose family is not a prefix of the direction table (horizon below 3 spacings:
    # |n|^2 <= 4 ends inside the table's first group) keeps the general layout and still follows
    # the oracle (the mixed form's stated bound after 100 steps)
    w4 = W.plate_vibration(nx=20, ny=20, nsteps=100, ratio=2.015, dt=1e-7)  # well inside the stable step
    sim = Simulation(w4, s0=0.0, precision=PD_MIXED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 0
    ref = oracle_for(w4, 0.0)
    sim.step(100)
    ref.step(100)
    assert float(np.linalg.norm(sim.state()[0] - ref.u) / np.linalg.norm(ref.u)) <= 2e-5
    sim.close()


@pytest.mark.parametrize("lo", [0, 1])
@pytest.mark.parametrize("case", ["cracked_plate", "notched_block", "plane_strain"])
def test_lattice_decisions_equal_fp64_and_follow_the_oracle(case, lo):
    """Breaking runs: zero decisions differing from FP64 on the run's own state (validation mode),
    with the lattice and with the general mixed kernels.  The trajectory is held to the FP64 oracle
    (rel-L2(u) <= 1e-5, as the mixed form's stated bound of configuration 1 over its first 100
    steps) while the oracle's smallest stretch margin stays above 1e-5: once a bond comes closer to
    its threshold than the FP32 trajectory's distance from the FP64 one, the two runs may break it
    at different steps and their crack paths separate (a property of the fracture, the decisions on
    each run's own state being exact)."""
    w = CASES[case]()
    s0 = s0_of(w)
    ref = oracle_for(w, s0)
    sims = {lat: _mixed(w, s0, lat) for lat in ((1, 0) if not lo else (1,))}
    for sim in sims.values():
        sim.set_option(B.PD_OPT_VALIDATE, 1)
        sim.set_option(B.PD_OPT_SHADOW_LO, lo)
        assert sim.get_option(B.PD_OPT_SHADOW_LO) == (lo if sim.get_option(B.PD_OPT_LATTICE) else 0)
    compared, done = 0, 0
    while done < w.nsteps:
        margins, _ = ref.step(25)
        for sim in sims.values():
            sim.step(25)
        done += 25
        if margins.min() <= 1e-5:
            break
        for sim in sims.values():
            assert rel(sim.state()[0], ref.u) <= 1e-5, (case, done)
        compared = done
    assert compared >= 25, case
    for sim in sims.values():
        sim.step(w.nsteps - done)
    for lat, sim in sims.items():
        st = sim.stats()
        assert st["broken_bonds"] > 0 and st["validate_mismatches"] == 0, (case, lat, st)
        sim.close()


def _mixed(w, s0, lattice):
    prm = B.make_params(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, PD_MIXED, 0.0, 0, None, B.PD_ORDER_BRICKS,
                        B.PD_LINEARIZED)
    sim = Simulation.__new__(Simulation)
    sim.w, sim.n, sim.dim, sim.s0 = w, w.n, w.dim, s0
    sim.h = B.pd_create_particles(prm, w.x, w.y, w.z, w.vol)
    B.pd_set_option(sim.h, B.PD_OPT_LATTICE, lattice)
    B.pd_build_neighbors(sim.h, w.cracks)
    assert B.pd_get_option(sim.h, B.PD_OPT_LATTICE) == lattice
    if w.flag is not None or w.b is not None:
        B.pd_set_bc(sim.h, w.dim, w.n, w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0))
    if getattr(w, "vp", None) is not None:
        B.pd_set_prescribed_velocity(sim.h, w.dim, w.n, w.vp)
    B.pd_set_state(sim.h, w.dim, w.n, w.initial_u(), w.initial_v())
    return sim


def test_lattice_config1_error_bound():
    """Configuration 1 (free vibration, 1000 steps) against the FP64 oracle: the stated bounds of
    the mixed form, 2e-5 after 100 steps and 1e-4 over 1000."""
    w = W.config1()
    sim = Simulation(w, s0=0.0, precision=PD_MIXED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 1
    ref = oracle_for(w, 0.0)
    errs = []
    for _ in range(10):
        ref.step(100)
        sim.step(100)
        errs.append(rel(sim.state()[0], ref.u))
    sim.close()
    print("lattice config1 rel-L2(u) per 100 steps:", ["%.2e" % e for e in errs])
    assert errs[0] <= 2e-5 and max(errs) <= 1e-4, errs


def test_lattice_graph_chunks_and_batch_are_bitwise():
    w = CASES["cracked_plate"]()
    s0 = s0_of(w)
    res = []
    for chunk in (0, 100, 7):
        sim = Simulation(w, s0=s0, precision=PD_MIXED, graph_chunk=chunk)
        sim.step(250)
        res.append((sim.state()[0], sim.neighbors()[2]))
        sim.close()
    for u, st in res[1:]:
        assert np.array_equal(u, res[0][0]) and np.array_equal(st, res[0][1])
    bw = W.plate_batch(nplates=5, seed=4, side_lo=20, side_hi=60)
    s0s = [s0_of(b) for b in bw.bodies]
    bs = BatchSimulation(bw, s0s, precision=PD_MIXED)
    assert bs.get_option(B.PD_OPT_LATTICE) == 1
    bs.step(150)
    ub = bs.state()[0]
    broken = bs.stats()["broken_bonds"]
    bs.close()
    for k, b in enumerate(bw.bodies):
        sim = Simulation(b, s0=s0s[k], precision=PD_MIXED)
        sim.step(150)
        u = sim.state()[0]
        sim.close()
        assert np.array_equal(u, ub[:, bw.offsets[k]:bw.offsets[k + 1]]), k
    assert broken >= 0


@pytest.mark.parametrize("kin", ["linearized", "nonlinear"])
def test_lattice_benchmark_block_validation_whole_run(kin):
    """The benchmark's block (configuration 3, 1M particles, ~1.17e8 bonds) in the mixed form with
    every bond decision also taken in FP64 on the run's own state, through all 2000 steps of the
    configuration (bonds break from about step 23 on; millions by the end): no decision differs
    (Eq 1.30, zero spurious breaks), for linearized and for nonlinear bonds."""
    w = W.config3()
    sim = Simulation(w, precision=PD_MIXED, kinematics=B.PD_NONLINEAR if kin == "nonlinear" else B.PD_LINEARIZED)
    assert sim.get_option(B.PD_OPT_LATTICE) == 1
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    sim.step(w.nsteps)
    st = sim.stats()
    sim.close()
    print("config3 mixed (%s), %d steps with validation:" % (kin, w.nsteps),
          {k: st[k] for k in ("broken_bonds", "band_rechecks", "validate_mismatches")})
    assert st["broken_bonds"] > 1000000 and st["validate_mismatches"] == 0


def test_two_word_shadow_config1_and_bitwise_properties():
    """PD_OPT_SHADOW_LO on configuration 1: the stated bounds hold and the error is no larger than
    with one word; set mid-run it takes effect from the current state; graph chunks and a batch
    equal eager runs and separate bodies bit for bit; off again, it reports 0."""
    w = W.config1()
    errs = {}
    for lo in (0, 1):
        sim = Simulation(w, s0=0.0, precision=PD_MIXED, shadow_lo=lo)
        assert sim.get_option(B.PD_OPT_SHADOW_LO) == lo
        ref = oracle_for(w, 0.0)
        e = []
        for _ in range(10):
            ref.step(100)
            sim.step(100)
            e.append(rel(sim.state()[0], ref.u))
        sim.close()
        errs[lo] = e
    print("config1 rel-L2(u), one word / two words:", ["%.2e" % x for x in errs[0]], ["%.2e" % x for x in errs[1]])
    assert errs[1][0] <= 2e-5 and max(errs[1]) <= 1e-4
    assert max(errs[1]) <= max(errs[0])
    # graph chunks, eager, and the option switched on after 100 eager steps of the same run
    cw = CASES["cracked_plate"]()
    s0 = s0_of(cw)
    res = []
    for chunk, late in ((0, False), (100, False), (0, True)):
        sim = Simulation(cw, s0=s0, precision=PD_MIXED, graph_chunk=chunk, shadow_lo=0 if late else 1)
        if late:
            sim.step(100)
            sim.set_option(B.PD_OPT_SHADOW_LO, 1)
            sim.step(150)
        else:
            sim.step(250)
        res.append((sim.state()[0], sim.neighbors()[2]))
        sim.set_option(B.PD_OPT_SHADOW_LO, 0)
        assert sim.get_option(B.PD_OPT_SHADOW_LO) == 0
        sim.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert not np.array_equal(res[0][0], res[2][0])  # the first 100 steps ran with one word
    bw = W.plate_batch(nplates=4, seed=6, side_lo=20, side_hi=50)
    s0s = [s0_of(b) for b in bw.bodies]
    bs = BatchSimulation(bw, s0s, precision=PD_MIXED)
    bs.set_option(B.PD_OPT_SHADOW_LO, 1)
    assert bs.get_option(B.PD_OPT_SHADOW_LO) == 1
    bs.step(120)
    ub = bs.state()[0]
    bs.close()
    for k, b in enumerate(bw.bodies):
        sim = Simulation(b, s0=s0s[k], precision=PD_MIXED, shadow_lo=1)
        sim.step(120)
        assert np.array_equal(sim.state()[0], ub[:, bw.offsets[k]:bw.offsets[k + 1]]), k
        sim.close()



def test_autotune_mid_run_restores_the_lattice_state_bitwise():
    """pd_autotune in the middle of a breaking mixed run (its trial steps advance the state, break
    bonds and raise the shadow's per-body bound, then restore) leaves the run bitwise the one
    without it: the lattice kernels' arithmetic does not depend on the mapping, and the restore
    brings back u, v, the status bits, the FP32 shadow and its bound."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=300)
    s0 = s0_of(w)
    out = []
    for tune in (False, True):
        sim = Simulation(w, s0=s0, precision=PD_MIXED)
        assert sim.get_option(B.PD_OPT_LATTICE) == 1
        sim.step(150)
        if tune:
            B.pd_autotune(sim.h, 20)
        sim.step(150)
        u, v, _ = sim.state()
        out.append((u, v, sim.neighbors()[2], sim.stats()["broken_bonds"]))
        sim.close()
    assert out[0][3] > 0
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
