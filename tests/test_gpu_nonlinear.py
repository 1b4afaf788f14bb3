"""Geometrically nonlinear bonds (PD_NONLINEAR: Eqs 1.10, 1.13, 1.14) on the GPU against the oracle's
kin=NONLINEAR, element by element (GPU only).  Same bars as the linearized FP64 path
(tests/parity.py): u and v within 1e-12 at every checkpoint in rel-L2 and per particle, theta per
particle within the propagation of that bar, bond status exactly equal while the oracle's minimum
relative stretch margin stays above 1e-9."""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, PD_NONLINEAR, BatchSimulation, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


from parity import elem, elem_v, rel, theta_elem


def s0_of(w):
    return O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0


def run_pair(w, nsteps, every, rate=None, s0=None, u0=None, v0=None, **kw):
    s0 = s0_of(w) if s0 is None else s0
    sim = Simulation(w, s0=s0, rate=rate, kinematics=PD_NONLINEAR, **kw)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks,
                      kin=O.NONLINEAR)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0) if rate is None else rate)
    u0 = w.initial_u() if u0 is None else u0
    v0 = w.initial_v() if v0 is None else v0
    ref.set_state(u0, v0)
    sim.set_state(u0, v0)
    exact, out, done = True, [], 0
    while done < nsteps:
        k = min(every, nsteps - done)
        margins, _ = ref.step(k)
        sim.step(k)
        done += k
        if margins.size and margins.min() <= 1e-9:
            exact = False
        u, v, th = sim.state()
        rp, col, intact = sim.neighbors()
        out.append(dict(step=done, ru=rel(u, ref.u), rv=rel(v, ref.v), eu=elem(u, ref.u), ev=elem_v(v, ref),
                        et=theta_elem(th, ref),
                        status_equal=np.array_equal(intact, ref.status), exact=exact,
                        broken=int((ref.status == 0).sum())))
    phi = sim.damage()
    sim.close()
    return out, phi, ref


def assert_parity(out, phi=None, ref=None, tol_v=TOL):
    for c in out:
        assert c["ru"] <= TOL and c["rv"] <= tol_v and c["eu"] <= TOL and c["ev"] <= tol_v, c
        assert c["et"] <= TOL, c
        if c["exact"]:
            assert c["status_equal"], c
    if phi is not None and out[-1]["exact"]:
        assert np.array_equal(phi, ref.damage())


FORMS = {"pairs": dict(bond_cache=1, pairs=1), "tabled": dict(bond_cache=1, pairs=0), "recompute": dict(bond_cache=0)}


@pytest.mark.parametrize("form", sorted(FORMS))
def test_cracked_plate_breaking_nonlinear(form):
    """All kernel forms: per-slot tables with each bond's e and 1/|Y| formed once per pair (default)
    or once per entry, and recomputed geometry."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    out, phi, ref = run_pair(w, 400, 100, **FORMS[form])
    assert out[-1]["broken"] > 0
    assert_parity(out, phi, ref)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_notched_block_twist_nonlinear(form):
    """Clamped + twisted notched block (24 s0 rad over the 300 steps): progressive fracture."""
    w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    out, phi, ref = run_pair(w, 300, 100, **FORMS[form])
    assert out[-1]["broken"] > 10000
    assert_parity(out, phi, ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_random_cloud_nonuniform_volumes_nonlinear(dim):
    rng = np.random.default_rng(30 + dim)
    n = 1500 if dim == 2 else 3000
    pts = rng.uniform(0.0, 1e-2, size=(dim, n))
    vol = rng.uniform(0.5, 1.5, n) * (2.5e-4) ** dim
    w = W.Workload("cloud", W.MODEL_3D if dim == 3 else W.MODEL_PLANE_STRAIN, E=1e9, nu=0.25, rho=1000.0,
                   dx=2.5e-4, delta=8e-4, dt=1e-9, nsteps=50, x=pts[0], y=pts[1],
                   z=pts[2] if dim == 3 else None, vol=vol, u0=2e-6 * rng.normal(size=(dim, n)))
    out, _, _ = run_pair(w, 50, 25, s0=0.0)
    assert_parity(out)


def _rotation(dim, angle):
    if dim == 2:
        c, s = np.cos(angle), np.sin(angle)
        return np.array([[c, -s], [s, c]])
    a = np.array([0.3, -0.5, 0.8]); a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * K @ K


@pytest.mark.parametrize("dim", [2, 3])
def test_turned_spinning_body(dim):
    """Large rotation: the body starts turned by 35 degrees and spins.  GPU equals the oracle, and
    the angular momentum sum_i rho V_i (x_i + u_i) x v_i is conserved (central pair forces).

    v is held to 1e-11 here: the bonds of a nearly rigid motion carry a strain of ~1e-8 (centripetal),
    while |Y|^2 - |xi|^2 of a bond turned by 35 degrees is a difference of terms of size |xi|^2, known
    to ~1e-16 |xi|^2 whatever the evaluation order; the forces of two correct evaluations therefore
    agree to ~1e-8 of themselves, and v, dominated by the rigid spin, to ~1e-12 of itself."""
    if dim == 2:
        w = W.plate_vibration(nx=24, ny=20, nsteps=300, dt=2e-7, amp=0.0)
    else:
        x, y, z = W.grid_3d(12, 10, 8, 1e-3)
        w = W.Workload("block", W.MODEL_3D, E=30e9, nu=0.2, rho=2400.0, dx=1e-3, delta=3.015e-3, dt=2e-7,
                       nsteps=300, x=x, y=y, z=z, vol=np.full(x.size, 1e-9))
    P = np.stack([w.x, w.y] + ([w.z] if dim == 3 else []))
    c = P.mean(axis=1, keepdims=True)
    r = _rotation(dim, np.deg2rad(35.0)) @ (P - c)
    om = np.array([0.0, 0.0, 2e3]) if dim == 2 else np.array([300.0, -500.0, 800.0])
    r3 = np.vstack([r, np.zeros((1, w.n))]) if dim == 2 else r
    v0 = np.cross(om, r3.T).T[:dim]
    out, _, ref = run_pair(w, 300, 100, s0=0.0, rate=0.0, u0=r + c - P, v0=v0)
    assert_parity(out, tol_v=1e-11)
    sim = Simulation(w, s0=0.0, rate=0.0, kinematics=PD_NONLINEAR)
    sim.set_state(r + c - P, v0)
    mass = w.rho * w.vol

    def L():
        u, v, _ = sim.state()
        q = P + u
        if dim == 2:
            return np.array([(mass * (q[0] * v[1] - q[1] * v[0])).sum()])
        return (mass * np.cross(q.T, v.T).T).sum(axis=1)

    sim.step(1)
    L1 = L()
    sim.step(300)
    L2 = L()
    sim.close()
    assert np.linalg.norm(L2 - L1) <= 1e-12 * np.linalg.norm(L1)


def test_batch_nonlinear_equals_separate_runs_bitwise():
    bw = W.plate_batch(nplates=4, seed=4, side_lo=10, side_hi=40, nsteps=200)
    s0s = [s0_of(b) for b in bw.bodies]
    bs = BatchSimulation(bw, s0s, kinematics=PD_NONLINEAR)
    bs.step(200)
    ub = bs.state()[0]
    bs.close()
    for k, b in enumerate(bw.bodies):
        sim = Simulation(b, s0=s0s[k], kinematics=PD_NONLINEAR)
        sim.step(200)
        u = sim.state()[0]
        sim.close()
        assert np.array_equal(u, ub[:, bw.offsets[k]:bw.offsets[k + 1]]), k


def test_nonlinear_reads_between_steps_keep_the_trajectory():
    """The check before a read (nonlinear pair form: the criterion alone, with pass 1a's arithmetic)
    takes the decisions the next step's pass 1a would take: reading the state after every step or
    every 7 steps gives bitwise the u, v and bond status of the run that is read only at its end,
    while bonds break throughout."""
    w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    res = []
    for every in (1, 7, w.nsteps):
        sim = Simulation(w, s0=s0_of(w), kinematics=PD_NONLINEAR)
        done = 0
        while done < w.nsteps:
            k = min(every, w.nsteps - done)
            sim.step(k)
            done += k
            sim.state()
        res.append(sim.state()[:2] + (sim.neighbors()[2],))
        sim.close()
    assert not res[-1][2].all()  # bonds broke
    for got in res[:-1]:
        for a, b in zip(got, res[-1]):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("block,split", [(128, 2), (512, 4)])
def test_nonlinear_mapping_variants_agree(block, split):
    w = W.notched_block(nx=30, ny=14, nz=12, dx=1e-3, notch_cells=11.5, nsteps=60, seed=1, amp=2e-6)
    res = []
    for blk, sp in ((256, 1), (block, split)):
        sim = Simulation(w, s0=s0_of(w), rate=5e3, kinematics=PD_NONLINEAR)
        sim.set_option(B.PD_OPT_SPLIT, 1)
        sim.set_option(B.PD_OPT_BLOCK, blk)
        sim.set_option(B.PD_OPT_SPLIT, sp)
        sim.step(60)
        res.append(sim.state()[0])
        sim.close()
    assert rel(res[1], res[0]) <= 1e-13


# ------------------------------------------------------------------ mixed precision, nonlinear bonds
def _oracle_nl(w, s0, rate=0.0):
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks,
                      kin=O.NONLINEAR)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, rate)
    ref.set_state(w.initial_u(), w.initial_v())
    return ref


@pytest.mark.parametrize("lattice", [1, 0])
def test_mixed_nonlinear_error_bound(lattice):
    """FP32 nonlinear bonds with FP64 integration on the vibrating plate (configuration 1's
    geometry): rel-L2(u) against the oracle's FP64 nonlinear run <= 2e-5 after 100 steps and <= 1e-4
    over 1000 (the bounds of the linearized mixed form), on the lattice layout (default for lattice
    bodies) and on the general layout."""
    w = W.config1()
    sim = Simulation(w, s0=0.0, precision=PD_MIXED, kinematics=PD_NONLINEAR, lattice=lattice)
    assert sim.get_option(B.PD_OPT_LATTICE) == lattice
    ref = _oracle_nl(w, 0.0)
    errs = []
    for _ in range(10):
        ref.step(100)
        sim.step(100)
        errs.append(rel(sim.state()[0], ref.u))
    sim.close()
    assert errs[0] <= 2e-5 and max(errs) <= 1e-4, errs


@pytest.mark.parametrize("lattice", [1, 0])
def test_mixed_nonlinear_decisions_equal_fp64_on_own_state(lattice):
    """Zero spurious breaks for nonlinear bonds: with validation on, every decision of the FP32 +
    band path equals the FP64 nonlinear decision on the mixed run's own state; bonds do break.  Both
    layouts (the lattice kernels' band is LatBandNL of pd_lattice.h, the general kernels' the
    fixed-point one)."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    sim = Simulation(w, s0=s0_of(w), precision=PD_MIXED, kinematics=PD_NONLINEAR, lattice=lattice)
    assert sim.get_option(B.PD_OPT_LATTICE) == lattice
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    sim.step(400)
    st = sim.stats()
    u = sim.state()[0]
    sim.close()
    ref = _oracle_nl(w, s0_of(w))
    ref.step(400)
    assert st["broken_bonds"] > 0 and st["validate_mismatches"] == 0
    assert rel(u, ref.u) <= 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_mixed_nonlinear_turned_spinning_body(dim):
    """Large rotation in FP32 bonds: the body turned by 35 degrees and spinning follows the FP64
    oracle to 1e-5 in u (the rigid motion dominates u; the FP32 strain resolution, ~1e-7 of the bond
    length, bounds the accuracy of the small elastic forces)."""
    if dim == 2:
        w = W.plate_vibration(nx=24, ny=20, nsteps=300, dt=2e-7, amp=0.0)
    else:
        x, y, z = W.grid_3d(12, 10, 8, 1e-3)
        w = W.Workload("block", W.MODEL_3D, E=30e9, nu=0.2, rho=2400.0, dx=1e-3, delta=3.015e-3, dt=2e-7,
                       nsteps=300, x=x, y=y, z=z, vol=np.full(x.size, 1e-9))
    P = np.stack([w.x, w.y] + ([w.z] if dim == 3 else []))
    c = P.mean(axis=1, keepdims=True)
    r = _rotation(dim, np.deg2rad(35.0)) @ (P - c)
    om = np.array([0.0, 0.0, 2e3]) if dim == 2 else np.array([300.0, -500.0, 800.0])
    r3 = np.vstack([r, np.zeros((1, w.n))]) if dim == 2 else r
    v0 = np.cross(om, r3.T).T[:dim]
    w.u0, w.v0 = r + c - P, v0
    sim = Simulation(w, s0=0.0, rate=0.0, precision=PD_MIXED, kinematics=PD_NONLINEAR)
    ref = _oracle_nl(w, 0.0)
    sim.step(300)
    ref.step(300)
    assert rel(sim.state()[0], ref.u) <= 1e-5
    sim.close()


def test_mixed_nonlinear_full_size_block():
    """The 200 x 100 x 50 notched block under torsion with nonlinear bonds: the mixed form follows
    the FP64 GPU path (itself held to the oracle at 1e-12 above) to 1e-3 over the first tenth of the
    run, with zero decisions differing from FP64 on its own state."""
    w = W.config3()
    s0 = s0_of(w)
    ref = Simulation(w, s0=s0, kinematics=PD_NONLINEAR)
    sim = Simulation(w, s0=s0, precision=PD_MIXED, kinematics=PD_NONLINEAR)
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    ref.step(200)
    sim.step(200)
    e = rel(sim.state()[0], ref.state()[0])
    st = sim.stats()
    ref.close()
    sim.close()
    assert e <= 1e-3 and st["validate_mismatches"] == 0, (e, st)


def test_mixed_nonlinear_two_word_shadow():
    """PD_OPT_SHADOW_LO with nonlinear bonds on the lattice layout: configuration 1's plate stays
    within the stated bounds and no worse than one word; on the breaking cracked plate every
    decision equals the FP64 nonlinear decision on the run's own state (validation mode)."""
    w = W.config1()
    ref = _oracle_nl(w, 0.0)
    ref.step(1000)
    errs = {}
    for lo in (0, 1):
        sim = Simulation(w, s0=0.0, precision=PD_MIXED, kinematics=PD_NONLINEAR, shadow_lo=lo)
        assert sim.get_option(B.PD_OPT_LATTICE) == 1 and sim.get_option(B.PD_OPT_SHADOW_LO) == lo
        sim.step(1000)
        errs[lo] = rel(sim.state()[0], ref.u)
        sim.close()
    print("nonlinear config1 rel-L2(u) one / two words:", errs)
    assert errs[1] <= 1e-4 and errs[1] <= 1.5 * errs[0], errs
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    sim = Simulation(w, s0=s0_of(w), precision=PD_MIXED, kinematics=PD_NONLINEAR, shadow_lo=1)
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    sim.step(400)
    st = sim.stats()
    sim.close()
    assert st["broken_bonds"] > 0 and st["validate_mismatches"] == 0, st
