"""CUDA path vs the CPU oracle, element by element, on seeded synthetic workloads (GPU only).

Tolerances (tests/parity.py): FP64 path u and v within 1e-12 at every checkpoint both in rel-L2 and
per particle (max_i |u_i - u_ref,i| <= 1e-12 max_i |u_ref,i|); theta per particle within the
propagation of that bar and, globally, within 1e-12 of the size of the terms of its sum; bond status
(and so damage) exactly equal while the oracle's minimum relative stretch margin stays above 1e-9.
"""
import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import PD_FP64, PD_MIXED, BatchSimulation, Simulation
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import workloads as W

from parity import assert_fp64_close, compare, rel

pytestmark = pytest.mark.gpu
TOL = 1e-12


def s0_of(w):
    return O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0


def oracle_for(w, s0, rate=None):
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    ref.set_bc(w.flag, w.b, w.axis_point, w.axis_dir, w.rotation_rate(s0) if rate is None else rate)
    ref.set_state(w.initial_u(), w.initial_v())
    return ref


def run_pair(w, nsteps, every, precision=PD_FP64, rate=None, **kw):
    """Advance GPU and oracle side by side; returns per-checkpoint comparisons."""
    s0 = s0_of(w)
    sim = Simulation(w, s0=s0, precision=precision, rate=rate, **kw)
    ref = oracle_for(w, s0, rate)
    exact_status = True
    out = []
    done = 0
    while done < nsteps:
        k = min(every, nsteps - done)
        margins, broken = ref.step(k)
        sim.step(k)
        done += k
        if margins.size and margins.min() <= 1e-9:
            exact_status = False
        u, v, th = sim.state()
        rp, col, intact = sim.neighbors()
        out.append(dict(step=done, **compare(u, v, th, ref),
                        status_equal=np.array_equal(intact, ref.status), exact=exact_status,
                        broken=int((ref.status == 0).sum()), u=u, ref_u=ref.u.copy()))
    stats = sim.stats()
    phi = sim.damage()
    sim.close()
    return out, stats, phi, ref


def assert_fp64(out, ref_phi=None, phi=None):
    for c in out:
        assert_fp64_close({k: c[k] for k in ("ru", "rv", "eu", "ev", "et", "rt")}, TOL, "step %d" % c["step"])
        if c["exact"]:
            assert c["status_equal"], "bond status differs at step %d" % c["step"]
    if phi is not None and out[-1]["exact"]:
        assert np.array_equal(phi, ref_phi)


# ------------------------------------------------------------------------------------- family
FAMILY_CASES = {
    "cracked_plate": lambda: W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125),
    "notched_block": lambda: W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5),
    "ratio_4": lambda: W.plate_vibration(nx=30, ny=17, ratio=4.015),
}


@pytest.mark.parametrize("case", sorted(FAMILY_CASES))
def test_family_matches_oracle(case):
    w = FAMILY_CASES[case]()
    sim = Simulation(w, s0=0.0)
    rp, col, intact = sim.neighbors()
    sim.close()
    orp, ocol = O.family(w.x, w.y, w.z, w.delta, w.cracks)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    assert intact.all()


@pytest.mark.parametrize("dim", [2, 3])
def test_family_random_cloud_nonuniform_volumes(dim):
    rng = np.random.default_rng(10 + dim)
    n = 1500 if dim == 2 else 3000
    pts = rng.uniform(0.0, 1e-2, size=(dim, n))
    vol = rng.uniform(0.5, 1.5, n) * (2.5e-4) ** dim
    w = W.Workload("cloud", W.MODEL_3D if dim == 3 else W.MODEL_PLANE_STRAIN, E=1e9, nu=0.25, rho=1000.0,
                   dx=2.5e-4, delta=8e-4, dt=1e-9, nsteps=50, x=pts[0], y=pts[1],
                   z=pts[2] if dim == 3 else None, vol=vol,
                   u0=1e-7 * rng.normal(size=(dim, n)))
    s0 = 0.0
    sim = Simulation(w, s0=s0)
    rp, col, _ = sim.neighbors()
    orp, ocol = O.family(w.x, w.y, w.z, w.delta)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    ref = oracle_for(w, s0)
    ref.step(50)
    sim.step(50)
    u, v, th = sim.state()
    sim.close()
    assert_fp64_close(compare(u, v, th, ref), TOL)


# ------------------------------------------------------------------------------ FP64 dynamics
def test_config1_fp64_parity():
    """Configuration 1 in full: 40 x 40 plane stress plate, 1000 steps, checkpoints every 100."""
    w = W.config1()
    out, stats, phi, ref = run_pair(w, w.nsteps, 100)
    assert_fp64(out)
    assert stats["broken_bonds"] == 0 and stats["steps"] == w.nsteps


def test_cracked_plate_breaking_parity():
    """A small pre-cracked plate under traction: the crack grows from the pre-crack tip (about 1,400
    directed bonds break over 130 of the 400 steps, none in the loaded edge rows; the oracle's
    smallest stretch margin stays near 1e-7, so bond status is compared exactly throughout)."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    out, stats, phi, ref = run_pair(w, w.nsteps, 50)
    assert out[-1]["broken"] > 0
    assert_fp64(out, ref.damage(), phi)


def test_notched_block_twist_parity():
    """3D notched block, clamped + twisted ends (24 s0 rad over the run), small random initial
    displacement, breaking on: the fracture grows from step 23 on (about 50,000 of 263,000 directed
    bonds over 260 of the 300 steps) with the oracle's stretch margin above 4e-6 throughout."""
    w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    out, stats, phi, ref = run_pair(w, w.nsteps, 50)
    assert out[-1]["broken"] > 0
    assert_fp64(out, ref.damage(), phi)
    # prescribed particles follow the rigid rotation exactly
    pres = w.flag == W.PRESCRIBED
    assert np.array_equal(out[-1]["u"][:, pres], out[-1]["ref_u"][:, pres])


def test_plane_strain_breaking_parity():
    """Plane strain (Eq 1.8 / 1.15 / 1.28 plane-strain rows), steel-like material, breaking on."""
    w = W.cracked_plate(nx=50, ny=20, dx=2.5e-4, crack_cells=25.125, sigma=5e6, nsteps=300, dt=4.5e-8)
    w.model, w.E, w.nu, w.rho, w.Gc = W.MODEL_PLANE_STRAIN, 190e9, 0.25, 7800.0, 50.0
    out, stats, phi, ref = run_pair(w, w.nsteps, 50)
    assert out[-1]["broken"] > 0
    assert_fp64(out, ref.damage(), phi)


def test_config2_fp64_parity_first_1000_steps():
    """Configuration 2 at full size (64,000 particles), first 1000 of its 5000 steps."""
    w = W.config2()
    out, stats, phi, ref = run_pair(w, 1000, 250)
    assert_fp64(out, ref.damage(), phi)


def test_config3_quarter_scale_parity():
    """Configuration 3 geometry at quarter size (100 x 50 x 25), random u0, 40 steps."""
    w = W.notched_block(nx=100, ny=50, nz=25, dx=2e-3, nsteps=40, dt=3.790e-7 * 2, seed=5, amp=3e-6)
    out, stats, phi, ref = run_pair(w, w.nsteps, 20, rate=2e3)
    assert_fp64(out, ref.damage(), phi)


def _full_size_pair(w, s0, sim, nsteps):
    """nsteps of GPU and oracle from the same state: element-wise u, v, theta and, while the oracle's
    smallest stretch margin stays above 1e-9, the exact bond status."""
    ref = oracle_for(w, s0)
    assert ref.nbonds == sim.nbonds
    margins, broken = ref.step(nsteps)
    sim.step(nsteps)
    u, v, th = sim.state()
    rp, col, intact = sim.neighbors()
    assert_fp64_close(compare(u, v, th, ref, with_global_theta=False), TOL)
    assert int((ref.status == 0).sum()) > 0  # the random state stretches bonds near 2 s0: some break
    if margins.min() > 1e-9:
        assert np.array_equal(intact, ref.status)
    return ref


def test_config3_full_size_first_steps():
    """Configuration 3 at full size (1M particles, ~1.17e8 bonds): 2 steps from a random state,
    every particle compared (the oracle runs multi-threaded), bond status exactly."""
    w = W.notched_block(seed=7, amp=1e-6)
    s0 = s0_of(w)
    sim = Simulation(w, s0=s0)
    _full_size_pair(w, s0, sim, 2)
    sim.close()


def test_config3_full_size_autotuned_mapping():
    """The same full-size comparison with the launch mapping pd_autotune picks for this body (the
    mapping the benchmark times: threads per block, warps per slice, pair form), 3 steps."""
    w = W.notched_block(seed=8, amp=1e-6)
    s0 = s0_of(w)
    sim = Simulation(w, s0=s0)
    B.pd_autotune(sim.h, 5)
    sim.set_state(w.initial_u(), w.initial_v())  # autotune restores the state; start anew anyway
    mapping = {k: sim.get_option(o) for k, o in (("block", B.PD_OPT_BLOCK), ("split", B.PD_OPT_SPLIT),
                                                   ("pairs", B.PD_OPT_PAIRS))}
    _full_size_pair(w, s0, sim, 3)
    sim.close()
    print("autotuned mapping:", mapping)


# --------------------------------------------------------------------- launch-shape invariance
def test_graph_chunks_match_eager_launches():
    w = W.config1()
    res = []
    for chunk in (0, 100, 7):
        sim = Simulation(w, s0=0.0, graph_chunk=chunk)
        sim.step(250)
        res.append(sim.state()[0])
        sim.close()
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[0], res[2])


@pytest.mark.parametrize("block,split", [(128, 1), (512, 1), (256, 2), (128, 4), (512, 4)])
def test_mapping_variants_agree(block, split):
    w = W.notched_block(nx=30, ny=14, nz=12, dx=1e-3, notch_cells=11.5, nsteps=60, seed=1, amp=2e-6)
    base = Simulation(w, s0=s0_of(w), rate=5e3)
    base.step(60)
    ub = base.state()[0]
    base.close()
    sim = Simulation(w, s0=s0_of(w), rate=5e3)
    sim.set_option(B.PD_OPT_SPLIT, 1)
    sim.set_option(B.PD_OPT_BLOCK, block)
    sim.set_option(B.PD_OPT_SPLIT, split)
    sim.set_state(w.initial_u())
    sim.step(60)
    u = sim.state()[0]
    sim.close()
    assert rel(u, ub) <= 1e-13


@pytest.mark.parametrize("precision", [PD_FP64, PD_MIXED])
def test_orderings_and_bond_cache_agree(precision):
    """Internal particle order (bricks / Morton) and the FP64 geometry table change only rounding."""
    w = W.notched_block(nx=30, ny=14, nz=12, dx=1e-3, notch_cells=11.5, nsteps=60, seed=1, amp=2e-6)
    res = {}
    for order in (B.PD_ORDER_BRICKS, B.PD_ORDER_MORTON):
        for cache in ((1, 0) if precision == PD_FP64 else (1,)):
            sim = Simulation(w, s0=s0_of(w), rate=5e3, precision=precision, ordering=order, bond_cache=cache)
            sim.step(60)
            res[(order, cache)] = sim.state()[0]
            sim.close()
    ref = res[(B.PD_ORDER_BRICKS, 1)]
    tol = 1e-13 if precision == PD_FP64 else 1e-5
    for k, u in res.items():
        assert rel(u, ref) <= tol, (k, rel(u, ref))


def test_intact_sums_follow_the_status_bits():
    """The tabled FP64 force pass applies the i-end dilatation term of Eq 2.2 to a per-particle sum
    of V_j xi over the intact bonds, so that sum has to follow every change of the status bits: bonds
    broken by the tabled kernels, bonds broken while the table is switched off (untabled kernels), and
    bits restored by an autotune whose trial steps broke bonds.  Through all three the run equals the
    oracle (the cracked plate breaks bonds from step 40 to 180)."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    s0 = s0_of(w)
    sim = Simulation(w, s0=s0)
    ref = oracle_for(w, s0)
    exact = True
    for k, action in ((50, None), (40, "autotune"), (40, "untabled"), (270, "tabled")):
        if action == "autotune":
            B.pd_autotune(sim.h, 10)  # each trial advances 11 steps (breaking bonds), then restores
        elif action == "untabled":
            sim.set_option(B.PD_OPT_BOND_CACHE, 0)
        elif action == "tabled":
            sim.set_option(B.PD_OPT_BOND_CACHE, 1)
        margins, _ = ref.step(k)
        sim.step(k)
        exact = exact and (not margins.size or margins.min() > 1e-9)
    u, v, th = sim.state()
    _, _, intact = sim.neighbors()
    phi = sim.damage()
    sim.close()
    assert exact and (ref.status == 0).sum() > 1000
    assert_fp64_close(compare(u, v, th, ref), TOL)
    assert np.array_equal(intact, ref.status) and np.array_equal(phi, ref.damage())


@pytest.mark.parametrize("case,split", [("block", 1), ("block", 2), ("block", 4), ("plate", 1), ("plate", 2)])
def test_pair_form_is_bitwise_the_single_pass(case, split):
    """The tabled FP64 path forms each bond's xi.(u_j - u_i) once for both directed entries (the
    pair form, default) or once per entry: the two give bitwise the same u, v, bond status and
    damage, through bond breaking, with a state read (and its failure check) half way."""
    if case == "block":
        w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    else:
        w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    res = []
    for pairs in (1, 0):
        sim = Simulation(w, s0=s0_of(w))
        assert B.pd_get_option(sim.h, B.PD_OPT_PAIRS) == 1
        sim.set_option(B.PD_OPT_PAIRS, pairs)
        sim.set_option(B.PD_OPT_BLOCK, 128)
        sim.set_option(B.PD_OPT_SPLIT, split)
        sim.step(w.nsteps // 2)
        mid = sim.state()[0]
        sim.step(w.nsteps - w.nsteps // 2)
        u, v, _ = sim.state()
        res.append((mid, u, v, sim.neighbors()[2], sim.damage(), sim.stats()["broken_bonds"]))
        sim.close()
    assert res[0][5] > 0
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("split", [1, 2])
def test_checks_between_steps_with_form_switches_keep_the_trajectory(split):
    """A read between steps applies the pending failure check itself (the pair form by its own
    check kernel, the single pass by its check-only form) and the next step skips it.  Reading
    after every step, and switching between the pair form and the single pass after every read,
    gives bitwise the run that reads only at the end: bonds broken by a pair-form check and
    followed by a single-pass step leave no stale intact sum behind."""
    w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    ref = Simulation(w, s0=s0_of(w))
    ref.set_option(B.PD_OPT_BLOCK, 128)
    ref.set_option(B.PD_OPT_SPLIT, split)
    ref.step(w.nsteps)
    want = ref.state()[:2] + (ref.neighbors()[2], ref.damage())
    ref.close()
    sim = Simulation(w, s0=s0_of(w))
    sim.set_option(B.PD_OPT_BLOCK, 128)
    sim.set_option(B.PD_OPT_SPLIT, split)
    broken, pair_checks_broke = 0, 0
    for k in range(w.nsteps):
        pairs = B.pd_get_option(sim.h, B.PD_OPT_PAIRS)
        sim.step(1)
        now = sim.stats()["broken_bonds"]
        pair_checks_broke += pairs == 1 and now > broken
        broken = now
        sim.set_option(B.PD_OPT_PAIRS, 1 - pairs)
    got = sim.state()[:2] + (sim.neighbors()[2], sim.damage())
    sim.close()
    assert pair_checks_broke > 0
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", ["plate", "block"])
def test_screened_check_decides_near_threshold_bonds_in_fp64(shape):
    """The pair form's check before a read first decides each bond in FP32, with a bound on its
    distance from the FP64 value, and evaluates in FP64 only the bonds that bound cannot settle.
    Under a uniform stretch equal to the critical stretch every bond along x sits on its threshold
    (FP64 rounding decides it) and every other bond lies below: the screened check and the single
    pass's FP64 check break the same bonds, and the runs stay bitwise equal from there."""
    s0 = 1e-3
    if shape == "plate":
        w = W.plate_vibration(nx=40, ny=12, nsteps=10)
    else:
        w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=10)
    u0 = np.zeros((w.dim, w.n))
    u0[0] = s0 * w.x
    w.u0 = u0
    res = []
    for pairs in (1, 0):
        sim = Simulation(w, s0=s0)
        sim.set_option(B.PD_OPT_PAIRS, pairs)
        assert B.pd_get_option(sim.h, B.PD_OPT_PAIRS) == pairs
        sim.step(1)
        phi = sim.damage()  # the check of u^1, by the screened kernel in the pair form
        bits = sim.neighbors()[2]
        broken = sim.stats()["broken_bonds"]
        sim.step(5)
        res.append((phi, bits, broken) + sim.state()[:2] + (sim.neighbors()[2],))
        sim.close()
    assert 0 < res[0][2] < res[0][1].size
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [PD_FP64, PD_MIXED])
def test_state_round_trip_after_every_step_is_the_plain_run(precision):
    """Reading u and v after every step and writing them back before the next gives bitwise the
    run that never leaves the device, while bonds break throughout: the read's copies (and the
    write's upload and finiteness check) run on the library's transfer stream beside the failure
    check that the read leaves running, and the written state lands only after that check.  Host
    buffers alternate between pageable and pinned memory."""
    import torch
    w = W.notched_block(nx=24, ny=12, nz=10, dx=1e-3, notch_cells=9.5, nsteps=300, seed=3, amp=1e-7)
    ref = Simulation(w, s0=s0_of(w), precision=precision)
    ref.step(w.nsteps)
    want = ref.state()[:2] + (ref.neighbors()[2],)
    ref.close()
    sim = Simulation(w, s0=s0_of(w), precision=precision)
    dim, n = 3, w.n
    pinned = [torch.empty((dim, n), dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    for k in range(w.nsteps):
        sim.step(1)
        if k % 2:
            u, v = pinned
            B.pd_get_state(sim.h, dim, n, u, v, False)
        else:
            u, v, _ = B.pd_get_state(sim.h, dim, n, True, True, False)
        B.pd_set_state(sim.h, dim, n, u, v)
    got = sim.state()[:2] + (sim.neighbors()[2],)
    sim.close()
    assert not want[2].all()  # bonds broke
    for a, b in zip(got, want):
        assert np.array_equal(a, b)


# --------------------------------------------------------------------------------- edge cases
def test_single_particle_and_ragged_sizes():
    for nx, ny in ((1, 1), (33, 1), (7, 5)):
        w = W.plate_vibration(nx=nx, ny=ny, nsteps=20, amp=1e-6)
        out, stats, phi, ref = run_pair(w, 20, 10)
        assert_fp64(out)
        if nx * ny == 1:
            assert stats["bonds"] == 0 and np.all(phi == 0.0)


def test_crack_removing_every_bond():
    """A crack between every pair of columns leaves particles without bonds: no force, phi = 0."""
    w = W.plate_vibration(nx=4, ny=6, ratio=1.2, nsteps=10)
    w.cracks = [(x0, -1.0, 0, x0, 1.0, 0, 0, 0, 0) for x0 in (1e-3, 2e-3, 3e-3)]
    w.cracks += [(-1.0, y0, 0, 1.0, y0, 0, 0, 0, 0) for y0 in (1e-3, 2e-3, 3e-3, 4e-3, 5e-3)]
    out, stats, phi, ref = run_pair(w, 10, 10)
    assert stats["bonds"] == 0 and np.all(phi == 0.0)
    assert np.array_equal(out[-1]["u"], w.initial_u())


def test_state_errors_and_divergence_guard():
    w = W.plate_vibration(nx=8, ny=8)
    prm = B.make_params(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt)
    h = B.pd_create_particles(prm, w.x, w.y, None, w.vol)
    with pytest.raises(B.PDError) as e:
        B.pd_step(h, 1)
    assert e.value.status == B.PD_ERR_STATE
    B.pd_build_neighbors(h)
    u0 = w.initial_u()
    B.pd_set_state(h, 2, w.n, u0)
    assert B.pd_check_state(h, 1.0) == B.PD_OK
    assert B.pd_check_state(h, 1e-9) == B.PD_ERR_NUMERIC
    # a non-finite value anywhere in u or v is rejected and leaves the state as it was
    bad_u = u0.copy()
    bad_u[1, w.n - 1] = np.inf
    bad_v = np.zeros((2, w.n))
    bad_v[0, 3] = np.nan
    for args in ((np.full((2, w.n), np.nan),), (bad_u,), (2.0 * u0, bad_v)):
        with pytest.raises(B.PDError) as e:
            B.pd_set_state(h, 2, w.n, *args)
        assert e.value.status == B.PD_ERR_ARG
    u, v, _ = B.pd_get_state(h, 2, w.n)
    assert np.array_equal(u, u0) and np.all(v == 0.0)
    B.pd_destroy(h)


def test_unstable_time_step_trips_the_guard():
    """dt = 1.2 x the stable bound diverges: the guard reports PD_ERR_NUMERIC (no GPU fault)."""
    w = W.plate_vibration(dt=1.2 * 3.3693e-7)
    sim = Simulation(w, s0=0.0)
    sim.step(600)
    assert B.pd_check_state(sim.h, 1e-3) == B.PD_ERR_NUMERIC
    # run on until the state overflows: the next sync reports it without a device fault
    sim.step(20000)
    with pytest.raises(B.PDError) as e:
        sim.sync()
    assert e.value.status == B.PD_ERR_NUMERIC
    sim.close()


def test_expired_wait_reports_timeout_and_context_recovers():
    """Failure path of the bounded waits: with PD_OPT_EXPIRE_WAITS the staged kernels never issue
    each warp's first index copy, so that wait runs out (1 s of the GPU timer), the warps skip their
    outputs and the next pd_sync returns PD_ERR_TIMEOUT; the context stays usable and a clean rerun
    equals a fresh run bitwise."""
    w = W.plate_vibration(nx=16, ny=8, nsteps=20)
    sim = Simulation(w, s0=0.0, precision=PD_MIXED, graph_chunk=0)
    assert sim.get_option(B.PD_OPT_STAGE) == 1 and sim.get_option(B.PD_OPT_SPLIT) == 1
    sim.set_option(B.PD_OPT_EXPIRE_WAITS, 1)
    sim.step(1)
    with pytest.raises(B.PDError) as e:
        sim.sync()
    assert e.value.status == B.PD_ERR_TIMEOUT
    sim.set_option(B.PD_OPT_EXPIRE_WAITS, 0)
    sim.sync()  # the error word was cleared when it was reported
    sim.set_state(w.initial_u())
    sim.step(20)
    u = sim.state()[0]
    sim.close()
    ref = Simulation(w, s0=0.0, precision=PD_MIXED, graph_chunk=0)
    ref.step(20)
    assert np.array_equal(u, ref.state()[0])
    ref.close()


# ------------------------------------------------------------------------------------ batched
def _small_batch(n=5, seed=4):
    return W.plate_batch(nplates=n, seed=seed, side_lo=10, side_hi=40, nsteps=200)


def test_batch_equals_separate_runs_bitwise():
    bw = _small_batch()
    s0s = [s0_of(b) for b in bw.bodies]
    bs = BatchSimulation(bw, s0s)
    bs.step(200)
    ub = bs.state()[0]
    bs.close()
    for k, b in enumerate(bw.bodies):
        sim = Simulation(b, s0=s0s[k])
        sim.step(200)
        u = sim.state()[0]
        sim.close()
        assert np.array_equal(u, ub[:, bw.offsets[k]:bw.offsets[k + 1]]), k


def test_batch_pair_form_and_option_reporting():
    """A batch of uneven plates with breaking: the pair form (pairs never cross bodies) equals the
    single pass bitwise; PD_OPT_PAIRS reads back 1 for FP64 contexts and 0 for mixed ones."""
    bw = _small_batch(n=6, seed=11)
    s0s = [s0_of(b) for b in bw.bodies]
    res = []
    for pairs in (1, 0):
        bs = BatchSimulation(bw, s0s)
        assert B.pd_get_option(bs.h, B.PD_OPT_PAIRS) == 1
        B.pd_set_option(bs.h, B.PD_OPT_PAIRS, pairs)
        assert B.pd_get_option(bs.h, B.PD_OPT_PAIRS) == pairs
        bs.step(200)
        res.append((bs.state()[0], bs.neighbors()[2], bs.stats()["broken_bonds"]))
        bs.close()
    assert res[0][2] > 0 and res[0][2] == res[1][2]
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    bm = BatchSimulation(bw, s0s, precision=PD_MIXED)
    assert B.pd_get_option(bm.h, B.PD_OPT_PAIRS) == 0
    bm.close()


def test_batch_vs_oracle():
    bw = _small_batch(n=3, seed=9)
    s0s = [s0_of(b) for b in bw.bodies]
    bs = BatchSimulation(bw, s0s)
    bs.step(150)
    ub, vb, thb = bs.state()
    rp, col, intact = bs.neighbors()
    bs.close()
    for k, b in enumerate(bw.bodies):
        ref = oracle_for(b, s0s[k])
        margins, _ = ref.step(150)
        sl = slice(bw.offsets[k], bw.offsets[k + 1])
        assert_fp64_close(compare(ub[:, sl], vb[:, sl], thb[sl], ref), TOL, "body %d" % k)
        if margins.min() > 1e-9:
            lo, hi = rp[bw.offsets[k]], rp[bw.offsets[k + 1]]
            assert np.array_equal(intact[lo:hi], ref.status)


# -------------------------------------------------------------------------------------- mixed
def test_mixed_config1_error_bound():
    """FP32 bond arithmetic with FP64 integration: rel-L2(u) vs the FP64 oracle after 100 and 1000
    steps of configuration 1 (stated bound 2e-5 / 1e-4)."""
    w = W.config1()
    out, stats, phi, ref = run_pair(w, 1000, 100, precision=PD_MIXED)
    assert out[0]["ru"] <= 2e-5, out[0]["ru"]
    assert max(c["ru"] for c in out) <= 1e-4, [c["ru"] for c in out]


def test_mixed_decisions_equal_fp64_on_own_state():
    """Zero spurious breaks: with validation on, every bond decision of the FP32 + band path equals
    the pure FP64 decision on the mixed run's own state."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    sim = Simulation(w, s0=s0_of(w), precision=PD_MIXED)
    sim.set_option(B.PD_OPT_VALIDATE, 1)
    sim.step(400)
    st = sim.stats()
    sim.close()
    assert st["broken_bonds"] > 0
    assert st["validate_mismatches"] == 0


# ------------------------------------------------------------------------------- diagnostics
def _strain_energy_np(ref, u, status):
    """sum_i V_i [(K - G/3)/(2A) theta_i^2 + G/(2 m_i) sum_j e_ij^2 V_j], linearized e, from the
    oracle's family and coordinates (written out here, independently of both implementations)."""
    P = np.stack([ref.x, ref.y] + ([ref.z] if ref.dim == 3 else []))
    rows = np.repeat(np.arange(ref.n), np.diff(ref.row_ptr))
    xi = P[:, ref.col] - P[:, rows]
    xl = np.sqrt((xi * xi).sum(0))
    e = ((xi / xl) * (u[:, ref.col] - u[:, rows])).sum(0) * status
    vj = ref.vol[ref.col]
    th = ref.A / ref.m * np.bincount(rows, weights=xl * e * vj, minlength=ref.n)
    es = np.bincount(rows, weights=e * e * vj, minlength=ref.n)
    return float((ref.vol * ((ref.K - ref.G / 3) / (2 * ref.A) * th ** 2 + ref.G / (2 * ref.m) * es)).sum())


def test_shadow_energy_is_conserved():
    """Configuration 1 (no loads, constraints or breaking): pd_get_stats' shadow energy
    U(u^n) + 1/2 sum rho V v^n . v^{n+1} stays constant to 1e-12 over 1000 steps while the strain
    energy alone swings; the strain energy equals the one written out in the test to 1e-12."""
    w = W.config1()
    sim = Simulation(w, s0=0.0)
    ref = oracle_for(w, 0.0)
    H, Us = [], []
    for _ in range(10):
        sim.step(100)
        ref.step(100)
        st = sim.stats()
        H.append(st["shadow_energy"])
        Us.append(st["strain_energy"])
        u = sim.state()[0]
        assert st["strain_energy"] == pytest.approx(_strain_energy_np(ref, u, np.ones(ref.col.size)), rel=1e-12)
    sim.close()
    H = np.array(H)
    assert np.abs(H - H[0]).max() <= 1e-12 * abs(H[0])
    assert (max(Us) - min(Us)) > 1e-3 * max(Us)


def test_min_margin_matches_oracle():
    """The smallest relative stretch margin of pd_get_stats equals the oracle's after the same steps
    (cracked plate with crack growth)."""
    w = W.cracked_plate(nx=60, ny=24, dx=2.5e-4, crack_cells=30.125, sigma=2e6, nsteps=400)
    s0 = s0_of(w)
    sim = Simulation(w, s0=s0)
    ref = oracle_for(w, s0)
    for _ in range(4):
        margins, _ = ref.step(100)
        sim.step(100)
        st = sim.stats()
        assert st["min_rel_margin"] == pytest.approx(margins[-1], rel=1e-9)
    assert st["broken_bonds"] > 0
    sim.close()
