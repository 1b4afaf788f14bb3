"""pd_step_noalloc, the allocation-free single time step, against the context API and the oracle.

Callers that cannot allocate device memory -- code running inside a framework whose allocator owns
the device, or a real-time loop that must never allocate -- call pd_step_noalloc with buffers they
already own.  Its result must equal what the allocating context API (pd_create_particles,
pd_build_neighbors, pd_set_state, pd_step) produces on the same state, on two calls in a row, and
the oracle's step from that state, within the FP64 parity tolerance used by the other GPU tests
(element by element and in rel-L2).  Cases: a 3D body with every bond intact, a 2D plate, and a
3D body whose bond status (read back from a context run that broke bonds) has zeros.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _close(a, ref, what):
    """rel-L2 and the per-particle bar: max_i |a_i - ref_i| <= TOL * max_i |ref_i|."""
    scale = max(np.abs(ref).max(), 1e-300)
    assert _rel(a, ref) <= TOL, (what, _rel(a, ref))
    assert np.abs(a - ref).max() <= TOL * scale, (what, np.abs(a - ref).max() / scale)


def _free(w, seed=5, vamp=1e-3):
    w.flag = None  # free body: no constraints, no loads
    w.b = None
    w.axis_point = w.axis_dir = None
    w.twist_in_s0 = 0.0
    w.v0 = vamp * np.random.default_rng(seed).normal(size=(w.dim, w.n))
    return w


def _block(amp=1e-6):
    from paper_2309_11273_gb300 import workloads as W
    return _free(W.notched_block(nx=20, ny=12, nz=10, dx=1e-3, notch_cells=7.5, seed=2, amp=amp))


def _plate():
    from paper_2309_11273_gb300 import workloads as W
    w = W.plate_vibration(nx=37, ny=21, dx=1e-3, seed=3)
    return _free(w, seed=6)


def _noalloc_twice(w, u0, v0, rp, col, intact):
    import torch

    from paper_2309_11273_gb300 import _binding as B
    dev = torch.device("cuda", torch.cuda.current_device())

    def d(a, dtype=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)

    x, y, vol = d(w.x), d(w.y), d(w.vol)
    z = d(w.z) if w.dim == 3 else None
    rp_d, col_d = d(rp, torch.int64), d(col, torch.int32)
    intact_d = d(intact, torch.uint8) if intact is not None else None
    u, v = d(u0), d(v0)
    stream = torch.cuda.current_stream()
    out = []
    for _ in range(2):
        u_out, v_out = torch.empty_like(u), torch.empty_like(v)
        theta = torch.empty(w.n, dtype=torch.float64, device=dev)
        st = B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, w.n, x.data_ptr(), y.data_ptr(),
                               z.data_ptr() if z is not None else None, vol.data_ptr(), rp_d.data_ptr(),
                               col_d.data_ptr(), intact_d.data_ptr() if intact_d is not None else None,
                               u.data_ptr(), v.data_ptr(), u_out.data_ptr(), v_out.data_ptr(),
                               theta.data_ptr(), stream.cuda_stream)
        assert st == B.PD_OK, B.pd_last_error()
        stream.synchronize()
        out.append((u_out.cpu().numpy(), v_out.cpu().numpy(), theta.cpu().numpy()))
        u, v = u_out, v_out
    return out


def _oracle_steps(w, u0, v0, status, nsteps=2):
    """The oracle's explicit steps from (u0, v0) with the given bond status and no breaking; per step
    (u, v, theta, per-particle theta bar scale)."""
    import oracle as O
    from parity import theta_scale
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, 0.0, w.dt, w.x, w.y, w.z, w.vol, w.cracks)
    if status is not None:
        assert status.size == ref.status.size
        ref.status[:] = status
    ref.set_state(u0, v0)
    res = []
    for _ in range(nsteps):
        ref.step(1)
        res.append((ref.u.copy(), ref.v.copy(), ref.theta.copy(), theta_scale(ref)))
    return ref, res


def _check_against(w, results, ctx_results, oracle_results):
    for k in range(2):
        un, vn, thn = results[k]
        for uc, vc, who in ((ctx_results[k][0], ctx_results[k][1], "context"),
                            (oracle_results[k][0], oracle_results[k][1], "oracle")):
            _close(un, uc.reshape(un.shape), (who, k, "u"))
            _close(vn, vc.reshape(vn.shape), (who, k, "v"))
        # theta (a cancelling sum): per particle within the propagation of the displacement bar
        th_ref, T = oracle_results[k][2], oracle_results[k][3]
        err = np.abs(thn - th_ref)
        assert np.all(err <= TOL * T), (k, float((err / np.where(T > 0, T, np.inf)).max()))
        assert np.abs(un - w.initial_u().reshape(un.shape)).max() > 0


def test_noalloc_step_matches_context_and_oracle_3d():
    from paper_2309_11273_gb300 import Simulation

    w = _block()
    sim = Simulation(w, s0=0.0)
    rp, col, intact = sim.neighbors()
    u0, v0 = w.initial_u(), w.initial_v()
    results = _noalloc_twice(w, u0, v0, rp, col, intact)
    ctx = []
    for _ in range(2):
        sim.step(1)
        ctx.append(sim.state())
    sim.close()
    ref, orc = _oracle_steps(w, u0, v0, intact)
    assert np.array_equal(ref.row_ptr, rp) and np.array_equal(ref.col, col)
    _check_against(w, results, ctx, orc)


def test_noalloc_step_matches_context_and_oracle_2d_plate():
    from paper_2309_11273_gb300 import Simulation

    w = _plate()
    sim = Simulation(w, s0=0.0)
    rp, col, intact = sim.neighbors()
    u0, v0 = w.initial_u(), w.initial_v()
    results = _noalloc_twice(w, u0, v0, rp, col, intact)
    ctx = []
    for _ in range(2):
        sim.step(1)
        ctx.append(sim.state())
    sim.close()
    ref, orc = _oracle_steps(w, u0, v0, intact)
    _check_against(w, results, ctx, orc)


def test_noalloc_step_with_broken_bonds():
    """Status with zeros: a free block whose random initial displacement (stretches near 2 s0)
    breaks bonds during a context run.  From the state and status read back, the context's next
    step (its head re-applies the failure check the read already applied, on the same u, and the
    step breaks nothing before the following step) equals the first pd_step_noalloc call; both
    calls equal the oracle's steps with that status and breaking off."""
    from paper_2309_11273_gb300 import Simulation

    w = _block(amp=1e-6)
    sim = Simulation(w, s0=1e-3)
    sim.step(3)
    u0, v0, _ = sim.state()
    rp, col, intact = sim.neighbors()
    assert (intact == 0).sum() > 100, (intact == 0).sum()
    results = _noalloc_twice(w, u0, v0, rp, col, intact)
    sim.step(1)
    uc, vc, thc = sim.state()
    sim.close()
    _close(results[0][0], uc.reshape(results[0][0].shape), ("context", 0, "u"))
    _close(results[0][1], vc.reshape(results[0][1].shape), ("context", 0, "v"))
    ref, orc = _oracle_steps(w, u0, v0, intact)
    for k in range(2):
        un, vn, _ = results[k]
        _close(un, orc[k][0].reshape(un.shape), ("oracle", k, "u"))
        _close(vn, orc[k][1].reshape(vn.shape), ("oracle", k, "v"))


def test_noalloc_rejects_oversized_host_foreign_and_overlapping_inputs():
    import torch

    from paper_2309_11273_gb300 import _binding as B

    w = _block()
    st = B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, (1 << 20) + 1, None, None, None, None, None, None,
                           None, None, None, None, None)
    assert st == B.PD_ERR_ARG and "1048576" in B.pd_last_error()
    n, dim = w.n, 3
    dev = torch.device("cuda", torch.cuda.current_device())

    def z(k, dtype=torch.float64):
        return torch.zeros(k, dtype=dtype, device=dev)

    x, y, zz, vol = z(n), z(n), z(n), z(n)
    rp = z(n + 1, torch.int64)
    col = z(8, torch.int32)
    intact = z(8, torch.uint8)
    u, v, uo, vo, th = z(dim * n), z(dim * n), z(dim * n), z(dim * n), z(n)

    def call(**kw):
        a = dict(x=x.data_ptr(), y=y.data_ptr(), z=zz.data_ptr(), vol=vol.data_ptr(), rp=rp.data_ptr(),
                 col=col.data_ptr(), intact=intact.data_ptr(), u=u.data_ptr(), v=v.data_ptr(),
                 uo=uo.data_ptr(), vo=vo.data_ptr(), th=th.data_ptr())
        a.update(kw)
        return B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, n, a["x"], a["y"], a["z"], a["vol"], a["rp"],
                                 a["col"], a["intact"], a["u"], a["v"], a["uo"], a["vo"], a["th"], None)

    host = np.zeros(3 * n)
    host_u8 = np.zeros(8, dtype=np.uint8)
    for kw in (dict(x=host.ctypes.data), dict(z=host.ctypes.data), dict(intact=host_u8.ctypes.data),
               dict(th=host.ctypes.data), dict(u=host.ctypes.data)):
        st = call(**kw)
        assert st == B.PD_ERR_ARG and "device" in B.pd_last_error(), kw
    for kw in (dict(vo=u.data_ptr()), dict(uo=v.data_ptr()), dict(vo=uo.data_ptr()),
               dict(uo=u.data_ptr() + 8), dict(th=vo.data_ptr() + 16), dict(th=x.data_ptr()),
               dict(uo=col.data_ptr() - 8)):
        st = call(**kw)
        assert st == B.PD_ERR_ARG and "overlap" in B.pd_last_error(), kw
    # a valid call on the same arrays still works (zero state: zero result)
    assert call() == B.PD_OK, B.pd_last_error()
    torch.cuda.synchronize()
    assert float(uo.abs().max()) == 0.0
