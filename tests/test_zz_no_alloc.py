"""pd_step_noalloc, the allocation-free single time step, against the context API.

Callers that cannot allocate device memory -- code running inside a framework whose allocator owns
the device, or a real-time loop that must never allocate -- call pd_step_noalloc with buffers they
already own.  Its result must equal what the allocating context API (pd_create_particles,
pd_build_neighbors, pd_set_state, pd_step) produces, on two calls in a row, within the FP64 parity
tolerance used by the other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _body():
    from paper_2309_11273_gb300 import workloads as W
    w = W.notched_block(nx=20, ny=12, nz=10, dx=1e-3, notch_cells=7.5, seed=2, amp=1e-6)
    w.flag = None  # free body: no constraints, no loads, no breaking
    w.axis_point = w.axis_dir = None
    w.twist_in_s0 = 0.0
    w.v0 = 1e-3 * np.random.default_rng(5).normal(size=(3, w.n))
    return w


def test_noalloc_step_matches_context_api_twice():
    import torch

    from paper_2309_11273_gb300 import Simulation
    from paper_2309_11273_gb300 import _binding as B

    w = _body()
    sim = Simulation(w, s0=0.0)
    rp, col, intact = sim.neighbors()
    dev = torch.device("cuda", torch.cuda.current_device())

    def d(a, dtype=torch.float64):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)

    x, y, z, vol = d(w.x), d(w.y), d(w.z), d(w.vol)
    rp_d, col_d, intact_d = d(rp, torch.int64), d(col, torch.int32), d(intact, torch.uint8)
    u, v = d(w.initial_u()), d(w.initial_v())
    stream = torch.cuda.current_stream()
    results = []
    for _ in range(2):
        u_out, v_out = torch.empty_like(u), torch.empty_like(v)
        theta = torch.empty(w.n, dtype=torch.float64, device=dev)
        st = B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, w.n, x.data_ptr(), y.data_ptr(), z.data_ptr(),
                               vol.data_ptr(), rp_d.data_ptr(), col_d.data_ptr(), intact_d.data_ptr(),
                               u.data_ptr(), v.data_ptr(), u_out.data_ptr(), v_out.data_ptr(),
                               theta.data_ptr(), stream.cuda_stream)
        assert st == B.PD_OK, B.pd_last_error()
        stream.synchronize()
        results.append((u_out.cpu().numpy(), v_out.cpu().numpy(), theta.cpu().numpy()))
        u, v = u_out, v_out
    for k in range(2):
        sim.step(1)
        uc, vc, thc = sim.state()
        un, vn, thn = results[k]
        assert _rel(un, uc) <= TOL and _rel(vn, vc) <= TOL, (k, _rel(un, uc), _rel(vn, vc))
        assert np.linalg.norm(thn - thc) <= TOL * max(np.linalg.norm(thc), 1e-300) * 10, k
        assert np.abs(un - w.initial_u()).max() > 0
    sim.close()


def test_noalloc_rejects_oversized_and_host_inputs():
    import torch

    from paper_2309_11273_gb300 import _binding as B

    w = _body()
    st = B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, (1 << 20) + 1, None, None, None, None, None, None,
                           None, None, None, None, None)
    assert st == B.PD_ERR_ARG and "1048576" in B.pd_last_error()
    host = np.zeros(3 * w.n)
    dev = torch.zeros(3 * w.n, dtype=torch.float64, device="cuda")
    p = host.ctypes.data
    st = B.pd_step_noalloc(w.model, w.E, w.nu, w.rho, w.dt, w.n, p, p, p, p, p, p, None, p, p, dev.data_ptr(),
                           dev.data_ptr() + 8, None)
    assert st == B.PD_ERR_ARG and "device" in B.pd_last_error()
