"""The paper's own matrix-based scheme on this GPU: a same-box baseline for the fused kernels.

Section 3.1 writes one step of linearized OSB-PD as four sparse matrix-vector products over global
matrices assembled once (Eqs 2.4-2.10) and the solver loop of Appendix B:

    E = CE U,   Theta = CTH E,   PDF = KTH Theta + KE E,   RF = EXF + PDF,
    VEL = VEL + dt RF / M,   U(free) = U(free) + dt VEL(free)

with U, VEL, PDF, EXF node-major (3 entries per node), one row of CE per undirected bond.  Here the
four matrices are FP64 CSR with 32-bit indices on the GPU and every product runs through the sparse
library behind ``torch.sparse`` (cuSPARSE); the update and the boundary conditions (fixed /
prescribed linearized rotation, as the library's) are elementwise tensor operations.  This module is
a baseline for measurement, not part of the library's path: nothing in ``libosbpd.so`` calls it.
Bond failure is not included (Appendix B elides its failure block; with assembled matrices a broken
bond would require re-assembling KTH), so it runs the no-breaking form of a workload.
"""
from __future__ import annotations

import warnings

import numpy as np


class MatrixScheme:
    """Assembles CE, CTH, KTH, KE for a workload's family and advances its state step by step.

    ``row_ptr``/``col``: the family as CSR in caller order (e.g. from ``Simulation.neighbors()``);
    ``A, K, G``: material constants of Eqs 1.8, 1.15, 1.16.
    """

    def __init__(self, w, row_ptr, col, A, K, G, rate=0.0, device="cuda"):
        import torch
        self.torch = torch
        dev = torch.device(device)
        f64 = torch.float64
        self.dim = d = w.dim
        self.n = n = w.n
        self.dt = float(w.dt)
        self.rate = float(rate)
        P = torch.tensor(np.stack([w.x, w.y] + ([w.z] if d == 3 else [])), dtype=f64, device=dev)
        V = torch.tensor(w.vol, dtype=f64, device=dev)
        rp = torch.tensor(row_ptr, dtype=torch.int64, device=dev)
        cj = torch.tensor(col, dtype=torch.int64, device=dev)
        ci = torch.repeat_interleave(torch.arange(n, device=dev), rp[1:] - rp[:-1])
        # weighted volume over the directed family (Eq 1.9, w = 1)
        xi_d = P[:, cj] - P[:, ci]
        m = torch.zeros(n, dtype=f64, device=dev).index_add_(0, ci, (xi_d * xi_d).sum(0) * V[cj])
        del xi_d
        keep = ci < cj  # one row per undirected bond
        bi, bj = ci[keep], cj[keep]
        del ci, cj, keep
        nb = bi.numel()
        xi = P[:, bj] - P[:, bi]
        xl = torch.sqrt((xi * xi).sum(0))
        M = xi / xl
        del xi
        Vi, Vj, mi, mj = V[bi], V[bj], m[bi], m[bj]
        b_ar = torch.arange(nb, device=dev)
        comps = torch.arange(d, device=dev)

        def csr(rows, cols, vals, shape):
            with warnings.catch_warnings():
                warnings.simplefilter("ignore", UserWarning)  # "sparse CSR support is in beta"
                t = torch.sparse_coo_tensor(torch.stack([rows, cols]), vals, shape,
                                            check_invariants=False).coalesce().to_sparse_csr()
                return torch.sparse_csr_tensor(t.crow_indices().to(torch.int32), t.col_indices().to(torch.int32),
                                               t.values(), shape, check_invariants=False)

        # CE (Eq 2.7): row b, columns (i, c) -> -M_c and (j, c) -> +M_c
        r = b_ar.repeat_interleave(2 * d)
        cc = torch.cat([d * bi[:, None] + comps, d * bj[:, None] + comps], dim=1).reshape(-1)
        vv = torch.cat([-M.T, M.T], dim=1).reshape(-1)
        self.CE = csr(r, cc, vv, (nb, d * n))
        # CTH (Eq 2.10): theta_i += A x V_j / m_i e_b, theta_j += A x V_i / m_j e_b
        self.CTH = csr(torch.cat([bi, bj]), torch.cat([b_ar, b_ar]),
                       torch.cat([A * xl * Vj / mi, A * xl * Vi / mj]), (n, nb))
        # KE (Eq 2.9): column b, rows (i, c) -> +g M_c and (j, c) -> -g M_c, g = G V_i V_j (1/m_i + 1/m_j)
        g = G * Vi * Vj * (1.0 / mi + 1.0 / mj)
        rows = torch.cat([d * bi[:, None] + comps, d * bj[:, None] + comps], dim=1).reshape(-1)
        self.KE = csr(rows, b_ar.repeat_interleave(2 * d), torch.cat([(g * M).T, (-g * M).T], dim=1).reshape(-1),
                      (d * n, nb))
        # KTH (Eq 2.8): rows (i, c): [+k M_c / m_i at column i, +k M_c / m_j at column j];
        # rows (j, c): the same with the opposite sign; k = (K - G/3) x V_i V_j; summed over bonds
        k = (K - G / 3.0) * xl * Vi * Vj
        ri = (d * bi[:, None] + comps)
        rj = (d * bj[:, None] + comps)
        a_i = (k / mi)[:, None] * M.T
        a_j = (k / mj)[:, None] * M.T
        rows = torch.cat([ri, ri, rj, rj], dim=1).reshape(-1)
        cols = torch.cat([bi[:, None].expand(-1, d), bj[:, None].expand(-1, d),
                          bi[:, None].expand(-1, d), bj[:, None].expand(-1, d)], dim=1).reshape(-1)
        vals = torch.cat([a_i, a_j, -a_i, -a_j], dim=1).reshape(-1)
        self.KTH = csr(rows, cols, vals, (d * n, n))
        del rows, cols, vals, a_i, a_j, ri, rj
        self.nbonds_undirected = nb
        self.nnz = sum(int(t.values().numel()) for t in (self.CE, self.CTH, self.KE, self.KTH))
        self.matrix_bytes = sum(int(t.values().numel()) * 12 + int(t.crow_indices().numel()) * 4
                                for t in (self.CE, self.CTH, self.KE, self.KTH))
        # diagonal mass, external force, boundary conditions
        self.mass = (float(w.rho) * V).repeat_interleave(d)
        b = np.zeros((d, n)) if w.b is None else np.asarray(w.b, dtype=np.float64).reshape(d, n)
        self.EXF = (torch.tensor(b.T.reshape(-1), dtype=f64, device=dev) * V.repeat_interleave(d))
        flag = np.zeros(n, dtype=np.uint8) if w.flag is None else np.asarray(w.flag, dtype=np.uint8)
        fl = torch.tensor(flag, device=dev).repeat_interleave(d)
        self.free = fl == 0
        self.fixed = fl == 1
        self.presc = fl == 2
        self.has_fixed = bool(self.fixed.any())
        self.has_presc = bool(self.presc.any())
        if w.axis_point is not None and w.axis_dir is not None:
            a = torch.tensor(w.axis_dir, dtype=f64, device=dev)
            c = torch.tensor(w.axis_point, dtype=f64, device=dev)
            r3 = torch.zeros(3, n, dtype=f64, device=dev)
            r3[:d] = P - c[:d, None]
            if d == 2:
                r3[2] = -c[2]
            gv = torch.linalg.cross(a[:, None].expand(3, n), r3, dim=0)
            self.gvec = gv[:d].T.reshape(-1)
        else:
            self.gvec = torch.zeros(d * n, dtype=f64, device=dev)
        self.U = torch.zeros(d * n, dtype=f64, device=dev)
        self.VEL = torch.zeros(d * n, dtype=f64, device=dev)
        self.steps_done = 0

    def set_state(self, u, v=None):
        t = self.torch
        d, n = self.dim, self.n
        self.U = t.tensor(np.asarray(u, dtype=np.float64).reshape(d, n).T.reshape(-1), device=self.U.device)
        self.VEL = (t.zeros_like(self.U) if v is None else
                    t.tensor(np.asarray(v, dtype=np.float64).reshape(d, n).T.reshape(-1), device=self.U.device))
        self._bc(self.steps_done * self.dt)

    def _bc(self, t):
        if self.has_fixed:
            self.U = self.torch.where(self.fixed, 0.0, self.U)
            self.VEL = self.torch.where(self.fixed, 0.0, self.VEL)
        if self.has_presc:
            self.U = self.torch.where(self.presc, self.rate * t * self.gvec, self.U)
            self.VEL = self.torch.where(self.presc, self.rate * self.gvec, self.VEL)

    def step(self, nsteps: int):
        """The solver loop of Appendix B, nsteps iterations (boundary values at t_n and t_{n+1})."""
        mv = self.torch.mv
        for _ in range(int(nsteps)):
            self._bc(self.steps_done * self.dt)
            E = mv(self.CE, self.U)
            Th = mv(self.CTH, E)
            PDF = mv(self.KTH, Th) + mv(self.KE, E)
            ACC = (self.EXF + PDF) / self.mass
            self.VEL = self.torch.where(self.free, self.VEL + self.dt * ACC, self.VEL)
            self.U = self.torch.where(self.free, self.U + self.dt * self.VEL, self.U)
            self.steps_done += 1
            self._bc(self.steps_done * self.dt)

    def state(self):
        d, n = self.dim, self.n
        return (self.U.reshape(n, d).T.cpu().numpy(), self.VEL.reshape(n, d).T.cpu().numpy())
