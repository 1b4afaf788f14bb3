"""GB300 (sm_103a) hot path of linearized OSB-PD (Ni et al., arXiv 2309.11273).

The computation lives in the CUDA library ``libosbpd.so`` behind the C ABI of ``include/osbpd.h``;
``_binding`` exposes its entry points under the same names, and ``Simulation`` / ``BatchSimulation``
below only sequence those calls for a workload from ``workloads``.  There is no CPU fallback: if the
library is missing every call raises.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B
from ._binding import (PD_3D, PD_FP64, PD_LINEARIZED, PD_MIXED, PD_NONLINEAR, PD_PLANE_STRAIN, PD_PLANE_STRESS,
                       PD_W_INV, PD_W_ONE, PDError, pd_critical_stretch)

__all__ = ["Simulation", "BatchSimulation", "PDError", "PD_FP64", "PD_MIXED", "PD_LINEARIZED", "PD_NONLINEAR", "PD_3D",
           "PD_PLANE_STRESS", "PD_PLANE_STRAIN", "PD_W_ONE", "PD_W_INV", "pd_critical_stretch"]


class Simulation:
    """One body: create -> build family -> boundary conditions -> initial state, then step."""

    def __init__(self, w, s0=None, precision=PD_FP64, rate=None, device=0, stream=None,
                 band_safety=0.0, graph_chunk=None, ordering=B.PD_ORDER_BRICKS, bond_cache=None,
                 kinematics=B.PD_LINEARIZED, pairs=None, influence=B.PD_W_ONE, lattice=None,
                 shadow_lo=None):
        self.w = w
        self.n, self.dim = w.n, w.dim
        if s0 is None:
            s0 = pd_critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta) if w.Gc else 0.0
        self.s0 = float(s0)
        prm = B.make_params(w.model, w.E, w.nu, w.rho, w.delta, self.s0, w.dt, precision, band_safety,
                            device, stream, ordering, kinematics, influence)
        self.h = B.pd_create_particles(prm, w.x, w.y, w.z, w.vol)
        try:
            if lattice is not None:
                B.pd_set_option(self.h, B.PD_OPT_LATTICE, int(lattice))
            if shadow_lo is not None:
                B.pd_set_option(self.h, B.PD_OPT_SHADOW_LO, int(shadow_lo))
            if graph_chunk is not None:
                B.pd_set_option(self.h, B.PD_OPT_GRAPH_CHUNK, graph_chunk)
            if bond_cache is not None:
                B.pd_set_option(self.h, B.PD_OPT_BOND_CACHE, int(bond_cache))
            if pairs is not None:
                B.pd_set_option(self.h, B.PD_OPT_PAIRS, int(pairs))
            B.pd_build_neighbors(self.h, w.cracks)
            self.rate = w.rotation_rate(self.s0) if rate is None else float(rate)
            if w.flag is not None or w.b is not None:
                B.pd_set_bc(self.h, self.dim, self.n, w.flag, w.b, w.axis_point, w.axis_dir, self.rate)
            if getattr(w, "vp", None) is not None:
                B.pd_set_prescribed_velocity(self.h, self.dim, self.n, w.vp)
            B.pd_set_state(self.h, self.dim, self.n, w.initial_u(), w.initial_v())
        except Exception:
            B.pd_destroy(self.h)
            self.h = None
            raise

    @property
    def nbonds(self) -> int:
        return B.pd_num_bonds(self.h)

    def set_state(self, u, v=None):
        B.pd_set_state(self.h, self.dim, self.n, u, v)

    def step(self, nsteps: int):
        B.pd_step(self.h, nsteps)

    def sync(self):
        B.pd_sync(self.h)

    def state(self):
        return B.pd_get_state(self.h, self.dim, self.n)

    def damage(self):
        return B.pd_get_damage(self.h, self.n)

    def neighbors(self):
        return B.pd_get_neighbors(self.h, self.n)

    def stats(self):
        return B.pd_get_stats(self.h)

    def set_option(self, opt, value):
        B.pd_set_option(self.h, opt, value)

    def get_option(self, opt) -> int:
        return B.pd_get_option(self.h, opt)

    def save_state(self, path):
        """Checkpoint (u, v, bond status, step count) to a file; see pd_save_state."""
        B.pd_save_state(self.h, path)

    def load_state(self, path):
        """Resume from a checkpoint of the same problem; see pd_load_state."""
        B.pd_load_state(self.h, path)

    def close(self):
        if self.h:
            B.pd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation(Simulation):
    """Many independent bodies (``workloads.BatchWorkload``) in one context and the same kernels."""

    def __init__(self, bw, s0s=None, precision=PD_FP64, device=0, stream=None, band_safety=0.0,
                 graph_chunk=None, ordering=B.PD_ORDER_BRICKS, bond_cache=None, kinematics=B.PD_LINEARIZED,
                 influence=B.PD_W_ONE):
        self.w = bw
        self.n, self.dim = bw.n, 2 if bw.bodies[0].z is None else 3
        if s0s is None:
            s0s = [pd_critical_stretch(b.model, b.E, b.nu, b.Gc, b.delta) if b.Gc else 0.0 for b in bw.bodies]
        self.s0s = [float(s) for s in s0s]
        prms = [B.make_params(b.model, b.E, b.nu, b.rho, b.delta, s, b.dt, precision, band_safety, device, stream,
                              ordering, kinematics, influence) for b, s in zip(bw.bodies, self.s0s)]
        z = bw.concat("z") if self.dim == 3 else None
        self.h = B.pd_create_batch(prms, bw.offsets, bw.concat("x"), bw.concat("y"), z, bw.concat("vol"))
        try:
            if graph_chunk is not None:
                B.pd_set_option(self.h, B.PD_OPT_GRAPH_CHUNK, graph_chunk)
            if bond_cache is not None:
                B.pd_set_option(self.h, B.PD_OPT_BOND_CACHE, int(bond_cache))
            B.pd_build_neighbors(self.h, [])
            bs = [b.b if b.b is not None else np.zeros((self.dim, b.n)) for b in bw.bodies]
            if any(b.b is not None for b in bw.bodies):
                B.pd_set_bc(self.h, self.dim, self.n, None, np.concatenate(bs, axis=1))
            u0 = np.concatenate([b.initial_u() for b in bw.bodies], axis=1)
            B.pd_set_state(self.h, self.dim, self.n, u0)
        except Exception:
            B.pd_destroy(self.h)
            self.h = None
            raise
