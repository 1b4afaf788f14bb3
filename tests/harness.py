"""One call sequence for both implementations: the GPU library through its C ABI binding (pd_*) and
the oracle through the same sequence (pdref_*).  ``drive(api, w, s0, rate, nsteps)`` creates the
context, builds the family, applies boundary conditions and loads, sets the state, steps and reads
u, v, theta, damage and the family back."""
from types import SimpleNamespace

import numpy as np


def gpu_api():
    from paper_2309_11273_gb300 import _binding as B
    return SimpleNamespace(
        create=lambda w, s0: B.pd_create_particles(B.make_params(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt),
                                                   w.x, w.y, w.z, w.vol),
        build=lambda h, cracks: B.pd_build_neighbors(h, cracks),
        set_bc=B.pd_set_bc, set_state=B.pd_set_state, step=B.pd_step, get_state=B.pd_get_state,
        get_damage=B.pd_get_damage, get_neighbors=B.pd_get_neighbors, destroy=B.pd_destroy)


def oracle_api():
    import oracle as O
    return SimpleNamespace(
        create=lambda w, s0: O.pdref_create_particles(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt,
                                                      w.x, w.y, w.z, w.vol),
        build=lambda h, cracks: O.pdref_build_neighbors(h, cracks),
        set_bc=O.pdref_set_bc, set_state=O.pdref_set_state, step=O.pdref_step, get_state=O.pdref_get_state,
        get_damage=O.pdref_get_damage, get_neighbors=O.pdref_get_neighbors, destroy=O.pdref_destroy)


def drive(api, w, s0, rate, nsteps):
    h = api.create(w, s0)
    try:
        api.build(h, w.cracks)
        if w.flag is not None or w.b is not None:
            api.set_bc(h, w.dim, w.n, w.flag, w.b, w.axis_point, w.axis_dir, rate)
        api.set_state(h, w.dim, w.n, w.initial_u(), w.initial_v())
        api.step(h, nsteps)
        u, v, th = api.get_state(h, w.dim, w.n)
        phi = api.get_damage(h, w.n)
        rp, col, intact = api.get_neighbors(h, w.n)
    finally:
        api.destroy(h)
    return dict(u=u, v=v, theta=th, phi=phi, row_ptr=rp, col=col, intact=np.asarray(intact))
