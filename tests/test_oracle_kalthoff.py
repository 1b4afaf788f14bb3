"""Prescribed-velocity boundary condition and the Kalthoff-Winkler-like impact workload (Section 4.3
in shape) in the oracle: impacted particles move exactly with the given velocity, and the
configuration's mirror symmetry about the centre line holds in the dynamics (CPU)."""
import numpy as np

import oracle as O
from paper_2309_11273_gb300 import workloads as W


def _small(v=22.0, nsteps=400):
    return W.kalthoff(nx=120, ny=60, dx=5e-4 * 402 / 120, notch_cells=30.125, gap_cells=30, v_imp=v,
                      nsteps=nsteps)


def _run(w, nsteps):
    s0 = O.critical_stretch(w.model, w.E, w.nu, w.Gc, w.delta)
    ref = O.OracleSim(w.model, w.E, w.nu, w.rho, w.delta, s0, w.dt, w.x, w.y, None, w.vol, w.cracks)
    ref.set_bc(w.flag, None, w.axis_point, w.axis_dir, 0.0, vp=w.vp)
    margins, broken = ref.step(nsteps)
    return ref, margins, broken


def test_impacted_particles_move_with_the_prescribed_velocity():
    w = _small()
    ref, _, _ = _run(w, 250)
    hit = w.flag == W.PRESCRIBED
    assert hit.sum() == 3 * 30  # three columns of the 30 rows between the notches
    t = 250 * w.dt
    assert np.array_equal(ref.u[:, hit], t * w.vp[:, hit]) and np.array_equal(ref.v[:, hit], w.vp[:, hit])
    free = ~hit
    assert ref.u[0, free].max() > 0.0  # the compressive wave has entered the plate


def test_mirror_symmetry_about_the_centre_line():
    """Notches at y = yc -+ 15 dx and the impact between them are mirror images about y = yc, so
    u_x(x, yc + s) = u_x(x, yc - s) and u_y(x, yc + s) = -u_y(x, yc - s) to rounding (the mirrored
    particles sum their bonds in mirrored order)."""
    w = _small()
    ref, _, _ = _run(w, 400)
    nx, ny = 120, 60
    ux = ref.u[0].reshape(ny, nx)
    uy = ref.u[1].reshape(ny, nx)
    scale = np.abs(ref.u).max()
    assert np.abs(ux - ux[::-1]).max() <= 1e-12 * scale
    assert np.abs(uy + uy[::-1]).max() <= 1e-12 * scale
    assert np.abs(uy).max() > 1e-3 * scale
