"""Element-wise comparison helpers shared by the GPU parity tests.

FP64 bar (Eqs 2.2, 2.3, 2.11): for displacement and velocity, both
  rel-L2:       ||a - ref||_2 <= tol ||ref||_2, and
  per particle: max_i ||u_i - u_ref,i||_inf <= tol max_i ||u_ref,i||_inf, and for the velocity the
                same displacement bar carried through Eq 2.11: v^{n+1} = (u^{n+1} - u^n) / dt, so two
                displacement levels each within tol max|u| give velocities within 2 tol max|u| / dt
                (the highest mode carries the rounding of u into v amplified by ~2 / dt: measured on
                configuration 2 after 1000 steps, per particle 3e-15 of max|u| in u and 1.25e-12 of
                max|v| = 1.6e-15 of max|u| / dt in v); the bar is the larger of that and tol max|v|.
For the dilatation theta_i (Eq 1.6), a sum over the family whose terms cancel, the per-particle bar
is the propagation of the displacement bar: theta_i is linear in u, with
|d theta_i| <= (A/m_i) sum_j V_j |xi_ij| (|du_j| + |du_i|) <= (A/m_i) delta D_i 2 max_k |du_k|
(D_i = sum_j V_j, |xi| <= delta), so particle i is held to tol (A delta D_i / m_i) 2 max_k ||u_k||.
The global bar of theta (L2 relative to the L2 size S of its terms) is kept beside it.
"""
from __future__ import annotations

import numpy as np


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def elem(a, ref):
    """max_i ||a_i - ref_i||_inf / max_i ||ref_i||_inf for (dim, n) arrays (0 when both are 0)."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64).reshape(a.shape)
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    err = float(np.abs(a - ref).max()) if ref.size else 0.0
    if scale == 0.0:
        return 0.0 if err == 0.0 else np.inf
    return err / scale


def elem_v(v, ref):
    """max_i ||v_i - v_ref,i||_inf / max(max_i ||v_ref,i||_inf, 2 max_i ||u_ref,i||_inf / dt)."""
    v = np.asarray(v, dtype=np.float64)
    vr = np.asarray(ref.v, dtype=np.float64).reshape(v.shape)
    scale = max(float(np.abs(vr).max()) if vr.size else 0.0,
                2.0 * float(np.abs(ref.u).max()) / ref.dt if ref.u.size else 0.0)
    err = float(np.abs(v - vr).max()) if vr.size else 0.0
    if scale == 0.0:
        return 0.0 if err == 0.0 else np.inf
    return err / scale


def theta_scale(ref):
    """Per-particle bar scale T_i = (A delta D_i / m_i) 2 max_k ||u_k||_inf of an OracleSim."""
    umax = float(np.abs(ref.u).max()) if ref.u.size else 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        T = np.where(ref.m > 0, ref.A * ref.delta * ref.D / ref.m, 0.0) * 2.0 * umax
    return T


def theta_elem(th, ref):
    """max_i |theta_i - theta_ref,i| / T_i (particles without bonds must agree exactly: both 0)."""
    T = theta_scale(ref)
    d = np.abs(np.asarray(th, dtype=np.float64) - ref.theta)
    pos = T > 0
    if np.any(d[~pos] != 0.0):
        return np.inf
    return float((d[pos] / T[pos]).max()) if pos.any() else 0.0


def theta_global(th, ref):
    """L2 error of theta relative to the L2 size of the terms it sums, S_i = (A/m_i) sum_j V_j |xi.du|.
    theta_i is a cancelling sum (Eq 1.6), so two correct evaluations agree to eps * S_i."""
    P = np.stack([ref.x, ref.y] + ([ref.z] if ref.dim == 3 else []))
    rows = np.repeat(np.arange(ref.n), np.diff(ref.row_ptr))
    xi = P[:, ref.col] - P[:, rows]
    du = ref.u[:, ref.col] - ref.u[:, rows]
    t = np.abs((xi * du).sum(0)) * ref.vol[ref.col]
    S = ref.A * np.bincount(rows, weights=t, minlength=ref.n) / np.where(ref.m > 0, ref.m, np.inf)
    return float(np.linalg.norm(th - ref.theta) / max(np.linalg.norm(S), 1e-300))


def compare(u, v, th, ref, with_global_theta=True):
    """All FP64 error measures of a GPU state (u, v, theta) against an OracleSim at the same step."""
    out = dict(ru=rel(u, ref.u), rv=rel(v, ref.v), eu=elem(u, ref.u), ev=elem_v(v, ref),
               et=theta_elem(th, ref))
    if with_global_theta:
        out["rt"] = theta_global(th, ref)
    return out


def assert_fp64_close(errs, tol=1e-12, what=""):
    """Every measure in ``errs`` (from ``compare``) within tol."""
    bad = {k: v for k, v in errs.items() if k in ("ru", "rv", "eu", "ev", "et", "rt") and not (v <= tol)}
    assert not bad, (what, bad)


def rigid_split(err, P):
    """Split an error field into its best-fit rigid motion and the rest.

    err, P: (dim, n) arrays (displacement error, reference positions).  Least squares over the
    translations and infinitesimal rotations about the centroid (3 fields in 2D, 6 in 3D).  Returns
    (rigid, deformation): the L2 norms of the fitted rigid field and of the residual.  An internal
    force field whose bond forces are exactly antisymmetric and parallel to the bond moves no rigid
    mode; FP32 accumulation of those forces does (each particle's sum is rounded on its own), so on a
    free body the mixed form's error splits into a rigid drift that grows with time and a deformation
    error that measures the force arithmetic."""
    err = np.asarray(err, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    dim, n = err.shape
    X = P - P.mean(axis=1, keepdims=True)
    cols = []
    for a in range(dim):  # translations
        c = np.zeros((dim, n))
        c[a] = 1.0
        cols.append(c)
    for a, b in ((0, 1),) if dim == 2 else ((0, 1), (1, 2), (2, 0)):  # rotations in the (a, b) plane
        c = np.zeros((dim, n))
        c[a] = -X[b]
        c[b] = X[a]
        cols.append(c)
    M = np.stack([c.reshape(-1) for c in cols], axis=1)
    coef, *_ = np.linalg.lstsq(M, err.reshape(-1), rcond=None)
    fit = M @ coef
    return float(np.linalg.norm(fit)), float(np.linalg.norm(err.reshape(-1) - fit))
