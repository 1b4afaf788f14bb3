"""Plain FP64 CPU oracle for linearized OSB-PD (Ni et al., arXiv 2309.11273).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA library
never calls it and it never calls the CUDA library; the two share only the seeded input generators
(``paper_2309_11273_gb300.workloads``), which contain none of the method's arithmetic.

The arithmetic lives in ``osb_oracle.c`` (plain C, compiled with ``-ffp-contract=off`` so that x86 and
Arm hosts round identically).  This module only builds it, marshals numpy arrays through ctypes and
sequences the calls.  Equation references are to the paper:

* Eq 1.8 / 1.15 / 1.16  -> :func:`constants`
* Eqs 1.24-1.29         -> :func:`critical_stretch`
* Section 2.1 horizon   -> :func:`family`
* Eq 1.9                -> :func:`weighted_volume`
* Eq 1.6 / 2.3          -> :func:`dilatation`
* Eq 2.2                -> :func:`force`
* Eqs 1.10, 1.13, 1.14  -> the same functions with ``kin=NONLINEAR`` (geometrically exact bonds)
* Eqs 1.17, 1.30        -> :func:`failure`
* Eq 1.31               -> :func:`damage`
* Eq 1.9's influence function w: 1 (the paper's choice, Section 2.3) or ``infl=W_INV``, w = delta / |xi|
  (a form of the published catalogue the paper cites at Eq 1.9), in every function above
* Eq 2.11 + Appendix B  -> :class:`OracleSim`
* adaptive dynamic relaxation (Section 4.4's quasi-static solver) -> :func:`adr_lambda`,
  :meth:`OracleSim.adr_step`
* ``pdref_*``: the oracle behind the GPU library's call sequence (create, build, boundary
  conditions, state, step, read back), so that one harness drives both

Parity unpinned: none (every function is pinned by the ``-m "not gpu"`` tests).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libosb_oracle.so")
_lock = threading.Lock()
_lib = None

MODEL_3D, MODEL_PLANE_STRESS, MODEL_PLANE_STRAIN = 0, 1, 2
FREE, FIXED, PRESCRIBED = 0, 1, 2
LINEARIZED, NONLINEAR = 0, 1  # bond kinematics: Eqs 2.4/2.7 (the paper's method) or Eqs 1.10/1.13
W_ONE, W_INV = 0, 1  # influence function w of Eqs 1.6, 1.9, 1.14, 1.31: 1 (the paper's) or delta / |xi|

_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def build_oracle(force: bool = False) -> str:
    """Compile ``osb_oracle.c`` into ``_build/libosb_oracle.so`` (plain gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build_oracle())
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            L.orc_constants.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double] + [_d] * 5
            L.orc_critical_stretch.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4
            L.orc_critical_stretch.restype = ctypes.c_double
            fam = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, ctypes.c_double, ctypes.c_int, _d, _i64,
                   _i64, _i32]
            L.orc_family_bruteforce.argtypes = fam
            L.orc_family_bruteforce.restype = ctypes.c_int64
            L.orc_family_binned.argtypes = fam
            L.orc_family_binned.restype = ctypes.c_int64
            L.orc_weighted_volume.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32,
                                              ctypes.c_int, ctypes.c_double, _d]
            L.orc_damage_denominator.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32,
                                                 ctypes.c_int, ctypes.c_double, _d]
            L.orc_dilatation.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32, _u8,
                                         _d, ctypes.c_double, ctypes.c_int, ctypes.c_double, _d, _d, _d, _d]
            L.orc_force.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32, _u8, _d,
                                    _d, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    _d, _d, _d, _d, _d, _d]
            L.orc_failure.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, _d, _d, _d, _i64, _i32, _u8,
                                      ctypes.c_double, _d, _d, _d, _d]
            L.orc_failure.restype = ctypes.c_int64
            L.orc_damage.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32, _u8, ctypes.c_int,
                                     ctypes.c_double, _d]
            L.orc_run.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_int, _d, _d,
                                   _d, _d, _i64, _i32, _u8, _d]
                                  + [ctypes.c_double] * 6
                                  + [_u8, _d, _d, _d, _d, _d, ctypes.c_double, _d, _d, _d, ctypes.c_int64,
                                     ctypes.c_int64]
                                  + [_d] * 10 + [_d, _i64])
            L.orc_adr_lambda.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32, _d, _d,
                                         _d, _d, _d]
            L.orc_adr_run.argtypes = ([ctypes.c_int, ctypes.c_int64, ctypes.c_int, _d, _d, _d, _d, _i64, _i32,
                                       _u8, _d, _d, _d, _d, _d, ctypes.c_double, _u8, _d, _d, _d, _d, _d,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                       ctypes.c_int]
                                      + [_d] * 13 + [_d, _d, _i64])
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _p(a, ptype):
    if a is None:
        return ctypes.cast(None, ptype)
    return a.ctypes.data_as(ptype)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def constants(model: int, E: float, nu: float) -> dict:
    """A (Eq 1.8), K (Eq 1.15), G (Eq 1.16) and the classical kappa, mu they are built from."""
    out = [ctypes.c_double() for _ in range(5)]
    lib().orc_constants(int(model), float(E), float(nu), *[ctypes.byref(o) for o in out])
    return dict(zip(("A", "K", "G", "kappa", "mu"), (o.value for o in out)))


def critical_stretch(model: int, E: float, nu: float, Gc: float, delta: float) -> float:
    """s_c from G_c: Eq 1.26 with beta, beta' (3D, beta' read as 5 delta/24) or Eqs 1.28-1.29 (2D)."""
    return float(lib().orc_critical_stretch(int(model), float(E), float(nu), float(Gc), float(delta)))


def _crack_array(cracks):
    if cracks is None or len(cracks) == 0:
        return 0, None
    arr = np.zeros((len(cracks), 9), dtype=np.float64)
    for k, c in enumerate(cracks):
        pts = np.asarray(c, dtype=np.float64).reshape(-1)
        arr[k, :pts.size] = pts
    return len(cracks), np.ascontiguousarray(arr.reshape(-1))


def family(x, y, z, delta, cracks=(), method="binned"):
    """Family of every particle (Section 2.1 closed horizon, minus cracked bonds) as CSR.

    Returns ``(row_ptr int64[n+1], col int32[nb])`` with neighbours ascending within each row.
    """
    x, y, z = _f64(x), _f64(y), _f64(z)
    n = x.size
    dim = 3 if z is not None else 2
    nc, carr = _crack_array(cracks)
    fn = lib().orc_family_binned if method == "binned" else lib().orc_family_bruteforce
    counts = np.zeros(n, dtype=np.int64)
    zz = z if z is not None else x
    fn(n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), float(delta), nc, _p(carr, _d), _p(counts, _i64),
       _p(None, _i64), _p(None, _i32))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = np.zeros(int(row_ptr[-1]), dtype=np.int32)
    fn(n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), float(delta), nc, _p(carr, _d), _p(counts, _i64),
       _p(row_ptr, _i64), _p(col, _i32))
    return row_ptr, col


def weighted_volume(x, y, z, vol, row_ptr, col, infl=W_ONE, delta=0.0):
    """m_i = sum_j w x_ij^2 V_j (Eq 1.9; w = 1, or delta / |xi| with infl=W_INV)."""
    x, y, z, vol = _f64(x), _f64(y), _f64(z), _f64(vol)
    n = x.size
    dim = 3 if z is not None else 2
    m = np.zeros(n)
    lib().orc_weighted_volume(n, dim, _p(x, _d), _p(y, _d), _p(z if z is not None else x, _d),
                              _p(vol, _d), _p(row_ptr, _i64), _p(col, _i32), int(infl), float(delta), _p(m, _d))
    return m


def damage_denominator(vol, row_ptr, col, x=None, y=None, z=None, infl=W_ONE, delta=0.0):
    """D_i = sum_j w V_j over the built family (denominator of Eq 1.31)."""
    vol = _f64(vol)
    n = vol.size
    if x is None:  # w = 1 needs no geometry
        x = y = np.zeros(n)
    x, y, z = _f64(x), _f64(y), _f64(z)
    dim = 3 if z is not None else 2
    D = np.zeros(n)
    lib().orc_damage_denominator(n, dim, _p(x, _d), _p(y, _d), _p(z if z is not None else x, _d), _p(vol, _d),
                                 _p(row_ptr, _i64), _p(col, _i32), int(infl), float(delta), _p(D, _d))
    return D


def dilatation(x, y, z, vol, row_ptr, col, status, m, A, u, kin=LINEARIZED, infl=W_ONE, delta=0.0):
    """theta_i (Eq 1.6 / 2.3) for displacement ``u`` of shape (dim, n)."""
    x, y, z, vol, m = _f64(x), _f64(y), _f64(z), _f64(vol), _f64(m)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n, dim = x.size, u.shape[0]
    th = np.zeros(n)
    zz = z if z is not None else x
    uz = u[2] if dim == 3 else u[0]
    lib().orc_dilatation(int(kin), n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), _p(vol, _d), _p(row_ptr, _i64),
                         _p(col, _i32), _p(status, _u8), _p(m, _d), float(A), int(infl), float(delta),
                         _p(np.ascontiguousarray(u[0]), _d), _p(np.ascontiguousarray(u[1]), _d),
                         _p(np.ascontiguousarray(uz), _d), _p(th, _d))
    return th


def force(x, y, z, vol, row_ptr, col, status, m, theta, K, G, u, kin=LINEARIZED, infl=W_ONE, delta=0.0):
    """Internal force F_i = sum_j F_i^{xi_ij} (Eq 2.2; Eqs 1.11-1.14 with kin=NONLINEAR), shape (dim, n)."""
    x, y, z, vol, m, theta = _f64(x), _f64(y), _f64(z), _f64(vol), _f64(m), _f64(theta)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n, dim = x.size, u.shape[0]
    f = np.zeros((3, n))
    zz = z if z is not None else x
    uz = u[2] if dim == 3 else u[0]
    lib().orc_force(int(kin), n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), _p(vol, _d), _p(row_ptr, _i64),
                    _p(col, _i32), _p(status, _u8), _p(m, _d), _p(theta, _d), float(K), float(G),
                    int(infl), float(delta), _p(np.ascontiguousarray(u[0]), _d), _p(np.ascontiguousarray(u[1]), _d),
                    _p(np.ascontiguousarray(uz), _d), _p(f[0], _d), _p(f[1], _d), _p(f[2], _d))
    return f[:dim].copy()


def failure(x, y, z, row_ptr, col, status, s0, u, kin=LINEARIZED):
    """Apply Eq 1.30 in place on ``status``; returns (newly broken, min relative margin)."""
    x, y, z = _f64(x), _f64(y), _f64(z)
    u = np.ascontiguousarray(u, dtype=np.float64)
    n, dim = x.size, u.shape[0]
    mm = ctypes.c_double()
    zz = z if z is not None else x
    uz = u[2] if dim == 3 else u[0]
    nb = lib().orc_failure(int(kin), n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), _p(row_ptr, _i64), _p(col, _i32),
                           _p(status, _u8), float(s0), _p(np.ascontiguousarray(u[0]), _d),
                           _p(np.ascontiguousarray(u[1]), _d), _p(np.ascontiguousarray(uz), _d),
                           ctypes.byref(mm))
    return int(nb), mm.value


def adr_lambda(x, y, z, vol, row_ptr, col, m, A, K, G):
    """Fictitious ADR density lambda_i = R_i / 4 (R_i: Gerschgorin bound of the force-density
    stiffness row sums); A, K, G per particle."""
    x, y, z, vol, m = _f64(x), _f64(y), _f64(z), _f64(vol), _f64(m)
    n = x.size
    A, K, G = (np.broadcast_to(np.asarray(t, dtype=np.float64), (n,)).copy() for t in (A, K, G))
    lam = np.zeros(n)
    dim = 3 if z is not None else 2
    zz = z if z is not None else x
    lib().orc_adr_lambda(n, dim, _p(x, _d), _p(y, _d), _p(zz, _d), _p(vol, _d), _p(row_ptr, _i64),
                         _p(col, _i32), _p(m, _d), _p(A, _d), _p(K, _d), _p(G, _d), _p(lam, _d))
    return lam


def damage(vol, row_ptr, col, status, x=None, y=None, z=None, infl=W_ONE, delta=0.0):
    """phi_i (Eq 1.31)."""
    vol = _f64(vol)
    n = vol.size
    if x is None:  # w = 1 needs no geometry
        x = y = np.zeros(n)
    x, y, z = _f64(x), _f64(y), _f64(z)
    dim = 3 if z is not None else 2
    phi = np.zeros(n)
    lib().orc_damage(n, dim, _p(x, _d), _p(y, _d), _p(z if z is not None else x, _d), _p(vol, _d),
                     _p(row_ptr, _i64), _p(col, _i32), _p(status, _u8), int(infl), float(delta), _p(phi, _d))
    return phi


class OracleSim:
    """Explicit OSB-PD dynamics exactly as the paper's solver loop (Eq 2.11, Appendix B).

    Holds the family (CSR, user order), m_i, the bond status (one byte per directed bond) and the
    state u, v (shape (dim, n)).  ``step(k)`` runs k iterations of the C loop ``orc_run``.
    """

    def __init__(self, model, E, nu, rho, delta, s0, dt, x, y, z=None, vol=None, cracks=(),
                 family_method="binned", kin=LINEARIZED, infl=W_ONE):
        self.model = int(model)
        self.kin = int(kin)
        self.infl = int(infl)
        self.dim = 3 if z is not None else 2
        self.x, self.y = _f64(x), _f64(y)
        self.z = _f64(z) if z is not None else None
        self.n = self.x.size
        self.vol = _f64(vol) if vol is not None else None
        if self.vol is None:
            raise ValueError("vol is required")
        self.rho, self.delta, self.s0, self.dt = float(rho), float(delta), float(s0), float(dt)
        c = constants(model, E, nu)
        self.A, self.K, self.G = c["A"], c["K"], c["G"]
        self.row_ptr, self.col = family(self.x, self.y, self.z, delta, cracks, family_method)
        self.m = weighted_volume(self.x, self.y, self.z, self.vol, self.row_ptr, self.col, self.infl, self.delta)
        self.D = damage_denominator(self.vol, self.row_ptr, self.col, self.x, self.y, self.z, self.infl, self.delta)
        self.status = np.ones(self.col.size, dtype=np.uint8)
        self.u = np.zeros((self.dim, self.n))
        self.v = np.zeros((self.dim, self.n))
        self.theta = np.zeros(self.n)
        self.f = np.zeros((self.dim, self.n))
        self.flag = None
        self.b = None
        self.axis_point = np.zeros(3)
        self.axis_dir = np.zeros(3)
        self.rate = 0.0
        self.steps_done = 0

    @property
    def nbonds(self) -> int:
        return int(self.col.size)

    def set_bc(self, flag=None, b=None, axis_point=None, axis_dir=None, rate=0.0, vp=None):
        """vp (dim, n), optional: a prescribed velocity for the prescribed particles (u = t vp,
        v = vp) in place of the rotation."""
        self.vp = None if vp is None else np.ascontiguousarray(np.asarray(vp, dtype=np.float64).reshape(self.dim, -1))
        self.flag = None if flag is None else np.ascontiguousarray(flag, dtype=np.uint8)
        self.b = None if b is None else np.ascontiguousarray(b, dtype=np.float64).reshape(self.dim, -1)
        self.axis_point = np.zeros(3) if axis_point is None else np.asarray(axis_point, dtype=np.float64)
        self.axis_dir = np.zeros(3) if axis_dir is None else np.asarray(axis_dir, dtype=np.float64)
        self.rate = float(rate)

    def set_state(self, u, v=None):
        self._adr_fresh = True
        self.u = np.array(u, dtype=np.float64).reshape(self.dim, self.n).copy()
        self.v = (np.zeros_like(self.u) if v is None
                  else np.array(v, dtype=np.float64).reshape(self.dim, self.n).copy())

    def step(self, nsteps: int):
        """Run ``nsteps`` iterations; returns (min margin per step, broken count per step)."""
        nsteps = int(nsteps)
        margins = np.zeros(max(nsteps, 1))
        broken = np.zeros(max(nsteps, 1), dtype=np.int64)
        ux = np.ascontiguousarray(self.u[0]); uy = np.ascontiguousarray(self.u[1])
        vx = np.ascontiguousarray(self.v[0]); vy = np.ascontiguousarray(self.v[1])
        uz = np.ascontiguousarray(self.u[2]) if self.dim == 3 else np.zeros(self.n)
        vz = np.ascontiguousarray(self.v[2]) if self.dim == 3 else np.zeros(self.n)
        fx, fy, fz = np.zeros(self.n), np.zeros(self.n), np.zeros(self.n)
        zz = self.z if self.z is not None else self.x
        b = self.b
        bx = b[0].copy() if b is not None else None
        by = b[1].copy() if b is not None else None
        bz = b[2].copy() if (b is not None and self.dim == 3) else None
        vp = getattr(self, "vp", None)
        vpx = vp[0].copy() if vp is not None else None
        vpy = vp[1].copy() if vp is not None else None
        vpz = vp[2].copy() if (vp is not None and self.dim == 3) else (np.zeros(self.n) if vp is not None else None)
        lib().orc_run(self.kin, self.infl, self.delta, self.n, self.dim, _p(self.x, _d), _p(self.y, _d), _p(zz, _d),
                      _p(self.vol, _d),
                      _p(self.row_ptr, _i64), _p(self.col, _i32), _p(self.status, _u8), _p(self.m, _d),
                      self.A, self.K, self.G, self.rho, self.dt, self.s0, _p(self.flag, _u8),
                      _p(bx, _d), _p(by, _d), _p(bz, _d), _p(self.axis_point, _d),
                      _p(self.axis_dir, _d), self.rate, _p(vpx, _d), _p(vpy, _d), _p(vpz, _d),
                      self.steps_done, nsteps, _p(ux, _d),
                      _p(uy, _d), _p(uz, _d), _p(vx, _d), _p(vy, _d), _p(vz, _d), _p(self.theta, _d),
                      _p(fx, _d), _p(fy, _d), _p(fz, _d), _p(margins, _d), _p(broken, _i64))
        self.u = np.stack([ux, uy, uz][:self.dim])
        self.v = np.stack([vx, vy, vz][:self.dim])
        self.f = np.stack([fx, fy, fz][:self.dim])
        self.steps_done += nsteps
        return margins[:nsteps], broken[:nsteps]

    def internal_force(self, u=None):
        """theta and F for displacement u (default: current state) with the current bond status."""
        u = self.u if u is None else np.asarray(u, dtype=np.float64).reshape(self.dim, self.n)
        th = dilatation(self.x, self.y, self.z, self.vol, self.row_ptr, self.col, self.status, self.m,
                        self.A, u, self.kin, self.infl, self.delta)
        f = force(self.x, self.y, self.z, self.vol, self.row_ptr, self.col, self.status, self.m, th,
                  self.K, self.G, u, self.kin, self.infl, self.delta)
        return th, f

    def damage(self):
        return damage(self.vol, self.row_ptr, self.col, self.status, self.x, self.y, self.z, self.infl, self.delta)

    def adr_step(self, nsteps: int):
        """Adaptive dynamic relaxation iterations (``orc_adr_run``) from the current state.  The first
        call after ``set_state`` starts from rest (v = 0); returns (damping c per iteration, min
        margin per iteration, broken count per iteration).  ``self.v`` holds v^{n-1/2}."""
        if self.infl != W_ONE:
            raise ValueError("adaptive dynamic relaxation is restated for w = 1 only")
        nsteps = int(nsteps)
        if getattr(self, "lam", None) is None:
            self.lam = adr_lambda(self.x, self.y, self.z, self.vol, self.row_ptr, self.col, self.m,
                                  self.A, self.K, self.G)
        first = 1 if getattr(self, "_adr_fresh", True) else 0
        if first:
            self.v = np.zeros_like(self.u)
            self.g = np.zeros((3, self.n))
        damping = np.zeros(max(nsteps, 1))
        margins = np.zeros(max(nsteps, 1))
        broken = np.zeros(max(nsteps, 1), dtype=np.int64)
        u = [np.ascontiguousarray(self.u[k]) if k < self.dim else np.zeros(self.n) for k in range(3)]
        v = [np.ascontiguousarray(self.v[k]) if k < self.dim else np.zeros(self.n) for k in range(3)]
        g = [np.ascontiguousarray(self.g[k]) for k in range(3)]
        f = [np.zeros(self.n) for _ in range(3)]
        zz = self.z if self.z is not None else self.x
        b = self.b
        bx = b[0].copy() if b is not None else None
        by = b[1].copy() if b is not None else None
        bz = b[2].copy() if (b is not None and self.dim == 3) else None
        A, K, G = (np.full(self.n, t) for t in (self.A, self.K, self.G))
        lib().orc_adr_run(self.kin, self.n, self.dim, _p(self.x, _d), _p(self.y, _d), _p(zz, _d),
                          _p(self.vol, _d), _p(self.row_ptr, _i64), _p(self.col, _i32), _p(self.status, _u8),
                          _p(self.m, _d), _p(A, _d), _p(K, _d), _p(G, _d), _p(self.lam, _d), self.s0,
                          _p(self.flag, _u8), _p(bx, _d), _p(by, _d), _p(bz, _d), _p(self.axis_point, _d),
                          _p(self.axis_dir, _d), self.rate, self.dt, self.steps_done, nsteps, first,
                          _p(u[0], _d), _p(u[1], _d), _p(u[2], _d), _p(v[0], _d), _p(v[1], _d), _p(v[2], _d),
                          _p(g[0], _d), _p(g[1], _d), _p(g[2], _d), _p(self.theta, _d), _p(f[0], _d),
                          _p(f[1], _d), _p(f[2], _d), _p(damping, _d), _p(margins, _d), _p(broken, _i64))
        self.u = np.stack(u[:self.dim])
        self.v = np.stack(v[:self.dim])
        self.g = np.stack(g)
        self.f = np.stack(f[:self.dim])
        self._adr_fresh = False
        self.steps_done += nsteps
        return damping[:nsteps], margins[:nsteps], broken[:nsteps]


# ------------------------------------------------------------------------------------ pdref_*
class _PdrefParams(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("E", ctypes.c_double),
                ("nu", ctypes.c_double), ("rho", ctypes.c_double), ("horizon", ctypes.c_double),
                ("s0", ctypes.c_double), ("dt", ctypes.c_double), ("band_safety", ctypes.c_double),
                ("device", ctypes.c_int32), ("ordering", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("kinematics", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class _PdrefCrack(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_double * 3), ("p1", ctypes.c_double * 3), ("p2", ctypes.c_double * 3),
                ("body", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def _pdref_lib():
    L = lib()
    if not getattr(L, "_pdref_ready", False):
        vp = ctypes.c_void_p
        L.pdref_create_particles.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_PdrefParams), ctypes.c_int64,
                                             _d, _d, _d, _d]
        L.pdref_build_neighbors.argtypes = [vp, ctypes.POINTER(_PdrefCrack), ctypes.c_int32]
        L.pdref_set_bc.argtypes = [vp, _u8, _d, _d, _d, ctypes.c_double]
        L.pdref_set_state.argtypes = [vp, _d, _d]
        L.pdref_step.argtypes = [vp, ctypes.c_int64]
        L.pdref_get_state.argtypes = [vp, _d, _d, _d]
        L.pdref_get_damage.argtypes = [vp, _d]
        L.pdref_num_bonds.argtypes = [vp, _i64]
        L.pdref_get_neighbors.argtypes = [vp, _i64, _i32, _u8]
        L.pdref_destroy.argtypes = [vp]
        L.pdref_destroy.restype = None
        L._pdref_ready = True
    return L


def _ok(st):
    if st != 0:
        raise RuntimeError("pdref call failed with status %d" % st)


def pdref_create_particles(model, E, nu, rho, horizon, s0, dt, x, y, z=None, vol=None, kinematics=LINEARIZED):
    """The oracle behind the GPU library's call sequence (``pdref_*`` in ``osb_oracle.c``)."""
    prm = _PdrefParams(int(model), 0, float(E), float(nu), float(rho), float(horizon), float(s0), float(dt), 0.0,
                       0, 0, None, int(kinematics), 0)
    x, y, z, vol = _f64(x), _f64(y), _f64(z), _f64(vol)
    h = ctypes.c_void_p()
    _ok(_pdref_lib().pdref_create_particles(ctypes.byref(h), ctypes.byref(prm), x.size, _p(x, _d), _p(y, _d),
                                            _p(z, _d), _p(vol, _d)))
    return h


def pdref_build_neighbors(h, cracks=()):
    arr = (_PdrefCrack * max(len(cracks), 1))()
    for k, c in enumerate(cracks):
        pts = np.zeros(9)
        q = np.asarray(c, dtype=np.float64).reshape(-1)
        pts[:q.size] = q
        arr[k].p0[:] = list(pts[0:3])
        arr[k].p1[:] = list(pts[3:6])
        arr[k].p2[:] = list(pts[6:9])
        arr[k].body = -1
    _ok(_pdref_lib().pdref_build_neighbors(h, arr, len(cracks)))


def pdref_set_bc(h, dim, n, flag=None, b=None, axis_point=None, axis_dir=None, rate=0.0):
    flag = None if flag is None else np.ascontiguousarray(flag, dtype=np.uint8)
    b = None if b is None else np.ascontiguousarray(np.asarray(b, dtype=np.float64).reshape(dim, n))
    ap = None if axis_point is None else np.ascontiguousarray(axis_point, dtype=np.float64)
    ad = None if axis_dir is None else np.ascontiguousarray(axis_dir, dtype=np.float64)
    _ok(_pdref_lib().pdref_set_bc(h, _p(flag, _u8), _p(b, _d), _p(ap, _d), _p(ad, _d), float(rate)))


def pdref_set_state(h, dim, n, u, v=None):
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(dim, n))
    v = None if v is None else np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(dim, n))
    _ok(_pdref_lib().pdref_set_state(h, _p(u, _d), _p(v, _d)))


def pdref_step(h, nsteps):
    _ok(_pdref_lib().pdref_step(h, int(nsteps)))


def pdref_get_state(h, dim, n):
    u, v, th = np.zeros((dim, n)), np.zeros((dim, n)), np.zeros(n)
    _ok(_pdref_lib().pdref_get_state(h, _p(u, _d), _p(v, _d), _p(th, _d)))
    return u, v, th


def pdref_get_damage(h, n):
    phi = np.zeros(n)
    _ok(_pdref_lib().pdref_get_damage(h, _p(phi, _d)))
    return phi


def pdref_get_neighbors(h, n):
    nb = ctypes.c_int64()
    _ok(_pdref_lib().pdref_num_bonds(h, ctypes.byref(nb)))
    rp = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(nb.value, 1), dtype=np.int32)
    intact = np.zeros(max(nb.value, 1), dtype=np.uint8)
    _ok(_pdref_lib().pdref_get_neighbors(h, _p(rp, _i64), _p(col, _i32), _p(intact, _u8)))
    return rp, col[:nb.value], intact[:nb.value]


def pdref_destroy(h):
    _pdref_lib().pdref_destroy(h)
