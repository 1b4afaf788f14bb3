"""ctypes binding of libosbpd (include/osbpd.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library.  Importing this module does not need a GPU; calling
``lib()`` loads ``_build/libosbpd.so`` and raises ``RuntimeError`` when the library is missing (no
fallback path exists).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libosbpd.so")

PD_OK, PD_ERR_ARG, PD_ERR_STATE, PD_ERR_OOM, PD_ERR_CUDA, PD_ERR_NUMERIC, PD_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6
PD_3D, PD_PLANE_STRESS, PD_PLANE_STRAIN = 0, 1, 2
PD_FP64, PD_MIXED = 0, 1
PD_ORDER_BRICKS, PD_ORDER_MORTON = 0, 1
PD_LINEARIZED, PD_NONLINEAR = 0, 1
PD_OPT_GRAPH_CHUNK, PD_OPT_PROFILE, PD_OPT_VALIDATE, PD_OPT_BLOCK, PD_OPT_SPLIT, PD_OPT_BOND_CACHE = 1, 2, 3, 4, 5, 6
PD_OPT_STAGE = 7
PD_OPT_EXPIRE_WAITS = 8
PD_OPT_SOLVER = 9
PD_OPT_PAIRS = 10
PD_OPT_LATTICE = 11
PD_OPT_LAT_STAGE = 12
PD_OPT_SHADOW_LO = 13
PD_W_ONE, PD_W_INV = 0, 1
PD_SOLVER_EXPLICIT, PD_SOLVER_ADR = 0, 1
PD_K_PASS1, PD_K_PASS2, PD_K_PASS1B = 0, 1, 2

STATUS_NAMES = {0: "PD_OK", -1: "PD_ERR_ARG", -2: "PD_ERR_STATE", -3: "PD_ERR_OOM", -4: "PD_ERR_CUDA",
                -5: "PD_ERR_NUMERIC", -6: "PD_ERR_TIMEOUT"}

# Every function the header declares (checked against the shared object by the CPU tests).
EXPORTED = ["pd_critical_stretch", "pd_material_constants", "pd_set_prescribed_velocity", "pd_create_particles", "pd_create_batch", "pd_build_neighbors",
            "pd_set_bc", "pd_set_state", "pd_step", "pd_sync", "pd_get_damage", "pd_get_state",
            "pd_num_bonds", "pd_get_neighbors", "pd_get_stats", "pd_check_state", "pd_autotune",
            "pd_set_option", "pd_get_option", "pd_get_profile", "pd_get_info", "pd_save_state",
            "pd_load_state", "pd_step_noalloc", "pd_probe_fp64", "pd_last_error", "pd_destroy"]


class pd_params(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("precision", ctypes.c_int32), ("E", ctypes.c_double),
                ("nu", ctypes.c_double), ("rho", ctypes.c_double), ("horizon", ctypes.c_double),
                ("s0", ctypes.c_double), ("dt", ctypes.c_double), ("band_safety", ctypes.c_double),
                ("device", ctypes.c_int32), ("ordering", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("kinematics", ctypes.c_int32), ("influence", ctypes.c_int32)]


class pd_crack(ctypes.Structure):
    _fields_ = [("p0", ctypes.c_double * 3), ("p1", ctypes.c_double * 3), ("p2", ctypes.c_double * 3),
                ("body", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pd_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("bonds", ctypes.c_int64), ("broken_bonds", ctypes.c_int64),
                ("band_rechecks", ctypes.c_int64), ("validate_mismatches", ctypes.c_int64),
                ("max_abs_u", ctypes.c_double), ("min_rel_margin", ctypes.c_double),
                ("strain_energy", ctypes.c_double), ("shadow_energy", ctypes.c_double)]


class PDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_d = ctypes.POINTER(ctypes.c_double)
_i64 = ctypes.POINTER(ctypes.c_int64)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)


def lib(path: str = LIB_PATH):
    """Load libosbpd.so (built by ``__graft_entry__.build()`` / ``build.build_library()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError("libosbpd.so not built (%s); run __graft_entry__.build()" % path)
            L = ctypes.CDLL(path)
            L.pd_critical_stretch.argtypes = [ctypes.c_int32] + [ctypes.c_double] * 4
            L.pd_critical_stretch.restype = ctypes.c_double
            L.pd_material_constants.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double] + [_d] * 3
            L.pd_set_prescribed_velocity.argtypes = [_vp, _d]
            L.pd_create_particles.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(pd_params), ctypes.c_int64,
                                              _d, _d, _d, _d]
            L.pd_create_batch.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32, ctypes.POINTER(pd_params), _i64,
                                          _d, _d, _d, _d]
            L.pd_build_neighbors.argtypes = [_vp, ctypes.POINTER(pd_crack), ctypes.c_int32]
            L.pd_set_bc.argtypes = [_vp, _u8, _d, _d, _d, ctypes.c_double]
            L.pd_set_state.argtypes = [_vp, _d, _d]
            L.pd_step.argtypes = [_vp, ctypes.c_int64]
            L.pd_sync.argtypes = [_vp]
            L.pd_get_damage.argtypes = [_vp, _d]
            L.pd_get_state.argtypes = [_vp, _d, _d, _d]
            L.pd_num_bonds.argtypes = [_vp, _i64]
            L.pd_get_neighbors.argtypes = [_vp, _i64, _i32, _u8]
            L.pd_get_stats.argtypes = [_vp, ctypes.POINTER(pd_stats)]
            L.pd_check_state.argtypes = [_vp, ctypes.c_double]
            L.pd_autotune.argtypes = [_vp, ctypes.c_int32, _i32, _i32]
            L.pd_set_option.argtypes = [_vp, ctypes.c_int32, ctypes.c_int64]
            L.pd_get_option.argtypes = [_vp, ctypes.c_int32, _i64]
            L.pd_get_profile.argtypes = [_vp, ctypes.c_int32, _d, _i64, ctypes.c_int32]
            L.pd_get_info.argtypes = [_vp, _i64, _i32, _i64]
            L.pd_save_state.argtypes = [_vp, ctypes.c_char_p]
            L.pd_load_state.argtypes = [_vp, ctypes.c_char_p]
            L.pd_step_noalloc.argtypes = ([ctypes.c_int32] + [ctypes.c_double] * 4 + [ctypes.c_int64]
                                          + [_vp] * 12 + [_vp])
            L.pd_probe_fp64.argtypes = [ctypes.c_int32, ctypes.c_int32, _d, _d]
            L.pd_last_error.restype = ctypes.c_char_p
            L.pd_destroy.argtypes = [_vp]
            L.pd_destroy.restype = None
            for name in EXPORTED:
                if name not in ("pd_critical_stretch", "pd_last_error", "pd_destroy"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st):
    if st != PD_OK:
        raise PDError(st, lib().pd_last_error().decode())


def _ptr(a, t):
    if a is None:
        return ctypes.cast(None, t)
    return a.ctypes.data_as(t)


def _soa(a, dim, n):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(dim, n))
    return a


# ------------------------------------------------------------------ entry points (same names as C)
def pd_material_constants(model, E, nu):
    """(A, K, G) of Eqs 1.8, 1.15, 1.16."""
    A, K, G = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pd_material_constants(int(model), float(E), float(nu), ctypes.byref(A), ctypes.byref(K),
                                       ctypes.byref(G)))
    return A.value, K.value, G.value


def pd_critical_stretch(model, E, nu, Gc, delta) -> float:
    return float(lib().pd_critical_stretch(int(model), float(E), float(nu), float(Gc), float(delta)))


def make_params(model, E, nu, rho, horizon, s0, dt, precision=PD_FP64, band_safety=0.0, device=0,
                stream=None, ordering=PD_ORDER_BRICKS, kinematics=PD_LINEARIZED, influence=0) -> pd_params:
    return pd_params(int(model), int(precision), float(E), float(nu), float(rho), float(horizon), float(s0),
                     float(dt), float(band_safety), int(device), int(ordering), stream, int(kinematics),
                     int(influence))


def pd_create_particles(prm: pd_params, x, y, z=None, vol=None):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
    vol = None if vol is None else np.ascontiguousarray(vol, dtype=np.float64)
    h = _vp()
    _check(lib().pd_create_particles(ctypes.byref(h), ctypes.byref(prm), x.size, _ptr(x, _d), _ptr(y, _d),
                                     _ptr(z, _d), _ptr(vol, _d)))
    return h


def pd_create_batch(prms, offsets, x, y, z=None, vol=None):
    arr = (pd_params * len(prms))(*prms)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = None if z is None else np.ascontiguousarray(z, dtype=np.float64)
    vol = None if vol is None else np.ascontiguousarray(vol, dtype=np.float64)
    h = _vp()
    _check(lib().pd_create_batch(ctypes.byref(h), len(prms), arr, _ptr(offsets, _i64), _ptr(x, _d), _ptr(y, _d),
                                 _ptr(z, _d), _ptr(vol, _d)))
    return h


def make_cracks(cracks, bodies=None):
    out = (pd_crack * max(len(cracks), 1))()
    for k, c in enumerate(cracks):
        p = np.zeros(9)
        v = np.asarray(c, dtype=np.float64).reshape(-1)
        p[:v.size] = v
        out[k].p0[:] = p[0:3]
        out[k].p1[:] = p[3:6]
        out[k].p2[:] = p[6:9]
        out[k].body = -1 if bodies is None else int(bodies[k])
    return out, len(cracks)


def pd_build_neighbors(h, cracks=(), bodies=None):
    arr, n = make_cracks(list(cracks), bodies)
    _check(lib().pd_build_neighbors(h, arr, n))


def pd_set_bc(h, dim, n, flag=None, b=None, axis_point=None, axis_dir=None, rate=0.0):
    flag = None if flag is None else np.ascontiguousarray(flag, dtype=np.uint8)
    b = _soa(b, dim, n)
    ap = None if axis_point is None else np.ascontiguousarray(axis_point, dtype=np.float64)
    ad = None if axis_dir is None else np.ascontiguousarray(axis_dir, dtype=np.float64)
    _check(lib().pd_set_bc(h, _ptr(flag, _u8), _ptr(b, _d), _ptr(ap, _d), _ptr(ad, _d), float(rate)))


def pd_set_prescribed_velocity(h, dim, n, vp):
    vp = _soa(vp, dim, n)
    _check(lib().pd_set_prescribed_velocity(h, _ptr(vp, _d)))


def pd_set_state(h, dim, n, u, v=None):
    u = _soa(u, dim, n)
    v = _soa(v, dim, n)
    _check(lib().pd_set_state(h, _ptr(u, _d), _ptr(v, _d)))


def pd_step(h, nsteps):
    _check(lib().pd_step(h, int(nsteps)))


def pd_sync(h):
    _check(lib().pd_sync(h))


def pd_get_damage(h, n, out=None):
    phi = np.empty(n) if out is None else out
    _check(lib().pd_get_damage(h, _ptr(phi, _d)))
    return phi


def pd_get_state(h, dim, n, u=True, v=True, theta=True):
    uo = np.empty((dim, n)) if u is True else (u if u is not False else None)
    vo = np.empty((dim, n)) if v is True else (v if v is not False else None)
    to = np.empty(n) if theta is True else (theta if theta is not False else None)
    _check(lib().pd_get_state(h, _ptr(uo, _d), _ptr(vo, _d), _ptr(to, _d)))
    return uo, vo, to


def pd_num_bonds(h) -> int:
    nb = ctypes.c_int64()
    _check(lib().pd_num_bonds(h, ctypes.byref(nb)))
    return int(nb.value)


def pd_get_neighbors(h, n):
    nb = pd_num_bonds(h)
    rp = np.empty(n + 1, dtype=np.int64)
    col = np.empty(max(nb, 1), dtype=np.int32)
    intact = np.empty(max(nb, 1), dtype=np.uint8)
    _check(lib().pd_get_neighbors(h, _ptr(rp, _i64), _ptr(col, _i32), _ptr(intact, _u8)))
    return rp, col[:nb], intact[:nb]


def pd_get_stats(h) -> dict:
    s = pd_stats()
    _check(lib().pd_get_stats(h, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in pd_stats._fields_}


def pd_check_state(h, max_abs_u):
    return lib().pd_check_state(h, float(max_abs_u))


def pd_autotune(h, trial_steps=5):
    b, s = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().pd_autotune(h, int(trial_steps), ctypes.byref(b), ctypes.byref(s)))
    return b.value, s.value


def pd_set_option(h, option, value):
    _check(lib().pd_set_option(h, int(option), int(value)))


def pd_get_option(h, option) -> int:
    v = ctypes.c_int64()
    _check(lib().pd_get_option(h, int(option), ctypes.byref(v)))
    return int(v.value)


def pd_get_profile(h, kernel, reset=False):
    ms, cnt = ctypes.c_double(), ctypes.c_int64()
    _check(lib().pd_get_profile(h, int(kernel), ctypes.byref(ms), ctypes.byref(cnt), int(bool(reset))))
    return ms.value, int(cnt.value)


def pd_save_state(h, path):
    _check(lib().pd_save_state(h, os.fsencode(path)))


def pd_load_state(h, path):
    _check(lib().pd_load_state(h, os.fsencode(path)))


def pd_probe_fp64(device=0, repeats=20):
    """Measured FP64 FMA throughput of a device: (flop/s, ms per launch)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().pd_probe_fp64(int(device), int(repeats), ctypes.byref(f), ctypes.byref(ms)))
    return f.value, ms.value


def pd_get_info(h):
    n, dim, by = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().pd_get_info(h, ctypes.byref(n), ctypes.byref(dim), ctypes.byref(by)))
    return int(n.value), int(dim.value), int(by.value)


def pd_step_noalloc(model, E, nu, rho, dt, n, x_dev, y_dev, z_dev, vol_dev, row_ptr_dev, col_dev,
                    intact_dev, u_dev, v_dev, u_out_dev, v_out_dev, theta_dev=None, stream=None):
    """Device pointers (ints, e.g. torch ``tensor.data_ptr()``) or None; returns the status code."""
    return lib().pd_step_noalloc(int(model), float(E), float(nu), float(rho), float(dt), int(n), x_dev, y_dev,
                                 z_dev, vol_dev, row_ptr_dev, col_dev, intact_dev, u_dev, v_dev, u_out_dev,
                                 v_out_dev, theta_dev, stream)


def pd_last_error() -> str:
    return lib().pd_last_error().decode()


def pd_destroy(h):
    if h:
        lib().pd_destroy(h)
