"""C-ABI checks that need no GPU: the library builds, loads and exports every declared entry point;
host-only entry points and argument validation behave as documented."""
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2309_11273_gb300 import _binding as B
from paper_2309_11273_gb300 import build as BL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BL.build_library()
    return B.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "osbpd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pd_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_match_binding():
    assert declared_functions() == sorted(B.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", BL.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(pd_[a-z0-9_]+)\b", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


@pytest.mark.parametrize("model,E,nu,Gc,delta", [(0, 30e9, 0.2, 50.0, 3.015e-3), (0, 35e9, 0.2, 80.0, 7.5e-3),
                                                  (1, 72e9, 0.22, 3.8, 7.5375e-4), (1, 72e9, 1 / 3, 380.0, 7.5e-4),
                                                  (2, 190e9, 0.25, 6.9e4, 1.5e-3)])
def test_critical_stretch_matches_oracle(lib, model, E, nu, Gc, delta):
    a = B.pd_critical_stretch(model, E, nu, Gc, delta)
    b = O.critical_stretch(model, E, nu, Gc, delta)
    assert a == pytest.approx(b, rel=1e-15)


def test_critical_stretch_rejects_bad_arguments(lib):
    assert B.pd_critical_stretch(7, 1e9, 0.2, 1.0, 1e-3) < 0
    assert B.pd_critical_stretch(0, -1.0, 0.2, 1.0, 1e-3) < 0
    assert B.pd_critical_stretch(1, 1e9, 0.6, 1.0, 1e-3) < 0


def _prm(**kw):
    base = dict(model=B.PD_PLANE_STRESS, E=72e9, nu=0.22, rho=2440.0, horizon=3e-3, s0=0.0, dt=1e-7)
    base.update(kw)
    return B.make_params(**base)


@pytest.mark.parametrize("kw,msg", [(dict(E=-1.0), "E"), (dict(nu=0.5), "nu"), (dict(rho=0.0), "rho"),
                                    (dict(horizon=0.0), "horizon"), (dict(dt=float("nan")), "dt"),
                                    (dict(model=5), "model"), (dict(precision=3), "precision"),
                                    (dict(kinematics=2), "kinematics")])
def test_create_rejects_bad_parameters(lib, kw, msg):
    with pytest.raises(B.PDError) as e:
        B.pd_create_particles(_prm(**kw), np.zeros(4), np.arange(4.0), None, np.ones(4))
    assert e.value.status == B.PD_ERR_ARG and msg in str(e.value)


def test_create_rejects_bad_arrays(lib):
    with pytest.raises(B.PDError) as e:
        B.pd_create_particles(_prm(), np.array([0.0, np.inf]), np.zeros(2), None, np.ones(2))
    assert e.value.status == B.PD_ERR_ARG
    with pytest.raises(B.PDError) as e:
        B.pd_create_particles(_prm(), np.zeros(2), np.zeros(2), None, np.array([1.0, -1.0]))
    assert e.value.status == B.PD_ERR_ARG
    with pytest.raises(B.PDError) as e:
        B.pd_create_particles(_prm(model=B.PD_3D), np.zeros(2), np.zeros(2), None, np.ones(2))
    assert e.value.status == B.PD_ERR_ARG


def test_null_context_is_an_argument_error(lib):
    assert lib.pd_step(None, 1) == B.PD_ERR_ARG
    assert lib.pd_sync(None) == B.PD_ERR_ARG
    lib.pd_destroy(None)  # no-op


def test_batch_bodies_must_share_kinematics(lib):
    prms = [_prm(), _prm(kinematics=B.PD_NONLINEAR)]
    with pytest.raises(B.PDError) as e:
        B.pd_create_batch(prms, [0, 2, 4], np.arange(4.0), np.zeros(4), None, np.ones(4))
    assert e.value.status == B.PD_ERR_ARG and "kinematics" in str(e.value)


@pytest.mark.parametrize("model,E,nu", [(0, 30e9, 0.2), (1, 72e9, 0.22), (2, 72e9, 0.33)])
def test_material_constants_match_oracle(lib, model, E, nu):
    A, K, G = B.pd_material_constants(model, E, nu)
    ref = O.constants(model, E, nu)
    assert (A, K, G) == pytest.approx((ref["A"], ref["K"], ref["G"]), rel=1e-15)
    with pytest.raises(B.PDError):
        B.pd_material_constants(5, E, nu)
