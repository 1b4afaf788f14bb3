"""Host test of the integer-pipe break test of the FP64 kernels (csrc/pd_order.h).

The FP64 step kernels decide Eq 1.30 in the sqrt-free form xi.du >= s0 |xi|^2 by comparing the
bit patterns of the two doubles.  The header is compiled here with the host compiler and its
decision is compared with IEEE `d >= t` (what the oracle evaluates) for special values -- zeros of
both signs, denormals, infinities, NaNs of both signs and with payloads -- and for random values of
every magnitude, against thresholds across the positive range.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2309_11273_gb300", "csrc")

SRC = r"""
#include "pd_order.h"
extern "C" void decide(const double* d, const double* t, long n, unsigned char* out) {
  for (long k = 0; k < n; ++k) out[k] = pd_ge_threshold(d[k], t[k]) ? 1 : 0;
}
"""


@pytest.fixture(scope="module")
def decide():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    tmp = tempfile.mkdtemp(prefix="pd_order_")
    src = os.path.join(tmp, "order.cc")
    lib = os.path.join(tmp, "order.so")
    with open(src, "w") as f:
        f.write(SRC)
    subprocess.run([cxx, "-O2", "-shared", "-fPIC", "-I" + HDR, src, "-o", lib], check=True)
    so = ctypes.CDLL(lib)
    so.decide.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_long, ctypes.c_void_p]

    def run(d, t):
        d = np.ascontiguousarray(d, dtype=np.float64)
        t = np.ascontiguousarray(np.broadcast_to(t, d.shape), dtype=np.float64)
        out = np.zeros(d.shape, dtype=np.uint8)
        so.decide(d.ctypes.data, t.ctypes.data, d.size, out.ctypes.data)
        return out.astype(bool)

    yield run
    shutil.rmtree(tmp, ignore_errors=True)


def _nan(sign, payload):
    bits = np.array([(0xFFF0000000000000 if sign else 0x7FF0000000000000) | payload], dtype=np.uint64)
    return bits.view(np.float64)[0]


def test_special_values_follow_ieee(decide):
    t = np.array([5e-324, 2.2250738585072014e-308, 1e-300, 6.7e-4, 1.0, 3.5e7, 1.7976931348623157e308])
    d = np.array([0.0, -0.0, 5e-324, -5e-324, 1e-310, 1e-300, 6.7e-4, np.nextafter(6.7e-4, 0), 1.0,
                  -1.0, 1.7976931348623157e308, np.inf, -np.inf, _nan(0, 1 << 51), _nan(1, 1 << 51),
                  _nan(0, 1), _nan(1, 1), _nan(0, (1 << 52) - 1), _nan(1, (1 << 52) - 1)])
    D, T = np.meshgrid(d, t, indexing="ij")
    with np.errstate(invalid="ignore"):
        want = D >= T
    got = decide(D.ravel(), T.ravel()).reshape(D.shape)
    assert np.array_equal(got, want)
    # a NaN extension never breaks a bond, whatever its sign or payload
    assert not got[13:].any()


def test_random_values_follow_ieee(decide):
    rng = np.random.default_rng(7)
    n = 200000
    t = 10.0 ** rng.uniform(-300, 300, n)
    # values near the threshold (within a few ulps), far on both sides, and of both signs
    near = t * (1.0 + rng.integers(-4, 5, n) * np.finfo(np.float64).eps)
    far = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-308, 308, n)
    for d in (near, far, -near, np.nextafter(t, np.inf), np.nextafter(t, 0.0), t):
        assert np.array_equal(decide(d, t), d >= t)
