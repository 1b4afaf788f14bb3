"""Host tests of the comparison helpers in tests/parity.py (no GPU)."""
import numpy as np

from parity import rigid_split
from paper_2309_11273_gb300 import workloads as W


def _grid(dim):
    if dim == 2:
        x, y = W.grid_2d(12, 12, 1e-3)
        return np.stack([x, y])
    x, y, z = W.grid_3d(6, 6, 6, 1e-3)
    return np.stack([x, y, z])


def _rigid(P, t, w):
    X = P - P.mean(axis=1, keepdims=True)
    if P.shape[0] == 2:
        return np.stack([t[0] - w[0] * X[1], t[1] + w[0] * X[0]])
    wx, wy, wz = w
    return np.stack([t[0] + wy * X[2] - wz * X[1], t[1] + wz * X[0] - wx * X[2], t[2] + wx * X[1] - wy * X[0]])


def test_rigid_motion_is_all_rigid():
    rng = np.random.default_rng(1)
    for dim in (2, 3):
        P = _grid(dim)
        e = _rigid(P, rng.normal(size=dim), rng.normal(size=1 if dim == 2 else 3))
        r, d = rigid_split(e, P)
        assert abs(r - np.linalg.norm(e)) <= 1e-12 * np.linalg.norm(e) and d <= 1e-12 * np.linalg.norm(e)


def test_uniform_strain_on_a_symmetric_grid_is_all_deformation():
    """u = eps X with eps symmetric is orthogonal to every rigid field on a grid symmetric about its
    centroid (zero mean, isotropic second moment), so nothing of it is fitted as rigid."""
    rng = np.random.default_rng(2)
    for dim in (2, 3):
        P = _grid(dim)
        X = P - P.mean(axis=1, keepdims=True)
        a = rng.normal(size=(dim, dim))
        e = (a + a.T) @ X
        r, d = rigid_split(e, P)
        assert r <= 1e-12 * np.linalg.norm(e) and abs(d - np.linalg.norm(e)) <= 1e-12 * np.linalg.norm(e)


def test_sum_splits_into_its_parts():
    rng = np.random.default_rng(3)
    for dim in (2, 3):
        P = _grid(dim)
        X = P - P.mean(axis=1, keepdims=True)
        a = rng.normal(size=(dim, dim))
        s = (a + a.T) @ X
        g = _rigid(P, rng.normal(size=dim), rng.normal(size=1 if dim == 2 else 3))
        r, d = rigid_split(s + g, P)
        assert abs(r - np.linalg.norm(g)) <= 1e-10 * np.linalg.norm(g)
        assert abs(d - np.linalg.norm(s)) <= 1e-10 * np.linalg.norm(s)
