"""Pins of the oracle's patch transfer (Sec. 3.1): Eq. 3 through the poses and
Eq. 4 in the plane, against identities and closed forms of the geometry."""
import numpy as np
import pytest

import oracle as O

F, CX, CY, W, H = 15625.0, 4088.0, 3066.0, 8176.0, 6132.0
INTR = np.array([F, CX, CY, 0.0, 0.0, 0.0, 0.0])
NADIR = np.diag([1.0, -1.0, -1.0])  # camera x = east, y = south, z = down


def _rot(axis, ang):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


@pytest.fixture(scope="module", autouse=True)
def _build():
    O.build()


def test_eq3_identity_transfer():
    """Image k = image 0: every patch stays where it is, whatever the depth."""
    rng = np.random.default_rng(1)
    p0 = rng.uniform([0, 0], [W, H], (50, 2))
    R = _rot([0.3, -0.2, 1.0], 0.4) @ NADIR
    T = np.array([120.0, -40.0, 480.0])
    for lam in (50.0, 480.0, 2e4):
        pk, inside = O.patch_transfer_poses(INTR, R, T, p0, lam, INTR, R, T, W, H)
        assert np.abs(pk - p0).max() < 1e-8
        assert inside.all()


def test_eq3_nadir_translation_closed_form():
    """Nadir cameras at height Hh over flat ground, lambda = Hh: a move of the
    camera by (dx, dy) shifts every patch by f/Hh * (-dx, +dy) pixels."""
    rng = np.random.default_rng(2)
    p0 = rng.uniform([0, 0], [W, H], (40, 2))
    for hh, dx, dy in ((500.0, 10.0, 0.0), (800.0, -3.5, 12.0), (350.0, 0.0, -7.25)):
        T0 = np.array([1000.0, 2000.0, hh])
        Tk = T0 + np.array([dx, dy, 0.0])
        pk, _ = O.patch_transfer_poses(INTR, NADIR, T0, p0, hh, INTR, NADIR, Tk)
        expect = p0 + F / hh * np.array([-dx, dy])
        assert np.abs(pk - expect).max() < 1e-7


def test_eq3_pure_rotation_is_independent_of_depth():
    """Same camera centre: the transfer is the rotation homography K R_k^T R_0
    K^-1, which does not depend on lambda."""
    rng = np.random.default_rng(3)
    p0 = rng.uniform([1000, 1000], [W - 1000, H - 1000], (30, 2))
    R0 = NADIR
    Rk = _rot([0.1, 0.2, 0.9], 0.05) @ NADIR
    T = np.array([0.0, 0.0, 600.0])
    a, _ = O.patch_transfer_poses(INTR, R0, T, p0, 100.0, INTR, Rk, T)
    b, _ = O.patch_transfer_poses(INTR, R0, T, p0, 1e5, INTR, Rk, T)
    assert np.abs(a - b).max() < 1e-7
    # and it equals the homography applied to homogeneous pixels
    K = np.array([[F, 0, CX], [0, F, CY], [0, 0, 1.0]])
    Hm = K @ Rk.T @ R0 @ np.linalg.inv(K)
    h = np.c_[p0, np.ones(len(p0))] @ Hm.T
    assert np.abs(a - h[:, :2] / h[:, 2:]).max() < 1e-6


def test_eq3_point_behind_target_is_not_inside():
    """A target camera looking up from below the ground point does not see it."""
    T0 = np.array([0.0, 0.0, 500.0])
    Tk = np.array([0.0, 0.0, -10.0])
    _, inside = O.patch_transfer_poses(INTR, NADIR, T0, [[CX, CY]], 500.0, INTR, NADIR, Tk)
    assert not inside[0]


def test_eq4_translation_rotation_and_composition():
    rng = np.random.default_rng(4)
    q0 = rng.uniform(-300, 300, (60, 2))
    c = np.array([12.0, -7.0])
    g0, g1, g2 = np.array([5.0, 1.0]), np.array([40.0, -3.0]), np.array([71.0, 9.5])
    # theta = 0: a pure translation by g_k - g_0
    assert np.abs(O.patch_transfer_planar(q0, c, 0.0, g0, g1) - (q0 + g1 - g0)).max() < 1e-12
    # a quarter turn: (dx, dy) -> (-dy, dx) about c
    q = O.patch_transfer_planar(q0, c, np.pi / 2, g0, g0)
    d = q0 - c
    assert np.abs(q - (c + np.c_[-d[:, 1], d[:, 0]])).max() < 1e-9
    # distances to the grid centre are kept
    q = O.patch_transfer_planar(q0, c, 0.7, g0, g1)
    assert np.abs(np.linalg.norm(q - (g1 - g0) - c, axis=1) - np.linalg.norm(q0 - c, axis=1)).max() < 1e-9
    # two transfers compose: theta1 then theta2 (about the moved centre) = theta1 + theta2
    t1, t2 = 0.3, -1.1
    a = O.patch_transfer_planar(q0, c, t1, g0, g1)
    b = O.patch_transfer_planar(a, c + g1 - g0, t2, g1, g2)
    direct = O.patch_transfer_planar(q0, c, t1 + t2, g0, g2)
    assert np.abs(b - direct).max() < 1e-9
