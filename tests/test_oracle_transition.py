"""Pins of the oracle's cluster transition (Sec. 3.2, Eq. 8): the weighted
average of an overlap image's two poses."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation, Slerp

import oracle as O


def _rand_rot(rng, scale=1.0):
    return Rotation.from_rotvec(rng.normal(size=3) * scale).as_matrix()


@pytest.mark.parametrize("seed", range(6))
def test_orientation_is_the_geodesic_point_scipy_slerp(seed):
    """For two rotations the weighted mean on SO(3) is the geodesic point at
    fraction w_new / (w_old + w_new): scipy's Slerp computes it independently."""
    rng = np.random.default_rng(seed)
    Ra, Rb = _rand_rot(rng), _rand_rot(rng)
    wa, wb = rng.uniform(1, 500), rng.uniform(1, 500)
    R, _ = O.transition(Ra, np.zeros(3), wa, Rb, np.zeros(3), wb)
    ref = Slerp([0.0, 1.0], Rotation.from_matrix([Ra, Rb]))([wb / (wa + wb)]).as_matrix()[0]
    np.testing.assert_allclose(R, ref, atol=1e-12)


def test_limits_and_symmetry():
    rng = np.random.default_rng(11)
    Ra, Rb = _rand_rot(rng, 0.3), _rand_rot(rng, 0.3)
    Ta, Tb = rng.normal(size=3) * 100, rng.normal(size=3) * 100
    R, T = O.transition(Ra, Ta, 5.0, Rb, Tb, 0.0)  # no matches in the new cluster: the old pose
    assert np.array_equal(R, Ra) and np.allclose(T, Ta, atol=1e-13)
    R, T = O.transition(Ra, Ta, 0.0, Rb, Tb, 7.0)  # no matches in the old cluster: the new pose
    np.testing.assert_allclose(R, Rb, atol=1e-14)
    np.testing.assert_allclose(T, Tb, atol=1e-12)
    # equal weights: halfway in angle and in position
    R, T = O.transition(Ra, Ta, 3.0, Rb, Tb, 3.0)
    ang = lambda A, B: np.linalg.norm(Rotation.from_matrix(A.T @ B).as_rotvec())
    assert ang(Ra, R) == pytest.approx(ang(R, Rb), abs=1e-13)
    assert ang(Ra, R) == pytest.approx(0.5 * ang(Ra, Rb), abs=1e-13)
    np.testing.assert_allclose(T, 0.5 * (Ta + Tb), atol=1e-12)


def test_position_on_the_segment_at_the_weight_fraction():
    rng = np.random.default_rng(12)
    Ta, Tb = rng.normal(size=3) * 50, rng.normal(size=3) * 50
    R0 = np.eye(3)
    _, T = O.transition(R0, Ta, 3.0, R0, Tb, 1.0)  # a quarter of the way from the old to the new
    d = Tb - Ta
    np.testing.assert_allclose(T, Ta + 0.25 * d, atol=1e-12)


def test_frame_invariance():
    """Rotating the world frame rotates the averaged orientation the same way."""
    rng = np.random.default_rng(13)
    Q, Ra, Rb = _rand_rot(rng), _rand_rot(rng), _rand_rot(rng)
    R1, _ = O.transition(Ra, np.zeros(3), 2.0, Rb, np.zeros(3), 5.0)
    R2, _ = O.transition(Q @ Ra, np.zeros(3), 2.0, Q @ Rb, np.zeros(3), 5.0)
    np.testing.assert_allclose(R2, Q @ R1, atol=1e-12)
