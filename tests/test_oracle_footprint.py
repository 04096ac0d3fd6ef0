"""Pins of the oracle's image footprints on a DSM (Sec. 3.1: the four image
corners projected onto the surface model) and of the footprint overlap used to
find adjacent-strip images (Sec. 3.1, Sec. 3.2 cluster formation)."""
import math

import numpy as np
import pytest

import oracle as O
import scenegen as sg

W, H = 8176.0, 6132.0
INTR = np.array([15625.0, W / 2, H / 2, 0.0, 0.0, 0.0, 0.0])


def _plane_dsm(a, b, c, x0=-800.0, y0=-800.0, n=801, d=2.0):
    xs = x0 + d * np.arange(n)
    X, Y = np.meshgrid(xs, y0 + d * np.arange(n))
    return O.Dsm(dict(h=a * X + b * Y + c, x0=x0, y0=y0, dx=d, dy=d))


def _ray_plane(R, T, u, v, a, b, c):
    """Closed form: T + t d on the plane z = a x + b y + c."""
    d = R @ np.array([(u - INTR[1]) / INTR[0], (v - INTR[2]) / INTR[0], 1.0])
    t = (a * T[0] + b * T[1] + c - T[2]) / (d[2] - a * d[0] - b * d[1])
    return T + t * d


@pytest.mark.parametrize("yaw,tilt,plane", [(0.0, 0.0, (0, 0, 12.0)), (0.7, 0.0, (0, 0, -5.0)),
                                            (1.1, 0.05, (0.03, -0.02, 4.0)), (3.0, 0.1, (-0.05, 0.01, 0.0))])
def test_footprint_on_planes_is_the_ray_plane_intersection(yaw, tilt, plane):
    """Bilinear interpolation reproduces a plane exactly, so every corner must
    be the closed-form ray-plane point."""
    from scipy.spatial.transform import Rotation
    R = sg.nadir_rotation(yaw) @ Rotation.from_rotvec([tilt, -0.5 * tilt, 0.0]).as_matrix()
    T = np.array([15.0, -20.0, 300.0])
    D = _plane_dsm(*plane)
    q = O.footprint(INTR, W, H, R, T, D)
    for c, (u, v) in enumerate([(0, 0), (W, 0), (W, H), (0, H)]):
        np.testing.assert_allclose(q[c], _ray_plane(R, T, u, v, *plane), atol=1e-7)


def test_nadir_footprint_on_flat_ground_is_the_sensor_rectangle():
    T = np.array([0.0, 0.0, 300.0])
    q = O.footprint(INTR, W, H, sg.nadir_rotation(0.0), T, _plane_dsm(0, 0, 0.0))
    assert O.quad_area(q) == pytest.approx((W * 300 / INTR[0]) * (H * 300 / INTR[0]), rel=1e-12)


def test_dsm_bilinear_nodes_and_midpoints():
    h = np.array([[0.0, 1.0, 4.0], [2.0, 3.0, 5.0]])
    D = O.Dsm(dict(h=h, x0=10.0, y0=20.0, dx=2.0, dy=3.0))
    assert O.dsm_height(D, 12.0, 23.0) == 3.0
    assert O.dsm_height(D, 11.0, 20.0) == 0.5
    assert O.dsm_height(D, 11.0, 21.5) == pytest.approx((0 + 1 + 2 + 3) / 4)
    assert O.dsm_height(D, -5.0, 100.0) == 2.0  # clamped to the corner node


def test_first_surface_hit_over_buildings():
    """On the synthetic terrain with buildings, each corner lies on the surface
    and no point of the ray before it lies below the surface (checked by dense
    sampling: the first hit, not a later one)."""
    fl = sg.flight(4003, n_strips=2, per_strip=6, pts_per_cam=50)
    dsm = sg.dsm_raster(fl, 2.0)
    D = O.Dsm(dsm)
    for k in range(fl["n_cams"]):
        R = fl["R_true"][k].reshape(3, 3)
        T = fl["T_true"][k]
        q = O.footprint(fl["intr"][k], W, H, R, T, D)
        for c, (u, v) in enumerate([(0, 0), (W, 0), (W, H), (0, H)]):
            P = q[c]
            assert abs(P[2] - O.dsm_height(D, P[0], P[1])) < 1e-6
            t_hit = np.linalg.norm(P - T)
            d = (P - T) / t_hit
            ts = np.linspace(0.0, t_hit - 0.5, 4000)
            z = T[2] + ts * d[2]
            hs = np.array([O.dsm_height(D, T[0] + t * d[0], T[1] + t * d[1]) for t in ts])
            assert np.all(z > hs - 1e-6)


def _rect(x0, x1, y0, y1):
    return np.array([[x0, y0, 0], [x1, y0, 0], [x1, y1, 0], [x0, y1, 0]], dtype=float)


def test_overlap_closed_forms():
    a = _rect(0, 4, 0, 3)
    assert O.quad_overlap(a, a) == pytest.approx(12.0)
    assert O.quad_overlap(a, _rect(2, 6, 1, 5)) == pytest.approx(2 * 2)
    assert O.quad_overlap(a, _rect(5, 6, 0, 1)) == 0.0
    assert O.quad_overlap(a, _rect(1, 2, 1, 2)) == pytest.approx(1.0)
    assert O.quad_overlap(_rect(1, 2, 1, 2), a) == pytest.approx(1.0)
    diamond = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0]], dtype=float)
    assert O.quad_overlap(_rect(-1, 1, -1, 1), diamond) == pytest.approx(2.0)
    half = _rect(0, 1, -1, 1)  # the right half of the diamond
    assert O.quad_overlap(half, diamond) == pytest.approx(1.0)
    # vertex order (orientation) does not matter
    assert O.quad_overlap(a[::-1].copy(), _rect(2, 6, 1, 5)[::-1].copy()) == pytest.approx(4.0)


def test_overlap_of_rotated_squares():
    """Two unit squares rotated by 45 degrees about the same centre intersect in
    a regular octagon of area 2 (sqrt(2) - 1)."""
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    sq = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0.5, 0.5, 0], [-0.5, 0.5, 0]])
    rot = sq.copy()
    rot[:, 0], rot[:, 1] = c * sq[:, 0] - s * sq[:, 1], s * sq[:, 0] + c * sq[:, 1]
    assert O.quad_overlap(sq, rot) == pytest.approx(2 * (math.sqrt(2) - 1), rel=1e-12)
