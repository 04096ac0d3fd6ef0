"""Pins of the oracle's model arithmetic against things other than itself:
library rotation routines, textbook special cases of the camera model,
closed forms of the Huber function, finite differences of the residual, and
the scene generator's independent forward model.

Eq. 5 (Sec. 3.2) projection, Eq. 6 robust cost on the squared 2-D norm.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
import scenegen as sg


def rand_rot(rng, scale=1.0):
    return Rotation.from_rotvec(rng.normal(size=3) * scale).as_matrix()


# ---------------------------------------------------------------- SO(3)

@pytest.mark.parametrize("scale", [1e-12, 1e-9, 1e-6, 1e-3, 0.5, 2.0, 3.1])
def test_so3_exp_matches_library(scale):
    rng = np.random.default_rng(1)
    for _ in range(20):
        w = rng.normal(size=3)
        w *= scale / np.linalg.norm(w)
        np.testing.assert_allclose(O.so3_exp(w), Rotation.from_rotvec(w).as_matrix(), atol=2e-15, rtol=0)


@pytest.mark.parametrize("scale", [1e-12, 1e-7, 1e-3, 0.5, 2.0, 3.0, math.pi - 1e-7])
def test_so3_log_matches_library(scale):
    rng = np.random.default_rng(2)
    for _ in range(20):
        w = rng.normal(size=3)
        w *= scale / np.linalg.norm(w)
        R = Rotation.from_rotvec(w).as_matrix()
        ref = Rotation.from_matrix(R).as_rotvec()
        got = O.so3_log(R)
        tol = 1e-6 if scale > 3.1 else 1e-12
        np.testing.assert_allclose(got, ref, atol=tol * max(1.0, scale), rtol=0)


def test_so3_log_of_z_rotation():
    for a in [0.0, 1e-10, 0.3, -1.2, 3.0]:
        c, s = math.cos(a), math.sin(a)
        R = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])
        np.testing.assert_allclose(O.so3_log(R), [0, 0, a], atol=1e-14)


@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-4, 0.3, 2.5])
def test_so3_jr_inv_finite_difference(scale):
    """d Log(Exp(phi) Exp(d)) / dd at d = 0 is J_r^-1(phi)."""
    rng = np.random.default_rng(3)
    w = rng.normal(size=3)
    w = w * (scale / np.linalg.norm(w)) if scale > 0 else np.zeros(3)
    R = Rotation.from_rotvec(w).as_matrix()
    h = 1e-6
    fd = np.zeros((3, 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        lp = Rotation.from_matrix(R @ Rotation.from_rotvec(e).as_matrix()).as_rotvec()
        lm = Rotation.from_matrix(R @ Rotation.from_rotvec(-e).as_matrix()).as_rotvec()
        fd[:, i] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(O.so3_jr_inv(w), fd, atol=1e-8)


# ---------------------------------------------------------------- camera model (Eq. 5 + Brown)

def nadir_cam(f=15625.0, cx=4088.0, cy=3066.0, k=(0, 0, 0, 0)):
    return np.array([f, cx, cy, *k]), sg.nadir_rotation(0.0), np.array([0.0, 0.0, 300.0])


def test_point_below_nadir_camera_lands_on_principal_point():
    # camera at (0,0,300) looking down sees (0,0,0) at the principal point, whatever the distortion
    intr, R, T = nadir_cam(k=(1e-3, -2e-3, 5e-4, -7e-4))
    uv, ok = O.project(intr, R, T, np.zeros(3))
    assert ok
    np.testing.assert_allclose(uv, [4088.0, 3066.0], atol=1e-12)


def test_pinhole_textbook_case():
    """k = p = 0: u = f x/z + cx, v = f y/z + cy in the camera frame."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        f, cx, cy = rng.uniform(1000, 20000), rng.uniform(1000, 5000), rng.uniform(1000, 5000)
        R = rand_rot(rng)
        T = rng.normal(size=3) * 10
        Xc = np.array([rng.uniform(-5, 5), rng.uniform(-5, 5), rng.uniform(5, 50)])
        X = R @ Xc + T  # camera->world
        uv, ok = O.project(np.array([f, cx, cy, 0, 0, 0, 0.0]), R, T, X)
        assert ok
        np.testing.assert_allclose(uv, [f * Xc[0] / Xc[2] + cx, f * Xc[1] / Xc[2] + cy], rtol=1e-13)


def test_nadir_axes_and_sign():
    """Image x follows world East and image y follows world South for a
    north-flying (yaw 0) nadir camera, so a point east of nadir has u > cx."""
    intr, R, T = nadir_cam()
    uv, _ = O.project(intr, R, T, np.array([10.0, 0.0, 0.0]))
    assert uv[0] == pytest.approx(4088.0 + 15625.0 * 10.0 / 300.0, rel=1e-13)
    assert uv[1] == pytest.approx(3066.0, abs=1e-12)
    uv, _ = O.project(intr, R, T, np.array([0.0, -10.0, 0.0]))
    assert uv[1] == pytest.approx(3066.0 + 15625.0 * 10.0 / 300.0, rel=1e-13)


@pytest.mark.parametrize("which", ["k1", "k2", "p1", "p2"])
def test_brown_terms_one_at_a_time(which):
    """Brown-Conrady model with a single non-zero coefficient, checked at
    normalised points on the axes and on the diagonal."""
    c = 3e-3
    k = dict(k1=0.0, k2=0.0, p1=0.0, p2=0.0)
    k[which] = c
    f, cx, cy = 1000.0, 500.0, 400.0
    intr = np.array([f, cx, cy, k["k1"], k["k2"], k["p1"], k["p2"]])
    R, T = np.eye(3), np.zeros(3)
    for a, b in [(0.2, 0.0), (0.0, -0.3), (0.15, 0.25)]:
        uv, _ = O.project(intr, R, T, np.array([a, b, 1.0]))
        r2 = a * a + b * b
        xd, yd = a, b
        if which == "k1":
            xd, yd = a * (1 + c * r2), b * (1 + c * r2)
        elif which == "k2":
            xd, yd = a * (1 + c * r2 * r2), b * (1 + c * r2 * r2)
        elif which == "p1":
            xd, yd = a + 2 * c * a * b, b + c * (r2 + 2 * b * b)
        else:
            xd, yd = a + c * (r2 + 2 * a * a), b + 2 * c * a * b
        np.testing.assert_allclose(uv, [f * xd + cx, f * yd + cy], rtol=1e-14)


def test_behind_camera_is_rejected():
    intr, R, T = nadir_cam()
    _, ok = O.project(intr, R, T, np.array([0.0, 0.0, 400.0]))
    assert not ok


def test_generator_forward_model_agrees_with_oracle():
    """Zero-noise observations come from the generator's own vectorised
    forward model; the oracle's Eq. 5 must reproduce them at the truth."""
    c = sg.cluster_c1(zero_noise_init=True)
    P = O.Problem(c)
    R, T, X = c["R_true"].reshape(-1, 3, 3), c["T_true"], c["X_true"]
    idx = np.random.default_rng(5).choice(c["n_obs"], 300, replace=False)
    for i in idx:
        k, j = c["obs_cam"][i], c["obs_pt"][i]
        uv, ok = O.project(c["intr"][k], R[k], T[k], X[j])
        assert ok
        np.testing.assert_allclose(uv, c["obs_uv"][i], atol=1e-8)
    assert O.cost(P, c["R_true"], c["T_true"], c["X_true"]) < 1e-12


# ---------------------------------------------------------------- Huber (Eq. 6)

@pytest.mark.parametrize("delta", [1.0, 0.5, 3.0])
def test_huber_closed_forms(delta):
    d2 = delta * delta
    assert O.huber_rho(0.0, delta) == 0.0
    assert O.huber_rho(d2, delta) == pytest.approx(d2, rel=1e-15)
    assert O.huber_rho(4 * d2, delta) == pytest.approx(3 * d2, rel=1e-15)   # 2 d (2 d) - d^2
    assert O.huber_rho(0.25 * d2, delta) == pytest.approx(0.25 * d2, rel=1e-15)
    assert O.huber_weight(0.0, delta) == 1.0
    assert O.huber_weight(d2, delta) == 1.0
    assert O.huber_weight(4 * d2, delta) == pytest.approx(0.5, rel=1e-15)
    # rho' is the derivative of rho (both branches)
    for s in [0.3 * d2, 2.0 * d2, 30.0 * d2]:
        h = 1e-6 * s
        fd = (O.huber_rho(s + h, delta) - O.huber_rho(s - h, delta)) / (2 * h)
        assert O.huber_weight(s, delta) == pytest.approx(fd, rel=1e-7)


def test_huber_acts_on_the_squared_norm_not_per_component():
    """A residual (0.8, 0.8) px has s = 1.28 > delta^2 = 1 although both
    components are below delta: it must fall in the linear branch."""
    s = 0.8 ** 2 * 2
    assert O.huber_rho(s, 1.0) == pytest.approx(2 * math.sqrt(s) - 1, rel=1e-15)
    assert O.huber_rho(s, 1.0) < s


# ---------------------------------------------------------------- Jacobians

def _retract(R, T, d6):
    return R @ Rotation.from_rotvec(d6[:3]).as_matrix(), T + d6[3:]


def _fd_obs(c, P, i, R, T, X, h_rot=1e-7, h_t=1e-5, h_x=1e-5):
    k, j = c["obs_cam"][i], c["obs_pt"][i]
    r0, Jc, Jp, s, ok = O.linearize_obs(P, R, T, X, i)
    scale = math.sqrt(O.huber_weight(s, c["huber_delta"])) / c["sigma_px"]
    Rk, Tk = R[k].reshape(3, 3), T[k]
    fdc = np.zeros((2, 6))
    for a in range(6):
        h = h_rot if a < 3 else h_t
        e = np.zeros(6)
        e[a] = h
        Rp, Tp = _retract(Rk, Tk, e)
        Rm, Tm = _retract(Rk, Tk, -e)
        up, _ = O.project(c["intr"][k], Rp, Tp, X[j])
        um, _ = O.project(c["intr"][k], Rm, Tm, X[j])
        fdc[:, a] = scale * (up - um) / (2 * h)
    fdp = np.zeros((2, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h_x
        up, _ = O.project(c["intr"][k], Rk, Tk, X[j] + e)
        um, _ = O.project(c["intr"][k], Rk, Tk, X[j] - e)
        fdp[:, a] = scale * (up - um) / (2 * h_x)
    uv, _ = O.project(c["intr"][k], Rk, Tk, X[j])
    np.testing.assert_allclose(r0, scale * (uv - c["obs_uv"][i]), rtol=1e-12, atol=1e-12)
    return Jc, Jp, fdc, fdp


def test_observation_jacobians_central_differences():
    c = sg.cluster_c1()
    P = O.Problem(c)
    R, T, X = c["R0"].reshape(-1, 9), c["T0"], c["X0"]
    rng = np.random.default_rng(6)
    idx = list(rng.choice(c["n_obs"], 60, replace=False)) + list(np.nonzero(c["outlier"])[0][:10])
    for i in idx:
        Jc, Jp, fdc, fdp = _fd_obs(c, P, i, R, T, X)
        np.testing.assert_allclose(Jc, fdc, rtol=1e-6, atol=1e-6 * np.abs(fdc).max())
        np.testing.assert_allclose(Jp, fdp, rtol=1e-6, atol=1e-6 * np.abs(fdp).max())


def test_observation_jacobians_strong_distortion_and_tilt():
    """Large Brown terms and a tilted camera exercise every term of the
    distortion Jacobian."""
    c = sg.tiny_cluster(11, n_points=20)
    c["intr"][:, 3:] = [0.3, -0.2, 0.01, -0.02]
    tilt = Rotation.from_rotvec([0.15, -0.1, 0.2]).as_matrix()
    R = np.stack([r.reshape(3, 3) @ tilt for r in c["R0"]]).reshape(-1, 9)
    P = O.Problem(c)
    for i in range(c["n_obs"]):
        Jc, Jp, fdc, fdp = _fd_obs(c, P, i, R, c["T0"], c["X0"])
        np.testing.assert_allclose(Jc, fdc, rtol=1e-6, atol=1e-6 * np.abs(fdc).max())
        np.testing.assert_allclose(Jp, fdp, rtol=1e-6, atol=1e-6 * np.abs(fdp).max())


def test_prior_residual_and_jacobian():
    c = sg.cluster_c1()
    P = O.Problem(c)
    R, T = c["R0"].reshape(-1, 9).copy(), c["T0"].copy()
    rng = np.random.default_rng(7)
    # move away from the prior so that Log is not ~0
    for k in range(c["n_cams"]):
        R[k] = (R[k].reshape(3, 3) @ Rotation.from_rotvec(rng.normal(size=3) * 0.01).as_matrix()).ravel()
        T[k] += rng.normal(size=3) * 0.2
    for k in range(c["n_cams"]):
        r, J = O.linearize_prior(P, R, T, k)
        Rk = R[k].reshape(3, 3)
        phi = Rotation.from_matrix(c["R_prior"][k].reshape(3, 3).T @ Rk).as_rotvec()
        np.testing.assert_allclose(r[:3], phi / c["sigma_imu"], rtol=1e-10)
        np.testing.assert_allclose(r[3:], (T[k] - c["T_prior"][k]) / c["sigma_gnss"], rtol=1e-12)
        fd = np.zeros((6, 6))
        h = 1e-7
        for a in range(6):
            e = np.zeros(6)
            e[a] = h
            out = []
            for sgn in (1, -1):
                Rp, Tp = _retract(Rk, T[k], sgn * e)
                Rs, Ts = R.copy(), T.copy()
                Rs[k], Ts[k] = Rp.ravel(), Tp
                out.append(O.linearize_prior(P, Rs, Ts, k)[0])
            fd[:, a] = (out[0] - out[1]) / (2 * h)
        np.testing.assert_allclose(J, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_priors_switch_off_with_zero_sigma():
    c = sg.tiny_cluster(12, priors=False)
    P = O.Problem(c)
    r, J = O.linearize_prior(P, c["R0"], c["T0"] + 1.0, 0)
    assert not r.any() and not J.any()


def test_cost_definition_on_a_two_observation_problem():
    """F = 1/2 sum rho(s)/sigma^2 + 1/2 sum ||prior||^2 written out by hand
    for one camera, one point, one inlier and one outlier observation."""
    intr, R, T = nadir_cam()
    X = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    u1, _ = O.project(intr, R, T, X[0])
    u2, _ = O.project(intr, R, T, X[1])
    obs = np.array([u1 + [0.3, -0.4], u2 + [6.0, 8.0]])  # s = 0.25 and 100
    c = dict(n_cams=1, n_pts=2, n_obs=2, intr=intr[None], R_prior=R.reshape(1, 9), T_prior=(T + [0.1, 0, 0])[None],
             fixed=np.zeros(1, np.uint8), obs_cam=np.array([0, 0], np.int32), obs_pt=np.array([0, 1], np.int32),
             obs_uv=obs, sigma_px=0.5, huber_delta=1.0, sigma_gnss=0.05, sigma_imu=1e-4)
    P = O.Problem(c)
    F = O.cost(P, R.reshape(1, 9), T[None], X)
    expect = 0.5 * 0.25 / 0.25 + 0.5 * (2 * 10.0 - 1.0) / 0.25 + 0.5 * (0.1 / 0.05) ** 2
    assert F == pytest.approx(expect, rel=1e-12)
