"""Pins of the oracle's solver: the Schur-complement step against a dense
normal-equation solve by LAPACK, the predicted reduction against the
linear model's decrease, zero-noise convergence to the generating poses,
monotone cost on accepted steps, the damping schedule's rules, and the
time-budget example of Eq. 1.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import scenegen as sg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_system(c, P, R, T, X):
    """Dense whitened Jacobian (rows: observations then free-camera priors;
    columns: 6 per free camera then 3 per point) assembled from the oracle's
    per-observation pieces, which the finite-difference tests pin."""
    free = [k for k in range(c["n_cams"]) if not c["fixed"][k]]
    col = {k: 6 * i for i, k in enumerate(free)}
    nfc = 6 * len(free)
    n = nfc + 3 * c["n_pts"]
    rows, rr = [], []
    for i in range(c["n_obs"]):
        r, Jc, Jp, s, ok = O.linearize_obs(P, R, T, X, i)
        k, j = c["obs_cam"][i], c["obs_pt"][i]
        J = np.zeros((2, n))
        if k in col:
            J[:, col[k]:col[k] + 6] = Jc
        J[:, nfc + 3 * j:nfc + 3 * j + 3] = Jp
        rows.append(J)
        rr.append(r)
    for k in free:
        r, Jk = O.linearize_prior(P, R, T, k)
        J = np.zeros((6, n))
        J[:, col[k]:col[k] + 6] = Jk
        rows.append(J)
        rr.append(r)
    return np.vstack(rows), np.concatenate(rr), free


def dense_step(J, r, mu):
    H = J.T @ J
    g = -J.T @ r
    D = np.clip(np.diag(H), 1e-6, 1e32)
    d = np.linalg.solve(H + mu * np.diag(D), g)
    return d, g, D


@pytest.mark.parametrize("seed,strips,per,npts,fixed,priors,mu", [
    (21, 1, 2, 8, None, True, 1e-4),
    (22, 1, 3, 15, None, True, 1e-2),
    (23, 2, 2, 20, (0,), True, 1.0),
    (24, 1, 3, 12, (0, 2), False, 1e-3),
    (25, 2, 2, 18, None, True, 1e-6),
])
def test_schur_step_equals_dense_normal_equations(seed, strips, per, npts, fixed, priors, mu):
    c = sg.tiny_cluster(seed, strips, per, npts, fixed=fixed, priors=priors)
    P = O.Problem(c)
    R, T, X = c["R0"], c["T0"], c["X0"]
    out = O.solve_damped(P, R, T, X, mu)
    assert out["status"] == 0
    J, r, free = dense_system(c, P, R, T, X)
    d, g, D = dense_step(J, r, mu)
    nfc = 6 * len(free)
    dc_ref = np.zeros((c["n_cams"], 6))
    for i, k in enumerate(free):
        dc_ref[k] = d[6 * i:6 * i + 6]
    dp_ref = d[nfc:].reshape(-1, 3)
    scale = np.abs(d).max()
    np.testing.assert_allclose(out["dc"], dc_ref, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(out["dp"], dp_ref, rtol=0, atol=1e-9 * scale)
    # gradient and damping diagonal, block by block
    gc = np.zeros((c["n_cams"], 6))
    Dc = np.zeros((c["n_cams"], 6))
    for i, k in enumerate(free):
        gc[k] = g[6 * i:6 * i + 6]
        Dc[k] = D[6 * i:6 * i + 6]
    np.testing.assert_allclose(out["gc"], gc, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(out["gp"], g[nfc:].reshape(-1, 3), rtol=1e-12, atol=1e-12 * np.abs(g).max())
    np.testing.assert_allclose(out["Dc"], Dc, rtol=1e-12)
    np.testing.assert_allclose(out["Dp"], D[nfc:].reshape(-1, 3), rtol=1e-12)
    if fixed:
        assert not out["dc"][list(fixed)].any()


def test_predicted_reduction_is_the_linear_models_decrease():
    """pred = 1/2 d^T (mu D d + g) equals 1/2||r||^2 - 1/2||r + J d||^2."""
    c = sg.tiny_cluster(31, 2, 2, 16)
    P = O.Problem(c)
    S = O.State(c, mu0=1e-3)
    J, r, free = dense_system(c, P, S.R, S.T, S.X)
    info = O.lm_step(P, S)
    d, g, D = dense_step(J, r, 1e-3)
    model = 0.5 * r @ r - 0.5 * np.sum((r + J @ d) ** 2)
    assert info["pred"] == pytest.approx(model, rel=1e-8)


def test_step_applies_right_perturbation():
    """apply_step: R <- R Exp(dtheta), T <- T + dT, X <- X + dX."""
    from scipy.spatial.transform import Rotation
    c = sg.tiny_cluster(32)
    P = O.Problem(c)
    rng = np.random.default_rng(0)
    dc = rng.normal(size=(c["n_cams"], 6)) * 0.01
    dp = rng.normal(size=(c["n_pts"], 3)) * 0.01
    Rn, Tn, Xn = O.apply_step(P, c["R0"], c["T0"], c["X0"], dc, dp)
    for k in range(c["n_cams"]):
        ref = c["R0"][k].reshape(3, 3) @ Rotation.from_rotvec(dc[k, :3]).as_matrix()
        np.testing.assert_allclose(Rn[k].reshape(3, 3), ref, atol=1e-15)
    np.testing.assert_allclose(Tn, c["T0"] + dc[:, 3:], rtol=1e-15)
    np.testing.assert_allclose(Xn, c["X0"] + dp, rtol=1e-15)


@pytest.mark.parametrize("fixed,priors", [(None, True), ((0, 3), False)])
def test_zero_noise_converges_to_generating_poses(fixed, priors):
    """Exact pixels and priors; poses start 0.3 m / 0.02 deg off, points 0.1 m
    off.  Camera centres must converge to the truth within 1e-9 m."""
    c = sg.cluster_c1(zero_noise_init=True, fixed=fixed, priors=priors)
    P = O.Problem(c)
    S = O.State(c)
    assert sg.centre_error(S.T, c["T_true"]) > 0.1 or fixed
    O.lm_run(P, S, 25)
    assert sg.centre_error(S.T, c["T_true"]) < 1e-9
    assert np.abs(S.X - c["X_true"]).max() < 1e-8


def test_accepted_steps_decrease_cost_and_damping_rules():
    c = sg.cluster_c1()
    P = O.Problem(c)
    S = O.State(c)
    trace = O.lm_run(P, S, 10)
    nu_prev, F_prev = 2.0, trace[0]["F"]
    n_rej = 0
    for t in trace:
        assert t["F"] == pytest.approx(F_prev, rel=1e-15)  # F(x) of the state the step started from
        if t["accepted"]:
            assert t["F_new"] < t["F"]
            assert t["nu"] == 2.0
            assert 1 / 3 - 1e-15 <= t["mu"] / t["mu_used"] <= 2.0 + 1e-15
            F_prev = t["F_new"]
        else:
            n_rej += 1
            assert t["mu"] == pytest.approx(t["mu_used"] * nu_prev, rel=1e-15)
            assert t["nu"] == 2 * nu_prev
        nu_prev = t["nu"]
    # noisy data still lands near the noise floor (sqrt(2) sigma for inliers far from outliers)
    assert trace[-1]["F_new"] < 0.2 * trace[0]["F"]


def test_rejection_path_multiplies_damping():
    """Force a rejected step with a huge starting damping ... then an absurdly
    small one on a problem far from its minimum; either way the rules hold."""
    c = sg.cluster_c1()
    P = O.Problem(c)
    S = O.State(c, mu0=1e-12)
    # overshooting: a tiny mu on the IRLS model of a far start can be rejected
    t = O.lm_step(P, S)
    if not t["accepted"]:
        assert t["mu"] == pytest.approx(1e-12 * 2.0) and t["nu"] == 4.0
    S2 = O.State(c, mu0=1e12)
    t2 = O.lm_step(P, S2)  # a damped-to-nothing step: gain is tiny but positive
    assert t2["status"] == 0
    assert abs(t2["F_new"] - t2["F"]) < 1e-3 * t2["F"]


def test_eq1_time_budget_example():
    """Eq. 1 worked example (Sec. 1): 20 m/s, 80 % overlap -> 2.08 s, which
    fixes the along-track footprint at 208 m."""
    with open(os.path.join(GOLDEN, "eq1_time_budget.json")) as f:
        g = json.load(f)
    t = sg.image_interval_s(g["footprint_along_m"], g["overlap_pct"], g["velocity_mps"])
    assert t == pytest.approx(g["t_s"], abs=5e-3)
