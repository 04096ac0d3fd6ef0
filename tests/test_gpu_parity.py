"""GPU path (through the C ABI) against the FP64 CPU oracle, step by step.

FP64 path: every LM step matches the oracle to a relative 1e-10 on the state
(rotation entries, centres and points; scale 1 m), on F, on the gain's
accept/reject decision and on the damping.  Mixed path: the final
reprojection RMS within 1e-3 px and camera centres within 1 mm of the
oracle's.  The batch path equals the single-cluster path bit for bit.
"""
import numpy as np
import pytest

import oracle as O
import scenegen as sg
from helpers import fp64_step_parity, rms_inliers

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-10


@pytest.fixture(scope="module")
def ba():
    import paper_2511_06152_gb300 as m
    m.lib()
    return m


def _step_parity(ba, scene, iters, min_steps, tol=TOL_STEP):
    """FP64 step parity against the oracle; at least `min_steps` steps must be
    compared (the oracle alone decides where the cost reaches rounding level,
    so the count is fixed by the scene)."""
    n = fp64_step_parity(ba, O, scene, iters, tol)
    assert n >= min_steps, (n, min_steps)
    return n


def behind_camera_cluster(seed=606, k=4):
    """A 2 x 3-image cluster whose image k is turned over (its camera z axis
    points up, prior attitude likewise): every point lies behind it, so each
    of its observations gets weight 0 in the cost, the normal equations and
    the back-substitution (reading R10 of the z <= 1e-6 m rule)."""
    c = sg.tiny_cluster(seed, 2, 3, 300, fixed=(0,))
    c = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in c.items()}
    flip = np.diag([1.0, -1.0, -1.0])
    for key in ("R0", "R_prior"):
        R = np.asarray(c[key]).reshape(-1, 3, 3).copy()
        R[k] = R[k] @ flip
        c[key] = R.reshape(np.shape(c[key]))
    return c


def unobserved_camera_cluster(seed=707, mu0=1e-320):
    """A 2 x 3-image cluster without priors (two fixed images hold the gauge)
    plus one free image that observes nothing: its block of the reduced
    system is exactly mu * D = mu * 1e-6, which underflows to 0 for mu below
    about 2.5e-318, so the damped system is not positive definite until the
    rejections have raised mu (exact doublings, in every implementation)."""
    c = sg.tiny_cluster(seed, 2, 3, 200, fixed=(0, 1), priors=False)
    c = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in c.items()}
    nc = int(c["n_cams"])
    for key in ("intr", "R0", "T0", "R_prior", "T_prior", "R_true", "T_true"):
        a = np.asarray(c[key])
        c[key] = np.concatenate([a, a[2:3]], axis=0)
    c["T0"][nc] += (5.0, 0.0, 0.0)
    c["T_prior"][nc] += (5.0, 0.0, 0.0)
    c["fixed"] = np.concatenate([c["fixed"], np.zeros(1, np.uint8)])
    c["strip"] = np.concatenate([c["strip"], c["strip"][2:3]])
    c["n_cams"] = nc + 1
    c["mu0"] = mu0
    return c


def test_fp64_step_parity_c1(ba):
    """6 images, ~7,000 observations, Huber outliers, GNSS/IMU priors, 10 steps."""
    _step_parity(ba, sg.cluster_c1(), sg.ITERS["c1"], min_steps=10)


@pytest.mark.parametrize("seed,strips,per,npts,fixed,priors,min_steps", [
    (101, 1, 2, 10, None, True, 5),
    (102, 2, 2, 40, (0,), True, 8),
    (103, 1, 4, 60, (0, 3), False, 8),
    (104, 2, 3, 200, (1, 4), True, 8),
    (105, 3, 3, 500, None, True, 8),
])
def test_fp64_step_parity_small_clusters(ba, seed, strips, per, npts, fixed, priors, min_steps):
    _step_parity(ba, sg.tiny_cluster(seed, strips, per, npts, fixed=fixed, priors=priors), 8, min_steps)


def test_fp64_step_parity_point_behind_an_image(ba):
    """One image turned over: all of its observations lie behind it (weight
    0 in both implementations); 8 steps compared."""
    _step_parity(ba, behind_camera_cluster(), 8, min_steps=8)


def test_fp64_not_positive_definite_steps_match_oracle(ba):
    """Damped systems that are not positive definite: the GPU reports
    BA_ERR_NOT_PD in the step status, rejects the step, keeps the state and
    raises mu by nu exactly as the oracle; the steps that follow (accepted,
    then not positive definite again) match as well."""
    c = unobserved_camera_cluster()
    n = _step_parity(ba, c, 8, min_steps=8)
    assert n == 8
    P, S = O.Problem(c), O.State(c, mu0=c["mu0"])
    st = [O.lm_step(P, S)["status"] for _ in range(8)]
    assert st[:4] == [ba.BA_ERR_NOT_PD] * 4 and st[4] == 0 and ba.BA_ERR_NOT_PD in st[5:]


def test_fp64_step_parity_c2_full_size(ba):
    """The paper-scale cluster (24 images, 40,000 points, ~230k observations)
    at full size, 20 steps."""
    _step_parity(ba, sg.cluster_c2(), sg.ITERS["c2"], min_steps=20)


def test_fp64_zero_noise_convergence(ba):
    c = sg.cluster_c1(zero_noise_init=True)
    with ba.Context(precision=ba.BA_FP64) as ctx:
        cid = ctx.create_cluster(c)
        ctx.run(cid, 25)
        R, T, X = ctx.get_state(cid)
    assert sg.centre_error(T, c["T_true"]) < 1e-9
    assert np.abs(X - c["X_true"]).max() < 1e-8


def test_run_equals_single_steps_bitwise(ba):
    c = sg.cluster_c1()
    with ba.Context(precision=ba.BA_FP64) as ctx:
        a = ctx.create_cluster(c)
        b = ctx.create_cluster(c)
        ta = ctx.run(a, 6)
        tb = [ctx.solve_step(b) for _ in range(6)]
        for x, y in zip(ta, tb):
            assert x == y
        for u, v in zip(ctx.get_state(a), ctx.get_state(b)):
            assert np.array_equal(u, v)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_alone_bitwise(ba, precision):
    prec = ba.BA_FP64 if precision == "fp64" else ba.BA_MIXED
    scenes = sg.batch_c3(replica=7, n_clusters=5, scale=0.1)
    with ba.Context(precision=prec) as ctx:
        ids = [ctx.create_cluster(s) for s in scenes]
        alone = []
        for i in ids:
            ctx.run(i, 4)
            alone.append(ctx.get_state(i))
            ctx.reset(i)
        res = ctx.solve_batch(ids, 4)
        for i, a, r in zip(ids, alone, res):
            got = ctx.get_state(i)
            for u, v in zip(got, a):
                assert np.array_equal(u, v)
            assert r["iters"] == 4


def test_reset_and_determinism(ba):
    c = sg.cluster_c1()
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        cid = ctx.create_cluster(c)
        t1 = ctx.run(cid, 5)
        s1 = ctx.get_state(cid)
        ctx.reset(cid)
        t2 = ctx.run(cid, 5)
        s2 = ctx.get_state(cid)
    assert t1 == t2
    for u, v in zip(s1, s2):
        assert np.array_equal(u, v)


def test_linearize_cost_and_gradient(ba):
    c = sg.cluster_c1(fixed=(2,))
    P = O.Problem(c)
    ref = O.solve_damped(P, c["R0"], c["T0"], c["X0"], 1e-4)
    F = O.cost(P, c["R0"], c["T0"], c["X0"])
    with ba.Context(precision=ba.BA_FP64) as ctx:
        cid = ctx.create_cluster(c)
        lin = ctx.linearize(cid)
    g = max(np.abs(ref["gc"]).max(), np.abs(ref["gp"]).max())
    assert lin["cost"] == pytest.approx(F, rel=1e-12)
    assert lin["grad_inf"] == pytest.approx(g, rel=1e-9)
    assert lin["n_free"] == 5


@pytest.mark.parametrize("fixed", [None, (1,)])
def test_mixed_cost_evaluation_matches_fp64(ba, fixed):
    """The mixed path evaluates F in double-float per observation and sums in
    binary64: it must agree with the oracle's binary64 F to ~1e-12."""
    c = sg.cluster_c1(fixed=fixed)
    P = O.Problem(c)
    F = O.cost(P, c["R0"], c["T0"], c["X0"])
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        cid = ctx.create_cluster(c)
        lin = ctx.linearize(cid)
        R, T, X = ctx.get_state(cid)
    assert lin["cost"] == pytest.approx(F, rel=1e-11)
    # the initial state round-trips exactly through the double-float representation
    assert np.array_equal(T, c["T0"]) and np.array_equal(R, c["R0"].reshape(-1, 9))
    assert np.abs(X - c["X0"]).max() <= 1e-12


def test_mixed_step_decisions_follow_fp64(ba):
    """Mixed and FP64 paths take the same accept/reject decisions on c1 and
    reach costs within 1e-6 relative after every step."""
    c = sg.cluster_c1()
    with ba.Context(precision=ba.BA_MIXED) as cm, ba.Context(precision=ba.BA_FP64) as cd:
        a, b = cm.create_cluster(c), cd.create_cluster(c)
        tm, td = cm.run(a, 10), cd.run(b, 10)
    for x, y in zip(tm, td):
        assert x["accepted"] == y["accepted"]
        assert x["F_after"] == pytest.approx(y["F_after"], rel=1e-6)


def test_reprojection_errors_match_oracle(ba):
    c = sg.tiny_cluster(7, 2, 2, 50)
    P = O.Problem(c)
    with ba.Context(precision=ba.BA_FP64) as ctx:
        cid = ctx.create_cluster(c)
        e = ctx.reprojection_errors(cid)
    ref = O.residual_stats(P, c["R0"], c["T0"], c["X0"])
    np.testing.assert_allclose(e, ref, rtol=1e-12, atol=1e-12)


def test_mixed_precision_against_oracle_c1(ba):
    """Mixed precision (FP32 per-observation work, FP64 solve and cost):
    final reprojection RMS within 1e-3 px and centres within 1 mm."""
    c = sg.cluster_c1()
    P, S = O.Problem(c), O.State(c)
    O.lm_run(P, S, sg.ITERS["c1"])
    ref_rms = rms_inliers(O.residual_stats(P, S.R, S.T, S.X), c["outlier"])
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        cid = ctx.create_cluster(c)
        ctx.run(cid, sg.ITERS["c1"])
        R, T, X = ctx.get_state(cid)
        rms = rms_inliers(ctx.reprojection_errors(cid), c["outlier"])
    assert abs(rms - ref_rms) < 1e-3
    assert sg.centre_error(T, S.T) < 1e-3


@pytest.mark.parametrize("bad", ["cam_range", "pt_range", "nan", "dup", "long_track", "all_fixed", "sigma"])
def test_invalid_clusters_are_rejected(ba, bad):
    c = sg.tiny_cluster(9, 1, 3, 10)
    c = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in c.items()}
    if bad == "cam_range":
        c["obs_cam"][0] = c["n_cams"]
    elif bad == "pt_range":
        c["obs_pt"][0] = -1
    elif bad == "nan":
        c["obs_uv"][3, 1] = np.nan
    elif bad == "dup":
        c["obs_cam"][1] = c["obs_cam"][0]
        c["obs_pt"][1] = c["obs_pt"][0]
    elif bad == "long_track":
        n = 33
        c["n_obs"] = n
        c["obs_cam"] = np.arange(n, dtype=np.int32) % c["n_cams"]
        c["obs_pt"] = np.zeros(n, dtype=np.int32)
        c["obs_uv"] = np.zeros((n, 2))
    elif bad == "all_fixed":
        c["fixed"] = np.ones(c["n_cams"], np.uint8)
    elif bad == "sigma":
        c["sigma_px"] = 0.0
    with ba.Context() as ctx:
        with pytest.raises(ba.BAError) as ei:
            ctx.create_cluster(c)
        assert ei.value.status == ba.BA_ERR_INVALID


def test_chunks_with_only_fixed_camera_observations(ba):
    """Points seen only by fixed cameras fill whole chunks that have no
    camera or pair to reduce; the step must still match the oracle."""
    c = sg.tiny_cluster(4242, 1, 8, 6000, fixed=(0, 1, 2, 3))
    seen = np.zeros(c["n_pts"], dtype=int)
    np.add.at(seen, c["obs_pt"], c["fixed"][c["obs_cam"]] == 0)
    # ~1800 points seen by fixed cameras only; in Morton order they fill
    # several whole chunks at both chunk sizes
    assert (seen == 0).sum() > 1500
    _step_parity(ba, c, 5, min_steps=5)
    P, S = O.Problem(c), O.State(c)
    O.lm_run(P, S, 5)
    ref_rms = rms_inliers(O.residual_stats(P, S.R, S.T, S.X), c["outlier"])
    with ba.Context(precision=ba.BA_MIXED) as ctx:
        cid = ctx.create_cluster(c)
        tr = ctx.run(cid, 5)
        assert all(t["status"] == 0 for t in tr)
        R, T, X = ctx.get_state(cid)
        rms = rms_inliers(ctx.reprojection_errors(cid), c["outlier"])
    assert abs(rms - ref_rms) < 1e-3
    assert sg.centre_error(T, S.T) < 1e-3


def test_fp64_step_parity_cluster_without_observations(ba):
    """Three free images with priors and no observation at all (no
    back-substitution tile): the LM step is still taken every iteration and
    matches the oracle (the poses move to the priors)."""
    c = sg.tiny_cluster(808, 1, 3, 20)
    c = {key: (v.copy() if isinstance(v, np.ndarray) else v) for key, v in c.items()}
    c["T0"] = np.asarray(c["T0"]) + np.array([0.3, -0.2, 0.1])
    c.update(n_pts=0, n_obs=0, X0=np.zeros((0, 3)), obs_cam=np.zeros(0, np.int32), obs_pt=np.zeros(0, np.int32),
             obs_uv=np.zeros((0, 2)), outlier=np.zeros(0, bool))
    assert _step_parity(ba, c, 4, min_steps=2) >= 2
