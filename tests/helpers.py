"""Shared test helpers: running the oracle and the GPU library on one scene,
and the parity measures used by the GPU tests."""
import numpy as np


def state_rel_err(Ra, Ta, Xa, Rb, Tb, Xb):
    """max |a - b| / max(|b|, s) with s = 1 m for positions and points and 1
    for rotation-matrix entries (which are bounded by 1)."""
    e = 0.0
    e = max(e, float(np.max(np.abs(np.asarray(Ra) - np.asarray(Rb)))))
    for a, b in ((Ta, Tb), (Xa, Xb)):
        a, b = np.asarray(a), np.asarray(b)
        if a.size:
            e = max(e, float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1.0))))
    return e


def rms_inliers(err, outlier):
    return float(np.sqrt(np.mean(np.asarray(err)[~np.asarray(outlier)] ** 2)))


def compare_steps(ctx, cid, O, P, S, iters, tol=1e-10):
    """Step the FP64 GPU path (cluster cid of ctx, through the C ABI) and the
    oracle (problem P, state S) side by side from the same state and compare
    every step: F before, the status, the accept/reject decision, F after,
    the damping and the state (relative `tol`, scale 1 m).  A step the oracle
    rejects as not positive definite must be rejected the same way, with the
    state unchanged.  Once the cost has converged to rounding level
    (|F - F(x+d)| <= 1e-10 F, or |gain| < 1e-8) the decision is not
    determined in binary64 and the comparison stops there.  Returns the
    number of steps compared."""
    import pytest
    compared = 0
    before = ctx.get_state(cid)
    for it in range(iters):
        io = O.lm_step(P, S)
        ig = ctx.solve_step(cid)
        R, T, X = ctx.get_state(cid)
        assert ig["F_before"] == pytest.approx(io["F"], rel=tol, abs=1e-300)
        assert ig["mu_used"] == io["mu_used"], (it, ig, io)
        assert ig["status"] == io["status"], (it, ig, io)
        if io["status"] != 0:
            assert ig["accepted"] == 0 and io["accepted"] == 0
            assert ig["mu"] == io["mu"] and ig["nu"] == io["nu"], (it, ig, io)
            for a, b in zip((R, T, X), before):  # a rejected step leaves the GPU's state as it was
                assert np.array_equal(a, b)
            compared += 1
            continue
        if abs(io["F"] - io["F_new"]) <= 1e-10 * abs(io["F"]) or abs(io["gain"]) < 1e-8:
            break
        assert ig["accepted"] == io["accepted"], (it, ig, io)
        assert ig["F_after"] == pytest.approx(io["F_new"], rel=tol, abs=1e-12)
        assert ig["mu"] == pytest.approx(io["mu"], rel=1e-9)
        e = state_rel_err(R, T, X, S.R, S.T, S.X)
        assert e < tol, (it, e)
        before = (R, T, X)
        compared += 1
    return compared


def fp64_step_parity(ba, O, scene, iters, tol=1e-10, min_free=None, flags=0):
    """compare_steps on a fresh FP64 context (with `flags`) and cluster made
    from `scene` (its initial damping scene["mu0"], default 1e-4).  Returns
    the number of steps compared."""
    P, S = O.Problem(scene), O.State(scene, mu0=scene.get("mu0", 1e-4))
    with ba.Context(precision=ba.BA_FP64, flags=flags) as ctx:
        cid = ctx.create_cluster(scene)
        if min_free is not None:
            assert ctx.cluster_info(cid)["n_free"] >= min_free
        return compare_steps(ctx, cid, O, P, S, iters, tol)
