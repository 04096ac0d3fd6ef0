"""Patch transfer on the GPU (Eq. 3 through the poses, Eq. 4 in the plane)
against the oracle, element by element."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

F, CX, CY, W, H = 15625.0, 4088.0, 3066.0, 8176.0, 6132.0
NADIR = np.diag([1.0, -1.0, -1.0])


def _rot(rng, max_ang):
    a = rng.normal(size=3)
    a /= np.linalg.norm(a)
    ang = rng.uniform(0, max_ang)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


@pytest.fixture(scope="module")
def ba():
    import paper_2511_06152_gb300 as m
    m.lib()
    O.build()
    return m


def test_poses_transfer_matches_oracle(ba):
    rng = np.random.default_rng(11)
    gu, gv = np.meshgrid(np.linspace(40, W - 40, 24), np.linspace(40, H - 40, 18))
    p0 = np.c_[gu.ravel(), gv.ravel()]                       # a 24 x 18 patch grid
    intr0 = np.array([F, CX, CY, 0, 0, 0, 0])
    R0, T0 = _rot(rng, 0.03) @ NADIR, np.array([0.0, 0.0, 500.0])
    m = 12
    intr = np.tile(intr0, (m, 1))
    intr[:, 0] *= rng.uniform(0.98, 1.02, m)
    R = np.stack([(_rot(rng, 0.08) @ NADIR).ravel() for _ in range(m)])
    T = np.c_[rng.uniform(-250, 250, m), rng.uniform(-250, 250, m), rng.uniform(420, 580, m)]
    T[m - 1] = [0.0, 0.0, -50.0]                              # below the ground: every point behind it
    lam = 500.0
    with ba.Context(precision=ba.BA_FP64) as ctx:
        p, inside = ctx.patch_transfer_poses(p0, intr0, R0, T0, lam, intr, R, T, W, H)
        assert ctx.patch_transfer_poses(p0[:0], intr0, R0, T0, lam, intr, R, T, W, H)[0].shape == (m, 0, 2)
    n_in = 0
    for k in range(m):
        ref, ref_in = O.patch_transfer_poses(intr0, R0, T0, p0, lam, intr[k], R[k], T[k], W, H)
        front = ~np.isnan(ref[:, 0])
        assert np.array_equal(np.isnan(p[k, :, 0]), ~front)
        assert np.abs(p[k][front] - ref[front]).max(initial=0.0) < 1e-6
        assert np.array_equal(inside[k], ref_in)
        n_in += int(ref_in.sum())
    assert not inside[m - 1].any()
    assert 0 < n_in < (m - 1) * len(p0)  # some patches leave the frame, most stay


def test_planar_transfer_matches_oracle(ba):
    rng = np.random.default_rng(12)
    q0 = rng.uniform(-400, 400, (333, 2))
    c, g0 = np.array([3.0, -2.0]), np.array([100.0, 50.0])
    m = 7
    theta = rng.uniform(-np.pi, np.pi, m)
    g = g0 + rng.uniform(-60, 60, (m, 2))
    with ba.Context(precision=ba.BA_FP64) as ctx:
        q = ctx.patch_transfer_planar(q0, c, g0, theta, g)
    for k in range(m):
        ref = O.patch_transfer_planar(q0, c, theta[k], g0, g[k])
        assert np.abs(q[k] - ref).max() < 1e-9
