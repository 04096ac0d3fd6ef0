"""Footprints on the DSM and their overlaps on the GPU (ba_footprints,
ba_footprint_overlaps) against the oracle, and the adjacent-strip selection
they serve (Sec. 3.1 cross-strip overlap, Sec. 3.2 cluster formation)."""
import numpy as np
import pytest

import oracle as O
import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    fl = sg.flight(4011, n_strips=3, per_strip=12, pts_per_cam=60)
    return fl, sg.dsm_raster(fl, 2.0)


@pytest.mark.parametrize("pose", ["R_true", "R_prior"])
def test_footprints_match_oracle(scene, pose):
    import paper_2511_06152_gb300 as ba
    fl, dsm = scene
    Rk = fl[pose].reshape(-1, 9)
    Tk = fl["T_true"] if pose == "R_true" else fl["T_prior"]
    D = O.Dsm(dsm)
    with ba.Context() as ctx:
        q = ctx.footprints(fl["intr"], sg.SENSOR_W, sg.SENSOR_H, Rk, Tk, dsm)
    for k in range(fl["n_cams"]):
        ref = O.footprint(fl["intr"][k], sg.SENSOR_W, sg.SENSOR_H, Rk[k], Tk[k], D)
        np.testing.assert_allclose(q[k], ref, atol=1e-6)


def test_overlaps_match_oracle_and_select_adjacent_strip_images(scene):
    """Every footprint against every other: the GPU areas equal the oracle's.
    With 60 % side overlap, neighbouring strips share ~60 % of a footprint's
    width and strips two apart ~20 %: a 30 % threshold on the overlap ratio
    selects images of the neighbouring strip only."""
    import paper_2511_06152_gb300 as ba
    fl, dsm = scene
    with ba.Context() as ctx:
        q = ctx.footprints(fl["intr"], sg.SENSOR_W, sg.SENSOR_H, fl["R_true"], fl["T_true"], dsm)
        A = ctx.footprint_overlaps(q, q)
    n = fl["n_cams"]
    for i in range(n):
        for j in range(n):
            assert A[i, j] == pytest.approx(O.quad_overlap(q[i], q[j]), rel=1e-9, abs=1e-9)
        assert A[i, i] == pytest.approx(O.quad_area(q[i]), rel=1e-12)
    np.testing.assert_allclose(A, A.T, rtol=1e-9, atol=1e-9)
    strip = fl["strip"]
    window = np.nonzero(strip == 2)[0][:6]
    earlier = np.nonzero(strip < 2)[0]
    ratio = A[np.ix_(window, earlier)] / np.diag(A)[window][:, None]
    sel = earlier[(ratio >= 0.3).any(axis=0)]
    assert len(sel) > 0 and np.all(strip[sel] == 1)
    assert ratio[:, strip[earlier] == 0].max() < 0.3
