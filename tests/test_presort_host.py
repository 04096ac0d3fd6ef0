"""Host logic of cluster creation, on the CPU (no GPU): ba_presort_host runs
the presort ba_create_cluster runs and checks its tables itself; these tests
check its sizes against a brute-force derivation from the observations, that
the tables do not depend on the number of threads that build them, the
edge cases, and the input validation."""
import itertools

import numpy as np
import pytest

import scenegen as sg

ba = pytest.importorskip("paper_2511_06152_gb300")


def _scene(nc, X, obs_cam, obs_pt, fixed=None, uv=None):
    """A cluster with the given observation structure (poses and pixels only
    need to be finite: the presort reads X for the point order)."""
    X = np.asarray(X, float).reshape(-1, 3)
    obs_cam = np.asarray(obs_cam, np.int32)
    obs_pt = np.asarray(obs_pt, np.int32)
    R = np.tile(np.eye(3).ravel(), (nc, 1))
    T = np.c_[np.arange(nc, dtype=float), np.zeros(nc), np.full(nc, 500.0)]
    intr = np.tile([15625.0, 4088.0, 3066.0, 0, 0, 0, 0], (nc, 1))
    return dict(n_cams=nc, n_pts=len(X), n_obs=len(obs_cam), intr=intr, R0=R, T0=T, X0=X, R_prior=R, T_prior=T,
                obs_uv=np.zeros((len(obs_cam), 2)) if uv is None else uv, obs_cam=obs_cam, obs_pt=obs_pt,
                fixed=np.zeros(nc, np.uint8) if fixed is None else np.asarray(fixed, np.uint8),
                sigma_px=0.5, huber_delta=1.0, sigma_gnss=0.05, sigma_imu=1.745e-4)


def _spread(v):
    v = v.astype(np.uint32) & np.uint32(0xFFFF)
    for s, m in ((8, 0x00FF00FF), (4, 0x0F0F0F0F), (2, 0x33333333), (1, 0x55555555)):
        v = (v | (v << np.uint32(s))) & np.uint32(m)
    return v


def _expected(sc, tiles_per_chunk):
    """Sizes of the tables from the observations: points in Morton order of
    their initial (x, y) on a 16-bit grid over the points' bounding box (ties
    by index), a point's observations by camera, tiles as greedy runs of whole
    points of at most 32 observations, chunks of tiles_per_chunk tiles; per
    chunk one image job per free image and one pair job per co-visible pair of
    free images."""
    nc, npt = sc["n_cams"], sc["n_pts"]
    X = np.asarray(sc["X0"], float)
    cam = np.asarray(sc["obs_cam"], np.int64)
    pt = np.asarray(sc["obs_pt"], np.int64)
    free = np.asarray(sc["fixed"]) == 0
    fidx = np.cumsum(free) - 1
    inv = np.zeros(npt, np.int64)
    if npt:
        x, y = X[:, 0], X[:, 1]
        sx = 65535.0 / (x.max() - x.min()) if x.max() > x.min() else 0.0
        sy = 65535.0 / (y.max() - y.min()) if y.max() > y.min() else 0.0
        code = _spread(((x - x.min()) * sx).astype(np.uint32)) | (_spread(((y - y.min()) * sy).astype(np.uint32)) << np.uint32(1))
        order = np.argsort(code, kind="stable")
        inv[order] = np.arange(npt)
    ip = inv[pt]
    o = np.lexsort((cam, ip))
    ip, cam = ip[o], cam[o]
    counts = np.bincount(ip, minlength=npt) if npt else np.zeros(0, np.int64)
    tiles, tn = [], 0
    for L in counts:
        if L == 0:
            continue
        if tn + L > 32:
            tiles.append(tn)
            tn = 0
        tn += int(L)
    if tn:
        tiles.append(tn)
    n_chunks = -(-len(tiles) // tiles_per_chunk)
    starts = np.concatenate([[0], np.cumsum(tiles)]).astype(int)
    cam_jobs = pair_jobs = 0
    pairs = set()
    for c in range(n_chunks):
        a0, a1 = starts[c * tiles_per_chunk], starts[min(len(tiles), (c + 1) * tiles_per_chunk)]
        fc = set()
        fp = set()
        for j in np.unique(ip[a0:a1]):
            cs = [int(fidx[k]) for k in cam[a0:a1][ip[a0:a1] == j] if free[k]]
            fc.update(cs)
            fp.update(itertools.combinations(cs, 2))
        cam_jobs += len(fc)
        pair_jobs += len(fp)
        pairs |= fp
    kf = np.bincount(pt[free[np.asarray(sc["obs_cam"])]], minlength=max(npt, 1))
    return dict(n_free=int(free.sum()), n_tiles=len(tiles), n_chunks=n_chunks, n_pairs=len(pairs),
                n_cam_jobs=cam_jobs, n_pair_jobs=pair_jobs, n_free_obs=int(free[np.asarray(sc["obs_cam"])].sum()),
                n_pair_entries=int((kf * (kf - 1) // 2).sum()))


def _check(sc, precisions=(ba.BA_MIXED, ba.BA_FP64)):
    out = {}
    for prec in precisions:
        r1 = ba.presort_host(sc, prec, 1)
        r3 = ba.presort_host(sc, prec, 3)
        assert r1["checks_failed"] == 0, r1["message"]
        assert r3["checks_failed"] == 0, r3["message"]
        assert r1["digest"] == r3["digest"]  # the tables do not depend on the threads
        want = _expected(sc, r1["tiles_per_chunk"])
        assert {k: r1[k] for k in want} == want
        assert 0 < r1["max_lanes"] <= 256 or r1["n_chunks"] == 0
        out[prec] = r1
    return out


@pytest.mark.parametrize("seed,strips,per_strip,n_points,fixed", [
    (1, 1, 3, 12, None), (2, 2, 5, 400, None), (3, 3, 6, 2500, (0, 1)), (4, 2, 12, 6000, (0, 5, 11)),
    (7, 4, 12, 8000, (0, 1)),  # 46 free images: the global-memory solver's tables
])
def test_presort_tables_generated_clusters(seed, strips, per_strip, n_points, fixed):
    sc = sg.tiny_cluster(seed, strips, per_strip, n_points, fixed=fixed)
    r = _check(sc)
    assert r[ba.BA_MIXED]["tiles_per_chunk"] == 2 * r[ba.BA_FP64]["tiles_per_chunk"]


def test_presort_tables_batched_workload_cluster():
    """A cluster of the batched workload (8-32 images in 2-3 strips), scaled down."""
    sc = sg.cluster_from_spec(sg.batch_c3_specs(0, 3, scale=0.1)[2])
    _check(sc)


def test_presort_chunks_with_more_jobs_than_threads():
    """60 free images, points seen by 3 random images each: a chunk holds far
    more than 256 image and pair jobs and falls back to one lane per job."""
    rng = np.random.default_rng(5)
    npt, nc = 1500, 60
    cams = np.array([rng.choice(nc, 3, replace=False) for _ in range(npt)])
    sc = _scene(nc, rng.uniform(0, 100, (npt, 3)), cams.ravel(), np.repeat(np.arange(npt), 3))
    r = _check(sc)
    assert r[ba.BA_MIXED]["fallback_chunks"] > 0


def test_presort_longest_tracks_and_fixed_images():
    """Points seen by all 32 images (496 pairs each), half of the images fixed."""
    nc, npt = 32, 40
    rng = np.random.default_rng(6)
    fixed = np.zeros(nc, np.uint8)
    fixed[::2] = 1
    sc = _scene(nc, rng.uniform(0, 50, (npt, 3)), np.tile(np.arange(nc), npt), np.repeat(np.arange(npt), nc),
                fixed=fixed)
    r = _check(sc)[ba.BA_FP64]
    assert r["n_tiles"] == npt and r["n_pair_entries"] == npt * 16 * 15 // 2


def test_presort_empty_and_unobserved():
    """No observations at all, and points nobody observes, are valid clusters."""
    r = _check(_scene(3, np.zeros((0, 3)), [], []))
    assert r[ba.BA_MIXED]["n_tiles"] == 0 and r[ba.BA_MIXED]["n_chunks"] == 0
    sc = _scene(4, np.arange(30.0).reshape(10, 3), [0, 1, 2, 3], [2, 2, 7, 7])
    r = _check(sc)[ba.BA_MIXED]
    assert r["n_tiles"] == 1 and r["n_pairs"] == 2 and r["n_pair_entries"] == 2


@pytest.mark.parametrize("what,scene", [
    ("repeated (camera, point)", lambda: _scene(3, np.zeros((2, 3)), [0, 0, 1], [0, 0, 1])),
    ("more than 32 observations", lambda: _scene(40, np.zeros((1, 3)), np.arange(33), np.zeros(33))),
    ("index out of range", lambda: _scene(3, np.zeros((2, 3)), [0, 3], [0, 1])),
    ("no free camera", lambda: _scene(2, np.zeros((1, 3)), [0, 1], [0, 0], fixed=[1, 1])),
    ("non-finite", lambda: _scene(2, np.zeros((1, 3)), [0, 1], [0, 0], uv=np.array([[0.0, np.nan], [1.0, 1.0]]))),
])
def test_presort_rejects_invalid_clusters(what, scene):
    with pytest.raises(ba.BAError) as e:
        ba.presort_host(scene())
    assert e.value.status == ba.BA_ERR_INVALID
