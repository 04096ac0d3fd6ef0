"""Seeded synthetic aerial scenes for local bundle adjustment.

This module makes the inputs that both the CPU oracle and the CUDA library
consume: camera strips flown over a synthetic terrain with box buildings,
ground points, their pixel observations, and noisy GNSS/IMU pose priors.
It stands in for the paper's MACS imagery and patch tracker (Sec. 3.1, Sec. 4),
which are not available; only the shapes, the noise model and the cluster
structure of the paper's workload are reproduced.

It holds none of the bundle-adjustment arithmetic.  Measurements are
synthesised with its own vectorised forward camera model (a scene simulator,
written independently of the oracle and of the CUDA kernels); rotation noise
uses scipy's rotation-vector routine.  No residual, Jacobian, normal equation
or solver lives here.

Conventions (shared by every consumer, so they are data, not arithmetic):
  * world frame: local East-North-Up metres, origin at the cluster centre;
  * R[k] (3x3, row-major) maps camera axes to world axes, T[k] is the camera
    centre (Eq. 5 reads p = pi(K R^T (X - T)));
  * camera z points at the ground, image x to the right, image y down; image
    rows run along the flight line;
  * intr[k] = (f, cx, cy, k1, k2, p1, p2): one focal length for both axes and
    Brown radial (k1, k2) / tangential (p1, p2) coefficients;
  * observations are sorted by (point, camera).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial.transform import Rotation

# Sensor and flight geometry of the paper-shaped workload.
SENSOR_W = 8176
SENSOR_H = 6132
FOCAL_PX = 15625.0
ALTITUDE_M = 300.0
FORWARD_OVERLAP = 0.80
SIDE_OVERLAP = 0.60
GSD_M = ALTITUDE_M / FOCAL_PX                     # 1.92 cm / px
FOOT_ACROSS_M = SENSOR_W * GSD_M                  # 157.0 m (image x)
FOOT_ALONG_M = SENSOR_H * GSD_M                   # 117.7 m (image y)
BASE_M = (1.0 - FORWARD_OVERLAP) * FOOT_ALONG_M   # 23.5 m between exposures
STRIP_SPACING_M = (1.0 - SIDE_OVERLAP) * FOOT_ACROSS_M  # 62.8 m between strips

SIGMA_PX = 0.5
OUTLIER_FRAC = 0.02
OUTLIER_HALF_WIDTH_PX = 50.0
HUBER_DELTA_PX = 1.0
SIGMA_GNSS_M = 0.05
SIGMA_IMU_RAD = math.radians(0.01)
DIST_SIGMA = 1e-3
ATTITUDE_JITTER_RAD = math.radians(0.5)
POINT_INIT_SIGMA_M = 0.10
PATCH_SIDE_M = 150 * GSD_M                        # 150 px patch ~ 2.88 m on the ground


def rng_for(config_index: int, replica: int = 0) -> np.random.Generator:
    """PCG64 stream, seed = 1000 * config + replica."""
    return np.random.Generator(np.random.PCG64(1000 * config_index + replica))


# --------------------------------------------------------------------------
# terrain: DSM z = 20 * (sin(2 pi x/400) + sin(2 pi y/250) + sin(2 pi (x+y)/600)) / 3
# plus axis-aligned box buildings (5-30 m tall, 10-40 m wide, ~1 per 2500 m^2)
# --------------------------------------------------------------------------
def make_buildings(rng, xmin, xmax, ymin, ymax):
    area = (xmax - xmin) * (ymax - ymin)
    n = rng.poisson(area / 2500.0)
    cx = rng.uniform(xmin, xmax, n)
    cy = rng.uniform(ymin, ymax, n)
    hw = rng.uniform(10.0, 40.0, n) / 2
    hh = rng.uniform(10.0, 40.0, n) / 2
    h = rng.uniform(5.0, 30.0, n)
    return np.stack([cx - hw, cx + hw, cy - hh, cy + hh, h], axis=1)


def terrain_height(x, y, buildings):
    z = 20.0 * (np.sin(2 * np.pi * x / 400.0) + np.sin(2 * np.pi * y / 250.0)
                + np.sin(2 * np.pi * (x + y) / 600.0)) / 3.0
    if len(buildings):
        extra = np.zeros_like(z)
        for b in buildings:
            inside = (x >= b[0]) & (x <= b[1]) & (y >= b[2]) & (y <= b[3])
            extra = np.where(inside, np.maximum(extra, b[4]), extra)
        z = z + extra
    return z


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
def nadir_rotation(yaw):
    """Camera->world rotation of a nadir camera whose image x axis points at
    heading `yaw` (radians from East) and whose optical axis points down."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, s, 0.0], [s, -c, 0.0], [0.0, 0.0, -1.0]])


def strip_layout(n_strips, cams_per_strip, x0=0.0, y0=0.0):
    """Serpentine strips flown along +y / -y, centred on (x0, y0).  Returns
    centres (n,3), yaw (n,), strip index (n,), in time order."""
    cams, yaws, strip = [], [], []
    for s in range(n_strips):
        x = x0 + (s - (n_strips - 1) / 2.0) * STRIP_SPACING_M
        order = range(cams_per_strip) if s % 2 == 0 else range(cams_per_strip - 1, -1, -1)
        for i in order:
            y = y0 + (i - (cams_per_strip - 1) / 2.0) * BASE_M
            cams.append((x, y, ALTITUDE_M))
            yaws.append(0.0 if s % 2 == 0 else math.pi)
            strip.append(s)
    return np.array(cams), np.array(yaws), np.array(strip, dtype=np.int32)


def forward_model(intr, R, T, X):
    """Scene simulator: pixel coordinates of points X (n,3) seen by one camera
    (intr (7,), R (3,3) camera->world, T (3,)).  Returns (uv (n,2), depth (n,))."""
    Xc = (X - T) @ R            # rows are R^T (X - T)
    depth = Xc[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        a = Xc[:, 0] / depth
        b = Xc[:, 1] / depth
    f, cx, cy, k1, k2, p1, p2 = intr
    rr = a * a + b * b
    radial = 1.0 + k1 * rr + k2 * rr * rr
    ad = a * radial + 2.0 * p1 * a * b + p2 * (rr + 2.0 * a * a)
    bd = b * radial + p1 * (rr + 2.0 * b * b) + 2.0 * p2 * a * b
    return np.stack([f * ad + cx, f * bd + cy], axis=1), depth


def _visible(intr, R, T, X):
    uv, depth = forward_model(intr, R, T, X)
    ok = (depth > 1.0) & (uv[:, 0] >= 0) & (uv[:, 0] < SENSOR_W) & (uv[:, 1] >= 0) & (uv[:, 1] < SENSOR_H)
    return ok, uv


def visibility_matrix(intr, R, T, X):
    """Boolean (n_pts, n_cams) of points inside each image, and their pixels."""
    n_c = len(T)
    vis = np.zeros((len(X), n_c), dtype=bool)
    uv = np.zeros((len(X), n_c, 2))
    for k in range(n_c):
        # cheap ground-box cull before projecting
        m = (np.abs(X[:, 0] - T[k, 0]) < 0.75 * FOOT_ACROSS_M) & (np.abs(X[:, 1] - T[k, 1]) < 0.75 * FOOT_ACROSS_M)
        idx = np.nonzero(m)[0]
        if len(idx) == 0:
            continue
        ok, puv = _visible(intr[k], R[k], T[k], X[idx])
        vis[idx[ok], k] = True
        uv[idx[ok], k] = puv[ok]
    return vis, uv


# --------------------------------------------------------------------------
# cluster assembly
# --------------------------------------------------------------------------
def _sample_points(rng, n, bbox, buildings, intr, R, T, min_views=2, batch=None):
    """Uniform ground points over bbox, kept when seen by >= min_views images."""
    xmin, xmax, ymin, ymax = bbox
    out = []
    have = 0
    batch = batch or max(4096, 2 * n)
    while have < n:
        x = rng.uniform(xmin, xmax, batch)
        y = rng.uniform(ymin, ymax, batch)
        X = np.stack([x, y, terrain_height(x, y, buildings)], axis=1)
        vis, _ = visibility_matrix(intr, R, T, X)
        keep = vis.sum(1) >= min_views
        out.append(X[keep])
        have += int(keep.sum())
    return np.concatenate(out)[:n]


def _patch_points(rng, n_points, per_patch, bbox, buildings, intr, R, T):
    """Points in 150 px (2.88 m) ground patches laid on a regular grid over
    the footprint union (the paper's patch grid, Sec. 3.1)."""
    xmin, xmax, ymin, ymax = bbox
    n_patches = -(-n_points // per_patch)
    # grid spacing so that the grid cells seen twice are about n_patches
    spacing = math.sqrt((xmax - xmin) * (ymax - ymin) / n_patches)
    for _ in range(60):
        gx = np.arange(xmin + spacing / 2, xmax, spacing)
        gy = np.arange(ymin + spacing / 2, ymax, spacing)
        cx, cy = np.meshgrid(gx, gy, indexing="ij")
        cx, cy = cx.ravel(), cy.ravel()
        C = np.stack([cx, cy, terrain_height(cx, cy, buildings)], axis=1)
        vis, _ = visibility_matrix(intr, R, T, C)
        good = np.nonzero(vis.sum(1) >= 2)[0]
        if len(good) >= n_patches:
            break
        spacing *= 0.97
    sel = np.sort(rng.choice(good, n_patches, replace=False))
    pts = []
    half = PATCH_SIDE_M / 2
    for c in sel:
        got = np.zeros((0, 3))
        while len(got) < per_patch:
            x = rng.uniform(cx[c] - half, cx[c] + half, 2 * per_patch)
            y = rng.uniform(cy[c] - half, cy[c] + half, 2 * per_patch)
            X = np.stack([x, y, terrain_height(x, y, buildings)], axis=1)
            v, _ = visibility_matrix(intr, R, T, X)
            got = np.concatenate([got, X[v.sum(1) >= 2]])
        pts.append(got[:per_patch])
    return np.concatenate(pts)[:n_points]


def make_cluster(rng, n_strips, cams_per_strip, n_points, *, layout="uniform",
                 per_patch=30, track=None, noise=True, zero_noise_init=False,
                 fixed=None, priors=True, n_cams=None):
    """Build one local-BA cluster as a dict of numpy arrays.

    track: None -> every image containing a point observes it; otherwise
           (p, L_max): L - 2 ~ Geometric(p) failures, truncated to
           min(L_max, number of images that contain the point), the L images
           drawn uniformly among those.
    noise: pixel noise N(0, 0.5^2), 2 % outliers uniform +-50 px, GNSS
           N(0, 0.05^2) per axis, IMU Exp(N(0, (0.01 deg)^2)).
    zero_noise_init: exact pixels and priors; initial poses perturbed by
           0.3 m / 0.02 deg and initial points by 0.1 m.
    fixed: iterable of camera indices held fixed (their true pose is the
           initial value).
    priors: False switches the GNSS/IMU prior terms off (sigma = 0 means off).
    """
    C, yaw, strip = strip_layout(n_strips, cams_per_strip)
    if n_cams is not None:  # uneven strips: drop the last images in time order
        C, yaw, strip = C[:n_cams], yaw[:n_cams], strip[:n_cams]
    nc = len(C)
    jitter = Rotation.from_rotvec(rng.normal(0.0, ATTITUDE_JITTER_RAD, (nc, 3))).as_matrix()
    R_true = np.stack([nadir_rotation(yaw[k]) @ jitter[k] for k in range(nc)])
    T_true = C + np.column_stack([rng.normal(0, 0.5, nc), rng.normal(0, 0.5, nc), rng.normal(0, 1.0, nc)])
    intr = np.zeros((nc, 7))
    intr[:, 0] = FOCAL_PX
    intr[:, 1] = SENSOR_W / 2.0
    intr[:, 2] = SENSOR_H / 2.0
    intr[:, 3:7] = rng.normal(0.0, DIST_SIGMA, (nc, 4))

    pad = 10.0
    bbox = (T_true[:, 0].min() - FOOT_ACROSS_M / 2 - pad, T_true[:, 0].max() + FOOT_ACROSS_M / 2 + pad,
            T_true[:, 1].min() - FOOT_ACROSS_M / 2 - pad, T_true[:, 1].max() + FOOT_ACROSS_M / 2 + pad)
    buildings = make_buildings(rng, *bbox)
    if layout == "patches":
        X_true = _patch_points(rng, n_points, per_patch, bbox, buildings, intr, R_true, T_true)
    else:
        X_true = _sample_points(rng, n_points, bbox, buildings, intr, R_true, T_true)
    npt = len(X_true)

    vis, uv_true = visibility_matrix(intr, R_true, T_true, X_true)
    if track is not None:
        p, lmax = track
        nvis = vis.sum(1)
        L = 2 + (rng.geometric(p, npt) - 1)
        L = np.minimum(L, np.minimum(nvis, lmax))
        keys = np.where(vis, rng.random(vis.shape), np.inf)
        order = np.argsort(keys, axis=1)
        sel = np.zeros_like(vis)
        rows = np.repeat(np.arange(npt), L)
        cols = order[rows, np.concatenate([np.arange(l) for l in L])]
        sel[rows, cols] = True
        vis = sel
    obs_pt, obs_cam = np.nonzero(vis)          # row-major: sorted by (point, camera)
    obs_pt = obs_pt.astype(np.int32)
    obs_cam = obs_cam.astype(np.int32)
    uv_exact = uv_true[obs_pt, obs_cam]
    n_obs = len(obs_pt)

    outlier = np.zeros(n_obs, dtype=bool)
    if noise and not zero_noise_init:
        obs_uv = uv_exact + rng.normal(0.0, SIGMA_PX, (n_obs, 2))
        outlier = rng.random(n_obs) < OUTLIER_FRAC
        obs_uv[outlier] = uv_exact[outlier] + rng.uniform(-OUTLIER_HALF_WIDTH_PX, OUTLIER_HALF_WIDTH_PX,
                                                         (int(outlier.sum()), 2))
        T_prior = T_true + rng.normal(0.0, SIGMA_GNSS_M, (nc, 3))
        R_prior = np.stack([R_true[k] @ Rotation.from_rotvec(rng.normal(0.0, SIGMA_IMU_RAD, 3)).as_matrix()
                            for k in range(nc)])
        R0, T0 = R_prior.copy(), T_prior.copy()
        X0 = X_true + rng.normal(0.0, POINT_INIT_SIGMA_M, (npt, 3))
    else:
        obs_uv = uv_exact.copy()
        T_prior, R_prior = T_true.copy(), R_true.copy()
        if zero_noise_init:
            dirs = rng.normal(size=(nc, 3))
            dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
            T0 = T_true + 0.3 * dirs
            ax = rng.normal(size=(nc, 3))
            ax /= np.linalg.norm(ax, axis=1, keepdims=True)
            R0 = np.stack([R_true[k] @ Rotation.from_rotvec(math.radians(0.02) * ax[k]).as_matrix()
                           for k in range(nc)])
            X0 = X_true + rng.normal(0.0, 0.1, (npt, 3))
        else:
            R0, T0, X0 = R_true.copy(), T_true.copy(), X_true.copy()

    fixed_mask = np.zeros(nc, dtype=np.uint8)
    if fixed is not None:
        for k in fixed:
            fixed_mask[k] = 1
            R0[k], T0[k] = R_true[k], T_true[k]

    return dict(
        n_cams=nc, n_pts=npt, n_obs=n_obs,
        intr=intr, R0=R0.reshape(nc, 9).copy(), T0=T0.copy(), X0=X0.copy(),
        R_prior=R_prior.reshape(nc, 9).copy(), T_prior=T_prior.copy(),
        R_true=R_true.reshape(nc, 9).copy(), T_true=T_true.copy(), X_true=X_true.copy(),
        fixed=fixed_mask, obs_cam=obs_cam, obs_pt=obs_pt, obs_uv=obs_uv, outlier=outlier,
        sigma_px=SIGMA_PX, huber_delta=HUBER_DELTA_PX,
        sigma_gnss=SIGMA_GNSS_M if priors else 0.0, sigma_imu=SIGMA_IMU_RAD if priors else 0.0,
        strip=strip, origin=np.zeros(3), buildings=buildings, bbox=np.array(bbox, dtype=np.float64),
    )


# --------------------------------------------------------------------------
# the paper-shaped workloads
# --------------------------------------------------------------------------
ITERS = {"c1": 10, "c2": 20, "c3": 20, "c5": 15}


def cluster_c1(replica=0, **kw):
    """Plain FP64 single cluster: 2 strips x 3 images, 2,000 points, all
    visible projections observed (~8,000 observations)."""
    return make_cluster(rng_for(1, replica), 2, 3, 2000, **kw)


def cluster_c2(replica=0, **kw):
    """Paper-scale cluster: 3 strips x 8 images, 40,000 points in 2.88 m
    ground patches of 30 points, every image containing a point observes it."""
    return make_cluster(rng_for(2, replica), 3, 8, 40000, layout="patches", per_patch=30, **kw)


def batch_c3_specs(replica=0, n_clusters=256, scale=1.0):
    """Per-cluster parameters of the batched workload: U{8..32} images in 2-3
    strips, U[5k, 60k] points (times `scale`), and a sub-seed."""
    rng = rng_for(3, replica)
    specs = []
    for _ in range(n_clusters):
        nc = int(rng.integers(8, 33))
        ns = int(rng.integers(2, 4))
        npt = max(16, int(round(rng.uniform(5000, 60000) * scale)))
        specs.append((nc, ns, npt, int(rng.integers(1 << 62))))
    return specs


def cluster_from_spec(spec):
    """One batched-workload cluster: track length 2 + Geometric(0.5) failures
    truncated at min(8, images containing the point)."""
    nc, ns, npt, seed = spec
    sub = np.random.Generator(np.random.PCG64(seed))
    return make_cluster(sub, ns, -(-nc // ns), npt, track=(0.5, 8), n_cams=nc)


def batch_c3(replica=0, n_clusters=256, scale=1.0, pool=None):
    """Batched workload of 256 uneven clusters (see batch_c3_specs)."""
    specs = batch_c3_specs(replica, n_clusters, scale)
    if pool is not None:
        return list(pool.map(cluster_from_spec, specs))
    return [cluster_from_spec(s) for s in specs]


def cluster_c5(replica=0, n_points=2_000_000, **kw):
    """Large block: 10 strips x 40 images, 2 M points, track length
    2 + Geometric(1/4) failures truncated at 16 (mean ~5)."""
    return make_cluster(rng_for(5, replica), 10, 40, n_points, track=(0.25, 16), **kw)


def tiny_cluster(seed, n_strips=1, cams_per_strip=3, n_points=12, **kw):
    """A small cluster for brute-force checks."""
    return make_cluster(np.random.Generator(np.random.PCG64(seed)), n_strips, cams_per_strip, n_points, **kw)


# --------------------------------------------------------------------------
# accuracy summaries (plain statistics of arrays; no BA arithmetic)
# --------------------------------------------------------------------------
def centre_error(T_est, T_ref):
    return float(np.max(np.linalg.norm(np.asarray(T_est) - np.asarray(T_ref), axis=1)))


# --------------------------------------------------------------------------
# flight timing (Eq. 1, Sec. 1): the interval between exposures is the time
# budget for processing one image pair
# --------------------------------------------------------------------------
def image_interval_s(footprint_along_m, overlap_pct, velocity_mps):
    """t = h_im (1 - beta/100) / v  (Eq. 1)."""
    return footprint_along_m * (1.0 - overlap_pct / 100.0) / velocity_mps


# --------------------------------------------------------------------------
# serving workload: long flights cut into sliding windows (Sec. 3.2, cluster
# transition: the last 25 % of a window is reused by the next one, the first
# half of that overlap held fixed)
# --------------------------------------------------------------------------
def flight(seed, n_strips=3, per_strip=40, pts_per_cam=1667):
    """One flight: serpentine strips of images over terrain, points at the
    c2 density (1,667 per image), every image containing a point observes it."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_strips * per_strip
    return make_cluster(rng, n_strips, per_strip, pts_per_cam * n)


def dsm_raster(scene, spacing=2.0):
    """The scene's surface model (terrain plus buildings) sampled on a regular
    grid over its bounding box, as a DSM raster: heights h[iy, ix] at
    (x0 + ix * dx, y0 + iy * dy).  Scene data only (no method arithmetic)."""
    xmin, xmax, ymin, ymax = scene["bbox"]
    nx = int(math.ceil((xmax - xmin) / spacing)) + 1
    ny = int(math.ceil((ymax - ymin) / spacing)) + 1
    xs = xmin + spacing * np.arange(nx)
    ys = ymin + spacing * np.arange(ny)
    X, Y = np.meshgrid(xs, ys)
    h = terrain_height(X.ravel(), Y.ravel(), scene["buildings"]).reshape(ny, nx)
    return dict(h=np.ascontiguousarray(h, dtype=np.float64), x0=float(xmin), y0=float(ymin), dx=float(spacing),
                dy=float(spacing))


def window_plan(seed, n_images, m_lo=12, m_hi=32, overlap=0.25):
    """Window boundaries over a flight's images in time order: sizes
    M ~ U{m_lo..m_hi}; each window after the first starts with the last
    ceil(overlap * M_prev) images of the previous one, and the first half of
    those (ceil) are held fixed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out, start, prev = [], 0, None
    while True:
        m = int(rng.integers(m_lo, m_hi + 1))
        if prev is not None:
            n_ov = int(math.ceil(overlap * (prev[1] - prev[0])))
            start = prev[1] - n_ov
            n_fix = int(math.ceil(n_ov / 2))
        else:
            n_fix = 0
        end = min(start + m, n_images)
        if end - start < 4 or (prev is not None and end <= prev[1]):
            break
        out.append((start, end, n_fix))
        prev = (start, end)
        if end == n_images:
            break
    return out


def window_cluster(fl, start, end, n_fix):
    """The local-BA cluster of images [start, end) of a flight, with its first
    n_fix images fixed; points seen by >= 2 of its images.  Returns the cluster
    and the flight indices of its cameras and points."""
    cams = np.arange(start, end)
    obs_sel = (fl["obs_cam"] >= start) & (fl["obs_cam"] < end)
    pc = np.bincount(fl["obs_pt"][obs_sel], minlength=fl["n_pts"])
    pts = np.nonzero(pc >= 2)[0]
    pmap = -np.ones(fl["n_pts"], dtype=np.int64)
    pmap[pts] = np.arange(len(pts))
    keep = obs_sel & (pmap[fl["obs_pt"]] >= 0)
    nc = end - start
    c = dict(
        n_cams=nc, n_pts=len(pts), n_obs=int(keep.sum()),
        intr=fl["intr"][cams], R0=fl["R0"][cams].copy(), T0=fl["T0"][cams].copy(), X0=fl["X0"][pts].copy(),
        R_prior=fl["R_prior"][cams], T_prior=fl["T_prior"][cams],
        R_true=fl["R_true"][cams], T_true=fl["T_true"][cams], X_true=fl["X_true"][pts],
        fixed=np.zeros(nc, dtype=np.uint8),
        obs_cam=(fl["obs_cam"][keep] - start).astype(np.int32), obs_pt=pmap[fl["obs_pt"][keep]].astype(np.int32),
        obs_uv=fl["obs_uv"][keep], outlier=fl["outlier"][keep],
        sigma_px=fl["sigma_px"], huber_delta=fl["huber_delta"], sigma_gnss=fl["sigma_gnss"],
        sigma_imu=fl["sigma_imu"], origin=fl["origin"])
    c["fixed"][:n_fix] = 1
    return c, cams, pts


def warm_maps(prev_cams, prev_pts, cams, pts):
    """Index of each camera / point of a window in the previous window, or -1."""
    pc = {int(v): i for i, v in enumerate(prev_cams)}
    pp = np.full(int(max(prev_pts.max() if len(prev_pts) else 0, pts.max() if len(pts) else 0)) + 1, -1, np.int64)
    pp[prev_pts] = np.arange(len(prev_pts))
    cam_map = np.array([pc.get(int(v), -1) for v in cams], dtype=np.int32)
    pt_map = pp[pts].astype(np.int32)
    return cam_map, pt_map
