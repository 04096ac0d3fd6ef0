"""Plain FP64 CPU oracle for the local bundle-adjustment LM iteration.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  The CUDA library never
loads it and shares no code with it.

The arithmetic lives in ``ba_oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that x86 and Arm hosts round identically); this
module only builds it and marshals numpy arrays through ctypes.

Functions and the passages they follow:
  project         Eq. 5 (Sec. 3.2), pi from Sec. 3.1, Brown distortion terms
  huber_rho/weight  rho of Eq. 6 on the squared 2-D norm (Huber)
  linearize_obs   Eq. 7 residual, whitened and robust-weighted, with analytic
                  Jacobians for the right perturbation [dtheta, dT] and dX
  linearize_prior GNSS/IMU priors on the initial values of Sec. 3.2
  cost            Eq. 7 plus the prior terms, halved
  solve_damped    Levenberg-Marquardt step by the Schur complement
  lm_step/lm_run  LM with Nielsen's damping update
  patch_transfer_poses   Eq. 3 (Sec. 3.1): patch centres through the poses
  patch_transfer_planar  Eq. 4 (Sec. 3.1): planar footprint-based transfer
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ba_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbaoracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_cams", ctypes.c_int), ("n_pts", ctypes.c_int), ("n_obs", ctypes.c_int),
        ("intr", _dp), ("R_prior", _dp), ("T_prior", _dp),
        ("fixed", ctypes.POINTER(ctypes.c_ubyte)),
        ("obs_cam", _ip), ("obs_pt", _ip), ("obs_uv", _dp),
        ("sigma_px", ctypes.c_double), ("huber_delta", ctypes.c_double),
        ("sigma_gnss", ctypes.c_double), ("sigma_imu", ctypes.c_double),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [
        ("accepted", ctypes.c_int), ("status", ctypes.c_int),
        ("F", ctypes.c_double), ("F_new", ctypes.c_double), ("pred", ctypes.c_double),
        ("gain", ctypes.c_double), ("mu_used", ctypes.c_double), ("mu", ctypes.c_double),
        ("nu", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile ba_oracle.c into _build/libbaoracle.so (plain gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ba_oracle.h"))):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_huber_rho.restype = ctypes.c_double
            L.orc_huber_weight.restype = ctypes.c_double
            L.orc_cost.restype = ctypes.c_double
            L.orc_dsm_height.restype = ctypes.c_double
            L.orc_quad_overlap.restype = ctypes.c_double
            L.orc_quad_area.restype = ctypes.c_double
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


class Problem:
    """Immutable problem data (intrinsics, priors, observations) held for the
    lifetime of the ctypes struct that points into it."""

    def __init__(self, c):
        self.n_cams, self.n_pts, self.n_obs = int(c["n_cams"]), int(c["n_pts"]), int(c["n_obs"])
        self.intr = _f64(c["intr"], (self.n_cams, 7))
        self.R_prior = _f64(c["R_prior"], (self.n_cams, 9))
        self.T_prior = _f64(c["T_prior"], (self.n_cams, 3))
        self.fixed = np.ascontiguousarray(c["fixed"], dtype=np.uint8)
        self.obs_cam = np.ascontiguousarray(c["obs_cam"], dtype=np.int32)
        self.obs_pt = np.ascontiguousarray(c["obs_pt"], dtype=np.int32)
        self.obs_uv = _f64(c["obs_uv"], (self.n_obs, 2))
        self.s = _Problem(self.n_cams, self.n_pts, self.n_obs, _d(self.intr), _d(self.R_prior), _d(self.T_prior),
                          self.fixed.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                          self.obs_cam.ctypes.data_as(_ip), self.obs_pt.ctypes.data_as(_ip), _d(self.obs_uv),
                          float(c["sigma_px"]), float(c["huber_delta"]), float(c["sigma_gnss"]),
                          float(c["sigma_imu"]))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def so3_exp(w):
    R = np.zeros(9)
    lib().orc_so3_exp(_d(_f64(w)), _d(R))
    return R.reshape(3, 3)


def so3_log(R):
    w = np.zeros(3)
    lib().orc_so3_log(_d(_f64(R, (9,))), _d(w))
    return w


def so3_jr_inv(w):
    J = np.zeros(9)
    lib().orc_so3_jr_inv(_d(_f64(w)), _d(J))
    return J.reshape(3, 3)


class _Dsm(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("h", _dp)]


class Dsm:
    """A DSM raster (dict h[ny, nx], x0, y0, dx, dy) held for the ctypes struct."""

    def __init__(self, d):
        self.h = _f64(d["h"])
        ny, nx = self.h.shape
        self.s = _Dsm(nx, ny, float(d["x0"]), float(d["y0"]), float(d["dx"]), float(d["dy"]), _d(self.h))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def dsm_height(dsm: Dsm, x, y):
    return lib().orc_dsm_height(dsm.ref, ctypes.c_double(x), ctypes.c_double(y))


def footprint(intr, width, height, R, T, dsm: Dsm):
    """Ground points of an image's four corners on the DSM, (4, 3); None for
    a ray that does not point down."""
    out = np.zeros(12)
    st = lib().orc_footprint(_d(_f64(intr, (7,))), ctypes.c_double(width), ctypes.c_double(height),
                             _d(_f64(R, (9,))), _d(_f64(T, (3,))), dsm.ref, _d(out))
    return None if st != 0 else out.reshape(4, 3)


def quad_overlap(qa, qb):
    """Area of the intersection of two convex footprints (ground plane)."""
    return lib().orc_quad_overlap(_d(_f64(qa, (12,))), _d(_f64(qb, (12,))))


def quad_area(q):
    return lib().orc_quad_area(_d(_f64(q, (12,))))


def transition(R_old, T_old, w_old, R_new, T_new, w_new):
    """Eq. 8: weighted average of an overlap image's poses from the previous
    and the new cluster (weights = its observations in each)."""
    R, T = np.zeros(9), np.zeros(3)
    lib().orc_transition(_d(_f64(R_old, (9,))), _d(_f64(T_old, (3,))), ctypes.c_double(w_old),
                         _d(_f64(R_new, (9,))), _d(_f64(T_new, (3,))), ctypes.c_double(w_new), _d(R), _d(T))
    return R.reshape(3, 3), T


def patch_transfer_poses(intr0, R0, T0, p0, lam, intrk, Rk, Tk, width=None, height=None):
    """Eq. 3: patch centres p0 (n, 2) of image 0 moved to image k at the
    nominal depth lam; returns (pk (n, 2), inside (n,) bool): inside = in
    front of image k and, when width/height are given, within the frame."""
    p0 = np.ascontiguousarray(np.asarray(p0, dtype=np.float64).reshape(-1, 2))
    out = np.zeros_like(p0)
    inside = np.zeros(len(p0), dtype=bool)
    L = lib()
    a = [_d(_f64(x, (s,))) for x, s in ((intr0, 7), (R0, 9), (T0, 3), (intrk, 7), (Rk, 9), (Tk, 3))]
    for i in range(len(p0)):
        row = np.zeros(2)
        front = L.orc_patch_transfer_poses(a[0], a[1], a[2], _d(p0[i]), ctypes.c_double(lam), a[3], a[4], a[5], _d(row))
        out[i] = row if front else np.nan
        ok = bool(front)
        if ok and width is not None:
            ok = 0.0 <= row[0] < width and 0.0 <= row[1] < height
        inside[i] = ok
    return out, inside


def patch_transfer_planar(q0, c, theta, g0, gk):
    """Eq. 4: patch centres q0 (n, 2) (ground plane) moved to image k."""
    q0 = np.ascontiguousarray(np.asarray(q0, dtype=np.float64).reshape(-1, 2))
    out = np.zeros_like(q0)
    L = lib()
    cc, a0, ak = _f64(c, (2,)), _f64(g0, (2,)), _f64(gk, (2,))
    for i in range(len(q0)):
        row = np.zeros(2)
        L.orc_patch_transfer_planar(_d(q0[i]), _d(cc), ctypes.c_double(theta), _d(a0), _d(ak), _d(row))
        out[i] = row
    return out


def project(intr, R, T, X):
    uv = np.zeros(2)
    ok = lib().orc_project(_d(_f64(intr)), _d(_f64(R, (9,))), _d(_f64(T)), _d(_f64(X)), _d(uv))
    return uv, bool(ok)


def huber_rho(s, delta):
    return lib().orc_huber_rho(ctypes.c_double(s), ctypes.c_double(delta))


def huber_weight(s, delta):
    return lib().orc_huber_weight(ctypes.c_double(s), ctypes.c_double(delta))


def linearize_obs(P: Problem, R, T, X, i):
    r, Jc, Jp, s = np.zeros(2), np.zeros(12), np.zeros(6), ctypes.c_double()
    R, T, X = _f64(R, (-1,)), _f64(T, (-1,)), _f64(X, (-1,))
    ok = lib().orc_linearize_obs(P.ref, _d(R), _d(T), _d(X), int(i), _d(r), _d(Jc), _d(Jp), ctypes.byref(s))
    return r, Jc.reshape(2, 6), Jp.reshape(2, 3), s.value, bool(ok)


def linearize_prior(P: Problem, R, T, k):
    r, J = np.zeros(6), np.zeros(36)
    lib().orc_linearize_prior(P.ref, _d(_f64(R, (-1,))), _d(_f64(T, (-1,))), int(k), _d(r), _d(J))
    return r, J.reshape(6, 6)


def cost(P: Problem, R, T, X):
    return lib().orc_cost(P.ref, _d(_f64(R, (-1,))), _d(_f64(T, (-1,))), _d(_f64(X, (-1,))))


def solve_damped(P: Problem, R, T, X, mu):
    dc, dp = np.zeros(6 * P.n_cams), np.zeros(3 * P.n_pts)
    gc, gp = np.zeros(6 * P.n_cams), np.zeros(3 * P.n_pts)
    Dc, Dp = np.zeros(6 * P.n_cams), np.zeros(3 * P.n_pts)
    st = lib().orc_solve_damped(P.ref, _d(_f64(R, (-1,))), _d(_f64(T, (-1,))), _d(_f64(X, (-1,))),
                                ctypes.c_double(mu), _d(dc), _d(dp), _d(gc), _d(gp), _d(Dc), _d(Dp))
    return dict(status=st, dc=dc.reshape(-1, 6), dp=dp.reshape(-1, 3), gc=gc.reshape(-1, 6),
                gp=gp.reshape(-1, 3), Dc=Dc.reshape(-1, 6), Dp=Dp.reshape(-1, 3))


def apply_step(P: Problem, R, T, X, dc, dp):
    Rn, Tn, Xn = np.zeros(9 * P.n_cams), np.zeros(3 * P.n_cams), np.zeros(3 * P.n_pts)
    lib().orc_apply_step(P.ref, _d(_f64(R, (-1,))), _d(_f64(T, (-1,))), _d(_f64(X, (-1,))),
                         _d(_f64(dc, (-1,))), _d(_f64(dp, (-1,))), _d(Rn), _d(Tn), _d(Xn))
    return Rn.reshape(-1, 9), Tn.reshape(-1, 3), Xn.reshape(-1, 3)


class State:
    """Mutable LM state (poses, points, damping) in FP64."""

    def __init__(self, c, mu0=1e-4):
        self.R = _f64(c["R0"], (-1, 9)).copy()
        self.T = _f64(c["T0"], (-1, 3)).copy()
        self.X = _f64(c["X0"], (-1, 3)).copy()
        self.mu = ctypes.c_double(mu0)
        self.nu = ctypes.c_double(2.0)


def lm_step(P: Problem, S: State):
    info = StepInfo()
    lib().orc_lm_step(P.ref, _d(S.R), _d(S.T), _d(S.X), ctypes.byref(S.mu), ctypes.byref(S.nu), ctypes.byref(info))
    return info.as_dict()


def lm_run(P: Problem, S: State, iters):
    trace = (StepInfo * max(1, iters))()
    lib().orc_lm_run(P.ref, _d(S.R), _d(S.T), _d(S.X), int(iters), ctypes.c_double(S.mu.value), trace)
    # lm_run starts from S.mu with nu = 2; leave the final damping in S
    if iters:
        S.mu = ctypes.c_double(trace[iters - 1].mu)
        S.nu = ctypes.c_double(trace[iters - 1].nu)
    return [trace[i].as_dict() for i in range(iters)]


def residual_stats(P: Problem, R, T, X, mask=None):
    """Reprojection error norms ||pi(...) - p|| per observation (pixels)."""
    R, T, X = _f64(R, (-1, 9)), _f64(T, (-1, 3)), _f64(X, (-1, 3))
    e = np.zeros(P.n_obs)
    for i in range(P.n_obs):
        k, j = P.obs_cam[i], P.obs_pt[i]
        uv, _ = project(P.intr[k], R[k], T[k], X[j])
        e[i] = np.hypot(*(uv - P.obs_uv[i]))
    return e
