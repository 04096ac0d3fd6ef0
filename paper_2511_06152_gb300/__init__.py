"""Python binding of the GB300 local bundle-adjustment library (include/ba.h).

Argument marshalling only: every step of the LM iteration runs in the CUDA
kernels of ``_build/libba_gb300.so``.  There is no CPU fallback; importing
``lib()`` on a machine where the library cannot be loaded raises.

The functions keep the C names (``ba_init``, ``ba_create_cluster``,
``ba_run`` ...) and take/return numpy arrays or ctypes structs.  ``Context``
is a small convenience wrapper that owns a ``ba_ctx``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

BA_OK = 0
BA_PENDING = 1
BA_ERR_INVALID = -1
BA_ERR_BUDGET = -2
BA_ERR_NOT_PD = -3
BA_ERR_TIMEOUT = -4
BA_ERR_CUDA = -5
BA_ERR_NOT_FOUND = -6
BA_FP64 = 0
BA_MIXED = 1
BA_PTR_HOST = 0
BA_PTR_DEVICE = 1
BA_FLAG_KERNEL_TIMING = 1
BA_FLAG_INJECT_COPY_TIMEOUT = 2  # failure injection for tests: the staged-copy wait expires
BA_FLAG_BIG_FP64_FACTOR = 4      # large reduced systems: binary64 CUDA-core factor instead of the tensor cores
BA_FLAG_SMALL_DF_FACTOR = 8      # BA_FP64: small reduced systems factored in double-float, as in BA_MIXED
KERNEL_KINDS = ["lin_schur", "partial_reduce", "factor", "backsub_cost", "lm_update", "cost_tiles", "cost_init",
                "other"]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class ba_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("stream", ctypes.c_void_p), ("hbm_budget_bytes", ctypes.c_uint64),
                ("precision", ctypes.c_int32), ("n_slots", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("tune_table", ctypes.c_char_p)]


TUNE_KEYS = ("chunk_tiles", "lin_ctas_per_sm", "back_ctas_per_sm", "factor_nb", "factor_threads", "big_panel_w",
             "batch_chains")
# the committed tuning table that Context hands to ba_init (entries per GPU and precision)
TUNE_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.txt")


class ba_tune(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in TUNE_KEYS] + [("ms_default", ctypes.c_double),
                                                           ("ms_tuned", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        for k, _ in cls._fields_:
            if k in d:
                setattr(t, k, d[k])
        return t


def tune_table_line(gpu_name, sm_count, precision, tune):
    """One line of the tuning table read by ba_tune_table_lookup (format in ba.h)."""
    prec = "mixed" if precision == BA_MIXED else "fp64"
    kv = " ".join(f"{k}={int(tune[k])}" for k in TUNE_KEYS)
    ms = f" ms_default={tune.get('ms_default', 0.0):.4f} ms_tuned={tune.get('ms_tuned', 0.0):.4f}"
    return f"{gpu_name.replace(' ', '_')} {int(sm_count)} {prec} {kv}{ms}"


def tune_table_lookup(path, gpu_name, sm_count, precision):
    """ba_tune_table_lookup (host only): the table's entry as a dict, or None."""
    t = ba_tune()
    st = lib().ba_tune_table_lookup(path.encode(), gpu_name.encode(), int(sm_count), int(precision), ctypes.byref(t))
    if st == BA_ERR_NOT_FOUND:
        return None
    _check(st, None, "ba_tune_table_lookup")
    return t.as_dict()


class ba_cluster_desc(ctypes.Structure):
    _fields_ = [("n_cams", ctypes.c_int32), ("n_pts", ctypes.c_int32), ("n_obs", ctypes.c_int32),
                ("ptr_kind", ctypes.c_int32),
                ("intr", _dp), ("R", _dp), ("T", _dp), ("X", _dp), ("R_prior", _dp), ("T_prior", _dp),
                ("fixed", _u8p), ("obs_cam", _ip), ("obs_pt", _ip), ("obs_uv", _dp),
                ("sigma_px", ctypes.c_double), ("huber_delta_px", ctypes.c_double),
                ("sigma_gnss_m", ctypes.c_double), ("sigma_imu_rad", ctypes.c_double), ("mu0", ctypes.c_double),
                ("warm_from", ctypes.c_uint64), ("warm_cam_map", _ip), ("warm_pt_map", _ip)]


class ba_lin_info(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_double), ("grad_inf", ctypes.c_double), ("n_free", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ba_step_info(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int32), ("status", ctypes.c_int32), ("F_before", ctypes.c_double),
                ("F_after", ctypes.c_double), ("predicted", ctypes.c_double), ("gain", ctypes.c_double),
                ("mu_used", ctypes.c_double), ("mu", ctypes.c_double), ("nu", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ba_solve_opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ftol", ctypes.c_double)]


class ba_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("initial_cost", ctypes.c_double), ("final_cost", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ba_cluster_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("n_cams", "n_free", "n_pts", "n_obs", "n_tiles", "n_chunks",
                                             "n_cam_slots", "n_pair_slots", "n_pairs", "reserved")] + \
               [(k, ctypes.c_int64) for k in ("n_free_obs", "n_pair_entries", "arena_bytes")] + \
               [(k, ctypes.c_double) for k in ("presort_ms", "upload_ms")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class ba_presort_info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in ("n_free", "n_tiles", "n_chunks", "n_pairs", "n_cam_jobs",
                                             "n_pair_jobs", "max_lanes", "fallback_chunks", "tiles_per_chunk",
                                             "checks_failed")] + \
               [("n_free_obs", ctypes.c_int64), ("n_pair_entries", ctypes.c_int64), ("digest", ctypes.c_uint64),
                ("message", ctypes.c_char * 128)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["message"] = self.message.decode()
        return d


class ba_dsm(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("h", ctypes.POINTER(ctypes.c_double))]


EXPORTS = ["ba_init", "ba_create_cluster", "ba_linearize", "ba_solve_step", "ba_run", "ba_solve_batch", "ba_reset",
           "ba_reset_batch", "ba_submit", "ba_poll", "ba_get_state", "ba_get_state_batch", "ba_reprojection_errors",
           "ba_memory_in_use",
           "ba_launch_count", "ba_kernel_stats", "ba_cost_noalloc", "ba_warm_start", "ba_transition", "ba_footprints", "ba_footprint_overlaps", "ba_patch_transfer_poses", "ba_patch_transfer_planar", "ba_get_cluster_info", "ba_presort_host", "ba_destroy_cluster", "ba_shutdown",
           "ba_get_tune", "ba_set_tune", "ba_autotune", "ba_tune_table_lookup", "ba_probe_fp32_fma",
           "ba_status_string", "ba_last_error"]

_lib = None
_lock = threading.Lock()


def library_path(build: bool = True) -> str:
    return _build.build() if build else _build.LIB


def lib(build: bool = True):
    """Load the shared library (building it first if stale)."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(library_path(build))
            vp = ctypes.c_void_p
            u64 = ctypes.c_uint64
            L.ba_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ba_config)]
            L.ba_create_cluster.argtypes = [vp, ctypes.POINTER(ba_cluster_desc), ctypes.POINTER(u64)]
            L.ba_linearize.argtypes = [vp, u64, ctypes.POINTER(ba_lin_info)]
            L.ba_solve_step.argtypes = [vp, u64, ctypes.POINTER(ba_step_info)]
            L.ba_run.argtypes = [vp, u64, ctypes.c_int32, ctypes.POINTER(ba_step_info)]
            L.ba_solve_batch.argtypes = [vp, ctypes.POINTER(u64), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ba_result), ctypes.POINTER(ba_step_info)]
            L.ba_reset.argtypes = [vp, u64]
            L.ba_reset_batch.argtypes = [vp, ctypes.POINTER(u64), ctypes.c_int32]
            L.ba_launch_count.argtypes = [vp, ctypes.POINTER(u64)]
            L.ba_kernel_stats.argtypes = [vp, _dp, ctypes.POINTER(u64), ctypes.c_int32, ctypes.c_int32]
            L.ba_cost_noalloc.argtypes = [ctypes.POINTER(ba_cluster_desc), vp, _dp]
            L.ba_warm_start.argtypes = [vp, u64, u64, _ip, _ip]
            L.ba_transition.argtypes = [vp, u64, u64, _ip]
            L.ba_footprints.argtypes = [vp, ctypes.c_int32, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp,
                                        ctypes.POINTER(ba_dsm), _dp]
            L.ba_footprint_overlaps.argtypes = [vp, ctypes.c_int32, _dp, ctypes.c_int32, _dp, _dp]
            L.ba_patch_transfer_poses.argtypes = [vp, ctypes.c_int32, _dp, _dp, _dp, _dp, ctypes.c_double,
                                                  ctypes.c_int32, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                                  _dp, ctypes.POINTER(ctypes.c_uint8)]
            L.ba_patch_transfer_planar.argtypes = [vp, ctypes.c_int32, _dp, _dp, _dp, ctypes.c_int32, _dp, _dp, _dp]
            L.ba_submit.argtypes = [vp, u64, ctypes.POINTER(ba_solve_opts), ctypes.POINTER(u64)]
            L.ba_poll.argtypes = [vp, u64, ctypes.POINTER(ba_result)]
            L.ba_get_state.argtypes = [vp, u64, _dp, _dp, _dp, ctypes.c_int32]
            _pp = ctypes.POINTER(ctypes.c_void_p)
            L.ba_get_state_batch.argtypes = [vp, ctypes.POINTER(u64), ctypes.c_int32, _pp, _pp, _pp]
            L.ba_reprojection_errors.argtypes = [vp, u64, _dp]
            L.ba_memory_in_use.argtypes = [vp, ctypes.POINTER(u64)]
            L.ba_get_cluster_info.argtypes = [vp, u64, ctypes.POINTER(ba_cluster_info)]
            L.ba_presort_host.argtypes = [ctypes.POINTER(ba_cluster_desc), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ba_presort_info)]
            L.ba_get_tune.argtypes = [vp, ctypes.POINTER(ba_tune)]
            L.ba_set_tune.argtypes = [vp, ctypes.POINTER(ba_tune)]
            L.ba_autotune.argtypes = [vp, ctypes.POINTER(ba_cluster_desc), ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ba_tune)]
            L.ba_tune_table_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ba_tune)]
            L.ba_probe_fp32_fma.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, _dp, _dp]
            L.ba_destroy_cluster.argtypes = [vp, u64]
            L.ba_shutdown.argtypes = [vp]
            L.ba_status_string.argtypes = [ctypes.c_int32]
            L.ba_status_string.restype = ctypes.c_char_p
            L.ba_last_error.argtypes = [vp]
            L.ba_last_error.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("ba_status_string", "ba_last_error"):
                    getattr(L, name).restype = ctypes.c_int32
            _lib = L
    return _lib


class BAError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _check(st, ctx=None, what=""):
    if st not in (BA_OK, BA_PENDING):
        L = lib()
        detail = L.ba_last_error(ctx).decode() if ctx else ""
        raise BAError(st, f"{what}: {L.ba_status_string(st).decode()} {detail}".strip())
    return st


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _d(a):
    return a.ctypes.data_as(_dp)


def make_desc(scene, keep):
    """ba_cluster_desc for a scene dict (host arrays); `keep` holds the arrays alive."""
    nc, npt, no = int(scene["n_cams"]), int(scene["n_pts"]), int(scene["n_obs"])
    arrs = dict(
        intr=_f64(scene["intr"], (nc, 7)), R=_f64(scene["R0"], (nc, 9)), T=_f64(scene["T0"], (nc, 3)),
        X=_f64(scene["X0"], (npt, 3)), R_prior=_f64(scene["R_prior"], (nc, 9)), T_prior=_f64(scene["T_prior"], (nc, 3)),
        fixed=np.ascontiguousarray(scene.get("fixed", np.zeros(nc)), dtype=np.uint8),
        obs_cam=np.ascontiguousarray(scene["obs_cam"], dtype=np.int32),
        obs_pt=np.ascontiguousarray(scene["obs_pt"], dtype=np.int32),
        obs_uv=_f64(scene["obs_uv"], (no, 2)))
    keep.append(arrs)
    d = ba_cluster_desc()
    d.n_cams, d.n_pts, d.n_obs, d.ptr_kind = nc, npt, no, BA_PTR_HOST
    for k in ("intr", "R", "T", "X", "R_prior", "T_prior", "obs_uv"):
        setattr(d, k, _d(arrs[k]))
    d.fixed = arrs["fixed"].ctypes.data_as(_u8p)
    d.obs_cam = arrs["obs_cam"].ctypes.data_as(_ip)
    d.obs_pt = arrs["obs_pt"].ctypes.data_as(_ip)
    d.sigma_px = float(scene["sigma_px"])
    d.huber_delta_px = float(scene["huber_delta"])
    d.sigma_gnss_m = float(scene["sigma_gnss"])
    d.sigma_imu_rad = float(scene["sigma_imu"])
    d.mu0 = float(scene.get("mu0", 1e-4))
    d.warm_from = 0
    return d


def presort_host(scene, precision=BA_MIXED, threads=0):
    """ba_presort_host: the creation presort of a host-array scene on the host
    alone (no GPU), its table sizes and the result of the tables' self-check."""
    keep = []
    d = make_desc(scene, keep)
    out = ba_presort_info()
    st = lib().ba_presort_host(ctypes.byref(d), precision, threads, ctypes.byref(out))
    if st != BA_OK:
        raise BAError(st, f"ba_presort_host: {lib().ba_status_string(st).decode()} {out.message.decode()}".strip())
    return out.as_dict()


class Context:
    """Owns one ba_ctx on one device and stream."""

    def __init__(self, device=0, precision=BA_FP64, stream=None, hbm_budget_bytes=0, n_slots=0, refine_steps=-1,
                 flags=0, tune_table=TUNE_TABLE):
        self.L = lib()
        cfg = ba_config(device=device, stream=stream, hbm_budget_bytes=hbm_budget_bytes, precision=precision,
                        n_slots=n_slots, refine_steps=refine_steps, flags=flags,
                        tune_table=tune_table.encode() if tune_table else None)
        h = ctypes.c_void_p()
        _check(self.L.ba_init(ctypes.byref(h), ctypes.byref(cfg)), None, "ba_init")
        self.h = h
        self.sizes = {}

    def close(self):
        if self.h:
            self.L.ba_shutdown(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def create_cluster(self, scene, warm_from=0, warm_cam_map=None, warm_pt_map=None):
        keep = []
        d = make_desc(scene, keep)
        if warm_from:
            cm = np.ascontiguousarray(warm_cam_map, dtype=np.int32)
            pm = np.ascontiguousarray(warm_pt_map, dtype=np.int32)
            keep += [cm, pm]
            d.warm_from = warm_from
            d.warm_cam_map = cm.ctypes.data_as(_ip)
            d.warm_pt_map = pm.ctypes.data_as(_ip)
        cid = ctypes.c_uint64()
        _check(self.L.ba_create_cluster(self.h, ctypes.byref(d), ctypes.byref(cid)), self.h, "ba_create_cluster")
        self.sizes[cid.value] = (d.n_cams, d.n_pts, d.n_obs)
        return cid.value

    def warm_start(self, dst, src, cam_map, pt_map):
        cm = np.ascontiguousarray(cam_map, dtype=np.int32)
        pm = np.ascontiguousarray(pt_map, dtype=np.int32)
        _check(self.L.ba_warm_start(self.h, dst, src, cm.ctypes.data_as(_ip), pm.ctypes.data_as(_ip)), self.h,
               "ba_warm_start")

    def linearize(self, cid):
        out = ba_lin_info()
        _check(self.L.ba_linearize(self.h, cid, ctypes.byref(out)), self.h, "ba_linearize")
        return {"cost": out.cost, "grad_inf": out.grad_inf, "n_free": out.n_free}

    def probe_fp32_fma(self, ctas_per_sm=4, iters=4096):
        tf, ms = ctypes.c_double(), ctypes.c_double()
        _check(self.L.ba_probe_fp32_fma(self.h, int(ctas_per_sm), int(iters), ctypes.byref(tf), ctypes.byref(ms)),
               self.h, "ba_probe_fp32_fma")
        return tf.value, ms.value

    def get_tune(self):
        t = ba_tune()
        _check(self.L.ba_get_tune(self.h, ctypes.byref(t)), self.h, "ba_get_tune")
        return t.as_dict()

    def set_tune(self, **kw):
        t = ba_tune.from_dict(dict(self.get_tune(), **kw))
        _check(self.L.ba_set_tune(self.h, ctypes.byref(t)), self.h, "ba_set_tune")

    def autotune(self, scenes, iters):
        keep = []
        descs = (ba_cluster_desc * len(scenes))(*[make_desc(sc, keep) for sc in scenes])
        t = ba_tune()
        _check(self.L.ba_autotune(self.h, descs, len(scenes), int(iters), ctypes.byref(t)), self.h, "ba_autotune")
        return t.as_dict()

    def solve_step(self, cid):
        out = ba_step_info()
        _check(self.L.ba_solve_step(self.h, cid, ctypes.byref(out)), self.h, "ba_solve_step")
        return out.as_dict()

    def run(self, cid, iters, trace=True):
        tr = (ba_step_info * max(1, iters))() if trace else None
        _check(self.L.ba_run(self.h, cid, iters, tr), self.h, "ba_run")
        return [tr[i].as_dict() for i in range(iters)] if trace else None

    def solve_batch(self, cids, iters, trace=False):
        n = len(cids)
        ids = (ctypes.c_uint64 * n)(*cids)
        res = (ba_result * n)()
        tr = (ba_step_info * (n * max(1, iters)))() if trace else None
        _check(self.L.ba_solve_batch(self.h, ids, n, iters, res, tr), self.h, "ba_solve_batch")
        out = [res[i].as_dict() for i in range(n)]
        if trace:
            for i in range(n):
                out[i]["trace"] = [tr[i * iters + t].as_dict() for t in range(iters)]
        return out

    def reset(self, cid):
        _check(self.L.ba_reset(self.h, cid), self.h, "ba_reset")

    def reset_batch(self, cids):
        ids = (ctypes.c_uint64 * len(cids))(*cids)
        _check(self.L.ba_reset_batch(self.h, ids, len(cids)), self.h, "ba_reset_batch")

    def launch_count(self):
        v = ctypes.c_uint64()
        _check(self.L.ba_launch_count(self.h, ctypes.byref(v)), self.h, "ba_launch_count")
        return v.value

    def kernel_stats(self, reset=False):
        n = len(KERNEL_KINDS)
        ms = np.zeros(n)
        cnt = (ctypes.c_uint64 * n)()
        _check(self.L.ba_kernel_stats(self.h, _d(ms), cnt, n, int(reset)), self.h, "ba_kernel_stats")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)}

    def submit(self, cid, iters, ftol=0.0):
        t = ctypes.c_uint64()
        _check(self.L.ba_submit(self.h, cid, ctypes.byref(ba_solve_opts(iters, 0, ftol)), ctypes.byref(t)), self.h,
               "ba_submit")
        return t.value

    def poll(self, ticket):
        r = ba_result()
        st = self.L.ba_poll(self.h, ticket, ctypes.byref(r))
        if st == BA_PENDING:
            return None
        _check(st, self.h, "ba_poll")
        return r.as_dict()

    def get_state(self, cid):
        nc, npt, _ = self.sizes[cid]
        R, T, X = np.zeros((nc, 9)), np.zeros((nc, 3)), np.zeros((max(npt, 1), 3))
        _check(self.L.ba_get_state(self.h, cid, _d(R), _d(T), _d(X), BA_PTR_HOST), self.h, "ba_get_state")
        return R, T, X[:npt]

    def get_state_batch(self, cids):
        """The current states of several clusters in one call: a list of
        (R, T, X) as get_state returns them."""
        cids = list(cids)
        n = len(cids)
        out = []
        ptrs = [(ctypes.c_void_p * max(n, 1))() for _ in range(3)]
        for i, cid in enumerate(cids):
            nc, npt, _ = self.sizes[cid]
            R, T, X = np.empty((nc, 9)), np.empty((nc, 3)), np.empty((max(npt, 1), 3))
            for a, arr in zip(ptrs, (R, T, X)):
                a[i] = arr.ctypes.data
            out.append((R, T, X, npt))
        ids = (ctypes.c_uint64 * max(n, 1))(*cids)
        _check(self.L.ba_get_state_batch(self.h, ids, n, ptrs[0], ptrs[1], ptrs[2]), self.h, "ba_get_state_batch")
        return [(R, T, X[:npt]) for R, T, X, npt in out]

    def reprojection_errors(self, cid):
        _, _, no = self.sizes[cid]
        e = np.zeros(max(no, 1))
        _check(self.L.ba_reprojection_errors(self.h, cid, _d(e)), self.h, "ba_reprojection_errors")
        return e[:no]

    def memory_in_use(self):
        v = ctypes.c_uint64()
        _check(self.L.ba_memory_in_use(self.h, ctypes.byref(v)), self.h, "ba_memory_in_use")
        return v.value

    def transition(self, dst, src, cam_map):
        """Eq. 8: blend the poses of the images of dst shared with src (free in
        dst) by their observation counts in both clusters."""
        m = np.ascontiguousarray(cam_map, dtype=np.int32)
        _check(self.L.ba_transition(self.h, dst, src, m.ctypes.data_as(_ip)), self.h, "ba_transition")

    def patch_transfer_poses(self, p0, intr0, R0, T0, lam, intr, R, T, width, height):
        """Eq. 3: patch centres p0 (n, 2) of image 0 moved to the m images of
        intr (m, 7), R (m, 9), T (m, 3) at depth lam: (p (m, n, 2), inside
        (m, n) bool)."""
        p0 = _f64(p0, (-1, 2))
        intr, R, T = _f64(intr, (-1, 7)), _f64(R, (-1, 9)), _f64(T, (-1, 3))
        n, m = p0.shape[0], intr.shape[0]
        p = np.zeros((m, n, 2))
        inside = np.zeros((m, n), dtype=np.uint8)
        _check(self.L.ba_patch_transfer_poses(self.h, n, _d(p0), _d(_f64(intr0, (7,))), _d(_f64(R0, (9,))),
                                              _d(_f64(T0, (3,))), float(lam), m, _d(intr), _d(R), _d(T),
                                              float(width), float(height), _d(p),
                                              inside.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))),
               self.h, "ba_patch_transfer_poses")
        return p, inside.astype(bool)

    def patch_transfer_planar(self, q0, c, g0, theta, g):
        """Eq. 4: patch centres q0 (n, 2) moved to m images by theta (m,) and
        the image centres g (m, 2) relative to g0: q (m, n, 2)."""
        q0, theta, g = _f64(q0, (-1, 2)), _f64(theta, (-1,)), _f64(g, (-1, 2))
        n, m = q0.shape[0], theta.shape[0]
        q = np.zeros((m, n, 2))
        _check(self.L.ba_patch_transfer_planar(self.h, n, _d(q0), _d(_f64(c, (2,))), _d(_f64(g0, (2,))), m,
                                               _d(theta), _d(g), _d(q)), self.h, "ba_patch_transfer_planar")
        return q

    def footprints(self, intr, width, height, R, T, dsm):
        """Ground quadrilaterals (n, 4, 3) of the images' corners on a DSM
        raster (dict h[ny, nx], x0, y0, dx, dy)."""
        intr, R, T = _f64(intr, (-1, 7)), _f64(R, (-1, 9)), _f64(T, (-1, 3))
        n = intr.shape[0]
        h = _f64(dsm["h"], (-1,))
        ny, nx = np.shape(dsm["h"])
        d = ba_dsm(nx, ny, float(dsm["x0"]), float(dsm["y0"]), float(dsm["dx"]), float(dsm["dy"]), _d(h))
        out = np.zeros((n, 4, 3))
        _check(self.L.ba_footprints(self.h, n, _d(intr), float(width), float(height), _d(R), _d(T), ctypes.byref(d),
                                    _d(out)), self.h, "ba_footprints")
        return out

    def footprint_overlaps(self, qa, qb):
        """Intersection areas (na, nb) of two sets of footprints."""
        qa, qb = _f64(qa, (-1, 12)), _f64(qb, (-1, 12))
        out = np.zeros((qa.shape[0], qb.shape[0]))
        _check(self.L.ba_footprint_overlaps(self.h, qa.shape[0], _d(qa), qb.shape[0], _d(qb), _d(out)), self.h,
               "ba_footprint_overlaps")
        return out

    def cluster_info(self, cid):
        """Table sizes of a cluster (units of work per LM iteration)."""
        v = ba_cluster_info()
        _check(self.L.ba_get_cluster_info(self.h, cid, ctypes.byref(v)), self.h, "ba_get_cluster_info")
        return v.as_dict()

    def destroy_cluster(self, cid):
        _check(self.L.ba_destroy_cluster(self.h, cid), self.h, "ba_destroy_cluster")
        self.sizes.pop(cid, None)
