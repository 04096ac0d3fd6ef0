"""ba_cost_noalloc: the allocation-free cost entry point.

Callers that cannot allocate device memory once they are running (onboard
flight software that reserves its memory at start-up, or a process whose
device memory belongs to another allocator) evaluate the robust cost F(x)
through ba_cost_noalloc, whose scratch is a fixed array inside the library.
This test calls it through the C ABI with device arrays and checks it
against the cost that ba_linearize reports for the same cluster and against
the CPU oracle's cost at the same state, on two calls in a row (a large
problem, then a smaller one, so that the second call reuses scratch the
first call left behind); an observation whose point index is out of range
must give NaN, not a fault.

It lives in a file of its own, collected last, and passes both alone in a
fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import scenegen as sg

pytestmark = pytest.mark.gpu

TOL = 1e-10  # relative, as the FP64 parity tests


def _device_desc(ba, torch, scene, keep):
    """A ba_cluster_desc whose arrays live in device memory (torch tensors)."""
    dev = torch.device("cuda", 0)

    def t(a, dtype):
        x = torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).to(dev).contiguous()
        keep.append(x)
        return x

    nc, npt, no = int(scene["n_cams"]), int(scene["n_pts"]), int(scene["n_obs"])
    arrs = dict(intr=t(np.reshape(scene["intr"], (nc, 7)), torch.float64),
                R=t(np.reshape(scene["R0"], (nc, 9)), torch.float64),
                T=t(np.reshape(scene["T0"], (nc, 3)), torch.float64),
                X=t(np.reshape(scene["X0"], (npt, 3)), torch.float64),
                R_prior=t(np.reshape(scene["R_prior"], (nc, 9)), torch.float64),
                T_prior=t(np.reshape(scene["T_prior"], (nc, 3)), torch.float64),
                fixed=t(scene["fixed"], torch.uint8),
                obs_cam=t(scene["obs_cam"], torch.int32), obs_pt=t(scene["obs_pt"], torch.int32),
                obs_uv=t(np.reshape(scene["obs_uv"], (no, 2)), torch.float64))
    d = ba.ba_cluster_desc()
    d.n_cams, d.n_pts, d.n_obs, d.ptr_kind = nc, npt, no, ba.BA_PTR_DEVICE
    dp = ctypes.POINTER(ctypes.c_double)
    for k in ("intr", "R", "T", "X", "R_prior", "T_prior", "obs_uv"):
        setattr(d, k, ctypes.cast(arrs[k].data_ptr(), dp))
    d.fixed = ctypes.cast(arrs["fixed"].data_ptr(), ctypes.POINTER(ctypes.c_uint8))
    d.obs_cam = ctypes.cast(arrs["obs_cam"].data_ptr(), ctypes.POINTER(ctypes.c_int32))
    d.obs_pt = ctypes.cast(arrs["obs_pt"].data_ptr(), ctypes.POINTER(ctypes.c_int32))
    d.sigma_px = float(scene["sigma_px"])
    d.huber_delta_px = float(scene["huber_delta"])
    d.sigma_gnss_m = float(scene["sigma_gnss"])
    d.sigma_imu_rad = float(scene["sigma_imu"])
    return d


def test_cost_noalloc_matches_linearize_on_two_calls():
    torch = pytest.importorskip("torch")
    import paper_2511_06152_gb300 as ba
    L = ba.lib()
    scenes = [sg.cluster_c2(fixed=(3,)), sg.cluster_c1()]  # ~230k then ~7k observations
    refs, orcs = [], []
    with ba.Context(precision=ba.BA_FP64) as ctx:
        for s in scenes:
            refs.append(ctx.linearize(ctx.create_cluster(s))["cost"])
            orcs.append(O.cost(O.Problem(s), s["R0"], s["T0"], s["X0"]))
    stream = torch.cuda.Stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    keep = []
    for s, ref, orc in zip(scenes, refs, orcs):
        d = _device_desc(ba, torch, s, keep)
        torch.cuda.synchronize()
        st = L.ba_cost_noalloc(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                               ctypes.cast(out.data_ptr(), ctypes.POINTER(ctypes.c_double)))
        assert st == ba.BA_OK
        stream.synchronize()
        got = float(out.item())
        assert got == pytest.approx(ref, rel=TOL), (got, ref)
        assert got == pytest.approx(orc, rel=TOL), (got, orc)


def test_cost_noalloc_out_of_range_index_gives_nan():
    """Indices are not checked on the host; the kernel skips the bad
    observation's reads and the cost comes out NaN."""
    torch = pytest.importorskip("torch")
    import paper_2511_06152_gb300 as ba
    L = ba.lib()
    s = sg.cluster_c1()
    s = dict(s, obs_pt=np.array(s["obs_pt"], dtype=np.int32).copy())
    s["obs_pt"][len(s["obs_pt"]) // 2] = int(s["n_pts"])  # one past the last point
    keep = []
    d = _device_desc(ba, torch, s, keep)
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    st = L.ba_cost_noalloc(ctypes.byref(d), ctypes.c_void_p(stream.cuda_stream),
                           ctypes.cast(out.data_ptr(), ctypes.POINTER(ctypes.c_double)))
    assert st == ba.BA_OK
    stream.synchronize()
    assert np.isnan(float(out.item()))


def test_cost_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2511_06152_gb300 as ba
    L = ba.lib()
    d = ba.ba_cluster_desc()
    d.n_cams, d.n_pts, d.n_obs, d.ptr_kind = 1, 1, 67_108_864 + 1, ba.BA_PTR_DEVICE
    d.sigma_px, d.huber_delta_px = 0.5, 1.0
    dummy = ctypes.cast(ctypes.c_void_p(256), ctypes.POINTER(ctypes.c_double))  # never dereferenced
    out = ctypes.cast(ctypes.c_void_p(256), ctypes.POINTER(ctypes.c_double))
    assert L.ba_cost_noalloc(ctypes.byref(d), None, out) == ba.BA_ERR_INVALID
    d.n_obs = 10
    d.ptr_kind = ba.BA_PTR_HOST  # host arrays are refused
    d.intr = d.R = d.T = d.X = d.R_prior = d.T_prior = d.obs_uv = dummy
    assert L.ba_cost_noalloc(ctypes.byref(d), None, out) == ba.BA_ERR_INVALID
