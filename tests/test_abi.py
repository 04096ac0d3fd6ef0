"""The C ABI library builds, loads without a GPU and exports every entry
point that include/ba.h declares; the Python binding carries the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    with open(os.path.join(ROOT, "include", "ba.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"BA_API\s+[\w\s\*]*?\b(ba_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for required in ["ba_init", "ba_create_cluster", "ba_linearize", "ba_solve_step", "ba_submit", "ba_poll",
                     "ba_get_state", "ba_destroy_cluster", "ba_shutdown", "ba_status_string", "ba_solve_batch"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import paper_2511_06152_gb300 as ba
    L = ctypes.CDLL(ba.library_path(build=True))
    for name in declared_entry_points():
        assert hasattr(L, name), name
    assert set(declared_entry_points()) <= set(ba.EXPORTS)


def test_status_strings_and_init_without_gpu():
    import paper_2511_06152_gb300 as ba
    L = ba.lib()
    assert L.ba_status_string(ba.BA_OK) == b"ok"
    assert L.ba_status_string(ba.BA_ERR_NOT_PD).startswith(b"damped")
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present; the no-GPU path is not reachable here")
    h = ctypes.c_void_p()
    cfg = ba.ba_config(device=0, stream=None, hbm_budget_bytes=0, precision=ba.BA_FP64, n_slots=0, refine_steps=-1)
    st = L.ba_init(ctypes.byref(h), ctypes.byref(cfg))
    assert st == ba.BA_ERR_CUDA  # fails loudly: no CPU fallback


def test_struct_layouts_match_header():
    """ctypes mirrors of the ABI structs have the C sizes (x86-64 / aarch64 LP64)."""
    import paper_2511_06152_gb300 as ba
    assert ctypes.sizeof(ba.ba_config) == 4 + 4 + 8 + 8 + 4 * 4
    assert ctypes.sizeof(ba.ba_step_info) == 8 + 7 * 8
    assert ctypes.sizeof(ba.ba_result) == 16 + 3 * 8
    assert ctypes.sizeof(ba.ba_lin_info) == 24
