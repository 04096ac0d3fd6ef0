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


STRUCTS = ["ba_config", "ba_cluster_desc", "ba_lin_info", "ba_step_info", "ba_solve_opts", "ba_result",
           "ba_cluster_info", "ba_dsm", "ba_presort_info"]


def test_struct_layouts_match_header(tmp_path):
    """ctypes mirrors of the ABI structs have the size and field offsets that
    the C compiler gives the declarations in include/ba.h."""
    import shutil
    import subprocess
    import paper_2511_06152_gb300 as ba
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "ba.h"', "int main(void) {"]
    for name in STRUCTS:
        st = getattr(ba, name)
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                              text=True).stdout.splitlines())
    for name in STRUCTS:
        st = getattr(ba, name)
        assert int(out[name]) == ctypes.sizeof(st), name
        for f, _ in st._fields_:
            assert int(out[f"{name}.{f}"]) == getattr(st, f).offset, (name, f)


def test_binding_constants_match_the_header():
    """Every BA_FLAG_*, BA_PTR_*, BA_FP64 / BA_MIXED and BA_ERR_* value the
    binding defines equals the header's."""
    import paper_2511_06152_gb300 as ba
    with open(os.path.join(ROOT, "include", "ba.h")) as f:
        src = f.read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(BA_\w+)\s+(-?\d+)\b", src)}
    enums = {k: int(v) for k, v in re.findall(r"\b(BA_\w+)\s*=\s*(-?\d+)\s*[,}]", src)}
    values = {**defines, **enums}
    checked = 0
    for name, v in values.items():
        if hasattr(ba, name):
            assert getattr(ba, name) == v, name
            checked += 1
    assert "BA_FLAG_SMALL_DF_FACTOR" in values and ba.BA_FLAG_SMALL_DF_FACTOR == values["BA_FLAG_SMALL_DF_FACTOR"]
    assert checked >= 8
