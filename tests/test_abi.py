"""The C-ABI library loads and exports every symbol include/gs.h declares
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import paper_2604_02851_b300 as gs
from paper_2604_02851_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:gs_status_t|size_t|int64_t|int32_t)\s+(gs_\w+)\s*\(", src, flags=re.M)))


def test_header_declarations_are_exported():
    from paper_2604_02851_b300 import build
    build.build()
    L = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(_lib.EXPORTS)


def test_struct_layouts_match_header():
    assert ctypes.sizeof(_lib.gs_camera) == 80
    assert gs.CAMERA_DTYPE.itemsize == 80
    assert ctypes.sizeof(_lib.gs_scene) == 48 and ctypes.sizeof(_lib.gs_precull) == 40
    assert ctypes.sizeof(_lib.gs_lighting) == 16 and ctypes.sizeof(_lib.gs_light_camera) == 72
    assert ctypes.sizeof(_lib.gs_dynamics) == 48
    assert _lib.gs_dynamics.ambient.offset == 40
    # gs_adam_cfg: 60 lr + 3 floats + step + pointer + 2 ints
    assert _lib.gs_adam_cfg.d_step.offset == 256
    assert ctypes.sizeof(_lib.gs_train_io) == 104 and _lib.gs_train_io.frozen.offset == 96
    assert ctypes.sizeof(_lib.gs_train_cfg) == 368 and _lib.gs_train_cfg.n_frozen.offset == 336
    assert _lib.gs_train_cfg.lighting.offset == 352 and _lib.gs_train_cfg.phases.offset == 360
    assert ctypes.sizeof(_lib.gs_tune_entry) == 28


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libgs.so")
    monkeypatch.setattr(_lib, "_lib", None)
    try:
        _lib.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected a failure without the CUDA library")


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """Sizes and field offsets of every struct as gcc lays out include/gs.h,
    against the ctypes mirrors of the binding."""
    import os
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        import pytest
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = ["gs_camera", "gs_dynamics", "gs_precull", "gs_lighting", "gs_scene", "gs_light_camera",
               "gs_tune_entry", "gs_adam_cfg", "gs_train_io", "gs_train_cfg"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', 'int main(void) {']
    expect = []
    for st in structs:
        lines.append(f'printf("%zu\\n", sizeof({st}));')
        expect.append(ctypes.sizeof(getattr(_lib, st)))
        for name, _ in getattr(_lib, st)._fields_:
            lines.append(f'printf("%zu\\n", offsetof({st}, {name}));')
            expect.append(getattr(getattr(_lib, st), name).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == expect
