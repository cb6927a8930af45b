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
    assert ctypes.sizeof(_lib.gs_scene) == 40 and ctypes.sizeof(_lib.gs_precull) == 40
    assert ctypes.sizeof(_lib.gs_dynamics) == 48
    assert _lib.gs_dynamics.ambient.offset == 40
    # gs_adam_cfg: 60 lr + 3 floats + step + pointer + 2 ints
    assert _lib.gs_adam_cfg.d_step.offset == 256
    assert ctypes.sizeof(_lib.gs_train_io) == 104 and _lib.gs_train_io.frozen.offset == 96
    assert ctypes.sizeof(_lib.gs_train_cfg) == 352 and _lib.gs_train_cfg.n_frozen.offset == 336
    assert ctypes.sizeof(_lib.gs_tune_entry) == 20


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(_lib, "LIB_PATH", "/nonexistent/libgs.so")
    monkeypatch.setattr(_lib, "_lib", None)
    try:
        _lib.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected a failure without the CUDA library")
