"""CPU checks of the boundary: libfire.so builds for sm_103a, loads without a
GPU, and exports every function include/fire.h declares (no compute call is
made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fire.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(fire_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fire_scene_create", "fire_bvh_build", "fire_bvh_refit", "fire_render",
                 "fire_render_batch", "fire_shade", "fire_shade_backward", "fire_debug_dump",
                 "fire_last_error"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2410_05095_b300 import _build, fire
    _build.build()
    lib = ctypes.CDLL(_build.LIB)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(fire.EXPORTS)
    assert fire.version().startswith("fire-b300")


def test_python_binding_has_no_cpu_path(monkeypatch, tmp_path):
    """Without the library the binding raises instead of falling back."""
    from paper_2410_05095_b300 import fire
    monkeypatch.setattr(fire, "_lib", None)
    monkeypatch.setattr(fire, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        fire.lib()


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2410_05095_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "fire_oracle" not in text, f
