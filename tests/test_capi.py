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


def test_ctypes_layouts_match_the_header(tmp_path):
    """The binding's ctypes structs have the C structs' sizes and field
    offsets, and its error codes the header's values (compiled with the host
    compiler; no GPU)."""
    import subprocess
    from paper_2410_05095_b300 import fire
    prog = tmp_path / "layout.c"
    prog.write_text('''
#include <stddef.h>
#include <stdio.h>
#include "fire.h"
#define P(T, F) printf(#T "." #F " %zu\\n", offsetof(T, F))
int main(void) {
  printf("fire_material %zu\\nfire_camera %zu\\nfire_light %zu\\nfire_render_opts %zu\\nfire_gbuffer_rec %zu\\n",
         sizeof(fire_material), sizeof(fire_camera), sizeof(fire_light), sizeof(fire_render_opts),
         sizeof(fire_gbuffer_rec));
  P(fire_camera, vfov_deg); P(fire_camera, spp); P(fire_light, intensity);
  P(fire_render_opts, blocks_per_sm); P(fire_render_opts, flags); P(fire_material, metallic);
  printf("errors %d %d %d %d %d %d\\n", FIRE_ERR_INVALID_ARG, FIRE_ERR_OOM, FIRE_ERR_CUDA,
         FIRE_ERR_STACK_OVERFLOW, FIRE_ERR_TIMEOUT, FIRE_ERR_NOT_BUILT);
  printf("srgb %d\\n", FIRE_MATERIALS_SRGB_ALBEDO);
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).splitlines()
               if not l.startswith(("errors", "srgb")))
    assert int(got["fire_material"]) == ctypes.sizeof(fire.Material)
    assert int(got["fire_camera"]) == ctypes.sizeof(fire.Camera)
    assert int(got["fire_light"]) == ctypes.sizeof(fire.Light)
    assert int(got["fire_render_opts"]) == ctypes.sizeof(fire.RenderOpts)
    assert int(got["fire_gbuffer_rec"]) == fire.GBUF_REC_BYTES
    assert int(got["fire_camera.vfov_deg"]) == fire.Camera.vfov_deg.offset
    assert int(got["fire_camera.spp"]) == fire.Camera.spp.offset
    assert int(got["fire_light.intensity"]) == fire.Light.intensity.offset
    assert int(got["fire_render_opts.blocks_per_sm"]) == fire.RenderOpts.blocks_per_sm.offset
    assert int(got["fire_render_opts.flags"]) == fire.RenderOpts.flags.offset
    assert int(got["fire_material.metallic"]) == fire.Material.metallic.offset
    out = subprocess.check_output([str(exe)], text=True)
    codes = [int(x) for x in next(l for l in out.splitlines() if l.startswith("errors")).split()[1:]]
    assert {c: fire.ERRORS[c] for c in codes} == fire.ERRORS
