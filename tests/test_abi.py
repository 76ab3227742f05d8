"""The C-ABI library builds, loads and exports every symbol include/dof.h declares,
and the binding's struct layouts match the header's (CPU only: no compute calls)."""

import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dof.h")


@pytest.fixture(scope="module")
def libdof():
    from paper_2210_06158_gb300 import _build, dof
    _build.build()
    return dof.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dof_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dof_ctx_create", "dof_scene_upload", "dof_frame", "dof_history_create", "dof_gbuffer",
                 "dof_gbuffer_raster",
                 "dof_last_error", "dof_frame_stats", "dof_debug_buffer"):
        assert must in names


def test_library_exports_every_declared_symbol(libdof):
    from paper_2210_06158_gb300 import dof
    for name in declared_functions():
        assert hasattr(libdof, name), name
        assert name in dof._SIGS, f"binding lacks {name}"


def test_struct_layouts_match_header():
    from paper_2210_06158_gb300 import dof
    probe = r'''
#include <stdio.h>
#include <stddef.h>
#include "dof.h"
#define S(t) printf(#t " %zu\n", sizeof(t));
#define O(t, f) printf(#t "." #f " %zu\n", offsetof(t, f));
int main(void) {
  S(DofCamera) S(DofParams) S(DofGBuffer) S(DofSceneInfo) S(DofFrameStats)
  O(DofParams, seed) O(DofParams, light_dir) O(DofParams, emit) O(DofParams, tile)
  O(DofCamera, frame_index) O(DofGBuffer, width) O(DofSceneInfo, device_bytes) O(DofFrameStats, device_status) O(DofFrameStats, tri_tests)
  return 0; }
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(probe)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    got = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    structs = dict(DofCamera=dof.DofCamera, DofParams=dof.DofParams, DofGBuffer=dof.DofGBuffer,
                   DofSceneInfo=dof.DofSceneInfo, DofFrameStats=dof.DofFrameStats)
    for k, v in got.items():
        if "." in k:
            s, f = k.split(".")
            assert getattr(structs[s], f).offset == int(v), k
        else:
            assert C.sizeof(structs[k]) == int(v), k


def test_defaults_match_paper_constants(libdof):
    from paper_2210_06158_gb300 import dof
    p = dof.DofParams()
    libdof.dof_params_default(C.byref(p))
    assert abs(p.s - 0.8) < 1e-7 and p.var_w_mask == 1e5 and abs(p.alpha - 0.95) < 1e-7
    assert p.var_w_recon == 2000.0 and abs(p.b_max - 0.9) < 1e-7 and abs(p.h_edge - 0.3) < 1e-7
    assert abs(p.lod_scale - 0.05) < 1e-8 and p.lod_max == 3.0 and abs(p.depth_range_m - 0.1) < 1e-8


def test_host_errors_without_device(libdof):
    """Argument checks run before any device work and report through dof_last_error."""
    ptr = C.c_void_p()
    rc = libdof.dof_ctx_create(0, 0, None)
    assert rc == -1 and b"NULL" in libdof.dof_last_error()
    rc = libdof.dof_frame(None, None, None, None, None, None, None, None)
    assert rc == -1
    rc = libdof.dof_history_create(None, 64, 64, 1, 0, C.byref(ptr))
    assert rc == -1
    rc = libdof.dof_scene_info(None, None)
    assert rc == -1


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2210_06158_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "or_frame" not in src and "oracle.h" not in src, f
