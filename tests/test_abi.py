"""The C ABI: the library loads without a GPU, exports every symbol that
include/*.h declares, and its host-only planning calls behave (CPU only)."""

import ctypes
import glob
import os
import re

import pytest

import synth
from paper_2410_04974_gb300 import _lib
from paper_2410_04974_gb300.render import camera_array, make_settings

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(sixdgs_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = _declared()
    assert "sixdgs_condition_project" in names and "sixdgs_raster_bwd" in names
    for name in names:
        assert hasattr(lib, name), name
    assert lib.sixdgs_version().decode().count(".") == 2
    assert lib.sixdgs_status_string(_lib.ERR_CAPACITY).decode() == "duplicate capacity exceeded"


def _plan(cams, n=1000, sh=3, dup=0, **kw):
    lib = _lib.load()
    st = make_settings(**kw)
    plan = _lib.Plan()
    code = lib.sixdgs_plan_init(n, sh, camera_array(cams), len(cams), ctypes.byref(st), dup, ctypes.byref(plan))
    return code, plan


def test_plan_layout_for_ring_of_eight():
    cams = synth.ring_cameras(8, 800, 800)
    code, plan = _plan(cams, n=300_000)
    assert code == _lib.OK
    assert plan.n_pairs == 8 * 300_000
    assert plan.total_tiles == 8 * 50 * 50
    assert plan.total_pixels == 8 * 800 * 800
    assert plan.depth_passes == 4 and plan.tile_passes == 2      # 20,000 tiles -> 15 bits
    assert plan.dup_capacity == 4 * plan.n_pairs + 4096
    offs = [plan.off[i] for i in range(11)]
    assert all(o % 256 == 0 for o in offs)
    assert plan.off[_lib.WS_REC] - plan.off[_lib.WS_CAMS] >= 8 * 128
    assert plan.ws_bytes >= plan.off[_lib.WS_SORTED] + 4 * plan.dup_capacity
    lib = _lib.load()
    assert lib.sixdgs_workspace_size(ctypes.byref(plan)) == plan.ws_bytes


def test_plan_mixed_resolutions_and_tile_shapes():
    w = synth.make_workload(3, n_override=1000)
    code, plan = _plan(w.cameras, n=1000, tile=(32, 8), batch=64)
    assert code == _lib.OK
    tiles = sum(((c.width + 31) // 32) * ((c.height + 7) // 8) for c in w.cameras)
    assert plan.total_tiles == tiles
    assert plan.total_pixels == sum(c.width * c.height for c in w.cameras)


@pytest.mark.parametrize("kw", [dict(tile=(12, 16)), dict(tile=(16, 32)), dict(batch=48), dict(batch=2048),
                                dict(lambda_opa=1.5)])
def test_plan_rejects_bad_settings(kw):
    code, _ = _plan(synth.ring_cameras(1, 64, 64), **kw)
    assert code == _lib.ERR_INVALID_ARG


def test_plan_rejects_unknown_footprint_and_inference_flags():
    lib = _lib.load()
    cams = camera_array(synth.ring_cameras(1, 64, 64))
    for field in ("alpha_footprint", "inference"):
        st = make_settings()
        setattr(st, field, 2)
        plan = _lib.Plan()
        assert lib.sixdgs_plan_init(10, 3, cams, 1, ctypes.byref(st), 0, ctypes.byref(plan)) == _lib.ERR_INVALID_ARG
    assert make_settings().alpha_footprint == 1 and make_settings(alpha_footprint=False).alpha_footprint == 0


def test_plan_rejects_bad_sizes():
    cams = synth.ring_cameras(1, 64, 64)
    assert _plan(cams, sh=4)[0] == _lib.ERR_INVALID_ARG
    assert _plan(cams, n=-1)[0] == _lib.ERR_INVALID_ARG
    assert _plan(cams, n=2 ** 31)[0] == _lib.ERR_INVALID_ARG
    assert _plan(cams, dup=2 ** 30)[0] == _lib.ERR_INVALID_ARG
    assert _plan(synth.ring_cameras(300, 64, 64))[0] == _lib.ERR_INVALID_ARG
    bad = synth.look_at_camera((4.0, 0.0, 0.0), 0, 64)
    assert _plan([bad])[0] == _lib.ERR_INVALID_ARG


def test_empty_scene_plan():
    code, plan = _plan(synth.ring_cameras(2, 33, 17), n=0)
    assert code == _lib.OK and plan.n_pairs == 0 and plan.total_tiles == 2 * 3 * 2


def test_stage_calls_reject_small_workspace_without_touching_the_gpu():
    lib = _lib.load()
    code, plan = _plan(synth.ring_cameras(1, 64, 64), n=10)
    assert code == _lib.OK
    # A workspace smaller than the plan is refused on the host, before any launch.
    fake = ctypes.c_void_p(256)
    assert lib.sixdgs_bin_sort(ctypes.byref(plan), fake, 16, None, None) == _lib.ERR_WORKSPACE
    assert lib.sixdgs_bin_sort(ctypes.byref(plan), ctypes.c_void_p(257), plan.ws_bytes, None, None) == \
        _lib.ERR_INVALID_ARG


def test_struct_layout_matches_header(tmp_path):
    """The ctypes mirrors have the size and field offsets of the C structs."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sixdgs_camera": _lib.Camera, "sixdgs_scene": _lib.Scene, "sixdgs_settings": _lib.Settings,
               "sixdgs_plan": _lib.Plan}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sixdgs.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, value = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert got == int(value), (cname, field)


def test_inference_plan_has_no_gradient_section():
    cams = synth.ring_cameras(2, 128, 128)
    code, train = _plan(cams, n=5000)
    code_i, inf = _plan(cams, n=5000, inference=True)
    assert code == _lib.OK and code_i == _lib.OK
    assert inf.off[_lib.WS_RANGES] == inf.off[_lib.WS_GRADREC]           # zero-sized section
    assert train.ws_bytes - inf.ws_bytes >= 48 * train.n_pairs - 256
    assert _plan(cams, n=5000, inference=True, store_aux=True)[0] == _lib.ERR_INVALID_ARG
    lib = _lib.load()
    # every backward entry point refuses an inference plan on the host
    fake = ctypes.c_void_p(256)
    sc = _lib.Scene()
    sc.n, sc.sh_degree = 5000, 3
    assert lib.sixdgs_blend_bwd(ctypes.byref(inf), fake, inf.ws_bytes, fake, fake, None, None) == \
        _lib.ERR_INVALID_ARG
    assert lib.sixdgs_raster_bwd(ctypes.byref(inf), ctypes.byref(sc), fake, inf.ws_bytes, fake, fake, fake,
                                 fake, fake, fake, fake, None, 0, None, None) == _lib.ERR_INVALID_ARG
    assert lib.sixdgs_project_bwd(ctypes.byref(inf), ctypes.byref(sc), fake, inf.ws_bytes, fake, fake, fake,
                                  fake, fake, None, 0, None, None) == _lib.ERR_INVALID_ARG


def test_header_constants_match_the_binding():
    text = open(os.path.join(ROOT, "include", "sixdgs.h")).read()
    defs = dict(re.findall(r"#define\s+(SIXDGS_[A-Z_]+)\s+(.+)", text))
    assert int(defs["SIXDGS_COND_CACHE_PLANES"]) == _lib.COND_CACHE_PLANES
    assert eval(defs["SIXDGS_STATIC_WS_BYTES"].replace("u", "")) == _lib.STATIC_WS_BYTES
    enums = dict((k, int(v)) for k, v in re.findall(r"(SIXDGS_ERR_[A-Z_]+)\s*=\s*(\d+)", text))
    for name, value in enums.items():
        assert getattr(_lib, name.replace("SIXDGS_", "")) == value, name
