"""Allocation-free forward render, checked against the staged entry points.

Some callers cannot allocate device memory: a plugin inside a host
application whose own allocator owns the GPU's memory, or a real-time loop
that must never call cudaMalloc.  They call sixdgs_render_fwd_static, whose
workspace is a fixed SIXDGS_STATIC_WS_BYTES array inside the library.  These
tests call it through the C ABI twice in a row (and a third time after a
differently sized frame left its contents in the array) and compare each
result with the images of sixdgs_condition_project + sixdgs_bin_sort +
sixdgs_raster_fwd run on a caller-allocated workspace.
"""

import ctypes
import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

sx = pytest.importorskip("paper_2410_04974_gb300")
from paper_2410_04974_gb300 import _lib  # noqa: E402
from paper_2410_04974_gb300.render import camera_array, make_settings  # noqa: E402

IMAGE_TOL = 2e-4   # the image tolerance of the parity tests


def _scene_struct(params, n, deg):
    s = _lib.Scene()
    s.n, s.sh_degree = n, deg
    for k in sx.PARAM_NAMES:
        setattr(s, k, params[k].data_ptr())
    return s


def _static_render(scene, cams, settings):
    lib = _lib.load()
    params = sx.params_to_device(scene)
    pixels = sum(c.width * c.height for c in cams)
    images = torch.full((3 * pixels,), -1.0, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sc = _scene_struct(params, scene.n, scene.sh_degree)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    code = lib.sixdgs_render_fwd_static(scene.n, scene.sh_degree, ctypes.byref(sc), camera_array(cams), len(cams),
                                        ctypes.byref(settings), ctypes.c_void_p(images.data_ptr()),
                                        ctypes.c_void_p(status.data_ptr()), stream)
    torch.cuda.synchronize()
    return code, images, int(status.item())


def _staged_render(scene, cams, **kw):
    r = sx.Renderer(scene.n, scene.sh_degree, cams, **kw)
    img = r.forward(sx.params_to_device(scene))
    torch.cuda.synchronize()
    return img


def test_static_workspace_render_matches_staged_calls_twice_in_a_row():
    frames = []
    a = synth.make_workload(0)
    frames.append((a.scene, a.cameras, dict(tile=(16, 16), batch=256)))
    b = synth.scene_shell(20_000, 77, dp_sigma=0.1)
    b.l_raw[:3] += math.log(3.0)
    cams_b = [synth.look_at_camera((4.0, 0.0, 0.3), 200, 136), synth.look_at_camera((0.0, 4.0, -0.5), 96, 256)]
    frames.append((b, cams_b, dict(tile=(8, 16), batch=64)))
    frames.append(frames[0])          # again, after frame b left its contents
    for scene, cams, kw in frames:
        settings = make_settings(**kw)
        code, got, status = _static_render(scene, cams, settings)
        assert code == _lib.OK, _lib.load().sixdgs_status_string(code)
        assert status == 0
        ref = _staged_render(scene, cams, **kw)
        assert got.shape == ref.shape
        err = float((got - ref).abs().max())
        assert err <= IMAGE_TOL, err


def test_static_workspace_refuses_frames_beyond_its_size():
    scene = synth.scene_shell(240_000, 3)
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 800, 800)]
    plan = sx.make_plan(scene.n, scene.sh_degree, cams, make_settings(inference=True))
    assert plan.ws_bytes > _lib.STATIC_WS_BYTES
    code, images, status = _static_render(scene, cams, make_settings())
    assert code == _lib.ERR_WORKSPACE
    assert torch.all(images == -1.0)          # nothing was launched


def test_static_workspace_fits_a_forward_only_frame_of_200k_gaussians():
    """The frame is planned forward-only (no gradient records), so 200,000
    Gaussians at 800x800 fit although a training plan of that frame would not."""
    scene = synth.scene_shell(200_000, 3)
    cams = [synth.look_at_camera((4.0, 0.0, 0.0), 800, 800)]
    assert sx.make_plan(scene.n, scene.sh_degree, cams, make_settings()).ws_bytes > _lib.STATIC_WS_BYTES
    settings = make_settings()
    code, got, status = _static_render(scene, cams, settings)
    assert code == _lib.OK and status == 0
    err = float((got - _staged_render(scene, cams)).abs().max())
    assert err <= IMAGE_TOL, err


def test_static_workspace_call_allocates_nothing():
    """After a first call (which looks up the array's address and loads the
    library's kernels), a call changes neither the device's free memory nor
    what PyTorch's allocator holds."""
    a = synth.make_workload(0)
    lib = _lib.load()
    params = sx.params_to_device(a.scene)
    images = torch.empty(3 * 128 * 128, dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sc = _scene_struct(params, a.scene.n, a.scene.sh_degree)
    cams = camera_array(a.cameras)
    settings = make_settings()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        code = lib.sixdgs_render_fwd_static(a.scene.n, a.scene.sh_degree, ctypes.byref(sc), cams, 1,
                                            ctypes.byref(settings), ctypes.c_void_p(images.data_ptr()),
                                            ctypes.c_void_p(status.data_ptr()), stream)
        torch.cuda.synchronize()
        assert code == _lib.OK and int(status.item()) == 0

    call()
    free0, held0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    call()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == held0
