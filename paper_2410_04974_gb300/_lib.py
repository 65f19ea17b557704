"""ctypes view of the C ABI in include/sixdgs.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int32, c_int64, c_float, c_void_p, c_size_t = (ctypes.c_int32, ctypes.c_int64, ctypes.c_float,
                                                  ctypes.c_void_p, ctypes.c_size_t)

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_CAPACITY, ERR_TIMEOUT, ERR_NONFINITE, ERR_WORKSPACE = range(7)

WS_CAMS, WS_REC, WS_NTILES, WS_RECT, WS_DEPTHKEY, WS_COUNTS, WS_SORTED, WS_RANGES, WS_NWALK, \
    WS_GRADREC, WS_SORTEDKEY = range(11)


class Camera(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("fx", c_float), ("fy", c_float),
                ("cx", c_float), ("cy", c_float), ("world_to_cam", c_float * 12),
                ("campos", c_float * 3), ("znear", c_float)]


class Scene(ctypes.Structure):
    _fields_ = [("n", c_int64), ("sh_degree", c_int32), ("_pad", c_int32), ("mu_p", c_void_p),
                ("mu_d", c_void_p), ("l_raw", c_void_p), ("opacity_logit", c_void_p), ("sh", c_void_p),
                ("lambda_raw", c_void_p), ("cond_cache", c_void_p)]


class Settings(ctypes.Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch", c_int32), ("lambda_opa", c_float),
                ("bg", c_float * 3), ("store_aux", c_int32), ("spin_budget", c_int64),
                ("loss_norm", c_float), ("count_pairs", c_int32), ("persistent", c_int32),
                ("inference", c_int32), ("alpha_footprint", c_int32), ("_pad", c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("n", c_int64), ("sh_degree", c_int32), ("n_cams", c_int32), ("settings", Settings),
                ("n_pairs", c_int64), ("total_tiles", c_int64), ("total_pixels", c_int64),
                ("dup_capacity", c_int64), ("depth_passes", c_int32), ("tile_passes", c_int32),
                ("ws_bytes", c_int64), ("off", c_int64 * 32)]


EXPORTS = {
    "sixdgs_version": (ctypes.c_char_p, []),
    "sixdgs_status_string": (ctypes.c_char_p, [c_int32]),
    "sixdgs_plan_init": (c_int32, [c_int64, c_int32, ctypes.POINTER(Camera), c_int32,
                                   ctypes.POINTER(Settings), c_int64, ctypes.POINTER(Plan)]),
    "sixdgs_workspace_size": (c_size_t, [ctypes.POINTER(Plan)]),
    "sixdgs_condition_project": (c_int32, [ctypes.POINTER(Plan), ctypes.POINTER(Scene),
                                           ctypes.POINTER(Camera), c_void_p, c_size_t, c_void_p, c_void_p]),
    "sixdgs_bin_sort": (c_int32, [ctypes.POINTER(Plan), c_void_p, c_size_t, c_void_p, c_void_p]),
    "sixdgs_raster_fwd": (c_int32, [ctypes.POINTER(Plan), c_void_p, c_size_t, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_void_p, c_void_p]),
    "sixdgs_raster_bwd": (c_int32, [ctypes.POINTER(Plan), ctypes.POINTER(Scene), c_void_p, c_size_t,
                                    c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "sixdgs_blend_bwd": (c_int32, [ctypes.POINTER(Plan), c_void_p, c_size_t, c_void_p, c_void_p,
                                   c_void_p, c_void_p]),
    "sixdgs_raster_fwd_bwd": (c_int32, [ctypes.POINTER(Plan), c_void_p, c_size_t] + [c_void_p] * 6),
    "sixdgs_render_batched": (c_int32, [ctypes.POINTER(Plan), ctypes.POINTER(Scene), ctypes.POINTER(Camera),
                                        c_void_p, c_size_t] + [c_void_p] * 12),
    "sixdgs_peak_probe": (c_int32, [c_int32, c_int64, c_void_p, c_int32, c_void_p]),
    "sixdgs_condition_cache": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sixdgs_scale_rotation": (c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "sixdgs_render_fwd_static": (c_int32, [c_int64, c_int32, ctypes.POINTER(Scene), ctypes.POINTER(Camera),
                                           c_int32, ctypes.POINTER(Settings), c_void_p, c_void_p, c_void_p]),
    "sixdgs_project_bwd": (c_int32, [ctypes.POINTER(Plan), ctypes.POINTER(Scene), c_void_p, c_size_t,
                                     c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                                     c_void_p, c_void_p]),
}

COND_CACHE_PLANES = 25
STATIC_WS_BYTES = 32 << 20   # SIXDGS_STATIC_WS_BYTES

_LIB = None


class SixDGSError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsixdgs.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise SixDGSError(f"libsixdgs.so not found at {path}; run paper_2410_04974_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(code: int, what: str) -> None:
    if code != OK:
        msg = load().sixdgs_status_string(code).decode()
        raise SixDGSError(f"{what} failed: {msg} ({code})")


def status_names(mask: int):
    lib = load()
    return [lib.sixdgs_status_string(c).decode() for c in range(1, 7) if mask & (1 << c)]
