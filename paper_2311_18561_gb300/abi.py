"""ctypes binding of the C ABI declared in ``include/pvg.h``.

Argument marshalling only: every step of the renderer runs in the CUDA
library ``_lib/libpvg.so``.  There is no fallback -- if the library is
missing or cannot be loaded, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_LIB = None

PVG_OK = 0
STATUS = {0: "PVG_OK", 1: "PVG_ERR_INVALID", 2: "PVG_ERR_OOM", 3: "PVG_ERR_BUSY", 4: "PVG_ERR_TIMEOUT",
          5: "PVG_ERR_CUDA", 6: "PVG_ERR_OVERFLOW", 7: "PVG_ERR_NOT_FOUND"}


class PVGError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        msg = "%s failed: %s" % (where, STATUS.get(self.status, str(status)))
        if self.status == 5 and _LIB is not None:
            msg += " (%s)" % _LIB.pvg_last_error().decode()
        super().__init__(msg)


class Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("sky_res", C.c_int32)] + [
        (k, C.c_void_p) for k in ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh", "sky",
                                  "sem")] + [("n_sem", C.c_int32), ("reserved0", C.c_int32)]


# extra composited channels (pvg_image_t.feat_mask)
FEAT_VBAR, FEAT_RHO, FEAT_SEM = 1, 2, 4
MAX_SEM = 32


class Camera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32), ("t", C.c_float),
                ("z_near", C.c_float), ("bg", C.c_float * 3), ("dt", C.c_float),
                ("sky_jitter", C.c_void_p)]


class Image(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p), ("feat", C.c_void_p),
                ("feat_mask", C.c_int32), ("reserved0", C.c_int32)]


class ImageGrad(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("depth", C.c_void_p), ("alpha", C.c_void_p), ("feat", C.c_void_p)]


class SceneGrad(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mu", "vel", "tau", "beta", "period", "scale", "quat", "opacity", "sh",
                                          "sky", "sem")]


class Config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("sync_sizes", C.c_int32),
                ("pixels_per_thread", C.c_int32), ("pair_capacity", C.c_int64), ("dilation", C.c_float),
                ("fov_clamp", C.c_float), ("reserved", C.c_float * 6)]


class ServeConfig(C.Structure):
    _fields_ = [("max_batch_views", C.c_int32), ("n_streams", C.c_int32), ("memory_budget", C.c_int64),
                ("max_pending", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("pixels_per_thread", C.c_int32), ("gate_timeout_us", C.c_int32), ("pipeline_depth", C.c_int32),
                ("pair_capacity", C.c_int32), ("reserved0", C.c_int32)]


class ReqStats(C.Structure):
    _fields_ = [("submit_ms", C.c_double), ("start_ms", C.c_double), ("done_ms", C.c_double),
                ("batch_views", C.c_int32), ("status", C.c_int32), ("gpu_ms", C.c_double),
                ("attempts", C.c_int32), ("reserved0", C.c_int32)]


# every symbol include/pvg.h declares, with (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "pvg_status_str": (C.c_char_p, [C.c_int]),
    "pvg_last_error": (C.c_char_p, []),
    "pvg_version": (C.c_int, []),
    "pvg_debug_fail_allocations": (None, [C.c_int32]),
    "pvg_config_default": (None, [C.POINTER(Config)]),
    "pvg_create": (C.c_int, [C.POINTER(_P), C.POINTER(Config)]),
    "pvg_destroy": (None, [_P]),
    "pvg_set_config": (C.c_int, [_P, C.POINTER(Config)]),
    "pvg_frame_create": (C.c_int, [C.POINTER(_P)]),
    "pvg_frame_destroy": (None, [_P]),
    "pvg_frame_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]),
    "pvg_render_fwd": (C.c_int, [_P, C.POINTER(Scene), C.POINTER(Camera), C.c_int32, C.POINTER(Image), _P, _P]),
    "pvg_render_fwd_multi": (C.c_int, [_P, C.POINTER(Scene), C.POINTER(Camera), C.c_int32, C.POINTER(Image), _P,
                                       _P]),
    "pvg_render_bwd": (C.c_int, [_P, C.POINTER(Scene), C.POINTER(Camera), C.c_int32, _P, C.POINTER(ImageGrad),
                                 C.POINTER(SceneGrad), _P]),
    "pvg_frame_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "pvg_serve_config_default": (None, [C.POINTER(ServeConfig)]),
    "pvg_serve_create": (C.c_int, [C.POINTER(_P), C.POINTER(ServeConfig)]),
    "pvg_serve_add_scene": (C.c_int, [_P, C.POINTER(Scene), C.POINTER(C.c_int32)]),
    "pvg_serve_submit": (C.c_int, [_P, C.c_int32, C.POINTER(Camera), C.POINTER(Image), C.POINTER(C.c_uint64)]),
    "pvg_serve_poll": (C.c_int, [_P, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(ReqStats)]),
    "pvg_serve_wait": (C.c_int, [_P, C.c_uint64, C.c_double, C.POINTER(ReqStats)]),
    "pvg_serve_release": (C.c_int, [_P, C.c_uint64]),
    "pvg_serve_counters": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64)]),
    "pvg_serve_arena": (C.c_int, [_P] + [C.POINTER(C.c_int64)] * 5),
    "pvg_serve_debug_withhold": (C.c_int, [_P, C.c_int32]),
    "pvg_serve_destroy": (C.c_int, [_P]),
    "pvg_sort_pairs": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.c_int32, _P]),
    "pvg_sort_pairs_noalloc": (C.c_int, [_P, _P, C.c_int64, C.c_int32, C.c_int32, _P]),
    "pvg_l1_loss": (C.c_int, [_P, _P, _P, C.c_int64, C.c_float, _P, _P, _P]),
    "pvg_rgb_loss": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_float, _P, _P, _P]),
    "pvg_kernel_launches": (C.c_uint64, []),
    "pvg_device_sm_count": (C.c_int32, []),
    "pvg_fma_probe": (C.c_int, [_P, C.c_int32, C.c_int64, C.c_float, C.c_float, _P]),
    "pvg_profile_enable": (C.c_int, [_P, C.c_int]),
    "pvg_profile_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "pvg_frame_eval_count": (C.c_int, [_P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}

STAGES = ("project", "depth_sort", "finalize", "pairs", "tile_sort", "composite", "composite_bwd",
          "preprocess_bwd")


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libpvg.so (building it first if asked and it is missing)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if build_if_missing and not os.path.exists(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libpvg.so is not built (run __graft_entry__.build()); there is no fallback")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def check(status, where):
    if status != PVG_OK:
        raise PVGError(status, where)


def config(tile=(16, 16), sync_sizes=True, pair_capacity=1 << 24, dilation=0.3, fov_clamp=1.3,
           pixels_per_thread=1) -> Config:
    c = Config()
    lib().pvg_config_default(C.byref(c))
    c.tile_w, c.tile_h = int(tile[0]), int(tile[1])
    c.pixels_per_thread = int(pixels_per_thread)
    c.sync_sizes = 1 if sync_sizes else 0
    c.pair_capacity = int(pair_capacity)
    c.dilation = float(dilation)
    c.fov_clamp = float(fov_clamp)
    return c


def camera(cam) -> Camera:
    """From a synth-style camera dict."""
    c = Camera()
    vm = [float(x) for x in list(__import__("numpy").asarray(cam["viewmat"], dtype="float32").reshape(12))]
    c.viewmat[:] = vm
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.t = float(cam["t"])
    c.z_near = float(cam.get("z_near", 0.2))
    bg = list(cam.get("bg", (0.0, 0.0, 0.0)))
    c.bg[:] = [float(b) for b in bg]
    c.dt = float(cam.get("dt", 0.0))
    jit = cam.get("sky_jitter")
    c.sky_jitter = jit.data_ptr() if jit is not None else None
    return c


def cameras(cams):
    arr = (Camera * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = camera(cam)
    return arr
