"""ctypes view of ``include/packuv.h``: structs, loader and signatures.

Argument marshalling only.  Loading fails loudly if the CUDA library has not
been built; nothing here computes any step of the render path.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

MAX_LEVELS = 16
RECORD_FLOATS = 12
GRAD2D_FLOATS = 12

PK_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid argument", 2: "invalid descriptor", 3: "capacity exceeded",
                4: "device wait timed out", 5: "CUDA error", 6: "unsupported",
                7: "larger than the allocation-free call's fixed scratch"}
DEV_CAPACITY = 1
DEV_LIVE_MISMATCH = 2
DEV_TIMEOUT = 4
DEV_BOUNDS = 8
BIN_RECT, BIN_ELLIPSE = 0, 1


class Level(C.Structure):
    _fields_ = [("w", C.c_int32), ("h", C.c_int32), ("x0", C.c_int32), ("y0", C.c_int32),
                ("rotated", C.c_int32)]


class AtlasDesc(C.Structure):
    _fields_ = [("atlas_w", C.c_int32), ("atlas_h", C.c_int32), ("num_levels", C.c_int32),
                ("level", Level * MAX_LEVELS), ("sh_degree", C.c_int32), ("frames", C.c_int32),
                ("texel_type", C.c_int32)]


class View(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("frame", C.c_int32)]


class Options(C.Structure):
    _fields_ = [("tile", C.c_int32), ("znear", C.c_float), ("bg", C.c_float * 3), ("max_dups", C.c_uint64),
                ("bin_mode", C.c_int32), ("batch", C.c_int32), ("stage_fwd", C.c_int32), ("stage_bwd", C.c_int32),
                ("batch_bwd", C.c_int32), ("sort_bits_tile", C.c_int32), ("sort_bits_depth", C.c_int32),
                ("count_evals", C.c_int32), ("first_wait_polls", C.c_int32)]


class Sizes(C.Structure):
    _fields_ = [("n_live", C.c_int64), ("n_gauss", C.c_int64), ("channels", C.c_int32),
                ("n_views", C.c_int32), ("n_pairs", C.c_int64), ("n_pixels", C.c_int64),
                ("n_tiles", C.c_int64), ("max_dups", C.c_uint64), ("workspace_bytes", C.c_uint64),
                ("mask_words", C.c_int64),
                ("bin_kernels", C.c_int32)]


class DeviceStatus(C.Structure):
    _fields_ = [("flags", C.c_uint32), ("live_seen", C.c_uint32), ("dups", C.c_uint64),
                ("dups_needed", C.c_uint64), ("valid_pairs", C.c_uint64), ("evals_fwd", C.c_uint64),
                ("evals_bwd", C.c_uint64), ("loss", C.c_double), ("ssim", C.c_double), ("nonfinite", C.c_uint64)]


P = C.c_void_p
ST = C.c_int

SIGNATURES = {
    "pk_version": (C.c_int32, []),
    "pk_status_string": (C.c_char_p, [ST]),
    "pk_atlas_layout": (ST, [C.c_int32, C.c_int32, C.POINTER(AtlasDesc)]),
    "pk_plan_create": (ST, [C.POINTER(AtlasDesc), C.POINTER(View), C.c_int32, C.c_int64,
                            C.POINTER(Options), C.POINTER(P)]),
    "pk_plan_sizes": (ST, [P, C.POINTER(Sizes)]),
    "pk_plan_options": (ST, [P, C.POINTER(Options)]),
    "pk_plan_destroy": (None, [P]),
    "pk_workspace_init": (ST, [P, P, P]),
    "pk_read_status": (ST, [P, P, P, C.POINTER(DeviceStatus)]),
    "pk_atlas_gather": (ST, [P, P, P, P, P, P, P, P, P]),
    "pk_project_and_sh": (ST, [P, P, P, P, P]),
    "pk_bin_and_sort": (ST, [P, P, P, P, P, P]),
    "pk_rasterize_fwd": (ST, [P, P, P, P, P, P, P, P, P]),
    "pk_rasterize_bwd": (ST, [P, P, P, P, P, P, P, P, P, P]),
    "pk_rasterize_bwd_accumulate": (ST, [P, P, P, P, P, P, P, P, P, P]),
    "pk_atlas_scatter_grad": (ST, [P, P, P, P, P, P, C.c_int32, P, P]),
    "pk_l1_loss_grad": (ST, [P, P, P, P, P, P]),
    "pk_rasterize_fwd_l1": (ST, [P, P, P, P, P, P, P, P, P, P, P]),
    "pk_rasterize_fwd_l1_clear": (ST, [P, P, P, P, P, P, P, P, P, P, P, P]),
    "pk_bin_and_sort_noalloc": (ST, [P, P, P, P, P, P]),
    "pk_motion_mask": (ST, [P, P, C.c_float, C.c_int32, P, P, P]),
    "pk_dynamic_mask": (ST, [P, P, P, P, C.c_float, P, C.c_int32, P, P]),
    "pk_lpo_minmax": (ST, [P, P, P, P, P, P]),
    "pk_lpo_encode": (ST, [P, P, P, P, P, P, P]),
    "pk_atlas_gather_lpo": (ST, [P, P, C.c_int32, P, P, P, P, P, P, P, P]),
    "pk_uv_max_k_scratch_bytes": (C.c_uint64, [C.c_int64, C.c_int32, C.c_int32]),
    "pk_uv_max_k": (ST, [P, C.c_int64, C.c_int64, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P]),
    "pk_photo_loss_grad": (ST, [P, P, P, C.c_float, P, P, P]),
    "pk_autotune": (ST, [P, P, P, P, P, P, P, P, P, P, P, P]),
    "pk_render_fwd": (ST, [P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]),
    "pk_render_bwd": (ST, [P, P, P, P, P, P, P, P, P, P, P, P, C.c_int32, P, P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load ``libpackuv.so``; raises if it is missing (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            if not build_if_missing:
                raise RuntimeError(
                    f"CUDA library {_build.LIB} is not built; run paper_2602_23040_gb300.build.build() "
                    "(nvcc, sm_103a). There is no CPU fallback.")
            _build.build()
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


class PackUVError(RuntimeError):
    def __init__(self, call: str, code: int):
        super().__init__(f"{call} failed: {STATUS_NAMES.get(code, code)} (status {code})")
        self.code = code


def check(call: str, code: int) -> None:
    if code != PK_OK:
        raise PackUVError(call, code)
