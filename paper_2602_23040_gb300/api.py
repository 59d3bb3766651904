"""Python binding of the C ABI (``include/packuv.h``), one function per call.

Every function only checks and marshals its torch tensors (device, dtype,
size, contiguity) and forwards raw pointers plus the current CUDA stream to
the library; all arithmetic runs in the library's kernels.  uint32 buffers
are carried in ``torch.int32`` tensors (same bits).
"""

from __future__ import annotations

import ctypes as C
from typing import Iterable, List, Optional, Sequence, Tuple

import torch

from . import _native as N

_I32 = torch.int32
_I64 = torch.int64


def _stream(stream) -> C.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: Optional[torch.Tensor], name: str, dtype=None, numel: Optional[int] = None, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise ValueError(f"{name} has dtype {t.dtype}, expected {dtype}")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} holds {t.numel()} elements, needs {numel}")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# Plan
# ---------------------------------------------------------------------------

def atlas_layout(S: int, K: int):
    """Pyramid levels of an S x S base packed into one atlas (Sec. 4.1)."""
    lib = N.load()
    d = N.AtlasDesc()
    N.check("pk_atlas_layout", lib.pk_atlas_layout(S, K, C.byref(d)))
    levels = [(d.level[k].w, d.level[k].h, d.level[k].x0, d.level[k].y0, d.level[k].rotated)
              for k in range(d.num_levels)]
    return levels, (d.atlas_w, d.atlas_h)


def _views_array(views) -> "C.Array":
    arr = (N.View * len(views))()
    for i, v in enumerate(views):
        R = [float(x) for x in getattr(v.R, "reshape", lambda *_: v.R)(-1)]
        arr[i].R[:] = R
        arr[i].t[:] = [float(x) for x in v.t]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
        arr[i].width, arr[i].height, arr[i].frame = int(v.width), int(v.height), int(getattr(v, "frame", 0))
    return arr


STAGE_MODES = {"loads": 0, "bulk": 1}


class Plan:
    """Host-side plan of one launch: atlas descriptor, views and options."""

    def __init__(self, levels: Sequence[Tuple[int, int, int, int, int]], atlas_wh: Tuple[int, int],
                 sh_degree: int, frames: int, texel_type: str, views, n_live: int, tile: int = 32,
                 znear: float = 0.01, bg=(0.0, 0.0, 0.0), max_dups: int = 0, bin_mode: str = "ellipse",
                 batch: int = 128, stage_fwd: str = "loads", stage_bwd: str = "loads", batch_bwd: int = None,
                 sort_bits_tile: int = 8, sort_bits_depth: int = 8, count_evals: bool = False,
                 first_wait_polls: int = 0):
        lib = N.load()
        self._args = dict(levels=list(levels), atlas_wh=tuple(atlas_wh), sh_degree=sh_degree, frames=frames,
                          texel_type=texel_type, views=list(views), n_live=n_live, tile=tile, znear=znear,
                          bg=tuple(bg), max_dups=max_dups, bin_mode=bin_mode, batch=batch, stage_fwd=stage_fwd,
                          stage_bwd=stage_bwd, batch_bwd=batch_bwd, sort_bits_tile=sort_bits_tile,
                          sort_bits_depth=sort_bits_depth, count_evals=count_evals,
                          first_wait_polls=first_wait_polls)
        if batch_bwd is None:
            batch_bwd = batch
        d = N.AtlasDesc()
        d.atlas_w, d.atlas_h = int(atlas_wh[0]), int(atlas_wh[1])
        d.num_levels = len(levels)
        for k, (w, h, x0, y0, rot) in enumerate(levels):
            d.level[k] = N.Level(w, h, x0, y0, rot)
        d.sh_degree = int(sh_degree)
        d.frames = int(frames)
        d.texel_type = {"f32": 0, "f16": 1}[texel_type]
        o = N.Options()
        o.tile, o.znear, o.max_dups = int(tile), float(znear), int(max_dups)
        o.bg[:] = [float(b) for b in bg]
        o.bin_mode = {"rect": N.BIN_RECT, "ellipse": N.BIN_ELLIPSE}[bin_mode]
        o.batch = int(batch)
        o.stage_fwd = STAGE_MODES[stage_fwd]
        o.stage_bwd = STAGE_MODES[stage_bwd]
        o.batch_bwd = int(batch_bwd)
        o.sort_bits_tile, o.sort_bits_depth = int(sort_bits_tile), int(sort_bits_depth)
        o.count_evals = 1 if count_evals else 0
        o.first_wait_polls = int(first_wait_polls)
        self.bin_mode = bin_mode
        self.batch = int(batch)
        self.batch_bwd = int(batch_bwd)
        self.stage_fwd, self.stage_bwd = stage_fwd, stage_bwd
        self.sort_bits_tile, self.sort_bits_depth = int(sort_bits_tile), int(sort_bits_depth)
        self._views = _views_array(views)
        h = C.c_void_p()
        N.check("pk_plan_create", lib.pk_plan_create(C.byref(d), self._views, len(views), int(n_live),
                                                     C.byref(o), C.byref(h)))
        self.handle = h
        self.desc = d
        self.texel_type = texel_type
        self.views = list(views)
        s = N.Sizes()
        N.check("pk_plan_sizes", lib.pk_plan_sizes(h, C.byref(s)))
        self.sizes = s
        self.view_pixels = [int(v.width) * int(v.height) for v in views]

    @classmethod
    def for_scene(cls, scene, views=None, **kw):
        F, D, H, W = scene.atlas.shape
        tt = "f16" if str(scene.atlas.dtype) == "float16" else "f32"
        tile = kw.pop("tile", scene.tile)
        return cls(scene.levels, (W, H), scene.sh_degree, F, tt, views if views is not None else scene.views,
                   scene.n_live, tile=tile, **kw)

    def with_capacity(self, max_dups: int) -> "Plan":
        """Same plan with another capacity of (pair, tile) entries."""
        return self.with_options(max_dups=int(max_dups))

    def with_options(self, **kw) -> "Plan":
        """Same plan with some options replaced (e.g. the tile side)."""
        a = dict(self._args)
        a.update(kw)
        return Plan(**a)

    @property
    def tile(self) -> int:
        return int(self._args["tile"])

    def close(self):
        if getattr(self, "handle", None):
            N.load().pk_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # sizes
    @property
    def N(self):
        return self.sizes.n_live

    @property
    def G(self):
        return self.sizes.n_gauss

    @property
    def D(self):
        return self.sizes.channels

    @property
    def V(self):
        return self.sizes.n_views

    @property
    def pairs(self):
        return self.sizes.n_pairs

    @property
    def P(self):
        return self.sizes.n_pixels

    @property
    def n_tiles(self):
        return self.sizes.n_tiles

    @property
    def max_dups(self):
        return self.sizes.max_dups

    @property
    def mask_words(self):
        return self.sizes.mask_words


def make_workspace(plan: Plan, device="cuda") -> torch.Tensor:
    return torch.empty(int(plan.sizes.workspace_bytes), dtype=torch.uint8, device=device)


def workspace_init(plan: Plan, ws: torch.Tensor, stream=None) -> None:
    N.check("pk_workspace_init", N.load().pk_workspace_init(plan.handle, _ptr(ws, "workspace"), _stream(stream)))


def read_status(plan: Plan, ws: torch.Tensor, stream=None, check: bool = False) -> dict:
    s = N.DeviceStatus()
    rc = N.load().pk_read_status(plan.handle, _ptr(ws, "workspace"), _stream(stream), C.byref(s))
    if rc not in (0, 3, 4):
        N.check("pk_read_status", rc)
    out = {f: getattr(s, f) for f, _ in N.DeviceStatus._fields_}
    out["rc"] = rc
    if check:
        N.check("device status", rc)
    return out


# ---------------------------------------------------------------------------
# The six calls of the render step (and the L1 loss helper)
# ---------------------------------------------------------------------------

def atlas_gather(plan: Plan, atlas, occ, dyn, soa, texel, dynflag, ws, stream=None) -> None:
    F, D = plan.desc.frames, plan.D
    W, H = plan.desc.atlas_w, plan.desc.atlas_h
    words = H * ((W + 31) // 32)
    adt = torch.float16 if plan.texel_type == "f16" else torch.float32
    rc = N.load().pk_atlas_gather(
        plan.handle, _ptr(atlas, "atlas", adt, F * D * H * W), _ptr(occ, "occ", _I32, words),
        _ptr(dyn, "dyn", _I32, words, allow_none=True), _ptr(soa, "soa", torch.float32, D * plan.G),
        _ptr(texel, "texel", _I32, plan.N), _ptr(dynflag, "dynflag", torch.uint8, plan.N),
        _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_atlas_gather", rc)


def project_and_sh(plan: Plan, soa, records, ws, stream=None) -> None:
    rc = N.load().pk_project_and_sh(plan.handle, _ptr(soa, "soa", torch.float32, plan.D * plan.G),
                                    _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
                                    _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_project_and_sh", rc)


def bin_and_sort(plan: Plan, records, sorted_vals, tile_ranges, ws, stream=None) -> None:
    rc = N.load().pk_bin_and_sort(plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
                                  _ptr(sorted_vals, "sorted_vals", _I32, plan.max_dups),
                                  _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
                                  _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_bin_and_sort", rc)


def rasterize_fwd(plan: Plan, records, sorted_vals, tile_ranges, image, T_final, n_contrib, ws,
                  stream=None) -> None:
    rc = N.load().pk_rasterize_fwd(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(image, "image", torch.float32, 3 * plan.P), _ptr(T_final, "T_final", torch.float32, plan.P),
        _ptr(n_contrib, "n_contrib", _I32, plan.P), _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_rasterize_fwd", rc)


def rasterize_bwd(plan: Plan, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d, ws,
                  stream=None) -> None:
    rc = N.load().pk_rasterize_bwd(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(T_final, "T_final", torch.float32, plan.P), _ptr(n_contrib, "n_contrib", _I32, plan.P),
        _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs), _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_rasterize_bwd", rc)


def rasterize_bwd_accumulate(plan: Plan, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage, grad2d,
                             ws, stream=None) -> None:
    """rasterize_bwd adding to grad2d instead of clearing it first."""
    rc = N.load().pk_rasterize_bwd_accumulate(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(T_final, "T_final", torch.float32, plan.P), _ptr(n_contrib, "n_contrib", _I32, plan.P),
        _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs), _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_rasterize_bwd_accumulate", rc)


def atlas_scatter_grad(plan: Plan, soa, grad2d, dynflag, texel, grad_atlas, accumulate: bool, ws,
                       stream=None) -> None:
    F, D = plan.desc.frames, plan.D
    W, H = plan.desc.atlas_w, plan.desc.atlas_h
    rc = N.load().pk_atlas_scatter_grad(
        plan.handle, _ptr(soa, "soa", torch.float32, D * plan.G),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs),
        _ptr(dynflag, "dynflag", torch.uint8, plan.N, allow_none=True), _ptr(texel, "texel", _I32, plan.N),
        _ptr(grad_atlas, "grad_atlas", torch.float32, F * D * H * W), int(bool(accumulate)),
        _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_atlas_scatter_grad", rc)


def l1_loss_grad(plan: Plan, image, target, dL_dimage, ws, stream=None) -> None:
    rc = N.load().pk_l1_loss_grad(plan.handle, _ptr(image, "image", torch.float32, 3 * plan.P),
                                  _ptr(target, "target", torch.float32, 3 * plan.P),
                                  _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
                                  _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_l1_loss_grad", rc)


def rasterize_fwd_l1(plan: Plan, records, sorted_vals, tile_ranges, target, image, T_final, n_contrib, dL_dimage,
                     ws, stream=None) -> None:
    """rasterize_fwd with the L1 loss gradient fused into its epilogue."""
    rc = N.load().pk_rasterize_fwd_l1(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(target, "target", torch.float32, 3 * plan.P), _ptr(image, "image", torch.float32, 3 * plan.P),
        _ptr(T_final, "T_final", torch.float32, plan.P), _ptr(n_contrib, "n_contrib", _I32, plan.P),
        _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P), _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_rasterize_fwd_l1", rc)


def rasterize_fwd_l1_clear(plan: Plan, records, sorted_vals, tile_ranges, target, image, T_final, n_contrib,
                           dL_dimage, grad2d, ws, stream=None) -> None:
    """rasterize_fwd_l1 that also sets grad2d to zero (for rasterize_bwd_accumulate)."""
    rc = N.load().pk_rasterize_fwd_l1_clear(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(target, "target", torch.float32, 3 * plan.P), _ptr(image, "image", torch.float32, 3 * plan.P),
        _ptr(T_final, "T_final", torch.float32, plan.P), _ptr(n_contrib, "n_contrib", _I32, plan.P),
        _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs), _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_rasterize_fwd_l1_clear", rc)


def photo_loss_grad(plan: Plan, image, target, dL_dimage, ws, lam: float = 0.2, stream=None) -> None:
    """(1 - lam) L1 + lam (1 - SSIM) and its gradient (loss and mean SSIM
    land in the status block)."""
    rc = N.load().pk_photo_loss_grad(plan.handle, _ptr(image, "image", torch.float32, 3 * plan.P),
                                     _ptr(target, "target", torch.float32, 3 * plan.P), float(lam),
                                     _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
                                     _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_photo_loss_grad", rc)


def render_fwd(plan: Plan, atlas, occ, dyn, soa, texel, dynflag, records, sorted_vals, tile_ranges, image, T_final,
               n_contrib, ws, stream=None) -> None:
    """gather -> project -> bin and sort -> composite, one C call."""
    F, D = plan.desc.frames, plan.D
    W, H = plan.desc.atlas_w, plan.desc.atlas_h
    words = H * ((W + 31) // 32)
    adt = torch.float16 if plan.texel_type == "f16" else torch.float32
    rc = N.load().pk_render_fwd(
        plan.handle, _ptr(atlas, "atlas", adt, F * D * H * W), _ptr(occ, "occ", _I32, words),
        _ptr(dyn, "dyn", _I32, words, allow_none=True), _ptr(soa, "soa", torch.float32, D * plan.G),
        _ptr(texel, "texel", _I32, plan.N), _ptr(dynflag, "dynflag", torch.uint8, plan.N),
        _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32, plan.max_dups), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(image, "image", torch.float32, 3 * plan.P), _ptr(T_final, "T_final", torch.float32, plan.P),
        _ptr(n_contrib, "n_contrib", _I32, plan.P), _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_render_fwd", rc)


def render_bwd(plan: Plan, soa, dynflag, texel, records, sorted_vals, tile_ranges, T_final, n_contrib, dL_dimage,
               grad2d, grad_atlas, accumulate: bool, ws, stream=None) -> None:
    """composite adjoint -> texel scatter, one C call."""
    F, D = plan.desc.frames, plan.D
    W, H = plan.desc.atlas_w, plan.desc.atlas_h
    rc = N.load().pk_render_bwd(
        plan.handle, _ptr(soa, "soa", torch.float32, D * plan.G),
        _ptr(dynflag, "dynflag", torch.uint8, plan.N, allow_none=True), _ptr(texel, "texel", _I32, plan.N),
        _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs), _ptr(sorted_vals, "sorted_vals", _I32),
        _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles), _ptr(T_final, "T_final", torch.float32, plan.P),
        _ptr(n_contrib, "n_contrib", _I32, plan.P), _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs),
        _ptr(grad_atlas, "grad_atlas", torch.float32, F * D * H * W), 1 if accumulate else 0, _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_render_bwd", rc)


def autotune(plan: Plan, records, sorted_vals, tile_ranges, image, T_final, n_contrib, dL_dimage, grad2d, ws,
             stream=None) -> int:
    """pk_autotune: time the compositing forward and backward for each
    staging batch and mode, and the sort for each radix digit width, on the
    current inputs; the plan keeps the fastest choices.  Returns the
    forward's batch."""
    chosen = C.c_int32(0)
    rc = N.load().pk_autotune(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32), _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles),
        _ptr(image, "image", torch.float32, 3 * plan.P), _ptr(T_final, "T_final", torch.float32, plan.P),
        _ptr(n_contrib, "n_contrib", _I32, plan.P), _ptr(dL_dimage, "dL_dimage", torch.float32, 3 * plan.P),
        _ptr(grad2d, "grad2d", torch.float32, N.GRAD2D_FLOATS * plan.pairs), _ptr(ws, "workspace"), _stream(stream),
        C.byref(chosen))
    N.check("pk_autotune", rc)
    o = N.Options()
    N.check("pk_plan_options", N.load().pk_plan_options(plan.handle, C.byref(o)))
    names = {v: k for k, v in STAGE_MODES.items()}
    plan.batch, plan.stage_fwd, plan.stage_bwd = int(o.batch), names[o.stage_fwd], names[o.stage_bwd]
    plan.batch_bwd = int(o.batch_bwd)
    plan.sort_bits_tile, plan.sort_bits_depth = int(o.sort_bits_tile), int(o.sort_bits_depth)
    plan._args.update(batch=plan.batch, stage_fwd=plan.stage_fwd, stage_bwd=plan.stage_bwd,
                      batch_bwd=plan.batch_bwd, sort_bits_tile=plan.sort_bits_tile,
                      sort_bits_depth=plan.sort_bits_depth)
    return plan.batch


def bin_and_sort_noalloc(plan: Plan, records, sorted_vals, tile_ranges, n_entries, stream=None) -> None:
    """``pk_bin_and_sort`` for callers that cannot provide a workspace (for
    example code running inside another framework's frame loop, where device
    allocation is not allowed).  The scratch is a fixed 64 MiB array inside
    the library; ``n_entries`` (one int32 on the device) receives the entry
    count, -1 (0xFFFFFFFF) if the entries exceeded ``plan.max_dups``, or -2
    (0xFFFFFFFE) if a bounded device wait gave up or an index check failed
    (nothing emitted).  Calls that overlap on the GPU share that array and
    must not run concurrently."""
    rc = N.load().pk_bin_and_sort_noalloc(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(sorted_vals, "sorted_vals", _I32, plan.max_dups),
        _ptr(tile_ranges, "tile_ranges", _I64, 2 * plan.n_tiles), _ptr(n_entries, "n_entries", _I32, 1),
        _stream(stream))
    N.check("pk_bin_and_sort_noalloc", rc)


# ---------------------------------------------------------------------------
# Motion masks and the dynamic mask D_i
# ---------------------------------------------------------------------------

def motion_mask(plan: Plan, flow, tau: float, dilate_r: int, mask_bits, ws, stream=None) -> None:
    """Binary motion masks of every view: flow magnitude above ``tau``, then
    a square dilation of radius ``dilate_r`` (``flow``: float32 ``[2 * P]``,
    per view ``[2][H][W]``; ``mask_bits``: int32 ``[plan.mask_words]``)."""
    rc = N.load().pk_motion_mask(plan.handle, _ptr(flow, "flow", torch.float32, 2 * plan.P), float(tau),
                                 int(dilate_r), _ptr(mask_bits, "mask_bits", _I32, plan.mask_words),
                                 _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_motion_mask", rc)


def dynamic_mask(plan: Plan, records, texel, mask_bits, dyn, ws, r_max: float = 0.0, accumulate: bool = False,
                 stream=None) -> None:
    """Covariance-aware dynamic mask: sets the texel bit of every Gaussian
    whose d^2 <= 9 ellipse covers a moving pixel in some view (``dyn``:
    int32 ``[H_A][ceil(W_A/32)]``, the layout ``atlas_gather`` reads)."""
    W, H = plan.desc.atlas_w, plan.desc.atlas_h
    rc = N.load().pk_dynamic_mask(
        plan.handle, _ptr(records, "records", torch.float32, N.RECORD_FLOATS * plan.pairs),
        _ptr(texel, "texel", _I32, plan.N), _ptr(mask_bits, "mask_bits", _I32, plan.mask_words), float(r_max),
        _ptr(dyn, "dyn", _I32, H * ((W + 31) // 32)), 1 if accumulate else 0, _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_dynamic_mask", rc)


# ---------------------------------------------------------------------------
# Low-precision proxy (16-bit position, 8-bit everything else)
# ---------------------------------------------------------------------------

LPO_CODES, LPO_MASTERS = 0, 1


def lpo_minmax(plan: Plan, atlas, occ, lohi, ws, stream=None) -> None:
    """Per-channel [lo, hi] over the live texels of every frame (``lohi``:
    float32 ``[D][2]``) of the FP32 atlas."""
    F, D, W, H = plan.desc.frames, plan.D, plan.desc.atlas_w, plan.desc.atlas_h
    rc = N.load().pk_lpo_minmax(plan.handle, _ptr(atlas, "atlas", torch.float32, F * D * H * W),
                                _ptr(occ, "occ", _I32, H * ((W + 31) // 32)), _ptr(lohi, "lohi", torch.float32, 2 * D),
                                _ptr(ws, "workspace"), _stream(stream))
    N.check("pk_lpo_minmax", rc)


def lpo_encode(plan: Plan, atlas, occ, lohi, codes, ws, stream=None) -> None:
    """8-bit code planes ``[F][D+3][H][W]`` (uint8) of the FP32 atlas."""
    F, D, W, H = plan.desc.frames, plan.D, plan.desc.atlas_w, plan.desc.atlas_h
    rc = N.load().pk_lpo_encode(plan.handle, _ptr(atlas, "atlas", torch.float32, F * D * H * W),
                                _ptr(occ, "occ", _I32, H * ((W + 31) // 32)), _ptr(lohi, "lohi", torch.float32, 2 * D),
                                _ptr(codes, "codes", torch.uint8, F * (D + 3) * H * W), _ptr(ws, "workspace"),
                                _stream(stream))
    N.check("pk_lpo_encode", rc)


def atlas_gather_lpo(plan: Plan, src, src_kind: int, lohi, occ, dyn, soa, texel, dynflag, ws, stream=None) -> None:
    """``atlas_gather`` on the low-precision proxy: ``src`` is the uint8 code
    planes (``LPO_CODES``) or the FP32 master atlas (``LPO_MASTERS``)."""
    F, D, W, H = plan.desc.frames, plan.D, plan.desc.atlas_w, plan.desc.atlas_h
    words = H * ((W + 31) // 32)
    if src_kind == LPO_CODES:
        sp = _ptr(src, "codes", torch.uint8, F * (D + 3) * H * W)
    else:
        sp = _ptr(src, "atlas", torch.float32, F * D * H * W)
    rc = N.load().pk_atlas_gather_lpo(
        plan.handle, sp, int(src_kind), _ptr(lohi, "lohi", torch.float32, 2 * D), _ptr(occ, "occ", _I32, words),
        _ptr(dyn, "dyn", _I32, words, allow_none=True), _ptr(soa, "soa", torch.float32, D * plan.G),
        _ptr(texel, "texel", _I32, plan.N), _ptr(dynflag, "dynflag", torch.uint8, plan.N), _ptr(ws, "workspace"),
        _stream(stream))
    N.check("pk_atlas_gather_lpo", rc)


# ---------------------------------------------------------------------------
# UV cells and Max-K UV pruning
# ---------------------------------------------------------------------------

def uv_max_k(soa, n: int, map_w: int, map_h: int, K: int, cell, rank, keep, count, scratch=None, stream=None):
    """Cells of eq. uvgs2 on a ``map_w`` (M, along u) x ``map_h`` (N, along v)
    map and the top-K Gaussians per cell by opacity, for the first ``n``
    columns of ``soa`` (float32 ``[D][stride]``).  Returns the scratch
    tensor (allocated if not given; reuse it)."""
    need = int(N.load().pk_uv_max_k_scratch_bytes(n, map_w, map_h))
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(max(need, 256), dtype=torch.uint8, device=soa.device)
    stride = soa.shape[1] if soa.dim() == 2 else n
    rc = N.load().pk_uv_max_k(_ptr(soa, "soa", torch.float32), int(n), int(stride), int(map_w), int(map_h), int(K),
                              _ptr(cell, "cell", _I32, n), _ptr(rank, "rank", _I32, n),
                              _ptr(keep, "keep", torch.uint8, n), _ptr(count, "count", _I32, map_w * map_h),
                              _ptr(scratch, "scratch"), _stream(stream))
    N.check("pk_uv_max_k", rc)
    return scratch
