"""Buffers for one render-step launch, the per-view baseline loop, and the
differentiable ``render`` (a ``torch.autograd.Function`` over the C ABI).

A ``Renderer`` owns the device buffers of every intermediate (SoA
attributes, projected records, sorted lists, images, per-pixel state, 2D
gradients) and runs the six calls on one stream; torch only provides the
memory and the stream.  All views of its plan are rendered by one sequence
of launches (one persistent launch per rasterisation pass), which can be
captured in a CUDA graph after the first call.
"""

from __future__ import annotations

from typing import List, Optional

import torch

from . import api
from .api import Plan


class Renderer:
    def __init__(self, plan: Plan, device="cuda", ws: Optional[torch.Tensor] = None):
        p = plan
        self.plan = p
        self.device = torch.device(device)
        f32, i32 = torch.float32, torch.int32
        self.ws = ws if ws is not None else api.make_workspace(p, self.device)
        api.workspace_init(p, self.ws)
        # Per-channel [lo, hi] of the low-precision proxy: when set, forward()
        # reads the FP32 masters through the LPO quantiser (16-bit position,
        # 8-bit other channels) and the gradients pass it straight through.
        self.lohi: Optional[torch.Tensor] = None
        # Forward passes run so far: the per-pixel state a backward reads
        # (T_final, n_contrib, records, sorted lists) belongs to the latest.
        self.generation = 0
        self._alloc()

    def _alloc(self):
        p = self.plan
        f32, i32 = torch.float32, torch.int32
        # (at least one element each: the library takes no null pointer, even for an empty array)
        self.soa = torch.empty(max(p.D * p.G, 4), dtype=f32, device=self.device)
        self.texel = torch.empty(max(p.N, 1), dtype=i32, device=self.device)
        self.dynflag = torch.empty(max(p.N, 1), dtype=torch.uint8, device=self.device)
        self.records = torch.empty(12 * max(p.pairs, 1), dtype=f32, device=self.device)
        self.sorted_vals = torch.empty(int(p.max_dups) + 64, dtype=i32, device=self.device)
        self.ranges = torch.empty(2 * p.n_tiles, dtype=torch.int64, device=self.device)
        self.image = torch.empty(3 * p.P, dtype=f32, device=self.device)
        self.T = torch.empty(p.P, dtype=f32, device=self.device)
        self.n_contrib = torch.empty(p.P, dtype=i32, device=self.device)
        self.grad2d = torch.empty(12 * max(p.pairs, 1), dtype=f32, device=self.device)
        self.dimage = torch.empty(3 * p.P, dtype=f32, device=self.device)
        self._has_dyn = False

    # forward: a1 .. a4 (target: the L1 loss gradient fused into a4)
    def _front(self, atlas, occ, dyn, stream):
        # a1 .. a3: gather, projection, binning + sort
        p = self.plan
        self.generation += 1
        self._has_dyn = dyn is not None
        if self.lohi is not None:
            api.atlas_gather_lpo(p, atlas, api.LPO_MASTERS, self.lohi, occ, dyn, self.soa, self.texel, self.dynflag,
                                 self.ws, stream)
        else:
            api.atlas_gather(p, atlas, occ, dyn, self.soa, self.texel, self.dynflag, self.ws, stream)
        api.project_and_sh(p, self.soa, self.records, self.ws, stream)
        api.bin_and_sort(p, self.records, self.sorted_vals, self.ranges, self.ws, stream)

    def forward(self, atlas, occ, dyn=None, stream=None, target=None):
        p = self.plan
        self._front(atlas, occ, dyn, stream)
        if target is None:
            api.rasterize_fwd(p, self.records, self.sorted_vals, self.ranges, self.image, self.T, self.n_contrib,
                              self.ws, stream)
        else:
            api.rasterize_fwd_l1(p, self.records, self.sorted_vals, self.ranges, target, self.image, self.T,
                                 self.n_contrib, self.dimage, self.ws, stream)
        return self.image

    # backward: a5 .. a6
    def backward(self, dL_dimage, grad_atlas, accumulate=False, stream=None):
        p = self.plan
        api.rasterize_bwd(p, self.records, self.sorted_vals, self.ranges, self.T, self.n_contrib, dL_dimage,
                          self.grad2d, self.ws, stream)
        api.atlas_scatter_grad(p, self.soa, self.grad2d, self.dynflag if self._has_dyn else None, self.texel,
                               grad_atlas, accumulate, self.ws, stream)
        return grad_atlas

    def l1_step(self, atlas, occ, dyn, target, grad_atlas, stream=None):
        """One fitting step: forward with the L1 loss gradient, backward.  The
        forward also clears the 2D gradient records, so the backward adds to
        them without a clearing pass of its own."""
        p = self.plan
        self._front(atlas, occ, dyn, stream)
        api.rasterize_fwd_l1_clear(p, self.records, self.sorted_vals, self.ranges, target, self.image, self.T,
                                   self.n_contrib, self.dimage, self.grad2d, self.ws, stream)
        api.rasterize_bwd_accumulate(p, self.records, self.sorted_vals, self.ranges, self.T, self.n_contrib,
                                     self.dimage, self.grad2d, self.ws, stream)
        api.atlas_scatter_grad(p, self.soa, self.grad2d, self.dynflag if self._has_dyn else None, self.texel,
                               grad_atlas, False, self.ws, stream)

    def photo_step(self, atlas, occ, dyn, target, grad_atlas, lam: float = 0.2, stream=None):
        """One fitting step with the paper's photometric objective
        (1 - lam) L1 + lam (1 - SSIM)."""
        self.forward(atlas, occ, dyn, stream)
        api.photo_loss_grad(self.plan, self.image, target, self.dimage, self.ws, lam, stream)
        self.backward(self.dimage, grad_atlas, False, stream)

    def autotune(self, atlas, occ, dyn, target, stream=None, tiles=None) -> int:
        """Pick the launch options on the given inputs.  With ``tiles`` (tile
        sides, e.g. (32, 16)) each side gets a plan of its own -- the binning
        and the buffers differ -- and the one whose sort + forward (with the
        L1 term) + backward takes least device time is kept; then
        pk_autotune picks that plan's compositing batch and staging and its
        radix digit widths.  Returns the forward's batch.  Host-synchronising:
        call it before graph capture."""
        if tiles:
            times = {}
            for side in tiles:
                if side != self.plan.tile:
                    self._replan(self.plan.with_options(tile=int(side)), atlas, occ, dyn, stream)
                times[side] = self._time_sort_and_composite(target, stream)
            best = min(times, key=times.get)
            self.tile_times_ms = times
            if best != self.plan.tile:
                self._replan(self.plan.with_options(tile=int(best)), atlas, occ, dyn, stream)
        self.forward(atlas, occ, dyn, stream)
        api.l1_loss_grad(self.plan, self.image, target, self.dimage, self.ws, stream)
        return api.autotune(self.plan, self.records, self.sorted_vals, self.ranges, self.image, self.T,
                            self.n_contrib, self.dimage, self.grad2d, self.ws, stream)

    def _replan(self, plan, atlas, occ, dyn, stream=None):
        """Adopt another plan (new workspace and buffers) sized for these inputs."""
        self.plan = plan
        self.ws = api.make_workspace(plan, self.device)
        api.workspace_init(plan, self.ws)
        self._alloc()
        self.ensure_capacity(atlas, occ, dyn, stream)

    def _time_sort_and_composite(self, target, stream=None, reps=2) -> float:
        """Device milliseconds of bin_and_sort + fused forward/L1 + backward
        on the current records (one warm-up, then the mean of ``reps``)."""
        p = self.plan
        st = stream if stream is not None else torch.cuda.current_stream(self.device)

        def once():
            api.bin_and_sort(p, self.records, self.sorted_vals, self.ranges, self.ws, st)
            api.rasterize_fwd_l1(p, self.records, self.sorted_vals, self.ranges, target, self.image, self.T,
                                 self.n_contrib, self.dimage, self.ws, st)
            api.rasterize_bwd(p, self.records, self.sorted_vals, self.ranges, self.T, self.n_contrib, self.dimage,
                              self.grad2d, self.ws, st)
        once()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            once()
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def status(self, stream=None) -> dict:
        return api.read_status(self.plan, self.ws, stream)

    def ensure_capacity(self, atlas, occ, dyn=None, stream=None, headroom: float = 1.15) -> dict:
        """Run one forward; if the (pair, tile) entries overflowed the plan's
        capacity, re-plan with room for them (plus headroom) and run again.
        A host-synchronising call: use it before graph capture."""
        self.forward(atlas, occ, dyn, stream)
        st = self.status(stream)
        if st["flags"] & 1:
            need = int(st["dups_needed"] * headroom) + 4096
            self.plan = self.plan.with_capacity(need)
            self.ws = api.make_workspace(self.plan, self.device)
            api.workspace_init(self.plan, self.ws)
            self._alloc()
            self.forward(atlas, occ, dyn, stream)
            st = self.status(stream)
        return st


class PerViewLoop:
    """Baseline of prior art: the same kernels run one view at a time.

    Each view has its own single-view plan (and small workspace); the large
    intermediate buffers are shared, image outputs are written into slices
    of full-size buffers, and texel gradients accumulate over the views.
    The atlas is gathered again for every view, as a per-view training loop
    would.
    """

    @classmethod
    def for_scene(cls, scene, device="cuda", **kw):
        F, D, H, W = scene.atlas.shape
        tt = "f16" if str(scene.atlas.dtype) == "float16" else "f32"
        kw.setdefault("tile", scene.tile)
        args = dict(levels=scene.levels, atlas_wh=(W, H), sh_degree=scene.sh_degree, frames=F,
                    texel_type=tt, n_live=scene.n_live, **kw)
        return cls(args, scene.views, device)

    def __init__(self, scene_like_plan_args: dict, views, device="cuda"):
        self.plans: List[Plan] = [Plan(views=[v], **scene_like_plan_args) for v in views]
        self.device = torch.device(device)
        f32, i32 = torch.float32, torch.int32
        p0 = self.plans[0]
        self.ws = [api.make_workspace(p, self.device) for p in self.plans]
        for p, w in zip(self.plans, self.ws):
            api.workspace_init(p, w)
        self.soa = torch.empty(max(p0.D * p0.G, 4), dtype=f32, device=self.device)
        self.texel = torch.empty(max(p0.N, 1), dtype=i32, device=self.device)
        self.dynflag = torch.empty(max(p0.N, 1), dtype=torch.uint8, device=self.device)
        self.records = torch.empty(12 * max(p0.pairs, 1), dtype=f32, device=self.device)
        self.grad2d = torch.empty(12 * max(p0.pairs, 1), dtype=f32, device=self.device)
        md = max(int(p.max_dups) for p in self.plans)
        self.sorted_vals = torch.empty(md + 64, dtype=i32, device=self.device)
        self.ranges = torch.empty(2 * max(p.n_tiles for p in self.plans), dtype=torch.int64, device=self.device)
        P = sum(p.P for p in self.plans)
        self.image = torch.empty(3 * P, dtype=f32, device=self.device)
        self.T = torch.empty(P, dtype=f32, device=self.device)
        self.n_contrib = torch.empty(P, dtype=i32, device=self.device)
        self.dimage = torch.empty(3 * P, dtype=f32, device=self.device)
        self.offsets = []
        o = 0
        for p in self.plans:
            self.offsets.append(o)
            o += p.P

    def ensure_capacity(self, atlas, occ, dyn, target, grad_atlas, headroom: float = 1.15) -> bool:
        """Run one step; re-plan every view whose entries overflowed, once.
        Host-synchronising.  Returns True when every view fits."""
        self.step(atlas, occ, dyn, target, grad_atlas, loss=target is not None)
        grown = False
        for i, (p, w) in enumerate(zip(self.plans, self.ws)):
            st = api.read_status(p, w)
            if st["flags"] & 1:
                p2 = p.with_capacity(int(st["dups_needed"] * headroom) + 4096)
                w2 = api.make_workspace(p2, self.device)
                api.workspace_init(p2, w2)
                self.plans[i], self.ws[i] = p2, w2
                grown = True
        if grown:
            md = max(int(p.max_dups) for p in self.plans)
            if self.sorted_vals.numel() < md + 64:
                self.sorted_vals = torch.empty(md + 64, dtype=torch.int32, device=self.device)
            self.step(atlas, occ, dyn, target, grad_atlas, loss=target is not None)
        return all(api.read_status(p, w)["flags"] == 0 for p, w in zip(self.plans, self.ws))

    def _slices(self, i):
        o, P = self.offsets[i], self.plans[i].P
        return (self.image[3 * o:3 * (o + P)], self.T[o:o + P], self.n_contrib[o:o + P],
                self.dimage[3 * o:3 * (o + P)])

    def step(self, atlas, occ, dyn, target, grad_atlas, stream=None, loss=True):
        for i, (p, ws) in enumerate(zip(self.plans, self.ws)):
            img, T, nc, dimg = self._slices(i)
            api.atlas_gather(p, atlas, occ, dyn, self.soa, self.texel, self.dynflag, ws, stream)
            api.project_and_sh(p, self.soa, self.records, ws, stream)
            api.bin_and_sort(p, self.records, self.sorted_vals, self.ranges, ws, stream)
            if loss:
                o = self.offsets[i]
                api.rasterize_fwd_l1(p, self.records, self.sorted_vals, self.ranges, target[3 * o:3 * (o + p.P)],
                                     img, T, nc, dimg, ws, stream)
            else:
                api.rasterize_fwd(p, self.records, self.sorted_vals, self.ranges, img, T, nc, ws, stream)
            api.rasterize_bwd(p, self.records, self.sorted_vals, self.ranges, T, nc, dimg, self.grad2d, ws, stream)
            api.atlas_scatter_grad(p, self.soa, self.grad2d, self.dynflag if dyn is not None else None, self.texel,
                                   grad_atlas, i > 0, ws, stream)


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, master, renderer: Renderer, proxy, occ, dyn):
        src = master if proxy is None else proxy
        renderer.forward(src.detach().contiguous(), occ, dyn)
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.shape = master.shape
        ctx.device = master.device
        # the renderer keeps the per-pixel state for the backward; hand out a copy of the image
        return renderer.image.clone()

    @staticmethod
    def backward(ctx, grad_image):
        r: Renderer = ctx.renderer
        if r.generation != ctx.generation:
            # the buffers now hold a later forward's state: its gradients
            # would be handed to this call's inputs
            raise RuntimeError("render(): the Renderer ran another forward before this render's backward; "
                               "call backward first or give each render its own Renderer")
        grad = torch.zeros(ctx.shape, dtype=torch.float32, device=ctx.device)
        r.backward(grad_image.contiguous().float(), grad, accumulate=False)
        return grad, None, None, None, None


def render(master: torch.Tensor, renderer: Renderer, occ: torch.Tensor, dyn: Optional[torch.Tensor] = None,
           proxy: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Differentiable render of every view of ``renderer.plan``.

    ``master`` is the FP32 atlas ``[F][D][H][W]`` (the parameter).  If
    ``proxy`` (the FP16 texels actually read) is given, the gradient passes
    straight through it to ``master``.  Returns the concatenated planar
    images ``[3 * P]``; the gradient is zero on texels that are not live or
    are frozen by ``dyn``.  The renderer keeps the per-pixel state of its
    latest forward only: a backward through an earlier ``render`` on the
    same renderer raises instead of returning another call's gradients.
    """
    return _RenderFn.apply(master, renderer, proxy, occ, dyn)
