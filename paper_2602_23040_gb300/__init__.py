"""PackUV-GS render step on GB300: C-ABI CUDA library + thin torch binding.

The hot path (atlas gather, EWA projection and SH colour, tile binning and
radix sort, compositing forward and backward, texel-gradient scatter) runs
entirely in the hand-written sm_103a kernels of ``libpackuv.so``; this
package only marshals torch tensors and streams into the C calls.
"""

from . import build  # noqa: F401
from .api import (  # noqa: F401
    Plan,
    atlas_gather,
    atlas_gather_lpo,
    atlas_layout,
    atlas_scatter_grad,
    autotune,
    bin_and_sort,
    bin_and_sort_noalloc,
    dynamic_mask,
    l1_loss_grad,
    lpo_encode,
    lpo_minmax,
    make_workspace,
    motion_mask,
    photo_loss_grad,
    project_and_sh,
    rasterize_bwd,
    rasterize_bwd_accumulate,
    rasterize_fwd,
    rasterize_fwd_l1,
    rasterize_fwd_l1_clear,
    read_status,
    render_bwd,
    render_fwd,
    uv_max_k,
    workspace_init,
)
from .render import PerViewLoop, Renderer, render  # noqa: F401

__all__ = [
    "Plan", "Renderer", "PerViewLoop", "render", "atlas_layout", "atlas_gather", "project_and_sh",
    "bin_and_sort", "bin_and_sort_noalloc", "rasterize_fwd", "rasterize_fwd_l1", "rasterize_fwd_l1_clear",
    "rasterize_bwd", "rasterize_bwd_accumulate",
    "atlas_scatter_grad", "l1_loss_grad", "photo_loss_grad", "motion_mask", "dynamic_mask", "lpo_minmax", "lpo_encode", "atlas_gather_lpo", "uv_max_k", "autotune",
    "render_fwd", "render_bwd",
    "make_workspace", "workspace_init", "read_status",
]
