"""Shared test helpers: small seeded scenes, GPU runs through the C ABI, and
tolerance checks against the oracle."""

from __future__ import annotations

import numpy as np

import synth

# FP32 image tolerance on non-borderline pixels (max abs), gradient tolerance
# (relative L2 error per attribute group).
IMG_TOL = 1e-4
GRAD_RTOL = 1e-3
GROUPS = {"position": (0, 3), "log_scale": (3, 6), "rotation": (6, 10), "opacity": (10, 11),
          "sh_dc": (11, 14), "sh_rest": (14, None)}


def scene_small_sh3(seed=101, dtype=np.float32, frames=1, dyn=0.0):
    """128^2 atlas at 60 %, SH degree 3, clustered means, three ragged views."""
    views = []
    for f in range(frames):
        views += [synth.scenes.pinhole((0.4, 0.3, -3.2), 200, 136, frame=f),
                  synth.scenes.pinhole((-2.6, -0.5, -1.8), 136, 200, frame=f),
                  synth.scenes.pinhole((2.0, 1.2, 2.5), 96, 72, frame=f)]
    return synth.make_scene([(128, 128, 0, 0, 0)], (128, 128), 0.6, views, sh_degree=3, frames=frames,
                            texel_dtype=dtype, seed=seed, dynamic_frac=dyn, log_scale=(-3.6, 0.5))


def scene_multilevel_f16(seed=202):
    """Three levels 96^2, 48^2, 24^2 packed as in the paper, FP16 texels, uneven views."""
    levels = [(96, 96, 48, 0, 0), (48, 48, 0, 0, 0), (24, 24, 0, 48, 0)]
    rng = np.random.default_rng(seed)
    sizes = [(64, 48), (96, 54), (128, 72), (160, 90)]
    views = synth.scenes.ring_views((2, 1, 1), (-1.0, 0.0, 1.0), 4.0, [sizes[i] for i in rng.integers(0, 4, 4)])
    return synth.make_scene(levels, (144, 96), "uniform", views, sh_degree=3, texel_dtype=np.float16, seed=seed,
                            log_scale=(-3.4, 0.5))


def upload(scene, device="cuda"):
    import torch
    atlas = torch.from_numpy(np.ascontiguousarray(scene.atlas)).to(device)
    occ = torch.from_numpy(scene.occ.view(np.int32)).to(device)
    dyn = None if scene.dyn is None else torch.from_numpy(scene.dyn.view(np.int32)).to(device)
    return atlas, occ, dyn


def u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def check_images(got_img, got_T, ora, tol=IMG_TOL, border_tol=0.05, max_border_frac=0.03):
    """Non-borderline pixels within tol; borderline pixels bounded and rare."""
    P = len(ora["T"])
    border = ora["border"].astype(bool)
    # per-channel mask in the planar-per-view layout
    b3 = np.zeros(3 * P, bool)
    off = 0
    for n in ora["view_pixels"]:
        for c in range(3):
            b3[3 * off + c * n:3 * off + (c + 1) * n] = border[off:off + n]
        off += n
    err = np.abs(got_img.astype(np.float64) - ora["img"])
    Terr = np.abs(got_T.astype(np.float64) - ora["T"])
    assert err[~b3].max(initial=0.0) <= tol, f"image max err {err[~b3].max()}"
    assert Terr[~border].max(initial=0.0) <= tol, f"T max err {Terr[~border].max()}"
    assert border.mean() <= max_border_frac, f"borderline fraction {border.mean()}"
    if b3.any():
        assert err[b3].max() <= border_tol
    return dict(max_err=float(err[~b3].max(initial=0.0)), border=int(border.sum()))


def rel_err(a, b):
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / den) if den > 0 else float(np.linalg.norm(a))


def check_grads(got, ref, rtol=GRAD_RTOL):
    """got/ref: [D][G] gradients.  Relative L2 error per attribute group."""
    out = {}
    for name, (a, b) in GROUPS.items():
        g, r = got[a:b], ref[a:b]
        if r.size == 0:
            continue
        e = rel_err(g, r)
        out[name] = e
        assert e <= rtol, f"{name}: rel err {e}"
    return out
