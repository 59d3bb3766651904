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


def i64(t) -> np.ndarray:
    """A device int64 tensor (tile ranges: 64-bit entry positions) on the host."""
    return t.cpu().numpy().astype(np.int64)


# Borderline bits of the oracle (oracle.B_*): image decisions only
B_Q, B_ALPHA, B_STOP, B_DEPTH, B_CULL = 1, 2, 4, 8, 16
IMAGE_BORDER = B_Q | B_ALPHA | B_STOP | B_DEPTH | B_CULL


def per_channel(values, view_pixels):
    """[P] per-pixel values -> [3P] in the planar-per-view image layout."""
    out = np.empty(3 * len(values), values.dtype)
    off = 0
    for n in view_pixels:
        for c in range(3):
            out[3 * off + c * n:3 * off + (c + 1) * n] = values[off:off + n]
        off += n
    return out


def check_images(got_img, got_T, ora, tol=IMG_TOL, max_border_frac=0.08, max_threshold_frac=0.012, label=""):
    """Every pixel within tol plus its own flip bound (the change the oracle
    computed for its borderline decisions going the other way; 0 off the
    borderline), colour and transmittance.  The borderline fraction is
    printed and bounded: all of it by max_border_frac, the threshold part
    (q, alpha, stop, cull) by max_threshold_frac.  Against the oracle's own
    FP64 projection most borderline pixels hold two contributors whose
    depths lie within their FP32 error bounds (a few 1e-6 world units), so
    the fraction grows with the contributors per pixel: 0.5-5 % at the
    full-size workloads, 0.03-0.06 % with identical FP32 records."""
    border = (ora["border"] & IMAGE_BORDER) != 0
    thresh = (ora["border"] & (IMAGE_BORDER & ~B_DEPTH)) != 0
    bound = ora["bound"]
    err = np.abs(got_img.astype(np.float64) - ora["img"])
    Terr = np.abs(got_T.astype(np.float64) - ora["T"])
    lim = tol + per_channel(bound[:, 0], ora["view_pixels"])
    over = err - lim
    b3 = per_channel(border, ora["view_pixels"])
    assert over.max(initial=-1.0) <= 0.0, \
        f"{label} image err {err[over.argmax()]:.3g} over its limit {lim[over.argmax()]:.3g} (borderline {b3[over.argmax()]})"
    overT = Terr - (tol + bound[:, 1])
    assert overT.max(initial=-1.0) <= 0.0, f"{label} T err {Terr[overT.argmax()]:.3g}"
    frac, tfrac = float(border.mean()), float(thresh.mean())
    print(f"{label} borderline pixels: {frac:.2e} (thresholds {tfrac:.2e}, depth order {frac - tfrac:.2e}); "
          f"max err off the borderline {err[~b3].max(initial=0.0):.2e}, on it {err[b3].max(initial=0.0):.2e} "
          f"(largest bound {bound[:, 0].max(initial=0.0):.2e})")
    assert frac <= max_border_frac, f"borderline fraction {frac}"
    assert tfrac <= max_threshold_frac, f"threshold-borderline fraction {tfrac}"
    return dict(max_err=float(err[~b3].max(initial=0.0)), max_err_border=float(err[b3].max(initial=0.0)),
                border=int(border.sum()), border_frac=frac, threshold_frac=tfrac)


def zero_on_borderline(w, ora):
    """dL/dimage w with every channel of the oracle's borderline pixels set
    to 0.  Where the two sides may take an image decision differently (a
    depth order or a threshold within FP32 error), the splats that pixel
    sends gradient to differ as well, so a gradient comparison leaves those
    pixels out on both sides; the images themselves are still checked
    there, against each pixel's flip bound."""
    border = (ora["border"] & IMAGE_BORDER) != 0
    w = np.array(w, copy=True)
    w[per_channel(border, ora["view_pixels"])] = 0
    return w


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


def oracle_views(orc, scene, vsel, dimg_by_view=None, tile=16, threads=None, soa_texel=None):
    """The FP64 oracle on the views vsel of a (large) scene, one thread per
    view (the oracle's C routines run without the interpreter lock): per
    view its own projection, lists, image with borderline bits and flip
    bounds, and, given dL/dimage of the view, its backward and texel
    gradient.  Returns images etc. concatenated over vsel in order, and
    the gradient [D][F*N] summed over the views."""
    import concurrent.futures as cf
    import os
    soa, texel, dynflag = soa_texel if soa_texel is not None else orc.gather(scene)
    N = len(texel)
    dyn = dynflag if scene.dyn is not None else None

    def one(i):
        v = vsel[i]
        va = orc.views_array([scene.views[v]])
        rec = orc.project(soa, N, scene.sh_degree, va)
        vals, ranges = orc.bin_sort(rec, va, tile)
        out = orc.render(rec, va, tile, vals, ranges)
        g = None
        if dimg_by_view is not None:
            g2 = orc.render_bwd(rec, va, tile, vals, ranges, np.asarray(dimg_by_view[i], np.float64))
            g = orc.scatter_grad(soa, N, scene.sh_degree, va, g2, dyn)
        return out, g

    n_thr = threads or min(len(vsel), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=n_thr) as ex:
        res = list(ex.map(one, range(len(vsel))))
    cat = lambda k: np.concatenate([r[0][k] for r in res])
    o = dict(img=cat("img"), T=cat("T"), last=cat("last"), border=cat("border"),
             bound=np.concatenate([r[0]["bound"] for r in res]),
             view_pixels=[scene.views[v].width * scene.views[v].height for v in vsel], texel=texel, N=N)
    if dimg_by_view is not None:
        o["grad_soa"] = sum(r[1] for r in res)
    return o


def view_slices(scene, vsel):
    """(image slice, pixel slice) of each view of vsel in the concatenated buffers."""
    poff = np.cumsum([0] + [v.width * v.height for v in scene.views])
    return [(slice(3 * poff[v], 3 * poff[v + 1]), slice(poff[v], poff[v + 1])) for v in vsel]
