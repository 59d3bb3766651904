"""Seeded generators for atlases, masks and cameras.

Channel layout of one texel (D = 11 + 3 (L+1)^2 channels):

    0..2   position xyz
    3..5   log-scale
    6..9   rotation quaternion (w, x, y, z)
    10     opacity logit
    11..   spherical-harmonic coefficients, coefficient j of colour c at 11 + 3 j + c

The atlas is planar, ``[F][D][H_A][W_A]``.  Occupancy and dynamic masks are
bit-packed rows, ``[H_A][ceil(W_A / 32)]`` uint32, texel x stored in bit
``x & 31`` of word ``x >> 5`` (least-significant bit first).

Cameras follow the usual computer-vision convention: camera space has x to
the right, y down and z forward; ``X_cam = R X_world + t``.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

CONFIG_NAMES = {
    1: "c1_64sq_atlas_1view_256sq_sh0",
    2: "c2_512sq_atlas_60pct_1view_1080p_sh3",
    3: "c3_1024sq_atlas_60pct_52view_rig_sh3",
    4: "c4_3level_fp16_atlas_16view_mixed_sh3",
    5: "c5_sequence_4frames_x_52view_dynamic30pct_sh3",
}

BASE_SEED = 20260223


def channel_count(sh_degree: int) -> int:
    return 11 + 3 * (sh_degree + 1) ** 2


@dataclasses.dataclass
class View:
    R: np.ndarray          # (3, 3) float64, world -> camera rotation
    t: np.ndarray          # (3,) float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    frame: int = 0         # which atlas frame this view renders


@dataclasses.dataclass
class Scene:
    name: str
    atlas: np.ndarray                  # [F][D][H][W] float32 or float16
    occ: np.ndarray                    # [H][Wp] uint32
    dyn: Optional[np.ndarray]          # [H][Wp] uint32 or None (all dynamic)
    levels: List[Tuple[int, int, int, int, int]]  # (w, h, x0, y0, rotated)
    sh_degree: int
    views: List[View]
    n_live: int                        # live texels per frame
    tile: int = 32                     # tile side of the binning (16 or 32; images do not depend on it)

    @property
    def frames(self) -> int:
        return int(self.atlas.shape[0])

    @property
    def channels(self) -> int:
        return int(self.atlas.shape[1])

    @property
    def atlas_hw(self) -> Tuple[int, int]:
        return int(self.atlas.shape[2]), int(self.atlas.shape[3])

    @property
    def pixels(self) -> int:
        return int(sum(v.width * v.height for v in self.views))


def pack_bits(mask: np.ndarray) -> np.ndarray:
    """Bool ``[H][W]`` -> uint32 ``[H][ceil(W/32)]``, bit x & 31 of word x >> 5."""
    h, w = mask.shape
    wp = (w + 31) // 32
    padded = np.zeros((h, wp * 32), dtype=bool)
    padded[:, :w] = mask
    by = np.packbits(padded.reshape(h, wp * 4, 8), axis=-1, bitorder="little")
    return np.ascontiguousarray(by.reshape(h, wp * 4)).view("<u4").reshape(h, wp).astype(np.uint32)


def unpack_bits(bits: np.ndarray, width: int) -> np.ndarray:
    h, wp = bits.shape
    by = np.ascontiguousarray(bits.astype("<u4")).view(np.uint8).reshape(h, wp * 4, 1)
    out = np.unpackbits(by, axis=-1, bitorder="little").reshape(h, wp * 32)
    return out[:, :width].astype(bool)


def look_at(eye: Sequence[float], target: Sequence[float] = (0.0, 0.0, 0.0),
            up: Sequence[float] = (0.0, 1.0, 0.0)) -> Tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) for a camera at ``eye`` looking at ``target``."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    return R, -R @ eye


def _f32(x):
    # cameras are generated in the precision the renderer's camera record carries (FP32)
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def pinhole(eye, width: int, height: int, fov_x_deg: float = 60.0, frame: int = 0) -> View:
    R, t = look_at(eye)
    fx = float(_f32((width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)))
    return View(R=_f32(R), t=_f32(t), fx=fx, fy=fx, cx=float(_f32(width / 2.0)), cy=float(_f32(height / 2.0)),
                width=width, height=height, frame=frame)


def ring_views(n_per_height: Sequence[int], heights: Sequence[float], radius: float,
               sizes: Sequence[Tuple[int, int]], frame: int = 0) -> List[View]:
    """Cameras on rings around the origin, all looking at it.

    ``sizes[i % len(sizes)]`` gives (width, height) of camera i.  The ring
    phase is offset so that no camera axis is aligned with a world axis
    (an aligned axis makes many depths tie exactly for quantised texels).
    """
    views = []
    i = 0
    for n, h in zip(n_per_height, heights):
        for k in range(n):
            phi = 2.0 * math.pi * (k + 0.5 * (h != 0) + 0.137) / n
            eye = (radius * math.cos(phi), h, radius * math.sin(phi))
            w, hh = sizes[i % len(sizes)]
            views.append(pinhole(eye, w, hh, frame=frame))
            i += 1
    return views


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    # QR of a Gaussian matrix, sign-fixed so the result is a proper rotation.
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _means(rng: np.random.Generator, n: int, kind: str) -> np.ndarray:
    if kind == "uniform":
        return rng.uniform(-1.0, 1.0, size=(n, 3))
    if kind == "clusters":
        k = 8
        centres = rng.uniform(-0.8, 0.8, size=(k, 3))
        sig = rng.uniform(0.05, 0.3, size=(k, 3))
        rots = [_random_rotation(rng) for _ in range(k)]
        lab = rng.integers(0, k, size=n)
        z = rng.standard_normal((n, 3))
        out = np.empty((n, 3))
        for c in range(k):
            sel = lab == c
            out[sel] = centres[c] + (z[sel] * sig[c]) @ rots[c].T
        return out
    raise ValueError(kind)


def _flow(rng: np.random.Generator, n_modes: int = 4):
    a = rng.standard_normal((n_modes, 3))
    a /= np.linalg.norm(a, axis=1).sum()          # max amplitude <= 1
    w = rng.normal(0.0, 2.0, size=(n_modes, 3))
    nu = rng.uniform(0.05, 0.2, size=n_modes)
    ph = rng.uniform(0, 2 * math.pi, size=n_modes)

    def f(mu: np.ndarray, t: float) -> np.ndarray:
        arg = mu @ w.T + nu[None, :] * t + ph[None, :]
        return np.sin(arg) @ a

    return f


def make_scene(levels: Sequence[Tuple[int, int, int, int, int]], atlas_wh: Tuple[int, int],
               occupancy, views: List[View], sh_degree: int = 3, frames: int = 1,
               texel_dtype=np.float32, means: str = "clusters", seed: int = BASE_SEED,
               dynamic_frac: float = 0.0, flow_amp: float = 0.05, frame_start: int = 0,
               name: str = "custom", tile: int = 32,
               log_scale: Tuple[float, float] = (-4.0, 0.5), mean_box: float = 1.0,
               uv_order: bool = True) -> Scene:
    """Generate one scene.

    ``occupancy`` is a fraction of texels per level (a float, applied to every
    level, or a sequence with one fraction per level, or ``"uniform"`` for
    U(0.4, 0.8) per level).  Exactly ``floor(fraction * level texels)``
    texels of each level are occupied.  ``log_scale`` is the (mean, std) of
    the log-scales and ``mean_box`` scales every mean (for small test scenes).
    ``uv_order``: live texels hold the means in the order of their spherical
    UV cells (as the method's maps do); False assigns them at random.
    """
    rng = np.random.default_rng(seed)
    aw, ah = atlas_wh
    D = channel_count(sh_degree)
    occ = np.zeros((ah, aw), dtype=bool)
    for li, (w, h, x0, y0, _rot) in enumerate(levels):
        if occupancy == "uniform":
            fr = rng.uniform(0.4, 0.8)
        elif isinstance(occupancy, (list, tuple)):
            fr = occupancy[li]
        else:
            fr = float(occupancy)
        n = int(math.floor(fr * w * h + 1e-9))
        sel = rng.permutation(w * h)[:n]
        m = np.zeros(w * h, dtype=bool)
        m[sel] = True
        occ[y0:y0 + h, x0:x0 + w] |= m.reshape(h, w)
    ys, xs = np.nonzero(occ)            # row-major order of live texels
    n_live = len(ys)

    mu0 = _means(rng, n_live, means) * mean_box
    if uv_order and n_live:
        # The method's maps hold each Gaussian at the texel of its UV cell
        # (the spherical cell of eq. uvgs2), so neighbouring texels hold
        # Gaussians of neighbouring directions.  The live texels are filled
        # in that order: means sorted by the row-major cell index of their
        # direction on the base level's w x h grid.
        w0, h0 = levels[0][0], levels[0][1]
        rho = np.linalg.norm(mu0, axis=1)
        theta = np.arctan2(mu0[:, 1], mu0[:, 0])
        phi = np.arccos(np.clip(mu0[:, 2] / np.maximum(rho, 1e-30), -1.0, 1.0))
        u = np.minimum(np.floor((np.pi + theta) / (2 * np.pi) * w0), w0 - 1).astype(np.int64)
        v = np.minimum(np.floor(phi / np.pi * h0), h0 - 1).astype(np.int64)
        mu0 = mu0[np.lexsort((u, v))]
    ls = rng.normal(log_scale[0], log_scale[1], size=(n_live, 3))
    q = rng.standard_normal((n_live, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = rng.standard_normal(n_live)
    nb = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.1, size=(n_live, nb, 3))
    sh[:, 0, :] = rng.normal(0.0, 0.5, size=(n_live, 3))

    dyn_mask = None
    is_dyn = np.ones(n_live, dtype=bool)
    if dynamic_frac > 0.0:
        actor = rng.uniform(-0.5, 0.5, size=3)
        dist = np.linalg.norm(mu0 - actor, axis=1)
        k = int(round(dynamic_frac * n_live))
        order = np.argsort(dist, kind="stable")
        is_dyn = np.zeros(n_live, dtype=bool)
        is_dyn[order[:k]] = True
        dm = np.zeros((ah, aw), dtype=bool)
        dm[ys[is_dyn], xs[is_dyn]] = True
        dyn_mask = pack_bits(dm)
    flow = _flow(rng) if dynamic_frac > 0.0 else None

    atlas = np.zeros((frames, D, ah, aw), dtype=np.float32)
    for f in range(frames):
        mu = mu0.copy()
        if flow is not None:
            mu[is_dyn] = mu0[is_dyn] + flow_amp * flow(mu0[is_dyn], float(frame_start + f))
        attrs = np.concatenate([mu, ls, q, logit[:, None], sh.reshape(n_live, nb * 3)], axis=1)
        atlas[f][:, ys, xs] = attrs.T.astype(np.float32)
    atlas = atlas.astype(texel_dtype)
    return Scene(name=name, atlas=np.ascontiguousarray(atlas), occ=pack_bits(occ), dyn=dyn_mask,
                 levels=[tuple(int(a) for a in l) for l in levels], sh_degree=sh_degree,
                 views=views, n_live=n_live, tile=tile)


def config_scene(k: int, n_views: Optional[int] = None, frame_start: int = 0, texel_dtype=None) -> Scene:
    """The five workload shapes, full size.  ``n_views`` truncates the view list;
    ``texel_dtype`` overrides the texel type (e.g. float32 gives the FP32
    masters of the FP16 workload: the same values before rounding)."""
    seed = BASE_SEED + k
    if k == 1:
        views = [pinhole((0.0, 0.0, -3.5), 256, 256)]
        sc = make_scene([(64, 64, 0, 0, 0)], (64, 64), 1.0, views, sh_degree=0,
                        means="uniform", seed=seed, name=CONFIG_NAMES[1])
    elif k == 2:
        views = [pinhole((0.0, 0.0, -4.0), 1920, 1080)]
        sc = make_scene([(512, 512, 0, 0, 0)], (512, 512), 0.6, views, seed=seed,
                        name=CONFIG_NAMES[2])
    elif k == 3:
        views = ring_views((18, 17, 17), (-1.0, 0.0, 1.0), 4.0, [(1920, 1080), (1280, 720)])
        sc = make_scene([(1024, 1024, 0, 0, 0)], (1024, 1024), 0.6, views[:n_views] if n_views else views,
                        seed=seed, name=CONFIG_NAMES[3])
    elif k == 4:
        rng = np.random.default_rng(seed + 1000)
        sizes = [(640, 480), (960, 540), (1280, 720), (1600, 900), (1920, 1080)]
        pick = [sizes[i] for i in rng.integers(0, len(sizes), size=16)]
        views = ring_views((6, 5, 5), (-1.0, 0.0, 1.0), 4.0, pick)
        levels = [(1024, 1024, 512, 0, 0), (512, 512, 0, 0, 0), (256, 256, 0, 512, 0)]
        sc = make_scene(levels, (1536, 1024), "uniform", views[:n_views] if n_views else views,
                        texel_dtype=np.float16 if texel_dtype is None else texel_dtype, seed=seed,
                        name=CONFIG_NAMES[4])
    elif k == 5:
        F = 4
        views = []
        for f in range(F):
            views += ring_views((18, 17, 17), (-1.0, 0.0, 1.0), 4.0, [(1920, 1080), (1280, 720)], frame=f)
        if n_views:
            views = [v for i, v in enumerate(views) if (i % 52) < n_views]
        sc = make_scene([(1024, 1024, 0, 0, 0)], (1024, 1024), 0.6, views, frames=F, seed=seed,
                        dynamic_frac=0.3, frame_start=frame_start, name=CONFIG_NAMES[5])
    else:
        raise ValueError(k)
    return sc


def actor_sphere(scene: Scene, frac: float = 0.3, seed: int = BASE_SEED + 76):
    """A moving "actor": a sphere around a random centre in [-0.5, 0.5]^3
    holding ``frac`` of the live Gaussians' frame-0 means."""
    rng = np.random.default_rng(seed)
    centre = rng.uniform(-0.5, 0.5, size=3)
    ys, xs = np.nonzero(unpack_bits(scene.occ, scene.atlas.shape[3]))
    mu = scene.atlas[0, 0:3][:, ys, xs].astype(np.float64).T
    radius = float(np.quantile(np.linalg.norm(mu - centre, axis=1), frac)) if len(mu) else 0.1
    return centre, radius


def motion_flow(views: Sequence[View], centre, radius: float, seed: int = BASE_SEED + 77, amp: float = 4.0,
                noise: float = 0.2) -> np.ndarray:
    """Synthetic optical-flow fields standing in for the per-camera flow maps.

    The moving region of each view is the silhouette of the actor sphere
    (``centre``, ``radius``): pixels whose viewing ray passes within
    ``radius`` of the centre.  There the flow has magnitude
    ``amp * sqrt(1 - dist^2 / radius^2)`` along a random direction per view;
    every component also carries i.i.d. N(0, ``noise``^2) flow.  Returned
    concatenated in view order, each view planar ``[2][H][W]`` (x component,
    then y), as one flat float32 array.
    """
    rng = np.random.default_rng(seed)
    centre = np.asarray(centre, np.float64)
    out = []
    for v in views:
        W, H = v.width, v.height
        f = rng.normal(0.0, noise, size=(2, H, W)).astype(np.float32)
        R = np.asarray(v.R, np.float64)
        eye = -R.T @ np.asarray(v.t, np.float64)
        xs = (np.arange(W) + 0.5 - v.cx) / v.fx
        ys = (np.arange(H) + 0.5 - v.cy) / v.fy
        d = np.empty((H, W, 3))
        d[..., 0] = xs[None, :]
        d[..., 1] = ys[:, None]
        d[..., 2] = 1.0
        d = d @ R                                    # camera ray -> world
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        w = centre - eye
        along = d @ w
        dist2 = float(w @ w) - along * along
        inside = (along > 0) & (dist2 < radius * radius)
        mag = np.where(inside, amp * np.sqrt(np.clip(1.0 - dist2 / (radius * radius), 0.0, 1.0)), 0.0)
        ang = rng.uniform(0.0, 2.0 * math.pi)
        f[0] += (mag * math.cos(ang)).astype(np.float32)
        f[1] += (mag * math.sin(ang)).astype(np.float32)
        out.append(f.reshape(-1))
    return np.concatenate(out) if out else np.zeros(0, np.float32)


def random_target(scene: Scene, seed: int = BASE_SEED + 99) -> np.ndarray:
    """U[0,1] target images, concatenated planar ``[V][3][H][W]`` as one flat float32 array."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=3 * scene.pixels).astype(np.float32)
