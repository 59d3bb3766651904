"""Pins of the oracle's motion masks and dynamic mask to facts outside it:
scipy's binary dilation, scipy's Mahalanobis distance over every pixel of
the image (the definition D_{i,c} = OR over the d^2 <= 9 ellipse, Sec. 4.2
"Covariance-Aware Gaussian Masking"), a closed-form isotropic footprint,
the OR over cameras and the r_max clamp of Alg. 1."""

import math

import numpy as np
import pytest

import synth
from synth.scenes import View

ndimage = pytest.importorskip("scipy.ndimage")
distance = pytest.importorskip("scipy.spatial.distance")


def _flow(rng, W, H, p_moving=0.05):
    f = rng.normal(0.0, 0.4, size=(2, H, W)).astype(np.float32)
    hot = rng.random((H, W)) < p_moving
    f[0][hot] += np.float32(3.0)
    return f


@pytest.mark.parametrize("W,H,r", [(37, 23, 0), (37, 23, 1), (64, 40, 3), (70, 9, 5), (33, 31, 40)])
def test_motion_mask_is_scipy_dilation_of_the_threshold(orc, W, H, r):
    rng = np.random.default_rng(W * 100 + H + r)
    f = _flow(rng, W, H)
    tau = np.float32(1.0)
    mag = np.sqrt(f[0] * f[0] + f[1] * f[1])            # float32 ops, IEEE rounded
    raw = mag > tau
    want = ndimage.binary_dilation(raw, structure=np.ones((2 * r + 1, 2 * r + 1), bool)) if r else raw
    got = orc.motion_mask(f, tau, r)
    assert got.dtype == np.uint8 and got.shape == (H, W)
    np.testing.assert_array_equal(got.astype(bool), want)


def test_motion_mask_non_finite_flow(orc):
    f = np.zeros((2, 4, 5), np.float32)
    f[0, 1, 1] = np.nan
    f[1, 2, 3] = np.inf
    got = orc.motion_mask(f, 0.5, 0)
    assert got[1, 1] == 0 and got[2, 3] == 1 and got.sum() == 1


def _small_scene(seed, views, log_scale=(-2.5, 0.5)):
    return synth.make_scene([(16, 12, 0, 0, 0)], (16, 12), 0.7, views, sh_degree=0, means="uniform",
                            seed=seed, log_scale=log_scale, mean_box=0.8)


def _brute_force(rec, va, masks):
    """OR over views and over EVERY pixel of the image: masked and
    mahalanobis(p, m, conic)^2 <= 9."""
    V, N, _ = rec.shape
    D = np.zeros(N, np.uint8)
    off = 0
    for v in range(V):
        W, H = int(va[v, 16]), int(va[v, 17])
        M = masks[off:off + W * H].reshape(H, W)
        ys, xs = np.nonzero(M)
        for g in range(N):
            r = rec[v, g]
            if not r[7] > 0:
                continue
            VI = np.array([[r[2], r[3]], [r[3], r[4]]])
            for x, y in zip(xs, ys):
                if distance.mahalanobis((x + 0.5, y + 0.5), (r[0], r[1]), VI) ** 2 <= 9.0:
                    D[g] = 1
                    break
        off += W * H
    return D


def test_dynamic_mask_equals_the_definition_over_all_pixels(orc):
    views = synth.scenes.ring_views((2, 1, 1), (-0.5, 0.0, 0.5), 3.0, [(48, 40), (37, 29)])
    sc = _small_scene(12, views, (-3.5, 0.4))
    va = orc.views_array(views)
    masks = orc.motion_masks(synth.motion_flow(views, *synth.actor_sphere(sc, 0.1, seed=5), seed=5), va, 1.0, 0)
    D, border, _, rec = orc.dynamic_mask_scene(sc, masks)
    want = _brute_force(rec, va, masks)
    ok = border == 0
    assert ok.mean() > 0.97
    np.testing.assert_array_equal(D[ok], want[ok])
    assert 0.3 < D.mean() < 0.7          # the case is not degenerate


def test_dynamic_mask_is_the_or_over_cameras(orc):
    views = synth.scenes.ring_views((2, 1, 1), (-0.5, 0.0, 0.5), 3.0, [(48, 40), (37, 29)])
    sc = _small_scene(12, views)
    va = orc.views_array(views)
    masks = orc.motion_masks(synth.motion_flow(views, *synth.actor_sphere(sc, 0.2, seed=6), seed=6), va, 1.0, 0)
    D, _, _, rec = orc.dynamic_mask_scene(sc, masks)
    acc = np.zeros_like(D)
    off = 0
    for v in range(len(views)):
        n = views[v].width * views[v].height
        Dv, _ = orc.dynamic_mask(rec[v:v + 1], va[v:v + 1], masks[off:off + n])
        acc |= Dv
        off += n
    np.testing.assert_array_equal(D, acc)


def _isotropic(orc, ls, d=4.0, W=64, H=48, f=60.0):
    """One isotropic Gaussian at the origin, camera on the -z axis looking
    along +z: Sigma2D = ((f s / d)^2 + 0.3) I and m = (cx, cy)."""
    D = 14
    soa = np.zeros((D, 1))
    soa[3:6, 0] = ls
    soa[6, 0] = 1.0
    view = View(R=np.eye(3), t=np.array([0.0, 0.0, d]), fx=f, fy=f, cx=W / 2, cy=H / 2, width=W, height=H)
    va = orc.views_array([view])
    rec = orc.project(soa, 1, 0, va)
    sig2 = (f * math.exp(ls) / d) ** 2 + 0.3
    return rec, va, sig2


@pytest.mark.parametrize("ls", [-3.0, -2.0, -1.5])
def test_dynamic_mask_closed_form_isotropic_footprint(orc, ls):
    rec, va, sig2 = _isotropic(orc, ls)
    W, H = 64, 48
    R9 = 3.0 * math.sqrt(sig2)              # d^2 = |p - m|^2 / sigma^2 <= 9
    hits = 0
    for dx in range(0, W // 2):
        for dy in (0, 3):
            dist2 = (dx + 0.5) ** 2 + (dy + 0.5) ** 2
            if abs(math.sqrt(dist2) - R9) < 1e-3:
                continue
            M = np.zeros(W * H, np.uint8)
            M[(H // 2 + dy) * W + W // 2 + dx] = 1
            Dg, b = orc.dynamic_mask(rec, va, M)
            assert b[0] == 0
            assert Dg[0] == (dist2 <= R9 * R9), (dx, dy, dist2, R9 * R9)
            hits += int(Dg[0])
    assert hits > 0


def test_dynamic_mask_r_max_clamps_the_scanned_square(orc):
    rec, va, sig2 = _isotropic(orc, -1.5)
    W, H = 64, 48
    assert 3.0 * math.sqrt(sig2) > 4.0       # the ellipse reaches pixels 3 away
    M = np.zeros(W * H, np.uint8)
    M[(H // 2) * W + W // 2 + 3] = 1         # centre 3.5 px right of m
    assert orc.dynamic_mask(rec, va, M)[0][0] == 1
    assert orc.dynamic_mask(rec, va, M, r_max=3.0)[0][0] == 0   # |dx| = 3.5 > 3
    assert orc.dynamic_mask(rec, va, M, r_max=4.0)[0][0] == 1
    r32 = rec.reshape(-1, 12).astype(np.float32)
    assert orc.dynamic_mask32(r32, va, M)[0] == 1
    assert orc.dynamic_mask32(r32, va, M, r_max=3.0)[0] == 0


def test_dynamic_mask_all_moving_marks_every_gaussian_inside_the_image(orc):
    """With M = 1 everywhere, a valid Gaussian whose mean lies inside the
    image always has a pixel centre within sqrt(0.5) of the mean, and its
    ellipse (smallest axis 3 sqrt(0.3) > 1.6 px) contains it."""
    views = synth.scenes.ring_views((1, 1, 1), (-0.5, 0.0, 0.5), 3.0, [(40, 30)])
    sc = _small_scene(13, views)
    va = orc.views_array(views)
    masks = np.ones(sum(v.width * v.height for v in views), np.uint8)
    D, border, _, rec = orc.dynamic_mask_scene(sc, masks)
    inside = np.zeros(len(D), bool)
    for v, view in enumerate(views):
        r = rec[v]
        inside |= (r[:, 7] > 0) & (r[:, 0] >= 0) & (r[:, 0] <= view.width) & (r[:, 1] >= 0) & \
            (r[:, 1] <= view.height)
    assert inside.any()
    assert np.all(D[inside] == 1)
    D0, _ = orc.dynamic_mask(rec, va, np.zeros_like(masks))
    assert D0.sum() == 0


def test_fp32_stage_agrees_with_fp64_away_from_the_borderline(orc):
    views = synth.scenes.ring_views((2, 2, 1), (-0.5, 0.0, 0.5), 3.0, [(48, 40), (37, 29)])
    sc = _small_scene(14, views)
    va = orc.views_array(views)
    masks = orc.motion_masks(synth.motion_flow(views, *synth.actor_sphere(sc, 0.3, seed=7), seed=7), va, 1.0, 2)
    D, border, _, rec = orc.dynamic_mask_scene(sc, masks)
    D32 = orc.dynamic_mask32(rec.reshape(-1, 12).astype(np.float32), va, masks)
    ok = border == 0
    np.testing.assert_array_equal(D32[ok], D[ok])
