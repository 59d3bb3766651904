"""Pins of the oracle's borderline rule (test infrastructure).

The rule marks a pixel borderline when an FP32 evaluation of one of its
decisions could go the other way, and bounds what the flip can do to the
pixel.  Two facts are pinned here against computations that do not go
through that code:

* the bound on the FP32 error of a projected mean holds for the mean
  evaluated in float32 arithmetic (numpy, several operation orders, with and
  without fused multiply-adds) on random Gaussians and cameras;
* on splats placed exactly at the thresholds (a footprint through a pixel
  centre, alpha at 1/255, a stack ending at T = 1e-4, equal FP32 depths),
  perturbations small enough to stay inside the rule's tolerances flip
  those decisions, and every pixel then moves by no more than the bound the
  oracle reported for it, while some pixels do move by far more than the
  continuous effect of the perturbation.
"""

import math

import numpy as np
import pytest

import synth


def _fma32(a, b, c):
    """float32 fused multiply-add: the exact a*b + c, rounded once (the
    float64 product of two float32 values is exact)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_mean_error_bound_holds_for_float32_evaluations(orc):
    rng = np.random.default_rng(5)
    views = synth.scenes.ring_views((6, 5, 5), (-1.0, 0.0, 1.0), 4.0, [(1920, 1080), (1280, 720)])
    va = orc.views_array(views)
    N = 4000
    mu = rng.uniform(-1.0, 1.0, (N, 3)).astype(np.float32)
    ratio_max = 0.0
    for v, vw in enumerate(views):
        R = np.asarray(vw.R, np.float32)
        t = np.asarray(vw.t, np.float32)
        fx, fy, cx, cy = (np.float32(a) for a in (vw.fx, vw.fy, vw.cx, vw.cy))
        X64 = mu.astype(np.float64) @ R.astype(np.float64).T + t.astype(np.float64)
        ok = X64[:, 2] > 0.5
        m64 = np.stack([fx * X64[:, 0] / X64[:, 2] + cx, fy * X64[:, 1] / X64[:, 2] + cy], 1)
        # the oracle's record fields the bound reads: m, z
        rec = np.zeros((1, N, 12))
        rec[0, :, 0:2] = m64
        rec[0, :, 6] = X64[:, 2]
        rec[0, :, 7] = np.where(ok, 1.0, 0.0)
        mt, zt = orc.mean_error_bounds(rec, va[v:v + 1])
        mt, zt = mt[0], zt[0]
        # float32 evaluations in several orders
        evals = []
        for order in range(3):
            X = np.zeros((N, 3), np.float32)
            for i in range(3):
                if order == 0:
                    X[:, i] = ((R[i, 0] * mu[:, 0] + R[i, 1] * mu[:, 1]) + R[i, 2] * mu[:, 2]) + t[i]
                elif order == 1:
                    X[:, i] = (R[i, 2] * mu[:, 2] + (R[i, 1] * mu[:, 1] + R[i, 0] * mu[:, 0])) + t[i]
                else:
                    X[:, i] = _fma32(np.full(N, R[i, 2], np.float32), mu[:, 2],
                                     _fma32(np.full(N, R[i, 1], np.float32), mu[:, 1],
                                            (R[i, 0] * mu[:, 0]).astype(np.float32))) + t[i]
            iz = (np.float32(1.0) / X[:, 2]).astype(np.float32)
            mx = [((fx * X[:, 0]) * iz) + cx, (fx * (X[:, 0] * iz)) + cx, (fx * X[:, 0]) / X[:, 2] + cx][order]
            my = [((fy * X[:, 1]) * iz) + cy, (fy * (X[:, 1] * iz)) + cy, (fy * X[:, 1]) / X[:, 2] + cy][order]
            evals.append((mx.astype(np.float64), my.astype(np.float64), X[:, 2].astype(np.float64)))
        for mx, my, z in evals:
            err = np.maximum(np.abs(mx - m64[:, 0]), np.abs(my - m64[:, 1]))
            assert np.all(err[ok] <= mt[ok]), (v, float((err[ok] / mt[ok]).max()))
            assert np.all(np.abs(z - X64[:, 2])[ok] <= zt[ok])
            ratio_max = max(ratio_max, float((err[ok] / mt[ok]).max()))
    # a bound, not a vacuous one: the worst observed error is a sizeable part of it
    assert ratio_max > 0.05, ratio_max


def _threshold_scene(seed):
    """Records of one 48 x 48 view built to sit on the compositing thresholds."""
    rng = np.random.default_rng(seed)
    W = H = 48
    recs = []

    def add(mx, my, a, b, c, o, z, rgb):
        r = np.zeros(12)
        r[0:2] = mx, my
        r[2:5] = a, b, c
        r[5] = o
        r[6] = z
        S = np.linalg.inv(np.array([[a, b], [b, c]]))
        tr, det = S[0, 0] + S[1, 1], np.linalg.det(S)
        r[7] = math.ceil(3 * math.sqrt(0.5 * (tr + math.sqrt(max(0.0, tr * tr - 4 * det))))) + 1
        r[8:11] = rgb
        recs.append(r)

    for k in range(40):
        # footprint boundary q = 9 through a pixel centre
        px, py = rng.integers(4, W - 4) + 0.5, rng.integers(4, H - 4) + 0.5
        s2 = rng.uniform(1.0, 4.0)
        th = rng.uniform(0, 2 * math.pi)
        add(px + 3 * math.sqrt(s2) * math.cos(th), py + 3 * math.sqrt(s2) * math.sin(th), 1 / s2, 0.0, 1 / s2,
            rng.uniform(0.4, 1.0), rng.uniform(1.0, 5.0), rng.uniform(0, 1, 3))
        # alpha = 1/255 at a pixel centre: q = 2 ln(255 o) < 9
        px, py = rng.integers(4, W - 4) + 0.5, rng.integers(4, H - 4) + 0.5
        o = rng.uniform(0.05, 0.3)
        qa = 2 * math.log(255 * o)
        th = rng.uniform(0, 2 * math.pi)
        add(px + math.sqrt(qa * s2) * math.cos(th), py + math.sqrt(qa * s2) * math.sin(th), 1 / s2, 0.0, 1 / s2, o,
            rng.uniform(1.0, 5.0), rng.uniform(0, 1, 3))
    # stacks of opaque splats (alpha clamped at 0.99): T = 1e-2, then about 1e-4
    for k in range(6):
        px, py = rng.integers(8, W - 8) + 0.5, rng.integers(8, H - 8) + 0.5
        z0 = rng.uniform(0.2, 0.9)
        for j in range(3):
            add(px, py, 0.25, 0.0, 0.25, 1.0, z0 + 0.01 * j, rng.uniform(0, 1, 3))
    # pairs at the same FP32 depth, different places
    for k in range(8):
        px, py = rng.integers(6, W - 6) + 0.5, rng.integers(6, H - 6) + 0.5
        z = float(np.float32(rng.uniform(1.0, 5.0)))
        add(px, py, 0.3, 0.05, 0.4, 0.8, z, rng.uniform(0, 1, 3))
        add(px + 0.7, py - 0.4, 0.35, -0.05, 0.3, 0.7, z, rng.uniform(0, 1, 3))
    rec = np.array(recs)[None]
    view = synth.View(R=np.eye(3), t=np.zeros(3), fx=40.0, fy=40.0, cx=24.0, cy=24.0, width=W, height=H)
    return rec, view


def test_flip_bound_covers_flipped_decisions(orc):
    rec, view = _threshold_scene(9)
    va = orc.views_array([view])
    q_rel = 1e-9
    vals, ranges = orc.bin_sort(rec, va, 16, orc.BIN_RECT)
    base = orc.render(rec, va, 16, vals, ranges, m_tol=0.0, q_rel=q_rel)
    P = 48 * 48
    assert (base["border"] & orc.IMAGE_BORDER).any()
    rng = np.random.default_rng(1)
    moved = 0.0
    for trial in range(12):
        r2 = rec.copy()
        n = r2.shape[1]
        # conics scaled within q_rel / 2: q crosses 9 where it sat on it
        r2[0, :, 2:5] *= (1.0 + rng.choice([-0.5, 0.5], n) * q_rel)[:, None]
        # opacities within the alpha band (ln alpha off by 5e-6 < 1e-5)
        r2[0, :, 5] *= np.exp(rng.choice([-5e-6, 5e-6], n))
        # equal FP32 depths split by one FP32 ulp either way
        z32 = r2[0, :, 6].astype(np.float32)
        step = rng.choice([-1, 0, 1], n)
        r2[0, :, 6] = np.where(step > 0, np.nextafter(z32, np.float32(np.inf)),
                               np.where(step < 0, np.nextafter(z32, np.float32(0)), z32)).astype(np.float64)
        v2, g2 = orc.bin_sort(r2, va, 16, orc.BIN_RECT)
        got = orc.render(r2, va, 16, v2, g2, m_tol=0.0, q_rel=q_rel)
        dimg = np.abs(got["img"] - base["img"]).reshape(3, P).max(0)
        dT = np.abs(got["T"] - base["T"])
        # the continuous effect of these perturbations is below 1e-5 everywhere
        assert np.all(dimg <= base["bound"][:, 0] + 1e-5), float((dimg - base["bound"][:, 0]).max())
        assert np.all(dT <= base["bound"][:, 1] + 1e-5)
        assert np.all(dimg[(base["border"] & orc.IMAGE_BORDER) == 0] <= 1e-5)
        moved = max(moved, float(dimg.max()))
    assert moved > 1e-3      # decisions did flip: the check is not vacuous


def test_flip_bound_is_zero_off_the_borderline(orc):
    sc = synth.make_scene([(48, 48, 0, 0, 0)], (48, 48), 0.6, [synth.scenes.pinhole((0.4, 0.3, -3.2), 96, 72)],
                          sh_degree=1, seed=3, log_scale=(-3.4, 0.5))
    f = orc.forward(sc)
    off = (f["border"] & orc.IMAGE_BORDER) == 0
    assert np.all(f["bound"][off] == 0.0)
    assert f["bound"][~off, 0].max(initial=0.0) < 1.0
