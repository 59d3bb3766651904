"""Pins of the oracle's photometric objective (Sec. 4.2 "Objective",
(1 - lambda) L1 + lambda (1 - SSIM)): scipy's correlation with zero padding
for the window sums, identical images (SSIM 1, zero gradient), the
closed form on constant images, symmetry, the two ends of lambda, and FP64
central differences of the loss for the gradient."""

import numpy as np
import pytest

ndimage = pytest.importorskip("scipy.ndimage")


def _views(*wh):
    va = np.zeros((len(wh), 20))
    for i, (w, h) in enumerate(wh):
        va[i, 16], va[i, 17] = w, h
    return va


def _window():
    k = np.arange(-5, 6, dtype=np.float64)
    g = np.exp(-k * k / (2 * 1.5 * 1.5))
    g /= g.sum()
    return np.outer(g, g)


def _planes(a, va):
    out, off = [], 0
    for w, h in va[:, 16:18].astype(int):
        n = w * h
        out.append(a[3 * off:3 * off + 3 * n].reshape(3, h, w))
        off += n
    return out


def test_ssim_map_from_scipy_window_sums(orc):
    va = _views((40, 23), (17, 31))
    rng = np.random.default_rng(1)
    P = int((va[:, 16] * va[:, 17]).sum())
    X, Y = rng.random(3 * P), rng.random(3 * P)
    out = orc.photo_loss(X, Y, va, ssim_map=True, grad=False)
    G = _window()
    C1, C2 = 0.01 ** 2, 0.03 ** 2
    for xs, ys, ms in zip(_planes(X, va), _planes(Y, va), _planes(out["map"], va)):
        for c in range(3):
            f = lambda a: ndimage.correlate(a, G, mode="constant", cval=0.0)
            m1, m2 = f(xs[c]), f(ys[c])
            s11, s22, s12 = f(xs[c] ** 2) - m1 ** 2, f(ys[c] ** 2) - m2 ** 2, f(xs[c] * ys[c]) - m1 * m2
            want = (2 * m1 * m2 + C1) * (2 * s12 + C2) / ((m1 ** 2 + m2 ** 2 + C1) * (s11 + s22 + C2))
            np.testing.assert_allclose(ms[c], want, rtol=1e-12, atol=1e-12)
    assert abs(out["ssim"] - out["map"].mean()) < 1e-12


def test_identical_images(orc):
    va = _views((30, 20))
    X = np.random.default_rng(2).random(3 * 600)
    out = orc.photo_loss(X, X, va)
    assert abs(out["ssim"] - 1.0) < 1e-12 and abs(out["loss"]) < 1e-12
    assert np.abs(out["grad"]).max() < 1e-12


def test_constant_images_closed_form(orc):
    """Away from the border every window sum is complete: m1 = a, m2 = b,
    no variance, SSIM = (2ab + C1) / (a^2 + b^2 + C1)."""
    va = _views((40, 40))
    a, b = 0.3, 0.7
    out = orc.photo_loss(np.full(4800, a), np.full(4800, b), va, ssim_map=True, grad=False)
    m = out["map"].reshape(3, 40, 40)[:, 5:35, 5:35]
    C1 = 0.01 ** 2
    np.testing.assert_allclose(m, (2 * a * b + C1) / (a * a + b * b + C1), rtol=1e-12)


def test_symmetry_and_lambda_ends(orc):
    va = _views((25, 19), (12, 7))
    rng = np.random.default_rng(3)
    P = 25 * 19 + 12 * 7
    X, Y = rng.random(3 * P), rng.random(3 * P)
    a, b = orc.photo_loss(X, Y, va), orc.photo_loss(Y, X, va)
    assert abs(a["ssim"] - b["ssim"]) < 1e-13
    assert abs(orc.photo_loss(X, Y, va, lam=0.0)["loss"] - np.abs(X - Y).mean()) < 1e-13
    assert abs(orc.photo_loss(X, Y, va, lam=1.0)["loss"] - (1.0 - a["ssim"])) < 1e-13


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_central_differences(orc, lam):
    va = _views((21, 16), (9, 13))
    rng = np.random.default_rng(4)
    P = 21 * 16 + 9 * 13
    X, Y = rng.random(3 * P), rng.random(3 * P)
    g = orc.photo_loss(X, Y, va, lam=lam)["grad"]
    h = 1e-6
    for p in rng.choice(3 * P, 40, replace=False):
        if abs(X[p] - Y[p]) < 10 * h:
            continue
        Xp, Xm = X.copy(), X.copy()
        Xp[p] += h
        Xm[p] -= h
        fd = (orc.photo_loss(Xp, Y, va, lam=lam, grad=False)["loss"] -
              orc.photo_loss(Xm, Y, va, lam=lam, grad=False)["loss"]) / (2 * h)
        assert abs(fd - g[p]) <= 1e-6 * max(1e-3, abs(g[p])), (p, fd, g[p])
