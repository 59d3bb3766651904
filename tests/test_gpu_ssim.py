"""The photometric objective (1 - lambda) L1 + lambda (1 - SSIM) on the
GPU against the FP64 oracle: loss, mean SSIM and gradient over several
views of ragged sizes (tiles cut by the image edges), identical images,
and the 1080p single-view workload."""

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_23040_gb300 as pk
    pk.build.build()
    return pk


def _plan(pk, sizes):
    views = [synth.scenes.pinhole((0.0, 0.0, -3.0), w, h) for w, h in sizes]
    sc = synth.make_scene([(16, 16, 0, 0, 0)], (16, 16), 0.5, views, sh_degree=0, seed=1)
    p = pk.Plan.for_scene(sc)
    ws = pk.make_workspace(p)
    pk.workspace_init(p, ws)
    return p, ws, sc


def _run(pk, p, ws, X, Y, lam):
    g = torch.empty(X.size, dtype=torch.float32, device="cuda")
    pk.photo_loss_grad(p, torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), g, ws, lam)
    st = pk.read_status(p, ws)
    return st["loss"], st["ssim"], g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("lam", [0.2, 1.0, 0.0])
def test_photo_loss_matches_oracle(pk, orc, lam):
    p, ws, sc = _plan(pk, [(100, 75), (33, 70), (64, 64), (7, 5)])
    rng = np.random.default_rng(2)
    X = rng.random(3 * sc.pixels).astype(np.float32)
    Y = (0.6 * X + 0.4 * rng.random(3 * sc.pixels)).astype(np.float32)
    loss, ssim, g = _run(pk, p, ws, X, Y, lam)
    o = orc.photo_loss(X.astype(np.float64), Y.astype(np.float64), orc.views_array(sc.views), lam=lam)
    assert abs(loss - o["loss"]) <= 1e-5 * max(1.0, abs(o["loss"]))
    if lam > 0:
        assert abs(ssim - o["ssim"]) <= 1e-5
    err = H.rel_err(g, o["grad"])
    assert err <= 1e-4, err


def test_identical_images_zero_gradient(pk, orc):
    p, ws, sc = _plan(pk, [(50, 40)])
    X = np.random.default_rng(3).random(3 * sc.pixels).astype(np.float32)
    loss, ssim, g = _run(pk, p, ws, X, X, 0.2)
    assert abs(ssim - 1.0) < 1e-5 and abs(loss) < 1e-5
    assert np.abs(g).max() < 1e-9


def test_photo_loss_1080p(pk, orc):
    p, ws, sc = _plan(pk, [(1920, 1080)])
    rng = np.random.default_rng(4)
    X = rng.random(3 * sc.pixels).astype(np.float32)
    Y = rng.random(3 * sc.pixels).astype(np.float32)
    loss, ssim, g = _run(pk, p, ws, X, Y, 0.2)
    # the oracle on a band of rows: window sums there need rows +-10 around it
    va = orc.views_array(sc.views)
    band = slice(500, 540)
    rows = slice(490, 550)
    Xs = X.reshape(3, 1080, 1920)[:, rows].reshape(-1)
    Ys = Y.reshape(3, 1080, 1920)[:, rows].reshape(-1)
    vb = va.copy()
    vb[0, 17] = 60
    o = orc.photo_loss(Xs.astype(np.float64), Ys.astype(np.float64), vb, lam=0.2)
    # interior rows of the band (the oracle's cut edges are 10 rows away)
    go = o["grad"].reshape(3, 60, 1920)[:, 10:50]
    gg = g.reshape(3, 1080, 1920)[:, band]
    # scale: the oracle normalises by its own 3 P
    gg = gg * (3.0 * 1920 * 1080) / (3.0 * 1920 * 60)
    assert H.rel_err(gg, go) <= 1e-4
