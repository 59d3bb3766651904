"""The differentiable render() (torch.autograd.Function over the C ABI):
gradients equal the library's backward, pass straight through the FP16 proxy,
agree with FP64 finite differences of the oracle on a C4-shaped subset, and
view shards summed equal the unsharded launch."""

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


def _renderer(pk, sc, views=None):
    r = pk.Renderer(pk.Plan.for_scene(sc, views=views))
    atlas, occ, dyn = H.upload(sc)
    assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    return r, atlas, occ, dyn


def test_autograd_matches_library_backward(pk):
    sc = H.scene_small_sh3(seed=505)
    r, atlas, occ, dyn = _renderer(pk, sc)
    w = torch.from_numpy(np.random.default_rng(1).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    master = atlas.clone().requires_grad_(True)
    img = pk.render(master, r, occ, dyn)
    (img * w).sum().backward()
    ref = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
    r.forward(atlas, occ, dyn)
    r.backward(w, ref)
    torch.cuda.synchronize()
    assert H.rel_err(master.grad.reshape(-1).cpu().numpy().astype(np.float64),
                     ref.cpu().numpy().astype(np.float64)) < 1e-5


def test_fp16_proxy_passes_gradient_straight_through(pk, orc):
    sc = H.scene_multilevel_f16()
    r, atlas16, occ, dyn = _renderer(pk, sc)
    master = atlas16.float().clone().requires_grad_(True)     # FP32 masters behind the FP16 proxy
    w = torch.from_numpy(np.random.default_rng(2).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    img = pk.render(master, r, occ, dyn, proxy=atlas16)
    (img * w).sum().backward()
    o = orc.forward(sc)
    b = orc.backward(sc, o, w.cpu().numpy().astype(np.float64))
    g = master.grad.reshape(1, sc.channels, -1)[0][:, o["texel"]].cpu().numpy().astype(np.float64)
    H.check_grads(g, b["grad_soa"])


def test_autograd_against_fp64_finite_differences_c4_subset(pk, orc):
    """C4 shapes: 3 FP16 levels, 16 uneven views (downscaled x4); 2,000 Gaussians live."""
    rng = np.random.default_rng(40)
    sizes = [(160, 120), (240, 135), (320, 180), (400, 225), (480, 270)]
    views = synth.scenes.ring_views((6, 5, 5), (-1.0, 0.0, 1.0), 4.0, [sizes[i] for i in rng.integers(0, 5, 16)])
    levels = [(64, 64, 32, 0, 0), (32, 32, 0, 0, 0), (16, 16, 0, 32, 0)]
    total = 64 * 64 + 32 * 32 + 16 * 16
    sc = synth.make_scene(levels, (96, 64), [2000 * 64 * 64 / total / 4096, 2000 * 32 * 32 / total / 1024,
                                             2000 * 16 * 16 / total / 256], views, texel_dtype=np.float16,
                          seed=41, log_scale=(-3.0, 0.4))
    r, atlas16, occ, dyn = _renderer(pk, sc)
    master = atlas16.float().clone().requires_grad_(True)
    w64 = np.random.default_rng(3).standard_normal(3 * sc.pixels)
    w = torch.from_numpy(w64.astype(np.float32)).cuda()
    (pk.render(master, r, occ, dyn, proxy=atlas16) * w).sum().backward()
    soa, texel, _ = orc.gather(sc)
    g = master.grad.reshape(1, sc.channels, -1)[0][:, texel].cpu().numpy().astype(np.float64)
    assert 1900 <= len(texel) <= 2000
    va = orc.views_array(sc.views)
    wq = w.cpu().numpy().astype(np.float64)

    def loss(s):
        rec = orc.project(s, len(texel), sc.sh_degree, va)
        vals, ranges = orc.bin_sort(rec, va, 16)
        out = orc.render(rec, va, 16, vals, ranges)
        return float(wq @ out["img"]), out["hash"]

    # one Gaussian per direction: a dense direction moves some of the
    # millions of threshold decisions (the decision hash then differs)
    live = np.flatnonzero(np.abs(g).sum(axis=0) > 0)
    ok = 0
    for gi in rng.choice(live, 24, replace=False):
        d = np.zeros_like(soa)
        d[:, gi] = rng.standard_normal(soa.shape[0])
        h = 1e-6
        lp, hp = loss(soa + h * d)
        lm, hm = loss(soa - h * d)
        if hp != hm:
            continue
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 2e-3 * max(1.0, abs(fd)), (fd, an)
        ok += 1
    assert ok >= 16


def test_view_shards_sum_to_the_unsharded_gradient(pk):
    """The multi-GPU split (views sharded, texel gradients summed) simulated on one GPU."""
    sc = H.scene_small_sh3(seed=606)
    w = np.random.default_rng(4).standard_normal(3 * sc.pixels).astype(np.float32)
    r, atlas, occ, dyn = _renderer(pk, sc)
    full = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
    r.forward(atlas, occ, dyn)
    r.backward(torch.from_numpy(w).cuda(), full)
    shard_sum = torch.zeros_like(full)
    off = 0
    for part in (sc.views[:1], sc.views[1:]):
        rs, _, _, _ = _renderer(pk, sc, views=part)
        n = sum(v.width * v.height for v in part)
        g = torch.zeros_like(full)
        rs.forward(atlas, occ, dyn)
        rs.backward(torch.from_numpy(w[3 * off:3 * (off + n)].copy()).cuda(), g)
        assert torch.equal(rs.image, r.image[3 * off:3 * (off + n)])
        shard_sum += g
        off += n
    torch.cuda.synchronize()
    assert H.rel_err(shard_sum.cpu().numpy().astype(np.float64), full.cpu().numpy().astype(np.float64)) < 1e-5
