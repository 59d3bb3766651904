"""Failure paths on the GPU, made on purpose without faulting anything:
bounded waits that give up (the plan's first-wait limit set to give up at
once, the draining waits keeping theirs), non-finite texels, and the
autograd wrapper refusing a backward through a stale forward."""

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


def _ready(pk, sc, **kw):
    r = pk.Renderer(pk.Plan.for_scene(sc, **kw))
    atlas, occ, dyn = H.upload(sc)
    assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    return r, atlas, occ, dyn


@pytest.mark.parametrize("which", ["fwd", "bwd"])
def test_compositing_wait_timeout_is_reported(pk, which):
    """Bulk staging with a first wait that gives up at once: the kernel
    drains its copies, leaves, and the status block reports the timeout;
    the context stays usable."""
    sc = H.scene_small_sh3(seed=515)
    r, atlas, occ, dyn = _ready(pk, sc)
    w = torch.from_numpy(np.random.default_rng(3).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    img0 = r.image.clone()
    p = pk.Plan.for_scene(sc, max_dups=r.plan.max_dups, stage_fwd="bulk", stage_bwd="bulk", first_wait_polls=-1)
    ws = pk.make_workspace(p)
    pk.workspace_init(p, ws)
    if which == "fwd":
        img, T, nc = torch.empty_like(r.image), torch.empty_like(r.T), torch.empty_like(r.n_contrib)
        pk.rasterize_fwd(p, r.records, r.sorted_vals, r.ranges, img, T, nc, ws)
    else:
        g2 = torch.empty_like(r.grad2d)
        pk.rasterize_bwd(p, r.records, r.sorted_vals, r.ranges, r.T, r.n_contrib, w, g2, ws)
    st = pk.read_status(p, ws)
    assert st["rc"] == 4 and st["flags"] & 4, st
    # the same call with the default limit: no timeout, the usual image
    q = pk.Plan.for_scene(sc, max_dups=r.plan.max_dups, stage_fwd="bulk", stage_bwd="bulk")
    ws2 = pk.make_workspace(q)
    pk.workspace_init(q, ws2)
    img, T, nc = torch.empty_like(r.image), torch.empty_like(r.T), torch.empty_like(r.n_contrib)
    pk.rasterize_fwd(q, r.records, r.sorted_vals, r.ranges, img, T, nc, ws2)
    assert pk.read_status(q, ws2)["flags"] == 0
    assert torch.equal(img, img0)


def test_sort_wait_timeout_emits_nothing(pk):
    """A radix pass whose first wait gives up: the call reports the timeout
    and leaves every tile range empty, so nothing reads a partial list;
    the regular plan then sorts the same records as before."""
    sc = H.scene_small_sh3(seed=525)
    r, atlas, occ, dyn = _ready(pk, sc)
    vals0, ranges0 = r.sorted_vals.clone(), r.ranges.clone()
    p = pk.Plan.for_scene(sc, max_dups=r.plan.max_dups, first_wait_polls=-1)
    ws = pk.make_workspace(p)
    pk.workspace_init(p, ws)
    vals = torch.full_like(r.sorted_vals, 7)
    ranges = torch.full_like(r.ranges, 7)
    pk.bin_and_sort(p, r.records, vals, ranges, ws)
    st = pk.read_status(p, ws)
    assert st["rc"] == 4 and st["flags"] & 4 and st["dups"] == 0, st
    assert int(torch.count_nonzero(ranges)) == 0
    pk.bin_and_sort(r.plan, r.records, r.sorted_vals, r.ranges, r.ws)
    assert r.status()["flags"] == 0
    assert torch.equal(r.ranges, ranges0)
    n = int(r.status()["dups"])
    assert torch.equal(r.sorted_vals[:n], vals0[:n])


def test_lists_naming_no_pair_are_skipped_and_flagged(pk):
    """A list entry past the plan's pairs (not a list this plan sorted) is
    staged as a splat that reaches nothing and flagged, never read."""
    sc = H.scene_small_sh3(seed=535)
    r, atlas, occ, dyn = _ready(pk, sc)
    n = int(r.status()["dups"])
    vals = r.sorted_vals.clone()
    vals[: n: 7] = 0x7ffffff0                      # far past V * N
    img, T, nc = torch.empty_like(r.image), torch.empty_like(r.T), torch.empty_like(r.n_contrib)
    pk.rasterize_fwd(r.plan, r.records, vals, r.ranges, img, T, nc, r.ws)
    st = r.status()
    assert st["flags"] & 8 and torch.isfinite(img).all()


def test_nonfinite_texels_are_culled_and_counted(pk, orc):
    """Gaussians with a NaN or infinite texel value (position, log-scale,
    quaternion, opacity logit, an SH coefficient) are counted by the gather,
    culled in every view and get a zero gradient; the rest renders as the
    oracle renders the same atlas."""
    sc = H.scene_small_sh3(seed=545)
    F, D, Hh, W = sc.atlas.shape
    occ = synth.scenes.unpack_bits(sc.occ, W)
    ys, xs = np.nonzero(occ)
    pick = np.random.default_rng(5).choice(len(ys), 6, replace=False)
    bad = [(0, np.nan), (4, np.inf), (7, np.nan), (10, -np.inf), (20, np.nan), (2, -np.inf)]
    for i, (c, val) in zip(pick, bad):
        sc.atlas[0, c, ys[i], xs[i]] = val
    r, atlas, occ_t, dyn = _ready(pk, sc)
    st = r.status()
    assert st["nonfinite"] == 6, st
    w = np.random.default_rng(6).standard_normal(3 * sc.pixels).astype(np.float32)
    grad = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
    r.backward(torch.from_numpy(w).cuda(), grad)
    torch.cuda.synchronize()
    rec = r.records.view(r.plan.V, r.plan.N, 12).cpu().numpy()
    texel = H.u32(r.texel[:r.plan.N])
    gidx = np.searchsorted(texel, ys[pick] * W + xs[pick])
    assert np.all(rec[:, gidx, 7] == 0)            # culled in every view
    o = orc.forward(sc)
    o["view_pixels"] = [v.width * v.height for v in sc.views]
    H.check_images(r.image.cpu().numpy(), r.T.cpu().numpy(), o, label="non-finite texels")
    b = orc.backward(sc, o, w.astype(np.float64))
    g = grad.view(F, D, Hh * W).cpu().numpy()[0][:, texel].astype(np.float64)
    assert np.all(np.isfinite(g)) and np.all(g[:, gidx] == 0)
    H.check_grads(g, b["grad_soa"])


def test_render_refuses_backward_through_a_stale_forward(pk):
    """Two render() calls on one Renderer, then the first one's backward:
    refused (its per-pixel state was overwritten); the latest call's
    backward, and forward/backward in turn, work."""
    sc = H.scene_small_sh3(seed=555)
    r, atlas, occ, dyn = _ready(pk, sc)
    w = torch.from_numpy(np.random.default_rng(7).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    m1 = atlas.clone().requires_grad_(True)
    m2 = atlas.clone().requires_grad_(True)
    img1 = pk.render(m1, r, occ, dyn)
    img2 = pk.render(m2, r, occ, dyn)
    with pytest.raises(RuntimeError, match="another forward"):
        (img1 * w).sum().backward()
    (img2 * w).sum().backward()
    ref = m2.grad.clone()
    for _ in range(2):   # forward, backward, forward, backward: each consistent
        m = atlas.clone().requires_grad_(True)
        (pk.render(m, r, occ, dyn) * w).sum().backward()
        assert H.rel_err(m.grad.cpu().numpy().astype(np.float64), ref.cpu().numpy().astype(np.float64)) < 1e-5
