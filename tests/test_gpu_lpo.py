"""Low-precision proxy on the GPU against the oracle: min/max and the 8-bit
code planes bit for bit, the proxy SoA value for value (from the codes and
from the FP32 masters), and a render step on the proxy whose gradients
pass the quantiser straight through to the masters."""

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


def _scene(W=128, frames=2, seed=901):
    views = [synth.scenes.pinhole((0.4, 0.3, -3.2), 160, 120, frame=f) for f in range(frames)]
    return synth.make_scene([(W, 96, 0, 0, 0)], (W, 96), 0.6, views, sh_degree=2, frames=frames, seed=seed,
                            dynamic_frac=0.3, log_scale=(-3.4, 0.5))


class Lpo:
    def __init__(self, pk, sc):
        self.pk, self.sc = pk, sc
        self.plan = pk.Plan.for_scene(sc)
        p = self.plan
        self.ws = pk.make_workspace(p)
        pk.workspace_init(p, self.ws)
        self.atlas, self.occ, self.dyn = H.upload(sc)
        F, D, Ha, Wa = sc.atlas.shape
        self.lohi = torch.empty(2 * D, dtype=torch.float32, device="cuda")
        self.codes = torch.empty(F * (D + 3) * Ha * Wa, dtype=torch.uint8, device="cuda")
        self.soa = torch.empty(p.D * p.G, dtype=torch.float32, device="cuda")
        self.texel = torch.empty(p.N, dtype=torch.int32, device="cuda")
        self.dynflag = torch.empty(p.N, dtype=torch.uint8, device="cuda")

    def run(self):
        p = self.plan
        self.pk.lpo_minmax(p, self.atlas, self.occ, self.lohi, self.ws)
        self.pk.lpo_encode(p, self.atlas, self.occ, self.lohi, self.codes, self.ws)
        torch.cuda.synchronize()
        F, D, Ha, Wa = self.sc.atlas.shape
        return self.lohi.cpu().numpy().reshape(D, 2), self.codes.cpu().numpy().reshape(F, D + 3, Ha, Wa)

    def gather(self, kind):
        p = self.plan
        src = self.codes if kind == self.pk.api.LPO_CODES else self.atlas
        self.pk.atlas_gather_lpo(p, src, kind, self.lohi, self.occ, self.dyn, self.soa, self.texel, self.dynflag,
                                 self.ws)
        torch.cuda.synchronize()
        return self.soa.cpu().numpy().reshape(p.D, p.G)


@pytest.mark.parametrize("W", [128, 125])
def test_minmax_and_codes_bit_exact(pk, orc, W):
    sc = _scene(W)
    a = sc.atlas
    a[1, 12, 5, 7] = np.nan                       # a NaN master texel
    a[0, 20][synth.scenes.unpack_bits(sc.occ, W)] = np.float32(0.75)   # a constant channel
    run = Lpo(pk, sc)
    lohi, codes = run.run()
    want_lohi = orc.lpo_minmax(a, sc.occ)
    np.testing.assert_array_equal(lohi.view(np.uint32), want_lohi.view(np.uint32))
    np.testing.assert_array_equal(codes, orc.lpo_encode(a, sc.occ, want_lohi))


@pytest.mark.parametrize("W", [128, 125])
def test_proxy_gather_from_codes_and_from_masters(pk, orc, W):
    sc = _scene(W, seed=902)
    run = Lpo(pk, sc)
    lohi, codes = run.run()
    proxy = orc.lpo_decode(codes, sc.occ, lohi)
    ref = synth.scenes.Scene(**{**sc.__dict__, "atlas": proxy})
    soa_ref, texel_ref, dyn_ref = orc.gather(ref)
    from_codes = run.gather(pk.api.LPO_CODES)
    np.testing.assert_array_equal(from_codes.astype(np.float64), soa_ref)
    np.testing.assert_array_equal(H.u32(run.texel), texel_ref)
    np.testing.assert_array_equal(run.dynflag.cpu().numpy(), dyn_ref)
    from_masters = run.gather(pk.api.LPO_MASTERS)
    np.testing.assert_array_equal(from_masters.view(np.uint32), from_codes.view(np.uint32))


def test_render_on_the_proxy_with_straight_through_gradients(pk, orc):
    sc = H.scene_small_sh3(seed=903)
    r = pk.Renderer(pk.Plan.for_scene(sc))
    atlas, occ, dyn = H.upload(sc)
    F, D, Ha, Wa = sc.atlas.shape
    r.lohi = torch.empty(2 * D, dtype=torch.float32, device="cuda")
    pk.lpo_minmax(r.plan, atlas, occ, r.lohi, r.ws)
    assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    lohi = r.lohi.cpu().numpy().reshape(D, 2)
    proxy = orc.lpo_decode(orc.lpo_encode(sc.atlas, sc.occ, lohi), sc.occ, lohi)
    ref = synth.scenes.Scene(**{**sc.__dict__, "atlas": proxy})
    o = orc.forward(ref)
    o["view_pixels"] = [v.width * v.height for v in sc.views]
    w = np.random.default_rng(6).standard_normal(3 * sc.pixels).astype(np.float32)
    grad = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
    r.forward(atlas, occ, dyn)
    r.backward(torch.from_numpy(w).cuda(), grad)
    torch.cuda.synchronize()
    H.check_images(r.image.cpu().numpy(), r.T.cpu().numpy(), o)
    b = orc.backward(ref, o, w.astype(np.float64))
    g = grad.reshape(F, D, -1)[0][:, o["texel"]].cpu().numpy().astype(np.float64)
    H.check_grads(g, b["grad_soa"])
    # the proxy differs from the masters (the quantiser is active)
    assert np.abs(proxy - sc.atlas).max() > 0
