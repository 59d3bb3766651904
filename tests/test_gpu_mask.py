"""Motion masks and the covariance-aware dynamic mask on the GPU, through
the C ABI, against the oracle: the masks bit for bit, D_i bit for bit
against the oracle's FP32 stage fed the GPU's own records, and against the
FP64 oracle end to end except on borderline Gaussians."""

import numpy as np
import pytest

import synth
from synth.scenes import unpack_bits
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


class Run:
    """Gather + project once; motion masks and the dynamic mask on demand."""

    def __init__(self, pk, sc):
        self.pk, self.sc = pk, sc
        self.plan = pk.Plan.for_scene(sc)
        p = self.plan
        self.ws = pk.make_workspace(p)
        pk.workspace_init(p, self.ws)
        self.atlas, self.occ, _ = H.upload(sc)
        self.soa = torch.empty(p.D * p.G, dtype=torch.float32, device="cuda")
        self.texel = torch.empty(p.N, dtype=torch.int32, device="cuda")
        self.dynflag = torch.empty(p.N, dtype=torch.uint8, device="cuda")
        self.rec = torch.empty(12 * p.pairs, dtype=torch.float32, device="cuda")
        pk.atlas_gather(p, self.atlas, self.occ, None, self.soa, self.texel, self.dynflag, self.ws)
        pk.project_and_sh(p, self.soa, self.rec, self.ws)
        self.bits = torch.empty(max(p.mask_words, 1), dtype=torch.int32, device="cuda")
        aw, ah = sc.atlas.shape[3], sc.atlas.shape[2]
        self.dyn = torch.empty(ah * ((aw + 31) // 32), dtype=torch.int32, device="cuda")
        self.va = None

    def masks(self, flow, tau, r):
        self.pk.motion_mask(self.plan, torch.from_numpy(flow).cuda(), tau, r, self.bits, self.ws)
        return self.unpack(H.u32(self.bits))

    def unpack(self, words):
        out, off = [], 0
        for v in self.sc.views:
            wpr = (v.width + 31) // 32
            out.append(unpack_bits(words[off:off + v.height * wpr].reshape(v.height, wpr), v.width).reshape(-1))
            off += v.height * wpr
        return np.concatenate(out).astype(np.uint8)

    def dynamic(self, r_max=0.0, accumulate=False):
        self.pk.dynamic_mask(self.plan, self.rec, self.texel, self.bits, self.dyn, self.ws, r_max=r_max,
                             accumulate=accumulate)
        torch.cuda.synchronize()
        aw = self.sc.atlas.shape[3]
        wp = (aw + 31) // 32
        words = H.u32(self.dyn)
        t = H.u32(self.texel).astype(np.int64)
        return ((words[(t // aw) * wp + (t % aw) // 32] >> (t % aw % 32)) & 1).astype(np.uint8)


def _scene(seed=808):
    views = [synth.scenes.pinhole((0.4, 0.3, -3.2), 200, 136), synth.scenes.pinhole((-2.6, -0.5, -1.8), 37, 200),
             synth.scenes.pinhole((2.0, 1.2, 2.5), 96, 72), synth.scenes.pinhole((0.1, 2.9, 1.0), 65, 33)]
    return synth.make_scene([(128, 128, 0, 0, 0)], (128, 128), 0.6, views, sh_degree=1, seed=seed,
                            log_scale=(-3.4, 0.6))


def _flow(sc, seed, frac=0.15):
    return synth.motion_flow(sc.views, *synth.actor_sphere(sc, frac, seed=seed), seed=seed)


@pytest.mark.parametrize("r", [0, 1, 7, 40])
def test_motion_mask_bit_exact(pk, orc, r):
    sc = _scene()
    run = Run(pk, sc)
    va = orc.views_array(sc.views)
    flow = _flow(sc, 31 + r)
    got = run.masks(flow, 1.0, r)
    want = orc.motion_masks(flow, va, 1.0, r)
    np.testing.assert_array_equal(got, want)
    # bits past each row's width stay clear
    words, off = H.u32(run.bits), 0
    for v in sc.views:
        wpr = (v.width + 31) // 32
        if v.width % 32:
            last = words[off:off + v.height * wpr].reshape(v.height, wpr)[:, -1]
            assert np.all(last >> (v.width % 32) == 0)
        off += v.height * wpr


def test_motion_mask_thresholds(pk, orc):
    sc = _scene()
    run = Run(pk, sc)
    va = orc.views_array(sc.views)
    flow = _flow(sc, 3)
    flow[::7] = np.float32(np.nan)
    for tau in (-1.0, 0.0, 0.7, 1e30):
        np.testing.assert_array_equal(run.masks(flow, tau, 2), orc.motion_masks(flow, va, tau, 2))


@pytest.mark.parametrize("r_max", [0.0, 2.5])
def test_dynamic_mask_bit_exact_on_gpu_records(pk, orc, r_max):
    sc = _scene()
    run = Run(pk, sc)
    va = orc.views_array(sc.views)
    masks = run.masks(_flow(sc, 9), 1.0, 2)
    got = run.dynamic(r_max)
    rec32 = run.rec.cpu().numpy()
    want = orc.dynamic_mask32(rec32, va, masks, r_max)
    np.testing.assert_array_equal(got, want)
    assert 0 < want.sum() < len(want)


def test_dynamic_mask_end_to_end_fp64(pk, orc):
    sc = _scene(809)
    run = Run(pk, sc)
    flow = _flow(sc, 10)
    masks = run.masks(flow, 1.0, 3)
    got = run.dynamic()
    D, border, texel, _ = orc.dynamic_mask_scene(sc, masks)
    np.testing.assert_array_equal(H.u32(run.texel), texel)
    ok = border == 0
    assert ok.mean() > 0.97
    np.testing.assert_array_equal(got[ok], D[ok])


def test_dynamic_mask_accumulate_and_degenerate_masks(pk, orc):
    sc = _scene(810)
    run = Run(pk, sc)
    zero = np.zeros(2 * sc.pixels, np.float32)
    run.masks(zero, 1.0, 1)
    run.dyn.fill_(-1)
    assert run.dynamic().sum() == 0                  # cleared, nothing moves
    assert H.u32(run.dyn).sum() == 0
    run.dyn.fill_(-1)
    assert run.dynamic(accumulate=True).sum() == len(H.u32(run.texel))   # kept
    run.masks(np.full(2 * sc.pixels, 5.0, np.float32), 1.0, 0)           # everything moves
    D = run.dynamic()
    va = orc.views_array(sc.views)
    rec = run.rec.cpu().numpy().reshape(len(sc.views), -1, 12)
    visible = np.zeros(D.shape, bool)
    for v, view in enumerate(sc.views):
        r = rec[v]
        visible |= (r[:, 7] > 0) & (r[:, 0] >= 0) & (r[:, 0] <= view.width) & (r[:, 1] >= 0) & \
            (r[:, 1] <= view.height)
    assert visible.any() and np.all(D[visible] == 1)
    np.testing.assert_array_equal(D, orc.dynamic_mask32(rec.reshape(-1, 12), va,
                                                        np.ones(sc.pixels, np.uint8)))


def test_dynamic_mask_feeds_the_gather(pk, orc):
    """The texel bits are the gather's dyn input: its dynflag equals D."""
    sc = _scene(811)
    run = Run(pk, sc)
    run.masks(_flow(sc, 12), 1.0, 2)
    D = run.dynamic()
    p = run.plan
    pk.atlas_gather(p, run.atlas, run.occ, run.dyn, run.soa, run.texel, run.dynflag, run.ws)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(run.dynflag.cpu().numpy(), D)


def test_dynamic_mask_full_size_52_view_rig_sampled(pk, orc):
    """The 52-view 1024^2-atlas workload: masks of three views bit for bit,
    D of 3,000 sampled Gaussians against the oracle's FP32 stage."""
    sc = synth.config_scene(3)
    run = Run(pk, sc)
    flow = synth.motion_flow(sc.views, *synth.actor_sphere(sc, 0.05), seed=77)
    run.pk.motion_mask(run.plan, torch.from_numpy(flow).cuda(), 1.0, 2, run.bits, run.ws)
    words = H.u32(run.bits)
    va = orc.views_array(sc.views)
    woff = np.concatenate([[0], np.cumsum([v.height * ((v.width + 31) // 32) for v in sc.views])])
    poff = np.concatenate([[0], np.cumsum([v.width * v.height for v in sc.views])])
    masks = np.zeros(sc.pixels, np.uint8)
    for v, view in enumerate(sc.views):
        wpr = (view.width + 31) // 32
        masks[poff[v]:poff[v + 1]] = unpack_bits(words[woff[v]:woff[v + 1]].reshape(view.height, wpr),
                                                 view.width).reshape(-1)
    for v in (0, 1, 51):
        want = orc.motion_mask(flow[2 * poff[v]:2 * poff[v + 1]].reshape(2, sc.views[v].height, -1), 1.0, 2)
        np.testing.assert_array_equal(masks[poff[v]:poff[v + 1]], want.reshape(-1))
    got = run.dynamic()
    N = run.plan.N
    pick = np.random.default_rng(5).choice(N, 3000, replace=False)
    rec = run.rec.cpu().numpy().reshape(len(sc.views), N, 12)[:, pick]
    want = orc.dynamic_mask32(rec.reshape(-1, 12), va, masks)
    np.testing.assert_array_equal(got[pick], want)
    assert 0.05 < got.mean() < 0.95
