"""Parity of the CUDA library (through the C ABI) with the FP64 oracle."""

import math

import numpy as np
import pytest

import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_23040_gb300 import build
    build.build()


def _pk():
    import paper_2602_23040_gb300 as pk
    return pk


def run_gpu(scene, dimg=None, **plan_kw):
    pk = _pk()
    plan = pk.Plan.for_scene(scene, **plan_kw)
    r = pk.Renderer(plan)
    atlas, occ, dyn = H.upload(scene)
    st = r.ensure_capacity(atlas, occ, dyn)
    assert st["flags"] == 0, st
    plan = r.plan
    grad = None
    if dimg is not None:
        F, D, Hh, W = scene.atlas.shape
        grad = torch.zeros(F * D * Hh * W, dtype=torch.float32, device="cuda")
        r.backward(torch.from_numpy(dimg.astype(np.float32)).cuda(), grad)
    torch.cuda.synchronize()
    return plan, r, grad


def oracle_run(orc, scene, dimg=None):
    o = orc.forward(scene)
    o["view_pixels"] = [v.width * v.height for v in scene.views]
    if dimg is not None:
        oracle_backward(orc, scene, o, dimg)
    return o


def oracle_backward(orc, scene, o, dimg):
    b = orc.backward(scene, o, dimg.astype(np.float32).astype(np.float64))
    o.update(b)
    o["grad_atlas"] = orc.grad_to_atlas(scene, b["grad_soa"], o["texel"])
    return o


def gpu_grad_soa(scene, grad, texel):
    F, D, Hh, W = scene.atlas.shape
    g = grad.view(F, D, Hh * W).cpu().numpy().astype(np.float64)
    return np.concatenate([g[f][:, texel] for f in range(F)], axis=1)


# ---------------------------------------------------------------------------
# a1 gather, a2 projection
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["f32", "f16", "frames_dyn"])
def test_gather_bit_exact(orc, which):
    sc = {"f32": lambda: H.scene_small_sh3(), "f16": lambda: H.scene_multilevel_f16(),
          "frames_dyn": lambda: H.scene_small_sh3(frames=2, dyn=0.3)}[which]()
    plan, r, _ = run_gpu(sc)
    soa, texel, dyn = orc.gather(sc)
    assert np.array_equal(r.soa.view(plan.D, plan.G).cpu().numpy().astype(np.float64), soa)
    assert np.array_equal(H.u32(r.texel[:plan.N]), texel)
    assert np.array_equal(r.dynflag[:plan.N].cpu().numpy(), dyn)
    st = r.status()
    assert st["flags"] == 0 and st["live_seen"] == plan.N


def test_project_matches_oracle(orc):
    sc = H.scene_small_sh3()
    plan, r, _ = run_gpu(sc)
    o = orc.forward(sc)
    got = r.records.view(plan.V, plan.N, 12).cpu().numpy().astype(np.float64)
    ref = o["rec"]
    live = ref[..., 7] > 0
    assert np.array_equal(got[..., 7] > 0, live)
    g, e = got[live], ref[live]
    assert np.abs(g[:, 0:2] - e[:, 0:2]).max() < 2e-3                               # mean, px
    assert (np.abs(g[:, 2:5] - e[:, 2:5]) / np.abs(e[:, 2:5]).max(1, keepdims=True)).max() < 1e-4
    assert np.abs(g[:, 5] - e[:, 5]).max() < 1e-6                                   # opacity
    assert (np.abs(g[:, 6] - e[:, 6]) / e[:, 6]).max() < 1e-6                      # depth
    assert np.abs(g[:, 8:11] - e[:, 8:11]).max() < 1e-5                             # colour
    # radius = ceil(3 sqrt(lambda_max)) may flip only where 3 sqrt(lambda) is an integer to FP32 precision
    assert np.mean(g[:, 7] != e[:, 7]) < 1e-3


# ---------------------------------------------------------------------------
# a3 binning and sort: bit-exact on identical FP32 inputs
# ---------------------------------------------------------------------------

def _synthetic_records(views, N, seed, huge=True):
    rng = np.random.default_rng(seed)
    V = len(views)
    rec = np.zeros((V, N, 12), np.float32)
    for v, vw in enumerate(views):
        rec[v, :, 0] = rng.uniform(-30, vw.width + 30, N)
        rec[v, :, 1] = rng.uniform(-30, vw.height + 30, N)
        # Sigma2D = L L^T + 0.3 I
        L = rng.normal(0, 1, (N, 2, 2)) * np.exp(rng.normal(0.8, 0.8, (N, 1, 1)))
        S = L @ L.transpose(0, 2, 1) + 0.3 * np.eye(2)
        det = S[:, 0, 0] * S[:, 1, 1] - S[:, 0, 1] ** 2
        rec[v, :, 2] = S[:, 1, 1] / det
        rec[v, :, 3] = -S[:, 0, 1] / det
        rec[v, :, 4] = S[:, 0, 0] / det
        rec[v, :, 5] = rng.uniform(0.02, 1.0, N)
        rec[v, :, 6] = rng.uniform(0.5, 8.0, N)
        tr = S[:, 0, 0] + S[:, 1, 1]
        lam = 0.5 * (tr + np.sqrt(np.maximum(0, tr * tr - 4 * det)))
        rec[v, :, 7] = np.ceil(3 * np.sqrt(lam))
        rec[v, :, 8:11] = rng.uniform(0, 1, (N, 3))
    rec[:, ::13, 7] = 0                          # culled pairs
    rec[:, 5::17, 6] = rec[:, 5, 6][:, None]     # exact depth ties
    if huge:
        rec[:, 7::29, 7] = 4000                  # footprints larger than the view
    return rec


def _records_plan(views, N, bin_mode="ellipse", tile=16, **kw):
    pk = _pk()
    side = int(math.ceil(math.sqrt(N)))
    return pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, bin_mode=bin_mode, tile=tile, **kw)


def _records_setup(seed, N=700, huge=True):
    views = [synth.scenes.pinhole((0, 0, -3), 150, 100), synth.scenes.pinhole((0, 0, -3), 67, 131),
             synth.scenes.pinhole((0, 0, -3), 16, 16)]
    rec = _synthetic_records(views, N, seed, huge)
    return views, rec


@pytest.mark.parametrize("seed,mode,tile,bits", [(1, "ellipse", 16, (8, 8)), (2, "ellipse", 16, (8, 8)),
                                                 (3, "rect", 16, (8, 8)), (4, "rect", 16, (8, 8)),
                                                 (1, "ellipse", 32, (8, 8)), (3, "rect", 32, (8, 8)),
                                                 (2, "ellipse", 16, (11, 11)), (5, "ellipse", 32, (11, 8)),
                                                 (6, "rect", 16, (8, 11))])
@pytest.mark.parametrize("huge", [True, False])
def test_bin_and_sort_bit_exact(orc, seed, mode, tile, bits, huge):
    """Every tile's list bit for bit, for either radix digit width of the
    depth sort and of the tile sort (bits = (depth, tile)); with footprints
    larger than the view among the pairs (warps walk their candidates
    together) or without (most warps walk them lane by lane)."""
    pk = _pk()
    views, rec = _records_setup(seed, huge=huge)
    V, N = rec.shape[:2]
    plan = _records_plan(views, N, mode, tile, sort_bits_depth=bits[0], sort_bits_tile=bits[1])
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    drec = torch.from_numpy(rec.reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, drec, vals, ranges, ws)
    st = pk.read_status(plan, ws)
    va = orc.views_array(views)
    r = rec.reshape(V * N, 12)
    ref_vals, ref_ranges = orc.bin_sort32(r[:, 0], r[:, 1], r[:, 7], r[:, 6], va, N, tile, r[:, 2], r[:, 3],
                                          r[:, 4], mode={"ellipse": orc.BIN_ELLIPSE, "rect": orc.BIN_RECT}[mode])
    assert st["dups"] == len(ref_vals) and st["flags"] == 0
    assert_same_tile_lists(H.u32(vals[:len(ref_vals)]), H.i64(ranges).reshape(-1, 2), ref_vals, ref_ranges)


def assert_same_tile_lists(vals, ranges, ref_vals, ref_ranges):
    """Every tile's list equal to the oracle's, bit for bit (the contract);
    the lists tile sorted_vals (disjoint, covering), in any order of tiles."""
    assert ranges.shape == ref_ranges.shape
    n = len(ref_vals)
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    assert np.array_equal(lens, ref_ranges[:, 1].astype(np.int64) - ref_ranges[:, 0])
    live = np.flatnonzero(lens > 0)
    if n == 0:
        assert len(live) == 0
        return
    starts = ranges[live, 0].astype(np.int64)
    order = np.argsort(starts)
    ends = starts[order] + lens[live][order]
    assert starts[order][0] == 0 and ends[-1] == n and np.array_equal(starts[order][1:], ends[:-1])
    for t in live:
        a, b = ranges[t]
        c, d = ref_ranges[t]
        assert np.array_equal(vals[a:b], ref_vals[c:d]), t


def test_bin_and_sort_capacity_overflow(orc):
    pk = _pk()
    views, rec = _records_setup(4)
    V, N = rec.shape[:2]
    side = int(math.ceil(math.sqrt(N)))
    plan = pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, max_dups=1024)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.full((2 * plan.n_tiles,), 7, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, torch.from_numpy(rec.reshape(-1)).cuda(), vals, ranges, ws)
    st = pk.read_status(plan, ws)
    assert st["flags"] & 1 and st["rc"] == 3 and st["dups"] == 0 and st["dups_needed"] > 1024
    assert int(ranges.abs().sum()) == 0


# valid pairs per view: the views' segments start at every residue mod 4 and
# several hold only 1-3 items, so a segment's only radix tile can start 1-3
# keys past a 16-byte boundary and end before the next one
RAGGED_COUNTS = [1, 2, 1, 1, 3, 2, 1, 2, 2, 1, 3, 3, 1, 2, 0, 1, 2, 3, 1]


def _ragged_records(tile, seed, spread):
    """Records with exactly RAGGED_COUNTS[v] valid pairs in view v, each a
    small footprint that reaches one tile, or (spread) one to four tiles
    when its mean sits on a tile edge or corner; the other pairs are culled."""
    rng = np.random.default_rng(seed)
    W = H_ = 64
    views = [synth.scenes.pinhole((0, 0, -3), W, H_) for _ in RAGGED_COUNTS]
    N = 8
    rec = np.zeros((len(views), N, 12), np.float32)
    nt = W // tile
    for v, c in enumerate(RAGGED_COUNTS):
        for i in rng.choice(N, c, replace=False):
            tx, ty = rng.integers(0, nt, 2)
            ox = oy = tile / 2
            if spread:
                ox = float(rng.choice([tile / 2, 0.0])) if tx else tile / 2
                oy = float(rng.choice([tile / 2, 0.0])) if ty else tile / 2
            rec[v, i, 0:2] = (tx * tile + ox, ty * tile + oy)
            rec[v, i, 2:5] = (4.0, 0.0, 4.0)          # conic: sigma^2 = 1/4, footprint radius 1.5 px
            rec[v, i, 5] = 0.5
            rec[v, i, 6] = rng.uniform(0.5, 8.0)
            rec[v, i, 7] = 2.0
            rec[v, i, 8:11] = rng.uniform(0, 1, 3)
    return views, rec


@pytest.mark.parametrize("tile,spread,bits", [(16, False, 8), (16, True, 8), (32, False, 8), (32, True, 8),
                                              (16, True, 11), (32, False, 11)])
def test_bin_and_sort_ragged_view_segments(orc, tile, spread, bits):
    """Per-view segments of 0-3 items at every start residue (both the depth
    passes and the tile passes run segmented by view here), 8- or 11-bit digits."""
    pk = _pk()
    views, rec = _ragged_records(tile, 11 + tile + spread, spread)
    V, N = rec.shape[:2]
    plan = _records_plan(views, N, "ellipse", tile, sort_bits_depth=bits, sort_bits_tile=bits)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    drec = torch.from_numpy(rec.reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, drec, vals, ranges, ws)
    st = pk.read_status(plan, ws)
    va = orc.views_array(views)
    r = rec.reshape(V * N, 12)
    ref_vals, ref_ranges = orc.bin_sort32(r[:, 0], r[:, 1], r[:, 7], r[:, 6], va, N, tile, r[:, 2], r[:, 3],
                                          r[:, 4], mode=orc.BIN_ELLIPSE)
    assert st["valid_pairs"] == sum(RAGGED_COUNTS)
    if not spread:
        assert len(ref_vals) == sum(RAGGED_COUNTS)
    assert st["dups"] == len(ref_vals) and st["flags"] == 0
    assert_same_tile_lists(H.u32(vals[:len(ref_vals)]), H.i64(ranges).reshape(-1, 2), ref_vals, ref_ranges)


# ---------------------------------------------------------------------------
# a4 / a5 on identical FP32 records
# ---------------------------------------------------------------------------

def _records_forward(seed, dimg_seed=None, tile=16):
    pk = _pk()
    views, rec = _records_setup(seed, N=500)
    V, N = rec.shape[:2]
    rec[..., 5] = np.minimum(rec[..., 5], 0.999)
    plan = _records_plan(views, N, tile=tile, count_evals=True)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    drec = torch.from_numpy(rec.reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    img = torch.empty(3 * plan.P, dtype=torch.float32, device="cuda")
    T = torch.empty(plan.P, dtype=torch.float32, device="cuda")
    nc = torch.empty(plan.P, dtype=torch.int32, device="cuda")
    pk.bin_and_sort(plan, drec, vals, ranges, ws)
    pk.rasterize_fwd(plan, drec, vals, ranges, img, T, nc, ws)
    out = dict(plan=plan, ws=ws, rec=rec, drec=drec, vals=vals, ranges=ranges, img=img, T=T, nc=nc, views=views)
    if dimg_seed is not None:
        w = np.random.default_rng(dimg_seed).standard_normal(3 * plan.P).astype(np.float32)
        g2 = torch.empty(12 * plan.pairs, dtype=torch.float32, device="cuda")
        pk.rasterize_bwd(plan, drec, vals, ranges, T, nc, torch.from_numpy(w).cuda(), g2, ws)
        out.update(w=w, g2=g2)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("seed", [5, 6])
def test_tile_side_leaves_images_unchanged(seed):
    """32 px tiles bin and composite the same splats per pixel in the same
    order (the extra splats of a larger tile fail the alpha test): images
    and transmittance bit for bit equal to 16 px tiles, the backward's
    gradients equal up to the order of their atomic sums."""
    a = _records_forward(seed, dimg_seed=seed + 3)
    b = _records_forward(seed, dimg_seed=seed + 3, tile=32)
    assert b["plan"].n_tiles < a["plan"].n_tiles
    assert torch.equal(a["img"].view(torch.int32), b["img"].view(torch.int32))
    assert torch.equal(a["T"].view(torch.int32), b["T"].view(torch.int32))
    ga, gb = a["g2"].cpu().numpy().astype(np.float64), b["g2"].cpu().numpy().astype(np.float64)
    assert np.abs(ga - gb).max() <= 1e-5 * max(1e-12, np.abs(ga).max())


@pytest.mark.parametrize("seed", [5, 6])
def test_rasterize_fwd_l1_matches_separate_calls(orc, seed):
    """The fused forward + L1: image, T, n_contrib and dL/dimage bit for bit
    equal to pk_rasterize_fwd then pk_l1_loss_grad, the loss equal up to
    summation order, and both equal to the L1 of the oracle's definition."""
    pk = _pk()
    o = _records_forward(seed)
    plan, ws = o["plan"], o["ws"]
    target = torch.from_numpy(np.random.default_rng(seed + 40).random(3 * plan.P).astype(np.float32)).cuda()
    # a few exact ties (zero gradient)
    target[::97] = o["img"][::97]
    g_ref = torch.empty_like(o["img"])
    pk.l1_loss_grad(plan, o["img"], target, g_ref, ws)
    loss_ref = pk.read_status(plan, ws)["loss"]
    img, T = torch.full_like(o["img"], -1.0), torch.full_like(o["T"], -1.0)
    nc, g = torch.full_like(o["nc"], -1), torch.full_like(o["img"], 7.0)
    pk.rasterize_fwd_l1(plan, o["drec"], o["vals"], o["ranges"], target, img, T, nc, g, ws)
    st = pk.read_status(plan, ws)
    assert st["flags"] == 0
    assert torch.equal(img.view(torch.int32), o["img"].view(torch.int32))
    assert torch.equal(T.view(torch.int32), o["T"].view(torch.int32))
    assert torch.equal(nc, o["nc"])
    assert torch.equal(g.view(torch.int32), g_ref.view(torch.int32))
    want = np.abs(o["img"].cpu().numpy().astype(np.float64) - target.cpu().numpy().astype(np.float64)).mean()
    assert abs(st["loss"] - loss_ref) <= 1e-6 * abs(want)
    assert abs(st["loss"] - want) <= 1e-6 * abs(want)


@pytest.mark.parametrize("seed,tile", [(5, 16), (5, 32)])
def test_clearing_forward_and_accumulating_backward(seed, tile):
    """pk_rasterize_fwd_l1_clear: the outputs of pk_rasterize_fwd_l1 bit for
    bit, and every float of grad2d (filled with garbage first) zero after
    it; pk_rasterize_bwd_accumulate then gives pk_rasterize_bwd's gradients
    (up to the order of their atomic sums), and a second call doubles them."""
    pk = _pk()
    o = _records_forward(seed, dimg_seed=seed + 9, tile=tile)
    plan, ws = o["plan"], o["ws"]
    target = torch.from_numpy(np.random.default_rng(seed + 41).random(3 * plan.P).astype(np.float32)).cuda()
    img0, T0, nc0, g0 = (torch.empty_like(o["img"]), torch.empty_like(o["T"]), torch.empty_like(o["nc"]),
                         torch.empty_like(o["img"]))
    pk.rasterize_fwd_l1(plan, o["drec"], o["vals"], o["ranges"], target, img0, T0, nc0, g0, ws)
    img, T = torch.full_like(o["img"], -1.0), torch.full_like(o["T"], -1.0)
    nc, g = torch.full_like(o["nc"], -1), torch.full_like(o["img"], 7.0)
    g2 = torch.full((12 * plan.pairs,), float("nan"), dtype=torch.float32, device="cuda")
    pk.rasterize_fwd_l1_clear(plan, o["drec"], o["vals"], o["ranges"], target, img, T, nc, g, g2, ws)
    torch.cuda.synchronize()
    assert pk.read_status(plan, ws)["flags"] == 0
    for a, b in ((img, img0), (T, T0), (g, g0)):
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    assert torch.equal(nc, nc0)
    assert torch.equal(g2.view(torch.int32), torch.zeros_like(g2).view(torch.int32))
    w = torch.from_numpy(o["w"]).cuda()
    pk.rasterize_bwd_accumulate(plan, o["drec"], o["vals"], o["ranges"], o["T"], o["nc"], w, g2, ws)
    torch.cuda.synchronize()
    ref = o["g2"].cpu().numpy().astype(np.float64)
    got = g2.cpu().numpy().astype(np.float64)
    scale = max(1e-12, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-5 * scale
    pk.rasterize_bwd_accumulate(plan, o["drec"], o["vals"], o["ranges"], o["T"], o["nc"], w, g2, ws)
    torch.cuda.synchronize()
    assert np.abs(g2.cpu().numpy().astype(np.float64) - 2.0 * ref).max() <= 2e-5 * scale


def test_l1_step_equals_forward_then_backward():
    """Renderer.l1_step (the clearing forward, the accumulating backward)
    against forward with the L1 target then backward: the same image and
    dL/dimage bit for bit, the same texel gradient up to the order of the
    atomic sums, whatever the 2D gradient buffer held before."""
    pk = _pk()
    sc = H.scene_small_sh3(seed=515)
    atlas, occ, dyn = H.upload(sc)
    F, D, Hh, W = sc.atlas.shape
    target = torch.from_numpy(synth.random_target(sc)).cuda()
    r = pk.Renderer(pk.Plan.for_scene(sc))
    r.ensure_capacity(atlas, occ, dyn)
    ga = torch.zeros(F * D * Hh * W, dtype=torch.float32, device="cuda")
    r.forward(atlas, occ, dyn, target=target)
    r.backward(r.dimage, ga)
    torch.cuda.synchronize()
    img0, dimg0 = r.image.clone(), r.dimage.clone()
    r.grad2d.fill_(float("nan"))
    gb = torch.zeros_like(ga)
    r.l1_step(atlas, occ, dyn, target, gb)
    torch.cuda.synchronize()
    assert r.status()["flags"] == 0
    assert torch.equal(r.image.view(torch.int32), img0.view(torch.int32))
    assert torch.equal(r.dimage.view(torch.int32), dimg0.view(torch.int32))
    a, b = ga.cpu().numpy().astype(np.float64), gb.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(b))
    assert np.abs(a - b).max() <= 1e-5 * max(1e-12, np.abs(a).max())


@pytest.mark.parametrize("seed,tile", [(5, 16), (6, 16), (5, 32)])
def test_rasterize_fwd_on_identical_records(orc, seed, tile):
    o = _records_forward(seed, tile=tile)
    rec64 = o["rec"].astype(np.float64)
    rec64[..., 11] = 0
    va = orc.views_array(o["views"])
    vals, ranges = orc.bin_sort(rec64, va, tile)
    # identical FP32 records on both sides: no mean error (m_tol 0), only the
    # rounding of the quadratic form; the depth order is the same (the sort
    # is bit-exact), so near-equal depths are not borderline here
    ref = orc.render(rec64, va, tile, vals, ranges, m_tol=0.0)
    ref["view_pixels"] = [v.width * v.height for v in o["views"]]
    ref["border"] = ref["border"] & ~np.uint8(H.B_DEPTH)
    H.check_images(o["img"].cpu().numpy(), o["T"].cpu().numpy(), ref, tol=2e-5, max_border_frac=1e-3,
                   max_threshold_frac=1e-3, label=f"identical records seed {seed} tile {tile}")
    ok = (ref["border"] & H.IMAGE_BORDER) == 0
    assert np.array_equal(H.u32(o["nc"])[ok], ref["last"][ok])
    st = _pk().read_status(o["plan"], o["ws"])
    assert st["evals_fwd"] > 0


@pytest.mark.parametrize("seed,tile", [(7, 16), (8, 16), (7, 32)])
def test_rasterize_bwd_on_identical_records(orc, seed, tile):
    o = _records_forward(seed, dimg_seed=seed + 100, tile=tile)
    rec64 = o["rec"].astype(np.float64)
    rec64[..., 11] = 0
    va = orc.views_array(o["views"])
    vals, ranges = orc.bin_sort(rec64, va, tile)
    ref = orc.render_bwd(rec64, va, tile, vals, ranges, o["w"].astype(np.float64))
    got = o["g2"].view(-1, 12).cpu().numpy().astype(np.float64)[:, :9]
    ref = ref.reshape(-1, 9)
    for name, sl in {"mean": slice(0, 2), "conic": slice(2, 5), "opacity": slice(5, 6),
                     "colour": slice(6, 9)}.items():
        assert H.rel_err(got[:, sl], ref[:, sl]) < 1e-3, name


# ---------------------------------------------------------------------------
# Whole step against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["sh3_small", "fp16_multilevel", "frames_dyn", "config1"])
def test_end_to_end(orc, which):
    sc = {"sh3_small": lambda: H.scene_small_sh3(), "fp16_multilevel": lambda: H.scene_multilevel_f16(),
          "frames_dyn": lambda: H.scene_small_sh3(frames=2, dyn=0.3),
          "config1": lambda: synth.config_scene(1)}[which]()
    P = sc.pixels
    o = oracle_run(orc, sc)
    w = H.zero_on_borderline(np.random.default_rng(11).standard_normal(3 * P).astype(np.float32), o)
    plan, r, grad = run_gpu(sc, dimg=w)
    oracle_backward(orc, sc, o, w)
    H.check_images(r.image.cpu().numpy(), r.T.cpu().numpy(), o)
    g = gpu_grad_soa(sc, grad, o["texel"])
    H.check_grads(g, o["grad_soa"])
    if sc.dyn is not None:
        frozen = np.tile(o["dynflag"] == 0, sc.frames)
        assert np.all(g[:, frozen] == 0)
    # texels that are not live receive nothing
    F, D, Hh, W = sc.atlas.shape
    live = np.zeros(Hh * W, bool)
    live[o["texel"]] = True
    assert np.all(grad.view(F, D, Hh * W).cpu().numpy()[:, :, ~live] == 0)


def test_end_to_end_degenerate_view_sizes(orc):
    """Views of 1 x 1, 1 x 37, 37 x 1, 17 x 15, 33 x 31 and 48 x 16 pixels
    (focal length 100 px each): rows and columns of tiles cut short on every
    side, compositing CTAs and warp blocks mostly past the view's edge.
    Images and gradients against the oracle, as for any scene."""
    sizes = [(1, 1), (1, 37), (37, 1), (17, 15), (33, 31), (48, 16)]
    eyes = [(0.4, 0.3, -3.2), (-2.6, -0.5, -1.8), (2.0, 1.2, 2.5), (0.3, -2.9, 1.1), (-1.7, 2.2, -2.0), (3.1, 0.2, 0.4)]
    views = [synth.scenes.pinhole(e, w, h, fov_x_deg=2.0 * math.degrees(math.atan(w / 200.0)))
             for e, (w, h) in zip(eyes, sizes)]
    sc = synth.make_scene([(128, 128, 0, 0, 0)], (128, 128), 0.6, views, sh_degree=3, seed=606,
                          log_scale=(-3.6, 0.5))
    P = sc.pixels
    o = oracle_run(orc, sc)
    w = H.zero_on_borderline(np.random.default_rng(21).standard_normal(3 * P).astype(np.float32), o)
    plan, r, grad = run_gpu(sc, dimg=w)
    oracle_backward(orc, sc, o, w)
    H.check_images(r.image.cpu().numpy(), r.T.cpu().numpy(), o, label="degenerate views")
    H.check_grads(gpu_grad_soa(sc, grad, o["texel"]), o["grad_soa"])


def test_rect_and_ellipse_binning_give_the_same_images(orc):
    sc = H.scene_small_sh3(seed=404)
    w = np.random.default_rng(15).standard_normal(3 * sc.pixels).astype(np.float32)
    _, r1, g1 = run_gpu(sc, dimg=w, bin_mode="ellipse")
    _, r0, g0 = run_gpu(sc, dimg=w, bin_mode="rect")
    assert r1.status()["dups"] < r0.status()["dups"]
    assert torch.equal(r1.image, r0.image) and torch.equal(r1.T, r0.T)
    assert H.rel_err(g1.cpu().numpy().astype(np.float64), g0.cpu().numpy().astype(np.float64)) < 1e-5


def test_config2_full_size(orc):
    """1080p single view, 157,286 Gaussians with SH degree 3: images and gradients in full."""
    sc = synth.config_scene(2)
    o = oracle_run(orc, sc)
    w = H.zero_on_borderline(np.random.default_rng(12).standard_normal(3 * sc.pixels).astype(np.float32), o)
    plan, r, grad = run_gpu(sc, dimg=w)
    oracle_backward(orc, sc, o, w)
    H.check_images(r.image.cpu().numpy(), r.T.cpu().numpy(), o)
    H.check_grads(gpu_grad_soa(sc, grad, o["texel"]), o["grad_soa"])


def test_batched_equals_per_view_loop(orc):
    pk = _pk()
    sc = H.scene_small_sh3()
    P = sc.pixels
    w = np.random.default_rng(14).standard_normal(3 * P).astype(np.float32)
    plan, r, grad = run_gpu(sc, dimg=w)
    loop = pk.PerViewLoop.for_scene(sc)
    atlas, occ, dyn = H.upload(sc)
    loop.dimage.copy_(torch.from_numpy(w))
    F, D, Hh, W = sc.atlas.shape
    g2 = torch.zeros(F * D * Hh * W, dtype=torch.float32, device="cuda")
    loop.step(atlas, occ, dyn, None, g2, loss=False)
    torch.cuda.synchronize()
    assert torch.equal(loop.image, r.image) and torch.equal(loop.T, r.T)
    assert torch.equal(loop.n_contrib, r.n_contrib)
    assert H.rel_err(g2.cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64)) < 1e-5


def test_cuda_graph_replay_matches_eager():
    pk = _pk()
    sc = H.scene_small_sh3(seed=303)
    plan = pk.Plan.for_scene(sc)
    r = pk.Renderer(plan)
    atlas, occ, dyn = H.upload(sc)
    tgt = torch.from_numpy(synth.random_target(sc)).cuda()
    F, D, Hh, W = sc.atlas.shape
    grad = torch.zeros(F * D * Hh * W, dtype=torch.float32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r.l1_step(atlas, occ, dyn, tgt, grad)
    torch.cuda.synchronize()
    img0, g0 = r.image.clone(), grad.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        r.l1_step(atlas, occ, dyn, tgt, grad)
    r.image.zero_()
    grad.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(r.image, img0)
    assert H.rel_err(grad.cpu().numpy(), g0.cpu().numpy()) < 1e-5
    st = r.status()
    assert st["flags"] == 0 and st["loss"] > 0


def test_live_count_mismatch_is_reported():
    pk = _pk()
    sc = H.scene_small_sh3()
    F, D, Hh, W = sc.atlas.shape
    plan = pk.Plan(sc.levels, (W, Hh), sc.sh_degree, F, "f32", sc.views, sc.n_live - 5)
    r = pk.Renderer(plan)
    atlas, occ, dyn = H.upload(sc)
    r.forward(atlas, occ, dyn)
    st = r.status()
    assert st["flags"] & 2 and st["live_seen"] == sc.n_live


def test_nothing_visible_gives_background():
    pk = _pk()
    sc = H.scene_small_sh3()
    # camera at z = +50 looking along +z: every mean is behind it
    views = [synth.View(R=np.eye(3), t=np.array([0.0, 0.0, -50.0]), fx=60.0, fy=60.0, cx=32.0, cy=20.0,
                        width=64, height=40)]
    F, D, Hh, W = sc.atlas.shape
    plan = pk.Plan(sc.levels, (W, Hh), sc.sh_degree, F, "f32", views, sc.n_live, bg=(0.25, 0.5, 1.0))
    r = pk.Renderer(plan)
    atlas, occ, dyn = H.upload(sc)
    r.forward(atlas, occ, dyn)
    torch.cuda.synchronize()
    img = r.image.view(3, -1).cpu().numpy()
    assert np.all(img[0] == 0.25) and np.all(img[1] == 0.5) and np.all(img[2] == 1.0)
    assert np.all(r.T.cpu().numpy() == 1.0) and r.status()["dups"] == 0


def test_empty_atlas_renders_background_and_leaves_gradients():
    """No live texel at all (N = 0): every call of the step still runs.  The
    image is the background, T = 1, no pixel has a contributor, no list
    entry is made, and the scatter writes nothing (it writes live texels
    only, so the gradient buffer keeps what it held)."""
    pk = _pk()
    views = [synth.scenes.pinhole((0.4, 0.3, -3.2), 64, 48), synth.scenes.pinhole((-2.6, -0.5, -1.8), 40, 56)]
    sc = synth.make_scene([(32, 32, 0, 0, 0)], (32, 32), 0.0, views, sh_degree=3, seed=3)
    assert sc.n_live == 0
    F, D, Hh, W = sc.atlas.shape
    plan = pk.Plan(sc.levels, (W, Hh), sc.sh_degree, F, "f32", sc.views, 0, bg=(0.25, 0.5, 1.0))
    r = pk.Renderer(plan)
    atlas, occ, dyn = H.upload(sc)
    r.forward(atlas, occ, dyn)
    grad = torch.full((F * D * Hh * W,), 7.0, dtype=torch.float32, device="cuda")
    r.backward(torch.ones(3 * sc.pixels, dtype=torch.float32, device="cuda"), grad)
    torch.cuda.synchronize()
    img = r.image.cpu().numpy()   # [view][3][H][W] concatenated
    off = 0
    for v in sc.views:
        n = v.width * v.height
        for c, b in enumerate((0.25, 0.5, 1.0)):
            assert np.all(img[3 * off + c * n:3 * off + (c + 1) * n] == b)
        off += n
    assert np.all(r.T.cpu().numpy() == 1.0)
    assert np.all(r.n_contrib.cpu().numpy() == 0)
    st = r.status()
    assert st["flags"] == 0 and st["dups"] == 0, st
    assert np.all(grad.cpu().numpy() == 7.0)


def test_every_batch_size_and_autotune():
    """The compositing batch (64, 128, 256 splats) and the staging mode (loads
    or bulk copies) change nothing but speed: images, transmittance and
    contributor counts are bit-identical, 2D gradients equal up to the order
    of their atomic sums; pk_autotune keeps one of the choices."""
    pk = _pk()
    sc = H.scene_small_sh3(seed=707)
    atlas, occ, dyn = H.upload(sc)
    w = torch.from_numpy(np.random.default_rng(8).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    out = {}
    for case in ((64, "loads", "bulk"), (128, "bulk", "loads"), (256, "loads", "loads"), (256, "bulk", "bulk")):
        b, mf, mb = case
        r = pk.Renderer(pk.Plan.for_scene(sc, batch=b, stage_fwd=mf, stage_bwd=mb))
        assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
        g = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
        r.backward(w, g)
        torch.cuda.synchronize()
        out[case] = (r.image.clone(), r.T.clone(), r.n_contrib.clone(), r.grad2d.clone())
    ref = out[(256, "loads", "loads")]
    for case, got in out.items():
        for k in range(3):
            assert torch.equal(got[k], ref[k]), case
        assert H.rel_err(got[3].cpu().numpy().astype(np.float64), ref[3].cpu().numpy().astype(np.float64)) < 1e-5
    r = pk.Renderer(pk.Plan.for_scene(sc))
    target = torch.from_numpy(synth.random_target(sc)).cuda()
    r.ensure_capacity(atlas, occ, dyn)
    chosen = r.autotune(atlas, occ, dyn, target)
    assert chosen in (64, 128, 256) and r.plan.batch == chosen
    assert torch.equal(r.image, ref[0])


def test_autotune_tile_side_and_digit_widths(orc):
    """The tuner over tile sides (a plan each) and radix digit widths: the
    tuned plan's images and transmittance are bit-identical to the default
    plan's, and its lists equal the oracle's tile by tile."""
    pk = _pk()
    sc = H.scene_small_sh3(seed=717)
    atlas, occ, dyn = H.upload(sc)
    target = torch.from_numpy(synth.random_target(sc)).cuda()
    ref = pk.Renderer(pk.Plan.for_scene(sc, tile=32))
    assert ref.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    r = pk.Renderer(pk.Plan.for_scene(sc, tile=32))
    r.ensure_capacity(atlas, occ, dyn)
    r.autotune(atlas, occ, dyn, target, tiles=(32, 16))
    p = r.plan
    assert p.tile in (16, 32) and set(r.tile_times_ms) == {16, 32}
    assert p.sort_bits_tile in (8, 11) and p.sort_bits_depth in (8, 11)
    r.forward(atlas, occ, dyn)
    torch.cuda.synchronize()
    st = r.status()
    assert st["flags"] == 0
    assert torch.equal(r.image, ref.image) and torch.equal(r.T, ref.T)
    V, N = p.V, p.N
    rec = r.records.cpu().numpy().reshape(V * N, 12)
    va = orc.views_array(sc.views)
    ref_vals, ref_ranges = orc.bin_sort32(rec[:, 0], rec[:, 1], rec[:, 7], rec[:, 6], va, N, p.tile, rec[:, 2],
                                          rec[:, 3], rec[:, 4], mode=orc.BIN_ELLIPSE)
    assert st["dups"] == len(ref_vals)
    assert_same_tile_lists(H.u32(r.sorted_vals[:len(ref_vals)]), H.i64(r.ranges).reshape(-1, 2), ref_vals,
                           ref_ranges)
    # either digit width, either sort: the same lists
    for bits in ((11, 11), (11, 8), (8, 11)):
        q = p.with_options(sort_bits_depth=bits[0], sort_bits_tile=bits[1])
        ws = pk.make_workspace(q)
        pk.workspace_init(q, ws)
        vals = torch.empty(q.max_dups + 64, dtype=torch.int32, device="cuda")
        ranges = torch.empty(2 * q.n_tiles, dtype=torch.int64, device="cuda")
        pk.bin_and_sort(q, r.records, vals, ranges, ws)
        assert pk.read_status(q, ws)["flags"] == 0
        assert_same_tile_lists(H.u32(vals[:len(ref_vals)]), H.i64(ranges).reshape(-1, 2), ref_vals, ref_ranges)


def test_render_fwd_bwd_convenience_calls():
    """pk_render_fwd / pk_render_bwd chain the six calls: same outputs."""
    pk = _pk()
    sc = H.scene_small_sh3(seed=708, dyn=0.3)
    atlas, occ, dyn = H.upload(sc)
    r = pk.Renderer(pk.Plan.for_scene(sc))
    assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    w = torch.from_numpy(np.random.default_rng(9).standard_normal(3 * sc.pixels).astype(np.float32)).cuda()
    g_ref = torch.zeros(atlas.numel(), dtype=torch.float32, device="cuda")
    r.backward(w, g_ref)
    img_ref = r.image.clone()
    p = r.plan
    img = torch.full_like(r.image, -1.0)
    pk.render_fwd(p, atlas, occ, dyn, r.soa, r.texel, r.dynflag, r.records, r.sorted_vals, r.ranges, img, r.T,
                  r.n_contrib, r.ws)
    g = torch.zeros_like(g_ref)
    pk.render_bwd(p, r.soa, r.dynflag, r.texel, r.records, r.sorted_vals, r.ranges, r.T, r.n_contrib, w, r.grad2d,
                  g, False, r.ws)
    torch.cuda.synchronize()
    assert torch.equal(img, img_ref)
    assert H.rel_err(g.cpu().numpy().astype(np.float64), g_ref.cpu().numpy().astype(np.float64)) < 1e-5


@pytest.mark.parametrize("mode", ["ellipse", "rect"])
def test_binning_from_fp64_projection_differs_only_at_borderline_pairs(orc, mode):
    """The sort is bit-exact as a function of the records; fed the oracle's
    own FP64 projection (rounded to FP32) instead of the GPU's, only pairs
    whose tile set sits on a threshold may differ: count them (a tiny
    fraction) and check that their summed entry counts nearly agree."""
    pk = _pk()
    sc = H.scene_small_sh3(seed=811)
    r = pk.Renderer(pk.Plan.for_scene(sc, bin_mode=mode))
    atlas, occ, dyn = H.upload(sc)
    assert r.ensure_capacity(atlas, occ, dyn)["flags"] == 0
    V, N = len(sc.views), r.plan.N
    gpu_rec = r.records.cpu().numpy().reshape(V * N, 12)
    o = orc.forward(sc, mode={"ellipse": orc.BIN_ELLIPSE, "rect": orc.BIN_RECT}[mode])
    ora_rec = o["rec"].reshape(V * N, 12).astype(np.float32)
    va = orc.views_array(sc.views)
    m = {"ellipse": orc.BIN_ELLIPSE, "rect": orc.BIN_RECT}[mode]

    def per_pair(rr):
        vals, _ = orc.bin_sort32(rr[:, 0], rr[:, 1], rr[:, 7], rr[:, 6], va, N, 16, rr[:, 2], rr[:, 3], rr[:, 4], mode=m)
        return np.bincount(vals, minlength=V * N)

    a, b = per_pair(gpu_rec), per_pair(ora_rec)
    differ = int(np.count_nonzero(a != b))
    print(f"{mode}: {differ} of {V * N} pairs have another tile count from the FP64 projection")
    assert differ <= max(3, 0.002 * V * N)
    assert abs(int(a.sum()) - int(b.sum())) <= 2 * max(1, differ)


def test_counting_variant_changes_nothing_but_the_counts():
    """The compositing kernels with and without the evaluation counters:
    bit-identical images, transmittance and contributor counts, 2D
    gradients equal up to their atomic order; only the counting plan
    reports evaluations."""
    pk = _pk()
    o = _records_forward(5, dimg_seed=9)
    plan, ws = o["plan"], o["ws"]
    st = pk.read_status(plan, ws)
    assert st["evals_fwd"] > 0 and st["evals_bwd"] > 0
    q = plan.with_options(count_evals=False)
    ws2 = pk.make_workspace(q)
    pk.workspace_init(q, ws2)
    img, T, nc = torch.empty_like(o["img"]), torch.empty_like(o["T"]), torch.empty_like(o["nc"])
    pk.rasterize_fwd(q, o["drec"], o["vals"], o["ranges"], img, T, nc, ws2)
    g2 = torch.empty_like(o["g2"])
    pk.rasterize_bwd(q, o["drec"], o["vals"], o["ranges"], T, nc, torch.from_numpy(o["w"]).cuda(), g2, ws2)
    st2 = pk.read_status(q, ws2)
    assert st2["evals_fwd"] == 0 and st2["evals_bwd"] == 0 and st2["flags"] == 0
    assert torch.equal(img, o["img"]) and torch.equal(T, o["T"]) and torch.equal(nc, o["nc"])
    a, b = g2.cpu().numpy().astype(np.float64), o["g2"].cpu().numpy().astype(np.float64)
    assert np.abs(a - b).max() <= 1e-5 * max(1e-12, np.abs(b).max())
