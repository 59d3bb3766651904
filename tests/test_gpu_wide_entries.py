"""More than 2^32 (pair, tile) entries in one launch.

Entry positions are 64-bit from the emission offsets to the tile ranges
that the compositing kernels read, so a plan may hold more entries than a
32-bit index reaches (Sec. 3's per-tile lists at a rig's scale).  65,536
tiles of 16 px (one 4096^2 view, or two 4096 x 2048 ones) reached by each
of 66,000 splats give 4.33e9 entries.  The splats are flat (zero
conic: alpha is the opacity at every pixel), so every tile's list is the
same depth order and every pixel composites the same sequence: a tile that
read its list at a wrong (truncated) position would come out different.
"""

import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = 66_000


def _flat_records(n, side, seed):
    """n splats with zero conic, opacity 0.5, a radius past the view's
    corners, distinct depths in shuffled order and distinct colours."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 12), np.float32)
    rec[:, 0] = rng.uniform(0, side, n)
    rec[:, 1] = rng.uniform(0, side, n)
    rec[:, 5] = 0.5
    rec[:, 6] = 1.0 + 1e-3 * rng.permutation(n).astype(np.float32)
    rec[:, 7] = 2.0 * side
    rec[:, 8:11] = rng.uniform(0, 1, (n, 3))
    return rec


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, _ = torch.cuda.mem_get_info()
    if free < 100 * 2**30:
        pytest.skip("needs about 90 GB of device memory")
    import paper_2602_23040_gb300 as pk
    pk.build.build()
    return pk


def _run(pk, sizes, n, max_dups, seed):
    """Binning, sort and forward of views of the given (width, height), each
    seeing the same n flat splats."""
    views = [synth.scenes.pinhole((0, 0, -3), w, h) for w, h in sizes]
    a = int(math.ceil(math.sqrt(n)))
    plan = pk.Plan([(a, a, 0, 0, 0)], (a, a), 0, 1, "f32", views, n, tile=16, bin_mode="rect",
                   max_dups=max_dups)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    one = _flat_records(n, max(max(wh) for wh in sizes), seed)
    rec = torch.from_numpy(np.concatenate([one] * len(sizes)).reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, rec, vals, ranges, ws)
    img = torch.empty(3 * plan.P, dtype=torch.float32, device="cuda")
    T = torch.empty(plan.P, dtype=torch.float32, device="cuda")
    nc = torch.empty(plan.P, dtype=torch.int32, device="cuda")
    pk.rasterize_fwd(plan, rec, vals, ranges, img, T, nc, ws)
    torch.cuda.synchronize()
    return dict(plan=plan, ws=ws, st=pk.read_status(plan, ws), vals=vals, ranges=ranges, img=img, T=T, nc=nc,
                rec=rec, sizes=sizes, n=n)


def _backward_of_tile(pk, r, t):
    """The backward with dL/dimage = 1 on the 16 x 16 pixels of global tile
    t, 0 elsewhere."""
    w = torch.zeros(3 * r["plan"].P, dtype=torch.float32, device="cuda")
    pix0, tile0 = 0, 0
    for wv, hv in r["sizes"]:
        tiles = (wv // 16) * (hv // 16)
        if t < tile0 + tiles:
            lt = t - tile0
            tx, ty = lt % (wv // 16), lt // (wv // 16)
            img = w[3 * pix0:3 * (pix0 + wv * hv)].view(3, hv, wv)
            img[:, 16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = 1.0
            break
        pix0, tile0 = pix0 + wv * hv, tile0 + tiles
    g2 = torch.empty(12 * r["plan"].pairs, dtype=torch.float32, device="cuda")
    pk.rasterize_bwd(r["plan"], r["rec"], r["vals"], r["ranges"], r["T"], r["nc"], w, g2, r["ws"])
    torch.cuda.synchronize()
    return g2.view(-1, 12)


# one 4096^2 view: global tile ids (16 bits) and pair indices (17) do not fit
# one word, so keys and values travel separately; two 4096 x 2048 views:
# local tile ids (15 bits) and local pair indices (17) share one word
@pytest.mark.parametrize("sizes", [[(4096, 4096)], [(4096, 2048), (4096, 2048)]], ids=["keys_and_values", "packed"])
def test_more_than_2_32_entries(pk, sizes):
    tiles = [(w // 16) * (h // 16) for w, h in sizes]
    total = N * sum(tiles)
    assert total > 2**32
    big = _run(pk, sizes, N, total + 1024, 5)
    st = big["st"]
    assert st["flags"] == 0 and st["dups"] == total, st
    # every tile's list: all N splats of its view, contiguous, in (depth, pair) order
    T_all = sum(tiles)
    rng = big["ranges"].view(T_all, 2)
    assert bool(torch.all(rng[:, 1] - rng[:, 0] == N))
    starts = torch.sort(rng[:, 0]).values
    assert torch.equal(starts, torch.arange(T_all, device="cuda", dtype=torch.int64) * N)
    last = int(torch.argmax(rng[:, 0]))
    assert int(rng[last, 0]) > 2**32                # a list that only a 64-bit position reaches
    z = big["rec"].view(-1, 12)[:N, 6]
    order = torch.argsort(z, stable=True).to(torch.int32)
    t0 = 0
    for v, tv in enumerate(tiles):
        for r0 in range(t0, t0 + tv, 1024):
            r1 = min(r0 + 1024, t0 + tv)
            s0 = rng[r0:r1, 0]
            idx = s0[:, None] + torch.arange(N, device="cuda", dtype=torch.int64)[None, :]
            assert torch.equal(big["vals"][idx], (order + v * N).expand(r1 - r0, N)), (v, r0)
        t0 += tv
    # one small view (a single tile at position 0) composites the same sequence
    small = _run(pk, [(16, 16)], N, N + 1024, 5)
    assert small["st"]["flags"] == 0 and small["st"]["dups"] == N
    assert torch.equal(small["vals"][:N], order)
    px0 = 0
    for w_, h_ in sizes:
        b = big["img"][3 * px0:3 * (px0 + w_ * h_)].view(3, -1)
        assert bool(torch.all(b == small["img"].view(3, -1)[:, :1]))
        px0 += w_ * h_
    assert bool(torch.all(big["T"] == small["T"][0])) and bool(torch.all(big["nc"] == small["nc"][0]))
    assert int(small["nc"][0]) > 1
    # the backward of the tile with the largest start equals the small view's, bit for bit, in the
    # opacity and colour gradients (a flat splat's terms do not depend on the pixel position)
    gb, gs = _backward_of_tile(pk, big, last), _backward_of_tile(pk, small, 0)
    v_last = int(np.searchsorted(np.cumsum(tiles), last, side="right"))
    assert int(torch.count_nonzero(gs[:, 5:9])) > 0
    assert torch.equal(gb[v_last * N:(v_last + 1) * N, 5:9], gs[:, 5:9])
    assert int(torch.count_nonzero(gb[:v_last * N])) == 0 and int(torch.count_nonzero(gb[(v_last + 1) * N:])) == 0
    assert bool(torch.all(gb[:, 0:2] == 0)) and bool(torch.all(gs[:, 0:2] == 0))
