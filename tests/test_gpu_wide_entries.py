"""More than 2^32 (pair, tile) entries in one launch.

Entry positions are 64-bit from the emission offsets to the tile ranges
that the compositing kernels read, so a plan may hold more entries than a
32-bit index reaches (Sec. 3's per-tile lists at a rig's scale).  One
4096 x 4096 view binned at 16 px has 65,536 tiles; 66,000 splats that
each reach every tile give 4.33e9 entries.  The splats are flat (zero
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

W = H = 4096
N = 66_000
TILES = (W // 16) * (H // 16)


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


def _run(pk, side, n, max_dups, seed):
    """Binning, sort and forward of one view."""
    views = [synth.scenes.pinhole((0, 0, -3), side, side)]
    a = int(math.ceil(math.sqrt(n)))
    plan = pk.Plan([(a, a, 0, 0, 0)], (a, a), 0, 1, "f32", views, n, tile=16, bin_mode="rect",
                   max_dups=max_dups)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    rec = torch.from_numpy(_flat_records(n, side, seed).reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, rec, vals, ranges, ws)
    img = torch.empty(3 * plan.P, dtype=torch.float32, device="cuda")
    T = torch.empty(plan.P, dtype=torch.float32, device="cuda")
    nc = torch.empty(plan.P, dtype=torch.int32, device="cuda")
    pk.rasterize_fwd(plan, rec, vals, ranges, img, T, nc, ws)
    torch.cuda.synchronize()
    return dict(plan=plan, ws=ws, st=pk.read_status(plan, ws), vals=vals, ranges=ranges, img=img, T=T, nc=nc,
                rec=rec, side=side, n=n)


def _backward_of_tile(pk, r, t):
    """The backward with dL/dimage = 1 on the 16 x 16 pixels of tile t, 0 elsewhere."""
    side, plan = r["side"], r["plan"]
    tx, ty = t % (side // 16), t // (side // 16)
    w = torch.zeros(3, side, side, dtype=torch.float32, device="cuda")
    w[:, 16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = 1.0
    g2 = torch.empty(12 * r["n"], dtype=torch.float32, device="cuda")
    pk.rasterize_bwd(plan, r["rec"], r["vals"], r["ranges"], r["T"], r["nc"], w.view(-1), g2, r["ws"])
    torch.cuda.synchronize()
    return g2.view(r["n"], 12)


def test_more_than_2_32_entries(pk):
    total = N * TILES
    assert total > 2**32
    big = _run(pk, W, N, total + 1024, 5)
    st = big["st"]
    assert st["flags"] == 0 and st["dups"] == total, st
    # every tile's list: all N splats, contiguous, in (depth, pair) order
    rng = big["ranges"].view(TILES, 2)
    assert bool(torch.all(rng[:, 1] - rng[:, 0] == N))
    starts = torch.sort(rng[:, 0]).values
    assert torch.equal(starts, torch.arange(TILES, device="cuda", dtype=torch.int64) * N)
    last = int(torch.argmax(rng[:, 0]))
    assert int(rng[last, 0]) > 2**32                # a list that only a 64-bit position reaches
    z = big["rec"].view(N, 12)[:, 6]
    order = torch.argsort(z, stable=True).to(torch.int32)
    lists = big["vals"][:total].view(TILES, N)
    for r0 in range(0, TILES, 2048):
        assert torch.equal(lists[r0:r0 + 2048], order.expand(min(2048, TILES - r0), N)), r0
    # one small view (a single tile at position 0) composites the same sequence
    small = _run(pk, 16, N, N + 1024, 5)
    assert small["st"]["flags"] == 0 and small["st"]["dups"] == N
    assert torch.equal(small["vals"][:N], order)
    assert bool(torch.all(big["img"].view(3, -1) == small["img"].view(3, -1)[:, :1]))
    assert bool(torch.all(big["T"] == small["T"][0])) and bool(torch.all(big["nc"] == small["nc"][0]))
    assert int(small["nc"][0]) > 1
    # the backward of the tile with the largest start equals the small view's, bit for bit, in the
    # opacity and colour gradients (a flat splat's terms do not depend on the pixel position)
    gb, gs = _backward_of_tile(pk, big, last), _backward_of_tile(pk, small, 0)
    assert int(torch.count_nonzero(gs[:, 5:9])) > 0
    assert torch.equal(gb[:, 5:9], gs[:, 5:9])
    assert bool(torch.all(gb[:, 0:2] == 0)) and bool(torch.all(gs[:, 0:2] == 0))
