"""The allocation-free binning call, checked against the regular one.

pk_bin_and_sort_noalloc serves callers that cannot give the library any
device memory (for instance a renderer driven from another framework's
frame callback, where that framework owns the allocations and allocating
would stall the frame): it keeps its scratch in a fixed array inside the
library.  Its sorted lists must be bit-identical to those of
pk_bin_and_sort, call after call and from one plan to another, although
every call reuses the same array.  This file is collected last on purpose.
"""

import math

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _records(views, N, seed):
    rng = np.random.default_rng(seed)
    rec = np.zeros((len(views), N, 12), np.float32)
    for v, vw in enumerate(views):
        rec[v, :, 0] = rng.uniform(-20, vw.width + 20, N)
        rec[v, :, 1] = rng.uniform(-20, vw.height + 20, N)
        L = rng.normal(0, 1, (N, 2, 2)) * np.exp(rng.normal(0.8, 0.7, (N, 1, 1)))
        S = L @ L.transpose(0, 2, 1) + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        rec[v, :, 2], rec[v, :, 3], rec[v, :, 4] = Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 1]
        rec[v, :, 5] = rng.uniform(0.05, 0.95, N)
        rec[v, :, 6] = rng.uniform(0.5, 8.0, N)
        rec[v, :, 7] = np.ceil(3 * np.sqrt(np.linalg.eigvalsh(S)[:, 1]))
    rec[:, ::11, 7] = 0
    rec[:, 3::13, 6] = rec[:, 3, 6][:, None]
    return rec


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_23040_gb300 as pk
    pk.build.build()
    return pk


def test_noalloc_matches_regular_call_twice(pk):
    views = [synth.scenes.pinhole((0, 0, -3), 301, 173), synth.scenes.pinhole((0, 0, -3), 128, 200)]
    N = 3000
    side = int(math.ceil(math.sqrt(N)))
    plan = pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, max_dups=400_000)
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    for seed in (1, 2):                       # two calls in a row on the shared array
        rec = torch.from_numpy(_records(views, N, seed).reshape(-1)).cuda()
        vals_ref = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
        rng_ref = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
        pk.bin_and_sort(plan, rec, vals_ref, rng_ref, ws)
        st = pk.read_status(plan, ws)
        assert st["flags"] == 0 and st["dups"] > 0
        vals = torch.full((plan.max_dups + 64,), -7, dtype=torch.int32, device="cuda")
        rng = torch.full((2 * plan.n_tiles,), -7, dtype=torch.int64, device="cuda")
        n = torch.zeros(1, dtype=torch.int32, device="cuda")
        pk.bin_and_sort_noalloc(plan, rec, vals, rng, n)
        torch.cuda.synchronize()
        d = int(st["dups"])
        assert int(n.item()) == d
        assert torch.equal(vals[:d], vals_ref[:d])
        assert torch.equal(rng, rng_ref)


def test_noalloc_reports_overflow_and_rejects_oversized_plans(pk):
    views = [synth.scenes.pinhole((0, 0, -3), 160, 120)]
    N = 2000
    side = int(math.ceil(math.sqrt(N)))
    plan = pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, max_dups=1024)
    rec = torch.from_numpy(_records(views, N, 3).reshape(-1)).cuda()
    vals = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    rng = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    pk.bin_and_sort_noalloc(plan, rec, vals, rng, n)
    torch.cuda.synchronize()
    assert int(n.item()) == -1 and int(rng.abs().sum()) == 0
    big = pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, max_dups=8_000_000)
    with pytest.raises(pk._native.PackUVError) as ei:
        pk.bin_and_sort_noalloc(big, rec, torch.empty(big.max_dups + 64, dtype=torch.int32, device="cuda"), rng, n)
    assert ei.value.code == 7


def _plan(pk, views, N, **kw):
    side = int(math.ceil(math.sqrt(N)))
    return pk.Plan([(side, side, 0, 0, 0)], (side, side), 0, 1, "f32", views, N, **kw)


def _both(pk, plan, rec):
    """The regular call on its own workspace and the allocation-free one:
    (entries, lists, ranges) of each."""
    ws = pk.make_workspace(plan)
    pk.workspace_init(plan, ws)
    vals_ref = torch.empty(plan.max_dups + 64, dtype=torch.int32, device="cuda")
    rng_ref = torch.empty(2 * plan.n_tiles, dtype=torch.int64, device="cuda")
    pk.bin_and_sort(plan, rec, vals_ref, rng_ref, ws)
    st = pk.read_status(plan, ws)
    vals = torch.full((plan.max_dups + 64,), -7, dtype=torch.int32, device="cuda")
    rng = torch.full((2 * plan.n_tiles,), -7, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    pk.bin_and_sort_noalloc(plan, rec, vals, rng, n)
    torch.cuda.synchronize()
    return st, (vals_ref, rng_ref), (int(n.item()), vals, rng)


def test_noalloc_after_calls_with_other_plans(pk):
    """Plan A (two views, segmented sorts), then plan B (one view, another N,
    unsegmented), then plan A again: whatever an earlier plan left in the
    shared array, each call equals the regular one bit for bit."""
    va = [synth.scenes.pinhole((0, 0, -3), 301, 173), synth.scenes.pinhole((0, 0, -3), 128, 200)]
    vb = [synth.scenes.pinhole((0, 0, -3), 220, 150)]
    pa = _plan(pk, va, 3000, max_dups=400_000)
    pb = _plan(pk, vb, 1700, max_dups=300_000)
    ra = torch.from_numpy(_records(va, 3000, 11).reshape(-1)).cuda()
    rb = torch.from_numpy(_records(vb, 1700, 12).reshape(-1)).cuda()
    for plan, rec in ((pa, ra), (pb, rb), (pa, ra)):
        st, (vals_ref, rng_ref), (n, vals, rng) = _both(pk, plan, rec)
        d = int(st["dups"])
        assert st["flags"] == 0 and d > 0 and n == d
        assert torch.equal(vals[:d], vals_ref[:d])
        assert torch.equal(rng, rng_ref)


def test_noalloc_reports_a_wait_that_gave_up(pk):
    """A radix pass whose first bounded wait gives up at once (the plan's
    test hook): the entry count comes back as 0xFFFFFFFE and every tile
    range is empty; the next regular call on the array is unaffected."""
    views = [synth.scenes.pinhole((0, 0, -3), 301, 173), synth.scenes.pinhole((0, 0, -3), 128, 200)]
    rec = torch.from_numpy(_records(views, 3000, 13).reshape(-1)).cuda()
    bad = _plan(pk, views, 3000, max_dups=400_000, first_wait_polls=-1)
    vals = torch.empty(bad.max_dups + 64, dtype=torch.int32, device="cuda")
    rng = torch.full((2 * bad.n_tiles,), 7, dtype=torch.int64, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    pk.bin_and_sort_noalloc(bad, rec, vals, rng, n)
    torch.cuda.synchronize()
    assert int(n.item()) == -2 and int(torch.count_nonzero(rng)) == 0
    good = _plan(pk, views, 3000, max_dups=400_000)
    st, (vals_ref, rng_ref), (n2, vals2, rng2) = _both(pk, good, rec)
    d = int(st["dups"])
    assert n2 == d and torch.equal(vals2[:d], vals_ref[:d]) and torch.equal(rng2, rng_ref)
