"""UV cells (eq. uvgs2) and Max-K UV pruning on the GPU against the
oracle: cells, ranks, keep flags and per-cell counts bit for bit, on
crowded cells with equal opacities, invalid Gaussians, and at the size of
the 1024^2 atlas's live set."""

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_23040_gb300 as pk
    pk.build.build()
    return pk


def _cloud(rng, n, M, N, crowd):
    cells = rng.integers(0, M * N, size=max(1, int(n / crowd)))
    pick = cells[rng.integers(0, len(cells), size=n)]
    u, v = pick % M, pick // M
    theta = (u + rng.uniform(0.02, 0.98, n)) / M * 2 * np.pi - np.pi
    phi = (v + rng.uniform(0.02, 0.98, n)) / N * np.pi
    rho = rng.uniform(0.2, 3.0, n)
    soa = np.zeros((14, n), np.float32)
    soa[0] = rho * np.sin(phi) * np.cos(theta)
    soa[1] = rho * np.sin(phi) * np.sin(theta)
    soa[2] = rho * np.cos(phi)
    soa[10] = np.round(rng.normal(0.0, 1.0, n), 1)
    return soa


def _run(pk, soa, M, N, K, n=None):
    n = soa.shape[1] if n is None else n
    d = torch.from_numpy(soa).cuda()
    cell = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    rank = torch.empty_like(cell)
    keep = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
    count = torch.empty(M * N, dtype=torch.int32, device="cuda")
    pk.uv_max_k(d, n, M, N, K, cell, rank, keep, count)
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32)
    return dict(cell=u32(cell)[:n], rank=u32(rank)[:n], keep=keep.cpu().numpy()[:n], count=u32(count))


@pytest.mark.parametrize("M,N,K,crowd", [(64, 32, 2, 4.0), (37, 19, 1, 12.0), (256, 128, 5, 1.5), (16, 8, 0, 3.0)])
def test_uv_max_k_bit_exact(pk, orc, M, N, K, crowd):
    rng = np.random.default_rng(M + K)
    soa = _cloud(rng, 5000, M, N, crowd)
    soa[:, 11] = 0.0                  # rho = 0
    soa[10, 12] = np.nan              # NaN opacity
    soa[0, 13] = np.inf
    soa[:3, 14] = (-1.0, 0.0, 0.0)    # theta = pi: u = M, outside the map
    got = _run(pk, soa, M, N, K)
    want = orc.uv_max_k(soa.astype(np.float64), M, N, K)
    # theta = pi sits exactly on the map's edge: the only borderline Gaussian
    assert np.flatnonzero(want["border"]).tolist() == [14]
    assert got["cell"][14] == want["cell"][14] == orc.INVALID
    for k in ("cell", "rank", "keep", "count"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_uv_max_k_live_set_of_the_1024_atlas(pk, orc):
    """629,145 Gaussians of the 1024^2 atlas (clustered means) on the
    1024 x 1024 base map, K = 4."""
    sc = synth.config_scene(3, n_views=1)
    soa, _, _ = orc.gather(sc)
    s32 = np.ascontiguousarray(soa.astype(np.float32))
    got = _run(pk, s32, 1024, 1024, 4)
    want = orc.uv_max_k(s32.astype(np.float64), 1024, 1024, 4)
    ok = want["border"] == 0
    assert ok.mean() > 0.999
    for k in ("cell", "rank", "keep"):
        np.testing.assert_array_equal(got[k][ok], want[k][ok], err_msg=k)
    np.testing.assert_array_equal(got["count"], want["count"])


def test_uv_max_k_empty(pk):
    got = _run(pk, np.zeros((14, 1), np.float32), 8, 4, 3, n=0)
    assert got["count"].sum() == 0
