"""Pins of the oracle's UV cells (eq. uvgs2) and Max-K UV pruning (Sec. 4.2
"UV-Based Pruning"): directions built at known spherical angles, cell
centres mapping back to their cell, the map's edges, and the per-cell
top-K against numpy's lexsort."""

import math

import numpy as np
import pytest


def _dir(theta, phi, rho=1.0):
    return (rho * math.sin(phi) * math.cos(theta), rho * math.sin(phi) * math.sin(theta), rho * math.cos(phi))


@pytest.mark.parametrize("M,N", [(64, 32), (37, 19), (1024, 512)])
def test_cell_centres_map_to_their_cell(orc, M, N):
    rng = np.random.default_rng(M)
    for _ in range(200):
        u, v = int(rng.integers(0, M)), int(rng.integers(0, N))
        theta = (u + 0.5) / M * 2 * math.pi - math.pi
        phi = (v + 0.5) / N * math.pi
        c, b = orc.uv_cell(*_dir(theta, phi, rng.uniform(0.1, 10.0)), M, N)
        assert b == 0 and c == v * M + u


def test_known_directions(orc):
    M, N = 8, 4
    assert orc.uv_cell(1.0, 0.0, 0.0, M, N)[0] == 2 * M + 4      # theta 0 -> u = M/2; phi pi/2 -> v = N/2
    assert orc.uv_cell(0.0, 1.0, 0.0, M, N)[0] == 2 * M + 6      # theta pi/2 -> u = 3M/4
    assert orc.uv_cell(-1.0, -1e-3, 0.3, M, N)[0] // M == 1      # phi = acos(0.3 / r) ~ 1.27 -> v = 1
    c, _ = orc.uv_cell(0.0, 0.0, 2.0, M, N)                       # phi = 0 -> v = 0, theta = atan2(0, 0) = 0
    assert c == 0 * M + 4
    assert orc.uv_cell(0.0, 0.0, -2.0, M, N)[0] == orc.INVALID    # phi = pi -> v = N: outside the map
    assert orc.uv_cell(-1.0, 0.0, 0.0, M, N)[0] == orc.INVALID    # theta = pi -> u = M: outside the map
    assert orc.uv_cell(0.0, 0.0, 0.0, M, N)[0] == orc.INVALID     # rho = 0
    assert orc.uv_cell(float("nan"), 0.0, 1.0, M, N)[0] == orc.INVALID


def _cloud(rng, n, M, N, crowd=3.0):
    """n Gaussians over about n / crowd cells (directions), random radii."""
    cells = rng.integers(0, M * N, size=max(1, int(n / crowd)))
    pick = cells[rng.integers(0, len(cells), size=n)]
    u, v = pick % M, pick // M
    theta = (u + rng.uniform(0.05, 0.95, n)) / M * 2 * np.pi - np.pi
    phi = (v + rng.uniform(0.05, 0.95, n)) / N * np.pi
    rho = rng.uniform(0.2, 3.0, n)
    soa = np.zeros((14, n))
    soa[0] = rho * np.sin(phi) * np.cos(theta)
    soa[1] = rho * np.sin(phi) * np.sin(theta)
    soa[2] = rho * np.cos(phi)
    soa[10] = np.round(rng.normal(0.0, 1.0, n), 1)          # rounded: many equal opacities
    return soa.astype(np.float32).astype(np.float64), pick


@pytest.mark.parametrize("K", [0, 1, 3, 1000])
def test_max_k_against_lexsort(orc, K):
    M, N = 16, 8
    rng = np.random.default_rng(10 + K)
    soa, pick = _cloud(rng, 600, M, N)
    out = orc.uv_max_k(soa, M, N, K)
    assert out["border"].sum() == 0
    np.testing.assert_array_equal(out["cell"], pick)
    # rank: order by (cell, -logit, index) with numpy's lexsort
    order = np.lexsort((np.arange(len(pick)), -soa[10], pick))
    rank = np.zeros(len(pick), np.int64)
    start = 0
    cs = pick[order]
    for i in range(1, len(order) + 1):
        if i == len(order) or cs[i] != cs[start]:
            rank[order[start:i]] = np.arange(i - start)
            start = i
    np.testing.assert_array_equal(out["rank"], rank)
    np.testing.assert_array_equal(out["keep"], (rank < K).astype(np.uint8))
    np.testing.assert_array_equal(out["count"], np.bincount(pick, minlength=M * N))
    assert out["keep"].sum() == np.minimum(np.bincount(pick, minlength=M * N), K).sum()


def test_max_k_invalid_and_permutation(orc):
    M, N = 16, 8
    rng = np.random.default_rng(3)
    soa, pick = _cloud(rng, 300, M, N)
    soa[:, 5] = 0.0                   # rho = 0
    soa[10, 7] = np.nan               # NaN opacity
    out = orc.uv_max_k(soa, M, N, 2)
    for i in (5, 7):
        assert out["cell"][i] == orc.INVALID and out["rank"][i] == orc.INVALID and out["keep"][i] == 0
    # the kept set does not depend on the input order (no equal opacities here)
    soa2, _ = _cloud(np.random.default_rng(4), 300, M, N)
    soa2[10] = rng.permutation(300) * 0.01
    a = orc.uv_max_k(soa2, M, N, 2)
    perm = rng.permutation(300)
    b = orc.uv_max_k(soa2[:, perm], M, N, 2)
    np.testing.assert_array_equal(b["keep"], a["keep"][perm])
    np.testing.assert_array_equal(b["rank"], a["rank"][perm])
