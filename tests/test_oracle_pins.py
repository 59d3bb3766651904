"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: a number the paper prints, a
closed form, a library routine, an invariant, or brute force on a tiny input.
"""

import math

import numpy as np
import pytest

import synth

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(f"{GOLDEN}/{name}") as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(x) for x in line.split()])
    return rows


def tiny_scene(seed=7, n_side=6, views=None, sh_degree=3, frames=1, dtype=np.float32, dyn=0.0,
               log_scale=(-2.2, 0.3), box=0.6):
    if views is None:
        views = [synth.scenes.pinhole((0.3, 0.2, -3.0), 40, 36)]
    return synth.make_scene([(n_side, n_side, 0, 0, 0)], (n_side, n_side), 1.0, views,
                            sh_degree=sh_degree, frames=frames, texel_dtype=dtype,
                            means="uniform", seed=seed, dynamic_frac=dyn,
                            log_scale=log_scale, mean_box=box)


# ---------------------------------------------------------------------------
# Pyramid and atlas (Sec. 4.1)
# ---------------------------------------------------------------------------

def test_pyramid_matches_printed_sequence(orc):
    # Sec. 4.1 prints the pattern {M0 x N0, M0 x N0/2, M0/2 x N0/2, M0/2 x N0/4, ...}
    rows = _read_golden("pyramid_1024_k8.txt")
    M, N = orc.pyramid_sizes(1024, 1024, 8)
    assert [[int(a), int(b)] for a, b in zip(M, N)] == rows


def test_atlas_efficiency_matches_paper(orc):
    # Sec. 4.1: the packing reaches 88.5 % (used texels / atlas texels), M0 = N0 = 1024, K = 8 (Sec. 5 setup)
    levels, (W, H) = orc.atlas_layout(1024, 8)
    used = sum(w * h for (w, h, *_r) in levels)
    assert round(used / (W * H), 3) == 0.885
    M, N = orc.pyramid_sizes(1024, 1024, 8)
    assert used == int(np.sum(M.astype(np.int64) * N))


def test_atlas_layout_structure(orc):
    for S, K in [(64, 1), (64, 2), (64, 3), (1024, 8), (256, 6)]:
        levels, (W, H) = orc.atlas_layout(S, K)
        cover = np.zeros((H, W), np.int32)
        for k, (w, h, x0, y0, rot) in enumerate(levels):
            assert 0 <= x0 and x0 + w <= W and 0 <= y0 and y0 + h <= H
            cover[y0:y0 + h, x0:x0 + w] += 1
            # odd levels rotated, even horizontal (Sec. 4.1)
            assert rot == (k % 2 == 1)
        assert cover.max() == 1, "levels overlap"
        if K > 1:
            w0, h0, x00, _y00, _ = levels[0]
            assert (w0, h0) == (S, S) and x00 + w0 == W, "L0 occupies the right region"


def test_texel_uv_round_trip(orc):
    levels, (W, H) = orc.atlas_layout(64, 8)
    seen = set()
    for y in range(H):
        for x in range(W):
            kuv = orc.texel_to_uv(levels, x, y)
            if kuv is None:
                continue
            k, u, v = kuv
            assert orc.uv_to_texel(levels, k, u, v) == (x, y)
            seen.add(kuv)
    M, N = orc.pyramid_sizes(64, 64, 8)
    assert len(seen) == int(np.sum(M * N))
    for k in range(8):   # every native (u, v) of every level is reachable
        assert all((k, u, v) in seen for u in range(M[k]) for v in range(N[k]))


# ---------------------------------------------------------------------------
# Gather
# ---------------------------------------------------------------------------

def test_half_decode_matches_numpy(orc):
    h = np.arange(65536, dtype=np.uint16)
    ref = h.view(np.float16).astype(np.float64)
    got = np.array([orc.half_to_double(int(x)) for x in h[::7]])
    r = ref[::7]
    assert np.array_equal(np.isnan(got), np.isnan(r))
    assert np.array_equal(got[~np.isnan(r)], r[~np.isnan(r)])


@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_gather_matches_numpy_indexing(orc, dtype):
    views = [synth.scenes.pinhole((0, 0, -3.0), 32, 32)]
    levels = [(40, 24, 20, 0, 0), (20, 40, 0, 0, 1), (16, 12, 0, 40, 0)]
    sc = synth.make_scene(levels, (60, 52), [0.5, 0.7, 0.3], views, sh_degree=1, frames=2,
                          texel_dtype=dtype, dynamic_frac=0.3, seed=3)
    soa, texel, dyn = orc.gather(sc)
    F, D, H, W = sc.atlas.shape
    occ = synth.scenes.unpack_bits(sc.occ, W)
    ys, xs = np.nonzero(occ)
    N = len(ys)
    assert N == sc.n_live and np.array_equal(texel, ys * W + xs)
    ref = np.concatenate([sc.atlas[f][:, ys, xs].astype(np.float64) for f in range(F)], axis=1)
    assert np.array_equal(soa, ref)
    dm = synth.scenes.unpack_bits(sc.dyn, W)
    assert np.array_equal(dyn.astype(bool), dm[ys, xs])


# ---------------------------------------------------------------------------
# Rotation and SH
# ---------------------------------------------------------------------------

def _hamilton(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def test_quaternion_rotation_is_the_sandwich_product(orc):
    rng = np.random.default_rng(1)
    for _ in range(50):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        R = orc.quat_rot(q)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-13
        v = rng.standard_normal(3)
        qc = q * np.array([1, -1, -1, -1])
        rv = _hamilton(_hamilton(q, np.r_[0.0, v]), qc)[1:]
        assert np.allclose(R @ v, rv, atol=1e-13)


def _real_sh_scipy(l, m, d):
    from scipy.special import sph_harm_y
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    am = abs(m)
    y = sph_harm_y(l, am, theta, phi)          # complex, Condon-Shortley phase included
    if m == 0:
        return y.real
    return math.sqrt(2) * (y.real if m > 0 else y.imag)


def test_sh_basis_matches_scipy(orc):
    rng = np.random.default_rng(2)
    for _ in range(40):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y, _ = orc.sh_basis(3, d)
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[l * l + l + m] - _real_sh_scipy(l, m, d)) < 1e-12


def test_sh_basis_orthonormal_and_y00(orc):
    # Gauss-Legendre in cos(theta) x uniform phi integrates products of degree <= 6 exactly.
    x, w = np.polynomial.legendre.leggauss(12)
    nphi = 16
    gram = np.zeros((16, 16))
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y, _ = orc.sh_basis(3, np.array([st * math.cos(ph), st * math.sin(ph), ct]))
            gram += wt * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(gram, np.eye(16), atol=1e-12)
    Y, _ = orc.sh_basis(0, np.array([0.0, 0.0, 1.0]))
    assert abs(Y[0] - 0.5 / math.sqrt(math.pi)) < 1e-15


def test_sh_gradient_tangential_part_by_differences(orc):
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y, dY = orc.sh_basis(3, d)
        for _k in range(3):
            t = rng.standard_normal(3)
            t -= d * (t @ d)
            t /= np.linalg.norm(t)
            h = 1e-5
            yp, _ = orc.sh_basis(3, (d + h * t) / np.linalg.norm(d + h * t))
            ym, _ = orc.sh_basis(3, (d - h * t) / np.linalg.norm(d - h * t))
            fd = (yp - ym) / (2 * h)
            assert np.allclose(dY @ t, fd, atol=1e-8)


# ---------------------------------------------------------------------------
# Projection (Alg. 1 steps 1-4)
# ---------------------------------------------------------------------------

def _one_gaussian_scene(mu, log_s, quat, logit, sh0, W=64, H=48, eye=(0.0, 0.0, -3.0), sh_degree=0):
    v = synth.scenes.pinhole(eye, W, H)
    D = synth.channel_count(sh_degree)
    atlas = np.zeros((1, D, 1, 1), np.float32)
    atlas[0, 0:3, 0, 0] = mu
    atlas[0, 3:6, 0, 0] = log_s
    atlas[0, 6:10, 0, 0] = quat
    atlas[0, 10, 0, 0] = logit
    atlas[0, 11:14, 0, 0] = sh0
    occ = synth.pack_bits(np.ones((1, 1), bool))
    return synth.Scene("one", atlas, occ, None, [(1, 1, 0, 0, 0)], sh_degree, [v], 1)


def test_isotropic_gaussian_closed_form(orc):
    s = math.exp(-3.0)
    sc = _one_gaussian_scene((0, 0, 0), (-3.0,) * 3, (0.3, 0.5, -0.1, 0.8), 0.7, (0.4, -0.2, 0.1))
    soa, _, _ = orc.gather(sc)
    va = orc.views_array(sc.views)
    rec = orc.project(soa, 1, 0, va)[0, 0]
    v = sc.views[0]
    fx = float(np.float32(v.fx))   # the camera the library receives is FP32
    z = 3.0
    var = (fx * s / z) ** 2 + 0.3
    assert abs(rec[0] - v.cx) < 1e-12 and abs(rec[1] - v.cy) < 1e-12
    assert np.allclose(rec[2:5], [1 / var, 0, 1 / var], rtol=1e-9, atol=1e-15)
    o = 1 / (1 + math.exp(-float(np.float32(0.7))))
    assert abs(rec[5] - o) < 1e-15
    assert abs(rec[6] - z) < 1e-12
    assert rec[7] == math.ceil(3 * math.sqrt(var))
    y00 = 0.5 / math.sqrt(math.pi)
    for c, k in enumerate((0.4, -0.2, 0.1)):
        assert abs(rec[8 + c] - max(0.0, float(np.float32(k)) * y00 + 0.5)) < 1e-12


def test_projected_covariance_matches_monte_carlo(orc):
    # The EWA covariance is the covariance of the projected point cloud to first order.
    rng = np.random.default_rng(4)
    views = [synth.scenes.pinhole((1.0, 0.5, -3.0), 80, 60)]
    v = views[0]
    for trial in range(5):
        mu = rng.uniform(-0.5, 0.5, 3)
        ls = rng.normal(-6.0, 0.3, 3)
        q = rng.standard_normal(4)
        sc = _one_gaussian_scene(mu, ls, q / np.linalg.norm(q), 0.0, (0, 0, 0), 80, 60, eye=(1.0, 0.5, -3.0))
        soa, _, _ = orc.gather(sc)
        rec = orc.project(soa, 1, 0, orc.views_array(views))[0, 0]
        Q = np.array([[rec[2], rec[3]], [rec[3], rec[4]]])
        S2 = np.linalg.inv(Q) - 0.3 * np.eye(2)
        # sample the 3D Gaussian with an independent rotation route (Hamilton product)
        qq = soa[6:10, 0] / np.linalg.norm(soa[6:10, 0])
        s = np.exp(soa[3:6, 0])
        n = 400000
        loc = rng.standard_normal((n, 3)) * s
        pts = np.empty_like(loc)
        qc = qq * np.array([1, -1, -1, -1])
        # rotate each sample: vectorised sandwich product
        w, x, y, z = qq
        Rm = np.array([[_hamilton(_hamilton(qq, np.r_[0.0, e]), qc)[1:] for e in np.eye(3)]]).reshape(3, 3).T
        pts = soa[0:3, 0] + loc @ Rm.T
        Xc = pts @ v.R.T + v.t
        uv = np.stack([v.fx * Xc[:, 0] / Xc[:, 2] + v.cx, v.fy * Xc[:, 1] / Xc[:, 2] + v.cy], 1)
        emp = np.cov(uv.T)
        assert np.allclose(S2, emp, rtol=0.02, atol=0.02 * np.abs(emp).max()), (trial, S2, emp)
        Xm = v.R @ soa[0:3, 0] + v.t
        assert abs(rec[0] - (v.fx * Xm[0] / Xm[2] + v.cx)) < 1e-9


def test_culling_behind_camera_and_near_plane(orc):
    sc = _one_gaussian_scene((0, 0, -3.2), (-3.0,) * 3, (1, 0, 0, 0), 0.0, (0, 0, 0))
    soa, _, _ = orc.gather(sc)
    rec = orc.project(soa, 1, 0, orc.views_array(sc.views))[0, 0]
    assert rec[7] == 0.0     # z = -0.2 <= znear: culled, radius 0
    sc = _one_gaussian_scene((0, 0, -3.0 + 0.005), (-3.0,) * 3, (1, 0, 0, 0), 0.0, (0, 0, 0))
    soa, _, _ = orc.gather(sc)
    rec = orc.project(soa, 1, 0, orc.views_array(sc.views))[0, 0]
    assert rec[7] == 0.0     # z = 0.005 <= 0.01


# ---------------------------------------------------------------------------
# Compositing (Supp. "Viewer")
# ---------------------------------------------------------------------------

def test_single_gaussian_image_and_footprint(orc):
    logit = 1.2
    sc = _one_gaussian_scene((0, 0, 0), (-2.5,) * 3, (1, 0, 0, 0), logit, (0.9, 0.3, -0.4), W=64, H=48)
    f = orc.forward(sc)
    v = sc.views[0]
    s = math.exp(float(np.float32(-2.5)))
    var = (v.fx * s / 3.0) ** 2 + 0.3
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    y00 = 0.5 / math.sqrt(math.pi)
    rgb = [max(0.0, float(np.float32(k)) * y00 + 0.5) for k in (0.9, 0.3, -0.4)]
    img = f["img"].reshape(3, v.height, v.width)
    count = 0
    for y in range(v.height):
        for x in range(v.width):
            r2 = (x + 0.5 - v.cx) ** 2 + (y + 0.5 - v.cy) ** 2
            q = r2 / var
            a = min(0.99, o * math.exp(-0.5 * q))
            inside = q <= 9 and a >= 1 / 255
            count += inside
            for c in range(3):
                exp = a * rgb[c] if inside else 0.0
                assert abs(img[c, y, x] - exp) < 1e-12
            assert abs(f["T"][y * v.width + x] - ((1 - a) if inside else 1.0)) < 1e-12
    # footprint in closed form: pixels with q <= min(9, 2 ln(255 o))
    rad2 = var * min(9.0, 2 * math.log(255 * o))
    closed = sum(1 for y in range(v.height) for x in range(v.width)
                 if (x + 0.5 - v.cx) ** 2 + (y + 0.5 - v.cy) ** 2 <= rad2)
    assert count == closed == int(np.count_nonzero(f["last"]))


def test_two_gaussians_hand_case(orc):
    # two isotropic splats on the optical axis: C = a1 c1 + (1 - a1) a2 c2 at the centre pixels
    v = synth.scenes.pinhole((0, 0, -3.0), 32, 32)
    D = synth.channel_count(0)
    atlas = np.zeros((1, D, 1, 2), np.float32)
    for i, (z, logit, k) in enumerate([(0.5, 0.4, (0.8, 0.1, 0.2)), (-0.5, -0.3, (0.1, 0.7, 0.3))]):
        atlas[0, 0:3, 0, i] = (0, 0, z)
        atlas[0, 3:6, 0, i] = -2.0
        atlas[0, 6, 0, i] = 1
        atlas[0, 10, 0, i] = logit
        atlas[0, 11:14, 0, i] = k
    sc = synth.Scene("two", atlas, synth.pack_bits(np.ones((1, 2), bool)), None, [(2, 1, 0, 0, 0)], 0, [v], 2)
    f = orc.forward(sc)
    rec = f["rec"][0]
    near, far = (1, 0) if rec[1, 6] < rec[0, 6] else (0, 1)
    x, y = 15, 15
    img = f["img"].reshape(3, 32, 32)

    def alpha(r):
        d = np.array([x + 0.5 - r[0], y + 0.5 - r[1]])
        q = r[2] * d[0] ** 2 + 2 * r[3] * d[0] * d[1] + r[4] * d[1] ** 2
        return min(0.99, r[5] * math.exp(-0.5 * q))

    a1, a2 = alpha(rec[near]), alpha(rec[far])
    for c in range(3):
        exp = a1 * rec[near, 8 + c] + (1 - a1) * a2 * rec[far, 8 + c]
        assert abs(img[c, y, x] - exp) < 1e-12


def test_tiled_render_equals_bruteforce_and_tile_size(orc):
    views = [synth.scenes.pinhole((0.3, 0.2, -3.0), 40, 36), synth.scenes.pinhole((-2.5, 0.4, -1.5), 24, 40)]
    sc = tiny_scene(views=views)
    f16 = orc.forward(sc, tile=16)
    # brute force over every splat of the view, per pixel
    pix = [(v, x, y) for v, vw in enumerate(views) for y in range(vw.height) for x in range(vw.width)]
    rgb, T, _, _ = orc.render_pixels(f16["rec"], f16["views"], 16, np.array(pix))
    P0 = views[0].width * views[0].height
    img = f16["img"]
    got = np.concatenate([img[:3 * P0].reshape(3, -1).T, img[3 * P0:].reshape(3, -1).T])
    assert np.array_equal(got, rgb)
    assert np.array_equal(f16["T"], T)
    for t in (8, 32, 1):
        for mode in (orc.BIN_ELLIPSE, orc.BIN_RECT):
            ft = orc.forward(sc, tile=t, mode=mode)
            assert np.array_equal(ft["img"], f16["img"]), (t, mode)
            assert np.array_equal(ft["T"], f16["T"]), (t, mode)
    assert (f16["T"] >= 1e-4).all() and (f16["T"] <= 1).all()
    assert f16["img"].min() >= 0


def test_permutation_invariance(orc):
    sc = tiny_scene(seed=11, n_side=5)
    f = orc.forward(sc)
    rng = np.random.default_rng(0)
    perm = rng.permutation(25)
    sc2 = tiny_scene(seed=11, n_side=5)
    a = sc2.atlas.reshape(1, sc2.channels, 25)
    sc2.atlas = np.ascontiguousarray(a[:, :, perm].reshape(sc.atlas.shape))
    f2 = orc.forward(sc2)
    assert np.allclose(f2["img"], f["img"], atol=1e-13, rtol=0)
    assert np.allclose(f2["T"], f["T"], atol=1e-13, rtol=0)


def test_background_adds_transmittance(orc):
    sc = tiny_scene(seed=5)
    f0 = orc.forward(sc)
    f1 = orc.forward(sc, bg=(1.0, 0.5, 0.25))
    P = len(f0["T"])
    d = (f1["img"] - f0["img"]).reshape(3, P)
    for c, b in enumerate((1.0, 0.5, 0.25)):
        assert np.allclose(d[c], b * f0["T"], atol=1e-14)


def test_early_stop_keeps_transmittance_above_cutoff(orc):
    # many opaque splats stacked on the axis: T must stop at >= 1e-4 and exclude the crossing splat
    v = synth.scenes.pinhole((0, 0, -3.0), 16, 16)
    n = 12
    D = synth.channel_count(0)
    atlas = np.zeros((1, D, 1, n), np.float32)
    for i in range(n):
        atlas[0, 0:3, 0, i] = (0, 0, -0.5 + 0.1 * i)
        atlas[0, 3:6, 0, i] = -1.0
        atlas[0, 6, 0, i] = 1
        atlas[0, 10, 0, i] = 1.5          # o = 0.82 -> 4 layers give T ~ 1e-3, 6 give < 1e-4
        atlas[0, 11:14, 0, i] = 0.5
    sc = synth.Scene("stack", atlas, synth.pack_bits(np.ones((1, n), bool)), None, [(n, 1, 0, 0, 0)], 0, [v], n)
    f = orc.forward(sc)
    c = 8 * 16 + 8
    T = f["T"][c]
    o = 1 / (1 + math.exp(-1.5))
    rec = f["rec"][0]
    d = np.array([8.5 - rec[0, 0], 8.5 - rec[0, 1]])
    # all splats have the same 2D footprint up to depth; compute the blended count by hand
    Tk, k = 1.0, 0
    for i in np.argsort(rec[:, 6]):
        r = rec[i]
        d = np.array([8.5 - r[0], 8.5 - r[1]])
        q = r[2] * d[0] ** 2 + 2 * r[3] * d[0] * d[1] + r[4] * d[1] ** 2
        a = min(0.99, r[5] * math.exp(-0.5 * q))
        if Tk * (1 - a) < 1e-4:
            break
        Tk *= 1 - a
        k += 1
    assert 0 < k < n and abs(T - Tk) < 1e-15 and T >= 1e-4
    assert f["last"][c] == k


# ---------------------------------------------------------------------------
# Binning and sort
# ---------------------------------------------------------------------------

def test_bin_sort_bruteforce_membership_and_order(orc):
    rng = np.random.default_rng(9)
    views = [synth.scenes.pinhole((0, 0, -3), 70, 45), synth.scenes.pinhole((0, 0, -3), 33, 50)]
    va = orc.views_array(views)
    V, N, T = 2, 300, 16
    mx = rng.uniform(-20, 90, V * N).astype(np.float32)
    my = rng.uniform(-20, 70, V * N).astype(np.float32)
    rad = rng.integers(0, 12, V * N).astype(np.float32)
    z = rng.uniform(0.5, 5, V * N).astype(np.float32)
    z[::17] = z[3]                     # exact depth ties across splats
    vals, ranges = orc.bin_sort32(mx, my, rad, z, va, N, T, mode=orc.BIN_RECT)
    ntiles, toff = orc.tiles_total(va, T)
    for v, vw in enumerate(views):
        tx_n, ty_n = -(-vw.width // T), -(-vw.height // T)
        for ty in range(ty_n):
            for tx in range(tx_n):
                t = toff[v] + ty * tx_n + tx
                got = vals[ranges[t, 0]:ranges[t, 1]].tolist()
                expect = []
                for g in range(N):
                    p = v * N + g
                    if rad[p] <= 0:
                        continue
                    cols = [i for i in range(tx * T, min(vw.width, tx * T + T))
                            if mx[p] - rad[p] <= i + 0.5 <= mx[p] + rad[p]]
                    rows = [j for j in range(ty * T, min(vw.height, ty * T + T))
                            if my[p] - rad[p] <= j + 0.5 <= my[p] + rad[p]]
                    if cols and rows:
                        expect.append(p)
                expect.sort(key=lambda p: (int(z[p].view(np.uint32)), p))
                assert got == expect, (v, tx, ty)
    assert ranges[:, 1].max() == len(vals)


def test_bin_sort_ellipse_rule_against_bounded_minimisation(orc):
    """Ellipse binning: a tile receives a splat iff min over the tile's pixel-centre rectangle of
    q = d^T conic d is <= 9 (1 + 2^-12).  The minimum is recomputed here with scipy's bounded
    L-BFGS-B; decisions must agree except inside a 1e-4 band around the cut."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(10)
    views = [synth.scenes.pinhole((0, 0, -3), 70, 45)]
    va = orc.views_array(views)
    N, T = 120, 16
    mx = rng.uniform(-10, 80, N).astype(np.float32)
    my = rng.uniform(-10, 55, N).astype(np.float32)
    L = rng.normal(0, 1, (N, 2, 2)) * np.exp(rng.normal(1.0, 0.7, (N, 1, 1)))
    S = L @ L.transpose(0, 2, 1) + 0.3 * np.eye(2)
    Q = np.linalg.inv(S).astype(np.float32)
    ca, cb, cc = Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 1]
    lam = np.linalg.eigvalsh(S)[:, 1]
    rad = np.ceil(3 * np.sqrt(lam)).astype(np.float32)
    z = rng.uniform(0.5, 5, N).astype(np.float32)
    vals, ranges = orc.bin_sort32(mx, my, rad, z, va, N, T, ca, cb, cc, mode=orc.BIN_ELLIPSE)
    rvals, rranges = orc.bin_sort32(mx, my, rad, z, va, N, T, mode=orc.BIN_RECT)
    assert len(vals) < len(rvals)
    W, H = views[0].width, views[0].height
    qcut = 9.0 * (1 + 2.0 ** -12)
    checked = 0
    for t in range(len(ranges)):
        ty, tx = divmod(t, -(-W // T))
        x0, x1 = tx * T + 0.5, min(W, tx * T + T) - 0.5
        y0, y1 = ty * T + 0.5, min(H, ty * T + T) - 0.5
        got = set(vals[ranges[t, 0]:ranges[t, 1]].tolist())
        cand = set(rvals[rranges[t, 0]:rranges[t, 1]].tolist())
        assert got <= cand
        for p in cand:
            A = np.array([[ca[p], cb[p]], [cb[p], cc[p]]], np.float64)
            m = np.array([mx[p], my[p]], np.float64)
            f = lambda x: float((x - m) @ A @ (x - m))
            x_init = np.clip(m, [x0, y0], [x1, y1])
            res = minimize(f, x_init, jac=lambda x: 2 * A @ (x - m), method="L-BFGS-B",
                           bounds=[(x0, x1), (y0, y1)], options=dict(ftol=1e-15, gtol=1e-12))
            qmin = min(res.fun, f(x_init))
            if abs(qmin - qcut) < 1e-4 * qcut:
                continue
            assert (p in got) == (qmin <= qcut), (t, p, qmin)
            checked += 1
    assert checked > 200


# ---------------------------------------------------------------------------
# Backward: central differences of the oracle's own forward
# ---------------------------------------------------------------------------

def _loss_and_hash(orc, sc, soa, N, w, tile=16):
    va = orc.views_array(sc.views)
    rec = orc.project(soa, N, sc.sh_degree, va)
    vals, ranges = orc.bin_sort(rec, va, tile)
    r = orc.render(rec, va, tile, vals, ranges)
    return float(w @ r["img"]), r["hash"]


@pytest.mark.parametrize("case", ["sh3_2views", "sh1_2frames_dyn", "sh2_fp16"])
def test_backward_matches_central_differences(orc, case):
    if case == "sh3_2views":
        views = [synth.scenes.pinhole((0.3, 0.2, -3.0), 40, 36), synth.scenes.pinhole((-2.5, 0.4, -1.5), 24, 40)]
        sc = tiny_scene(seed=21, views=views)
    elif case == "sh1_2frames_dyn":
        views = [synth.scenes.pinhole((0.3, 0.2, -3.0), 40, 36, frame=0),
                 synth.scenes.pinhole((2.5, -0.4, -1.5), 36, 30, frame=1)]
        sc = tiny_scene(seed=22, views=views, sh_degree=1, frames=2, dyn=0.5)
    else:
        sc = tiny_scene(seed=23, sh_degree=2, dtype=np.float16)
    f = orc.forward(sc)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(f["img"].shape)
    g = orc.backward(sc, f, w)["grad_soa"]
    soa, N = f["soa"], f["N"]
    if sc.dyn is not None:
        frozen = np.tile(f["dynflag"] == 0, sc.frames)
        assert np.count_nonzero(frozen) > 0 and np.all(g[:, frozen] == 0)
    checked = 0
    for _ in range(64):
        d = rng.standard_normal(soa.shape)
        if sc.dyn is not None:
            d[:, np.tile(f["dynflag"] == 0, sc.frames)] = 0
        h = 1e-6
        lp, hp = _loss_and_hash(orc, sc, soa + h * d, N, w)
        lm, hm = _loss_and_hash(orc, sc, soa - h * d, N, w)
        if hp != hm:
            continue
        fd = (lp - lm) / (2 * h)
        an = float(np.sum(g * d))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
        checked += 1
    assert checked >= 48
    # sampled scalar parameters of every attribute group
    D, G = soa.shape
    idx = [(c, gi) for c in range(D) for gi in rng.choice(G, 3, replace=False)]
    for c, gi in idx:
        if sc.dyn is not None and f["dynflag"][gi % N] == 0:
            continue
        h = 1e-6 * max(1.0, abs(soa[c, gi]))
        sp, sm = soa.copy(), soa.copy()
        sp[c, gi] += h
        sm[c, gi] -= h
        lp, hp = _loss_and_hash(orc, sc, sp, N, w)
        lm, hm = _loss_and_hash(orc, sc, sm, N, w)
        if hp != hm:
            continue
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[c, gi]) <= 1e-6 * max(1.0, abs(g[c, gi])), (c, gi, fd, g[c, gi])


def test_render_bwd_matches_differences_in_record_space(orc):
    sc = tiny_scene(seed=31)
    f = orc.forward(sc)
    rng = np.random.default_rng(6)
    w = rng.standard_normal(f["img"].shape)
    va, rec, vals, ranges = f["views"], f["rec"], f["vals"], f["ranges"]
    g2 = orc.render_bwd(rec, va, 16, vals, ranges, w)
    fields = [0, 1, 2, 3, 4, 5, 8, 9, 10]      # m, conic, opacity, rgb
    n_ok = 0
    for _ in range(120):   # directions whose step flips a decision are skipped
        if n_ok >= 40:
            break
        d = np.zeros_like(rec)
        d[..., fields] = rng.standard_normal(rec[..., fields].shape)
        d[rec[..., 7] == 0] = 0
        h = 1e-7
        rp = orc.render(rec + h * d, va, 16, vals, ranges)
        rm = orc.render(rec - h * d, va, 16, vals, ranges)
        if rp["hash"] != rm["hash"]:
            continue
        fd = (w @ rp["img"] - w @ rm["img"]) / (2 * h)
        an = float(np.sum(g2 * d[..., fields]))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        n_ok += 1
    assert n_ok >= 30


def test_images_do_not_depend_on_tile_side(orc):
    """A larger tile only adds splats whose footprint misses the pixel (they
    fail the alpha test), so the oracle's images and transmittance for 16
    and 32 px tiles are identical, while the lists differ."""
    rng = np.random.default_rng(21)
    V, N = 2, 150
    va = np.zeros((V, 20))
    for v, (w, h) in enumerate([(70, 45), (33, 50)]):
        va[v, 16], va[v, 17] = w, h
    rec = np.zeros((V, N, 12))
    for v in range(V):
        w, h = va[v, 16], va[v, 17]
        rec[v, :, 0] = rng.uniform(-5, w + 5, N)
        rec[v, :, 1] = rng.uniform(-5, h + 5, N)
        L = rng.normal(0, 1, (N, 2, 2)) * np.exp(rng.normal(0.8, 0.7, (N, 1, 1)))
        S = L @ L.transpose(0, 2, 1) + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        rec[v, :, 2], rec[v, :, 3], rec[v, :, 4] = Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 1]
        rec[v, :, 5] = rng.uniform(0.05, 0.99, N)
        rec[v, :, 6] = rng.uniform(1, 5, N)
        rec[v, :, 7] = np.ceil(3 * np.sqrt(np.linalg.eigvalsh(S)[:, 1]))
        rec[v, :, 8:11] = rng.uniform(0, 1, (N, 3))
    out = {}
    for tile in (16, 32):
        vals, ranges = orc.bin_sort(rec, va, tile)
        out[tile] = (len(vals), orc.render(rec, va, tile, vals, ranges))
    assert out[16][0] != out[32][0]
    assert np.array_equal(out[16][1]["img"], out[32][1]["img"])
    assert np.array_equal(out[16][1]["T"], out[32][1]["T"])


def test_nonfinite_texels_render_as_absent(orc):
    """A Gaussian with a non-finite texel value (any channel) is culled in
    every view: the oracle's images equal, bit for bit, those of the atlas
    with those texels removed from the occupancy mask, and its gradient
    there is zero."""
    import dataclasses
    sc = synth.make_scene([(40, 40, 0, 0, 0)], (40, 40), 0.6,
                          [synth.scenes.pinhole((0.4, 0.3, -3.2), 80, 60),
                           synth.scenes.pinhole((-2.6, -0.5, -1.8), 60, 72)],
                          sh_degree=2, seed=8, log_scale=(-3.2, 0.5))
    F, D, Hh, W = sc.atlas.shape
    occ = synth.scenes.unpack_bits(sc.occ, W)
    ys, xs = np.nonzero(occ)
    pick = np.random.default_rng(2).choice(len(ys), 5, replace=False)
    bad = sc.atlas.copy()
    for i, (c, v) in zip(pick, [(0, np.nan), (5, np.inf), (9, np.nan), (10, -np.inf), (D - 1, np.nan)]):
        bad[0, c, ys[i], xs[i]] = v
    with_bad = dataclasses.replace(sc, atlas=bad)
    occ2 = occ.copy()
    occ2[ys[pick], xs[pick]] = False
    without = dataclasses.replace(sc, occ=synth.pack_bits(occ2), n_live=sc.n_live - len(pick))
    a, b = orc.forward(with_bad), orc.forward(without)
    assert np.array_equal(a["img"], b["img"]) and np.array_equal(a["T"], b["T"])
    assert np.all(a["rec"][:, pick, 7] == 0)
    dimg = np.random.default_rng(3).standard_normal(len(a["img"]))
    g = orc.backward(with_bad, a, dimg)["grad_soa"]
    assert np.all(g[:, pick] == 0) and np.all(np.isfinite(g))
