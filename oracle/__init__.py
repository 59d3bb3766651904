"""FP64 CPU oracle of the PackUV-GS render step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``packuv_oracle.c`` (plain C,
double precision, single-threaded) through ctypes; it shares no code with the
CUDA library.  See the C file's header for the passage of the paper each
function follows.

Inputs are scene-like objects with the attributes ``atlas`` ([F][D][H][W]
float32/float16), ``occ`` / ``dyn`` (bit-packed rows), ``sh_degree``,
``views`` (objects with R, t, fx, fy, cx, cy, width, height, frame) and
``n_live``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "packuv_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_packuv.so")
_lock = threading.Lock()
_lib = None

VS = 20     # doubles per view
REC = 12    # doubles per projected record
G2D = 9     # doubles per per-view 2D gradient
ZNEAR = 0.01


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


P = C.c_void_p
I32, I64, U64, DBL = C.c_int32, C.c_int64, C.c_uint64, C.c_double


def _declare(L):
    sig = {
        "or_pyramid_sizes": (C.c_int, [C.c_int, C.c_int, C.c_int, P, P]),
        "or_atlas_layout": (C.c_int, [C.c_int, C.c_int, P, P]),
        "or_texel_to_uv": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P]),
        "or_uv_to_texel": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_int, P]),
        "or_half_to_double": (DBL, [C.c_uint16]),
        "or_count_live": (I64, [P, C.c_int, C.c_int]),
        "or_gather": (I64, [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, I64, P, P, P]),
        "or_quat_rot": (None, [P, P]),
        "or_sh_basis": (None, [C.c_int, P, P, P]),
        "or_project": (None, [P, I64, I64, C.c_int, C.c_int, P, C.c_int, DBL, P]),
        "or_tiles_total": (I64, [C.c_int, P, P, C.c_int, P]),
        "or_bin_sort": (I64, [P, P, P, P, P, P, P, C.c_int, C.c_int, I64, P, P, C.c_int, P, I64, P]),
        "or_render": (U64, [P, C.c_int, I64, P, C.c_int, P, P, P, DBL, DBL, P, P, P, P, P]),
        "or_render_bwd": (None, [P, C.c_int, I64, P, C.c_int, P, P, P, P, P]),
        "or_scatter_grad": (None, [P, I64, I64, C.c_int, C.c_int, P, C.c_int, DBL, P, P, P]),
        "or_mean_error_bounds": (None, [P, C.c_int, I64, P, P, P]),
        "or_render_pixels": (None, [P, C.c_int, I64, P, C.c_int, P, DBL, DBL, I64, P, P, P, P, P]),
        "or_motion_mask": (None, [P, C.c_int, C.c_int, C.c_float, C.c_int, P]),
        "or_dynamic_mask32": (None, [P, C.c_int, I64, P, P, P, C.c_float, P]),
        "or_dynamic_mask": (None, [P, C.c_int, I64, P, P, P, DBL, DBL, P, P]),
        "or_lpo_minmax": (None, [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P]),
        "or_lpo_encode": (None, [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]),
        "or_lpo_decode": (None, [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P]),
        "or_uv_cell": (C.c_uint32, [DBL, DBL, DBL, C.c_int, C.c_int, P]),
        "or_uv_max_k": (None, [P, I64, I64, C.c_int, C.c_int, C.c_int, P, P, P, P, P]),
        "or_photo_loss": (DBL, [P, P, C.c_int, P, P, DBL, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# Layout
# --------------------------------------------------------------------------

def pyramid_sizes(M0, N0, K):
    M = np.zeros(K, np.int32)
    N = np.zeros(K, np.int32)
    if lib().or_pyramid_sizes(M0, N0, K, _p(M), _p(N)):
        raise ValueError("invalid pyramid")
    return M, N


def atlas_layout(S, K):
    lv = np.zeros((K, 5), np.int32)
    wh = np.zeros(2, np.int32)
    if lib().or_atlas_layout(S, K, _p(lv), _p(wh)):
        raise ValueError("invalid layout")
    return [tuple(int(a) for a in r) for r in lv], (int(wh[0]), int(wh[1]))


def texel_to_uv(levels, x, y):
    lv = np.ascontiguousarray(np.asarray(levels, np.int32))
    out = np.zeros(3, np.int32)
    if lib().or_texel_to_uv(_p(lv), len(levels), x, y, _p(out)):
        return None
    return tuple(int(a) for a in out)


def uv_to_texel(levels, k, u, v):
    lv = np.ascontiguousarray(np.asarray(levels, np.int32))
    out = np.zeros(2, np.int32)
    if lib().or_uv_to_texel(_p(lv), len(levels), k, u, v, _p(out)):
        return None
    return int(out[0]), int(out[1])


def half_to_double(h: int) -> float:
    return lib().or_half_to_double(int(h))


# --------------------------------------------------------------------------
# Steps
# --------------------------------------------------------------------------

def views_array(views) -> np.ndarray:
    """Camera table; R, t, fx, fy, cx, cy rounded to FP32 first, the values
    the library's pk_view carries, so both sides render the same cameras."""
    a = np.zeros((len(views), VS), np.float64)
    f32 = lambda x: np.asarray(x, np.float64).astype(np.float32).astype(np.float64)
    for i, v in enumerate(views):
        a[i, 0:9] = f32(v.R).reshape(9)
        a[i, 9:12] = f32(v.t)
        a[i, 12:16] = f32([v.fx, v.fy, v.cx, v.cy])
        a[i, 16:19] = (v.width, v.height, v.frame)
    return a


def count_live(occ, H, W) -> int:
    occ = np.ascontiguousarray(occ, np.uint32)
    return int(lib().or_count_live(_p(occ), H, W))


def gather(scene):
    atlas = np.ascontiguousarray(scene.atlas)
    F, D, H, W = atlas.shape
    dtype = 1 if atlas.dtype == np.float16 else 0
    if dtype == 0:
        atlas = np.ascontiguousarray(atlas, np.float32)
    occ = np.ascontiguousarray(scene.occ, np.uint32)
    dyn = None if scene.dyn is None else np.ascontiguousarray(scene.dyn, np.uint32)
    N = count_live(occ, H, W)
    soa = np.zeros((D, F * N), np.float64)
    texel = np.zeros(N, np.uint32)
    dynflag = np.zeros(N, np.uint8)
    r = lib().or_gather(_p(atlas), dtype, F, D, H, W, _p(occ), _p(dyn), N, _p(soa), _p(texel), _p(dynflag))
    assert r == N
    return soa, texel, dynflag


def quat_rot(q):
    q = np.ascontiguousarray(q, np.float64)
    R = np.zeros(9, np.float64)
    lib().or_quat_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def sh_basis(deg, d):
    d = np.ascontiguousarray(d, np.float64)
    Y = np.zeros(16, np.float64)
    dY = np.zeros(48, np.float64)
    lib().or_sh_basis(deg, _p(d), _p(Y), _p(dY))
    nb = (deg + 1) ** 2
    return Y[:nb], dY.reshape(16, 3)[:nb]


def project(soa, N, sh_degree, views_arr, znear=ZNEAR):
    soa = np.ascontiguousarray(soa, np.float64)
    D, G = soa.shape
    V = views_arr.shape[0]
    rec = np.zeros((V, N, REC), np.float64)
    lib().or_project(_p(soa), G, N, D, sh_degree, _p(np.ascontiguousarray(views_arr)), V, znear, _p(rec))
    return rec


def tiles_total(views_arr, tile):
    vw = np.ascontiguousarray(views_arr[:, 16], np.int32)
    vh = np.ascontiguousarray(views_arr[:, 17], np.int32)
    toff = np.zeros(len(vw) + 1, np.int64)
    t = lib().or_tiles_total(len(vw), _p(vw), _p(vh), tile, _p(toff))
    return int(t), toff[:-1]


BIN_RECT, BIN_ELLIPSE = 0, 1


def bin_sort32(mx, my, rad, z, views_arr, N, tile, ca=None, cb=None, cc=None, mode=BIN_ELLIPSE):
    """Integer stage on FP32 inputs (each a flat [V*N] float32 array)."""
    mx, my, rad, z = (np.ascontiguousarray(a, np.float32).reshape(-1) for a in (mx, my, rad, z))
    if mode == BIN_ELLIPSE:
        ca, cb, cc = (np.ascontiguousarray(a, np.float32).reshape(-1) for a in (ca, cb, cc))
    else:
        ca = cb = cc = None
    V = views_arr.shape[0]
    vw = np.ascontiguousarray(views_arr[:, 16], np.int32)
    vh = np.ascontiguousarray(views_arr[:, 17], np.int32)
    ntiles, _ = tiles_total(views_arr, tile)
    ranges = np.zeros((ntiles, 2), np.uint32)
    args = (_p(mx), _p(my), _p(rad), _p(z), _p(ca), _p(cb), _p(cc), mode, V, N, _p(vw), _p(vh), tile)
    n = lib().or_bin_sort(*args, None, 0, _p(ranges))
    vals = np.zeros(max(n, 1), np.uint32)
    n2 = lib().or_bin_sort(*args, _p(vals), n, _p(ranges))
    assert n2 == n
    return vals[:n].copy(), ranges


def bin_sort(rec, views_arr, tile, mode=BIN_ELLIPSE):
    V, N, _ = rec.shape
    r = rec.reshape(V * N, REC)
    return bin_sort32(r[:, 0], r[:, 1], r[:, 7], r[:, 6], views_arr, N, tile, r[:, 2], r[:, 3], r[:, 4], mode)


# Borderline rule (see composite_pixel in packuv_oracle.c).  M_DERIVE: the
# mean's FP32 error bound is derived per record (records of the oracle's own
# FP64 projection, compared with a GPU that projected in FP32); a value >= 0
# is a fixed mean tolerance in pixels, 0 for identical FP32 records.
# Q_REL: relative rounding of the quadratic form (FP32, a few roundings per
# term; 2^-19 = 32 unit roundoffs), against |a| dx^2 + 2 |b dx dy| + |c| dy^2.
M_DERIVE = -1.0
Q_REL = 2.0 ** -19
B_Q, B_ALPHA, B_STOP, B_DEPTH, B_CULL, B_CLAMP = 1, 2, 4, 8, 16, 32
IMAGE_BORDER = B_Q | B_ALPHA | B_STOP | B_DEPTH | B_CULL   # B_CLAMP matters to gradients only


def render(rec, views_arr, tile, vals, ranges, bg=(0.0, 0.0, 0.0), m_tol=M_DERIVE, q_rel=Q_REL):
    """-> dict(img, T, last, border, bound [P][2] (colour, T flip bounds), hash)."""
    V, N, _ = rec.shape
    P = int(np.sum(views_arr[:, 16] * views_arr[:, 17]))
    img = np.zeros(3 * P, np.float64)
    T = np.zeros(P, np.float64)
    last = np.zeros(P, np.uint32)
    border = np.zeros(P, np.uint8)
    bound = np.zeros((P, 2), np.float64)
    bg = np.ascontiguousarray(bg, np.float64)
    h = lib().or_render(_p(np.ascontiguousarray(rec)), V, N, _p(np.ascontiguousarray(views_arr)), tile,
                        _p(np.ascontiguousarray(vals, np.uint32)), _p(np.ascontiguousarray(ranges, np.uint32)),
                        _p(bg), float(m_tol), float(q_rel), _p(img), _p(T), _p(last), _p(border), _p(bound))
    return dict(img=img, T=T, last=last, border=border, bound=bound, hash=int(h))


def render_bwd(rec, views_arr, tile, vals, ranges, dimg, bg=(0.0, 0.0, 0.0)):
    V, N, _ = rec.shape
    g2 = np.zeros((V, N, G2D), np.float64)
    bg = np.ascontiguousarray(bg, np.float64)
    lib().or_render_bwd(_p(np.ascontiguousarray(rec)), V, N, _p(np.ascontiguousarray(views_arr)), tile,
                        _p(np.ascontiguousarray(vals, np.uint32)), _p(np.ascontiguousarray(ranges, np.uint32)),
                        _p(bg), _p(np.ascontiguousarray(dimg, np.float64)), _p(g2))
    return g2


def scatter_grad(soa, N, sh_degree, views_arr, grad2d, dynflag=None, znear=ZNEAR):
    soa = np.ascontiguousarray(soa, np.float64)
    D, G = soa.shape
    V = views_arr.shape[0]
    out = np.zeros((D, G), np.float64)
    df = None if dynflag is None else np.ascontiguousarray(dynflag, np.uint8)
    lib().or_scatter_grad(_p(soa), G, N, D, sh_degree, _p(np.ascontiguousarray(views_arr)), V, znear,
                          _p(np.ascontiguousarray(grad2d, np.float64)), _p(df), _p(out))
    return out


def mean_error_bounds(rec, views_arr):
    """Per record: bound on the FP32 error of the projected mean (px) and depth."""
    V, N, _ = rec.shape
    mt = np.zeros(V * N, np.float64)
    zt = np.zeros(V * N, np.float64)
    lib().or_mean_error_bounds(_p(np.ascontiguousarray(rec)), V, N, _p(np.ascontiguousarray(views_arr)), _p(mt),
                               _p(zt))
    return mt.reshape(V, N), zt.reshape(V, N)


def render_pixels(rec, views_arr, tile, pix, bg=(0.0, 0.0, 0.0), m_tol=M_DERIVE, q_rel=Q_REL):
    """pix [n][3] = (view, x, y) -> (rgb [n][3], T [n], border [n], bound [n][2])."""
    V, N, _ = rec.shape
    pix = np.ascontiguousarray(pix, np.int32).reshape(-1, 3)
    n = pix.shape[0]
    rgb = np.zeros((n, 3), np.float64)
    T = np.zeros(n, np.float64)
    border = np.zeros(n, np.uint8)
    bound = np.zeros((n, 2), np.float64)
    lib().or_render_pixels(_p(np.ascontiguousarray(rec)), V, N, _p(np.ascontiguousarray(views_arr)), tile,
                           _p(np.ascontiguousarray(bg, np.float64)), float(m_tol), float(q_rel), n, _p(pix),
                           _p(rgb), _p(T), _p(border), _p(bound))
    return rgb, T, border, bound


# --------------------------------------------------------------------------
# Motion masks and the dynamic mask
# --------------------------------------------------------------------------

def motion_mask(flow, tau, r):
    """One view: flow [2][H][W] float32 -> mask [H][W] uint8 (0/1)."""
    flow = np.ascontiguousarray(flow, np.float32)
    _, H, W = flow.shape
    M = np.zeros((H, W), np.uint8)
    lib().or_motion_mask(_p(flow), W, H, float(tau), int(r), _p(M))
    return M


def motion_masks(flow_flat, views_arr, tau, r):
    """All views: flow concatenated as [V][2][H_v][W_v] -> masks concatenated [P] uint8."""
    out, off = [], 0
    for v in range(views_arr.shape[0]):
        W, H = int(views_arr[v, 16]), int(views_arr[v, 17])
        out.append(motion_mask(np.asarray(flow_flat[off:off + 2 * W * H]).reshape(2, H, W), tau, r).reshape(-1))
        off += 2 * W * H
    return np.concatenate(out)


def dynamic_mask32(rec32, views_arr, masks, r_max=0.0):
    """FP32 stage on float32 records [V*N][12] -> D [N] uint8."""
    V = views_arr.shape[0]
    rec32 = np.ascontiguousarray(rec32, np.float32).reshape(-1, REC)
    N = rec32.shape[0] // V
    vw = np.ascontiguousarray(views_arr[:, 16], np.int32)
    vh = np.ascontiguousarray(views_arr[:, 17], np.int32)
    D = np.zeros(N, np.uint8)
    lib().or_dynamic_mask32(_p(rec32), V, N, _p(vw), _p(vh), _p(np.ascontiguousarray(masks, np.uint8)),
                            float(r_max), _p(D))
    return D


def dynamic_mask(rec, views_arr, masks, r_max=0.0, m_tol=5e-4):
    """FP64 on the oracle's records [V][N][12] -> (D [N], border [N]) uint8."""
    V, N, _ = rec.shape
    vw = np.ascontiguousarray(views_arr[:, 16], np.int32)
    vh = np.ascontiguousarray(views_arr[:, 17], np.int32)
    D = np.zeros(N, np.uint8)
    border = np.zeros(N, np.uint8)
    lib().or_dynamic_mask(_p(np.ascontiguousarray(rec)), V, N, _p(vw), _p(vh),
                          _p(np.ascontiguousarray(masks, np.uint8)), float(r_max), m_tol, _p(D), _p(border))
    return D, border


def dynamic_mask_scene(scene, masks, r_max=0.0, znear=ZNEAR, m_tol=5e-4):
    """Gather, project (FP64) and mask: D and border per live texel, in gather order."""
    soa, texel, _ = gather(scene)
    va = views_array(scene.views)
    rec = project(soa, len(texel), scene.sh_degree, va, znear)
    D, border = dynamic_mask(rec, va, masks, r_max, m_tol)
    return D, border, texel, rec


# --------------------------------------------------------------------------
# Low-precision proxy
# --------------------------------------------------------------------------

def lpo_minmax(atlas, occ):
    """atlas [F][D][H][W] float32 -> lohi [D][2] float32 over live texels."""
    atlas = np.ascontiguousarray(atlas, np.float32)
    F, D, H, W = atlas.shape
    lohi = np.zeros((D, 2), np.float32)
    lib().or_lpo_minmax(_p(atlas), F, D, H, W, _p(np.ascontiguousarray(occ, np.uint32)), _p(lohi))
    return lohi


def lpo_encode(atlas, occ, lohi):
    """-> codes [F][D+3][H][W] uint8."""
    atlas = np.ascontiguousarray(atlas, np.float32)
    F, D, H, W = atlas.shape
    codes = np.zeros((F, D + 3, H, W), np.uint8)
    lib().or_lpo_encode(_p(atlas), F, D, H, W, _p(np.ascontiguousarray(occ, np.uint32)),
                        _p(np.ascontiguousarray(lohi, np.float32)), _p(codes))
    return codes


def lpo_decode(codes, occ, lohi):
    """codes [F][D+3][H][W] -> proxy atlas [F][D][H][W] float32."""
    codes = np.ascontiguousarray(codes, np.uint8)
    F, NP, H, W = codes.shape
    D = NP - 3
    proxy = np.zeros((F, D, H, W), np.float32)
    lib().or_lpo_decode(_p(codes), F, D, H, W, _p(np.ascontiguousarray(occ, np.uint32)),
                        _p(np.ascontiguousarray(lohi, np.float32)), _p(proxy))
    return proxy


# --------------------------------------------------------------------------
# UV cells and Max-K pruning
# --------------------------------------------------------------------------

INVALID = 0xFFFFFFFF


def uv_cell(x, y, z, M, N):
    """-> (cell id or INVALID, border flag)."""
    b = C.c_int(0)
    c = lib().or_uv_cell(float(x), float(y), float(z), int(M), int(N), C.byref(b))
    return int(c), int(b.value)


def uv_max_k(soa, M, N, K):
    """soa [D][n] -> dict(cell, rank, keep, count [M*N], border) for the n columns."""
    soa = np.ascontiguousarray(soa, np.float64)
    D, n = soa.shape
    cell = np.zeros(n, np.uint32)
    rank = np.zeros(n, np.uint32)
    keep = np.zeros(n, np.uint8)
    border = np.zeros(n, np.uint8)
    count = np.zeros(M * N, np.uint32)
    lib().or_uv_max_k(_p(soa), n, n, M, N, K, _p(cell), _p(rank), _p(keep), _p(count), _p(border))
    return dict(cell=cell, rank=rank, keep=keep, count=count, border=border)


# --------------------------------------------------------------------------
# Photometric objective
# --------------------------------------------------------------------------

SSIM_LAMBDA = 0.2


def photo_loss(img, tgt, views_arr, lam=SSIM_LAMBDA, grad=True, ssim_map=False):
    """-> dict(loss, ssim, grad [3P] or None, map [3P] or None)."""
    img = np.ascontiguousarray(img, np.float64)
    tgt = np.ascontiguousarray(tgt, np.float64)
    V = views_arr.shape[0]
    vw = np.ascontiguousarray(views_arr[:, 16], np.int32)
    vh = np.ascontiguousarray(views_arr[:, 17], np.int32)
    g = np.zeros_like(img) if grad else None
    m = np.zeros_like(img) if ssim_map else None
    s = C.c_double(0.0)
    L = lib().or_photo_loss(_p(img), _p(tgt), V, _p(vw), _p(vh), float(lam), _p(g), _p(m), C.byref(s))
    return dict(loss=float(L), ssim=float(s.value), grad=g, map=m)


# --------------------------------------------------------------------------
# Whole step
# --------------------------------------------------------------------------

def forward(scene, tile=16, znear=ZNEAR, bg=(0.0, 0.0, 0.0), m_tol=M_DERIVE, mode=BIN_ELLIPSE):
    soa, texel, dynflag = gather(scene)
    va = views_array(scene.views)
    N = len(texel)
    rec = project(soa, N, scene.sh_degree, va, znear)
    vals, ranges = bin_sort(rec, va, tile, mode)
    out = render(rec, va, tile, vals, ranges, bg, m_tol)
    out.update(soa=soa, texel=texel, dynflag=dynflag, views=va, rec=rec, vals=vals, ranges=ranges, N=N)
    return out


def backward(scene, fwd, dimg, tile=16, znear=ZNEAR, bg=(0.0, 0.0, 0.0)):
    g2 = render_bwd(fwd["rec"], fwd["views"], tile, fwd["vals"], fwd["ranges"], dimg, bg)
    gsoa = scatter_grad(fwd["soa"], fwd["N"], scene.sh_degree, fwd["views"], g2, fwd["dynflag"]
                        if scene.dyn is not None else None, znear)
    return dict(grad2d=g2, grad_soa=gsoa)


def grad_to_atlas(scene, grad_soa, texel):
    """Place [D][F*N] gradients at their texels: [F][D][H][W] (zeros elsewhere)."""
    F, D, H, W = scene.atlas.shape
    N = len(texel)
    out = np.zeros((F, D, H * W), np.float64)
    for f in range(F):
        out[f][:, texel] = grad_soa[:, f * N:(f + 1) * N]
    return out.reshape(F, D, H, W)
