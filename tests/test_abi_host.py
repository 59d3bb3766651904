"""C-ABI checks that need no GPU: exported symbols and the host-side logic
(atlas layout, plan validation, sizes) of libpackuv.so."""

import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_23040_gb300 import build, _native
    try:
        build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))
    return _native.load()


def declared_symbols():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(pk_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"pk_atlas_gather", "pk_project_and_sh", "pk_bin_and_sort", "pk_rasterize_fwd",
            "pk_rasterize_bwd", "pk_atlas_scatter_grad"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_version_and_status_strings(lib):
    assert lib.pk_version() == 1
    assert lib.pk_status_string(0) == b"ok"
    assert lib.pk_status_string(3) == b"device capacity exceeded"


@pytest.mark.parametrize("S,K", [(64, 1), (64, 2), (64, 3), (1024, 8), (256, 6), (512, 5)])
def test_atlas_layout_matches_oracle(lib, orc, S, K):
    from paper_2602_23040_gb300 import api
    levels, wh = api.atlas_layout(S, K)
    olevels, owh = orc.atlas_layout(S, K)
    assert levels == olevels and wh == owh


def _plan_args(**over):
    import synth
    v = synth.scenes.pinhole((0, 0, -3), 64, 48)
    a = dict(levels=[(32, 32, 0, 0, 0)], atlas_wh=(32, 32), sh_degree=3, frames=1, texel_type="f32",
             views=[v], n_live=500)
    a.update(over)
    return a


def test_plan_sizes_and_workspace(lib):
    from paper_2602_23040_gb300 import api
    p = api.Plan(**_plan_args())
    s = p.sizes
    assert (s.n_live, s.n_gauss, s.channels, s.n_views, s.n_pairs) == (500, 500, 59, 1, 500)
    assert s.n_pixels == 64 * 48 and s.n_tiles == 2 * 2           # 32 px tiles by default
    assert s.max_dups == max(1024, 32 * 500) and s.workspace_bytes > 0
    p.close()
    p16 = api.Plan(**_plan_args(tile=16))
    assert p16.sizes.n_tiles == 4 * 3
    p16.close()


@pytest.mark.parametrize("over,code", [
    (dict(levels=[(40, 32, 0, 0, 0)]), 2),                               # level outside the atlas
    (dict(levels=[(16, 16, 0, 0, 0), (16, 16, 8, 8, 0)]), 2),            # overlapping levels
    (dict(sh_degree=4), 2),
    (dict(n_live=32 * 32 + 1), 1),
    (dict(frames=0), 2),
    (dict(tile=8), 6),
    (dict(znear=0.0), 1),
])
def test_plan_validation(lib, over, code):
    from paper_2602_23040_gb300 import api, _native
    with pytest.raises(_native.PackUVError) as ei:
        api.Plan(**_plan_args(**over))
    assert ei.value.code == code


def test_plan_rejects_bad_view(lib):
    import synth
    from paper_2602_23040_gb300 import api, _native
    v = synth.scenes.pinhole((0, 0, -3), 64, 48)
    v.frame = 1                       # frame outside the single-frame atlas
    with pytest.raises(_native.PackUVError):
        api.Plan(**_plan_args(views=[v]))
    v = synth.scenes.pinhole((0, 0, -3), 0, 48)
    with pytest.raises(_native.PackUVError):
        api.Plan(**_plan_args(views=[v]))
