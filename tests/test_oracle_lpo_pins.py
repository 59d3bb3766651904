"""Pins of the oracle's low-precision proxy (Sec. 4.2 "Low Precision
Optimization", Supp. "Video Coding"): numpy's min/max over the live texels,
the closed form on an integer grid (Delta = 1), the error bound Delta / 2
of a uniform quantiser, the integer-exact round trip codes -> proxy ->
codes, the two-byte split of the 16-bit position codes, and the degenerate
cases."""

import numpy as np
import pytest

import synth


def _atlas(seed, F=2, D=14, H=20, W=37, frac=0.6):
    rng = np.random.default_rng(seed)
    occ = rng.random((H, W)) < frac
    a = rng.normal(0.0, 1.0, size=(F, D, H, W)).astype(np.float32) * rng.uniform(0.1, 5.0, size=(1, D, 1, 1)).astype(
        np.float32)
    return a, occ, synth.pack_bits(occ)


def test_minmax_is_numpy_over_live_texels_of_every_frame(orc):
    a, occ, bits = _atlas(1)
    a[1, 4, 3, 5] = np.nan          # ignored
    lohi = orc.lpo_minmax(a, bits)
    live = a[:, :, occ]             # [F][D][n]
    np.testing.assert_array_equal(lohi[:, 0], np.nanmin(live, axis=(0, 2)))
    np.testing.assert_array_equal(lohi[:, 1], np.nanmax(live, axis=(0, 2)))


def test_integer_grid_closed_form_and_byte_split(orc):
    """lo = 0, hi = 2^K - 1 gives Delta = 1: the code is x rounded half up,
    the proxy the integer itself; position codes are hi byte, lo byte."""
    F, D, H, W = 1, 14, 8, 16
    rng = np.random.default_rng(2)
    occ = np.ones((H, W), bool)
    bits = synth.pack_bits(occ)
    a = np.zeros((F, D, H, W), np.float32)
    for c in range(D):
        L = 65535 if c < 3 else 255
        k = rng.integers(0, L + 1, size=(H, W))
        off = rng.choice([-0.3, 0.0, 0.2, 0.49], size=(H, W))
        a[0, c] = np.clip(k + off, 0, L)
        a[0, c, 0, 0], a[0, c, 0, 1] = 0.0, float(L)      # pin the range
    lohi = orc.lpo_minmax(a, bits)
    codes = orc.lpo_encode(a, bits, lohi)
    proxy = orc.lpo_decode(codes, bits, lohi)
    for c in range(D):
        want = np.floor(a[0, c].astype(np.float64) + 0.5).astype(np.int64)
        if c < 3:
            q = codes[0, 2 * c].astype(np.int64) * 256 + codes[0, 2 * c + 1]
        else:
            q = codes[0, c + 3].astype(np.int64)
        np.testing.assert_array_equal(q, want)
        np.testing.assert_array_equal(proxy[0, c], want.astype(np.float32))


def test_error_within_half_a_step_and_endpoints(orc):
    a, occ, bits = _atlas(3)
    lohi = orc.lpo_minmax(a, bits)
    proxy = orc.lpo_decode(orc.lpo_encode(a, bits, lohi), bits, lohi)
    for c in range(a.shape[1]):
        L = 65535 if c < 3 else 255
        lo, hi = float(lohi[c, 0]), float(lohi[c, 1])
        delta = (hi - lo) / L
        err = np.abs(proxy[:, c][:, occ].astype(np.float64) - a[:, c][:, occ])
        assert err.max() <= 0.5 * delta * (1 + 1e-4) + 4 * np.finfo(np.float32).eps * max(abs(lo), abs(hi))
        assert err.mean() < 0.3 * delta + 1e-6       # uniform error: mean ~ Delta / 4
        # the extreme texels decode to the range's ends
        live = a[:, c][:, occ]
        p = proxy[:, c][:, occ]
        assert abs(float(p[live == live.min()][0]) - lo) <= 1e-6 * max(1.0, abs(lo))
        assert abs(float(p[live == live.max()][0]) - hi) <= 1e-5 * max(1.0, abs(hi))


def test_codes_round_trip_integer_exact(orc):
    a, occ, bits = _atlas(4, F=1)
    lohi = orc.lpo_minmax(a, bits)
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 256, size=(1, a.shape[1] + 3) + occ.shape).astype(np.uint8)
    codes[:, :, ~occ] = 0
    again = orc.lpo_encode(orc.lpo_decode(codes, bits, lohi), bits, lohi)
    np.testing.assert_array_equal(again, codes)


def test_degenerate_channel_nan_and_dead_texels(orc):
    a, occ, bits = _atlas(6, F=1)
    a[0, 5][occ] = 1.25             # constant channel: every code 0, proxy = lo
    a[0, 7, occ.nonzero()[0][0], occ.nonzero()[1][0]] = np.nan
    lohi = orc.lpo_minmax(a, bits)
    codes = orc.lpo_encode(a, bits, lohi)
    proxy = orc.lpo_decode(codes, bits, lohi)
    assert np.all(codes[0, 8] == 0) and np.all(proxy[0, 5][occ] == np.float32(1.25))
    y, x = occ.nonzero()[0][0], occ.nonzero()[1][0]
    assert codes[0, 10, y, x] == 0 and proxy[0, 7, y, x] == lohi[7, 0]
    assert np.all(codes[:, :, ~occ] == 0) and np.all(proxy[:, :, ~occ] == 0)
    with pytest.raises(AssertionError):
        np.testing.assert_array_equal(codes[0, 9], 0)   # other channels are not degenerate
