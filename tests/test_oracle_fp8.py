"""Pins of the float8 (E4M3) storage oracle, oracle/fp8.py: the code table
against the format's defining values and against an independent library
conversion (torch.float8_e4m3fn on the CPU), round-to-nearest-even against a
brute-force search of the table, and the per-slab power-of-two scaling
against its stated bounds."""

import numpy as np
import pytest

from oracle import fp8

torch = pytest.importorskip("torch")
if not hasattr(torch, "float8_e4m3fn"):
    pytest.skip("torch without float8_e4m3fn", allow_module_level=True)


def _torch_decode(codes):
    t = torch.from_numpy(np.asarray(codes, dtype=np.uint8).copy()).view(torch.float8_e4m3fn)
    return t.to(torch.float64).numpy()


def _torch_encode(vals):
    t = torch.from_numpy(np.asarray(vals, dtype=np.float64)).to(torch.float8_e4m3fn)
    return t.view(torch.uint8).numpy()


def test_code_table_defining_values():
    dec = fp8.e4m3_decode
    assert dec(0x00) == 0.0 and np.signbit(dec(0x80))
    assert dec(0x01) == 2.0 ** -9                   # smallest subnormal
    assert dec(0x07) == 7 * 2.0 ** -9               # largest subnormal
    assert dec(0x08) == 2.0 ** -6                   # smallest normal
    assert dec(0x38) == 1.0 and dec(0x3C) == 1.5 and dec(0xB8) == -1.0
    assert dec(0x7E) == 448.0 and dec(0xFE) == -448.0
    assert np.isnan(dec(0x7F)) and np.isnan(dec(0xFF))
    pos = dec(np.arange(0x7F))
    assert np.all(np.diff(pos) > 0)                 # codes 0..126 increase strictly
    finite = dec(np.arange(256))
    assert np.isfinite(finite).sum() == 254 and len(np.unique(finite[np.isfinite(finite)])) == 253


def test_code_table_equals_library_view():
    codes = np.arange(256, dtype=np.uint8)
    a, b = fp8.e4m3_decode(codes), _torch_decode(codes)
    assert np.array_equal(np.isnan(a), np.isnan(b))
    ok = ~np.isnan(a)
    assert np.array_equal(a[ok], b[ok]) and np.array_equal(np.signbit(a[ok]), np.signbit(b[ok]))


def test_rounding_fixes_grid_points_and_ties_to_even():
    codes = np.array([c for c in range(256) if (c & 0x7F) != 0x7F], dtype=np.uint8)
    assert np.array_equal(fp8.e4m3_round(fp8.e4m3_decode(codes)), codes)
    pos = fp8.e4m3_decode(np.arange(0x7F))
    mid = 0.5 * (pos[:-1] + pos[1:])               # exact in float64
    got = fp8.e4m3_round(mid)
    assert np.all((got & 1) == 0)                  # the even neighbour
    assert np.all((got == np.arange(0x7E)) | (got == np.arange(1, 0x7F)))
    assert np.array_equal(got, _torch_encode(mid))


def test_rounding_matches_brute_force_and_library():
    rs = np.random.default_rng(7)
    mag = np.exp2(rs.uniform(-12.0, np.log2(448.0), 20000))
    y = np.where(rs.random(20000) < 0.5, -mag, mag)
    got = fp8.e4m3_round(y)
    assert np.array_equal(got, _torch_encode(y))
    table = fp8.e4m3_decode(np.arange(0x7F))       # non-negative values, codes 0..126
    a = np.abs(y)
    dist = np.abs(a[:, None] - table[None, :])
    best = dist.min(axis=1)
    # nearest code; of two at the same distance the one with the even mantissa
    cand = dist == best[:, None]
    idx = np.array([np.flatnonzero(row)[0] if row.sum() == 1 else
                    [c for c in np.flatnonzero(row) if c % 2 == 0][0] for row in cand])
    want = (idx | np.where(y < 0, 0x80, 0)).astype(np.uint8)
    assert np.array_equal(got, want)
    assert fp8.e4m3_round(np.array([1000.0]))[0] == 0x7E   # saturated


def test_slab_scaling_bounds_and_layout():
    rs = np.random.default_rng(3)
    X = (rs.standard_normal((3, 2, 12, 20)) * np.exp2(rs.integers(-20, 20, (3, 2, 1, 1)))).astype(np.float32)
    X[1, 1] = 0.0                                  # an all-zero slab
    codes, scales = fp8.quantize(X)
    assert codes.shape == X.shape and codes.dtype == np.uint8 and scales.shape == (6,)
    Xs = X.astype(np.float64).reshape(6, 12, 20)
    for s in range(6):
        m, ex = np.frexp(scales[s])
        assert m == 0.5                            # a power of two
        amax = np.abs(Xs[s]).max()
        if amax == 0:
            assert scales[s] == 2.0 ** -8 and not codes.reshape(6, 12, 20)[s].any()
        else:
            assert 128.0 <= amax / scales[s] < 256.0
    Xd = fp8.dequantize(codes, scales).reshape(6, 12, 20)
    sc = scales.astype(np.float64)[:, None, None]
    err = np.abs(Xd - Xs)
    normal = np.abs(Xs) >= sc * 2.0 ** -6
    assert np.all(err[normal] <= 2.0 ** -4 * np.abs(Xs)[normal])   # half a spacing of 2^(E-3)
    assert np.all(err[~normal] <= sc.repeat(12, 1).repeat(20, 2)[~normal] * 2.0 ** -10)
    # d = 2: the whole matrix is one slab
    c2, s2 = fp8.quantize(X[0, 0])
    assert s2.shape == (1,) and np.array_equal(c2, codes[0, 0]) and s2[0] == scales[0]
