"""Float8 (E4M3) storage of X with one power-of-two scale per slab, in plain
float64 NumPy: the encoding behind the FP8 form of the pass over X.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper computes in the input's own precision; storing X in 8 bits is an
extension of its Alg. 1 (the core step and the sampled fibers read X), not a
step it prints.  Everything here is written from the E4M3 format definition
(OCP 8-bit floating point, E4M3 variant): 1 sign bit, 4 exponent bits with
bias 7, 3 mantissa bits; exponent field 0 holds the subnormals m * 2^-9; the
code S.1111.111 is NaN and there is no infinity, so the largest finite value is
1.110 * 2^8 = 448.

Encoding of a tensor X of order d >= 2: a *slab* is one matrix of the last two
modes (X[i_1, ..., i_{d-2}, :, :]; the whole matrix when d = 2).  Per slab:

* amax = max |x| over the slab; e is the exponent with amax = f * 2^e,
  0.5 <= f < 1 (e = 0 for an all-zero slab);
* the scale is the power of two sigma = 2^(e - 8), so |x| / sigma < 256;
* each code is the E4M3 value nearest to x / sigma, ties to the even mantissa.

Scaling by a power of two is exact, so every code is decided on the exact real
number x / sigma: both sides of a parity test take the same decision in any
precision.  The stored value of an element is code * sigma, again exact.
"""

import numpy as np

E4M3_MAX = 448.0
MIN_NORMAL_EXP = -6        # smallest normal: 2^-6
SUB_QUANTUM = 2.0 ** -9    # spacing of the subnormals


def e4m3_decode(code):
    """Value of each E4M3 code (uint8 array or int), from the bit fields."""
    c = np.asarray(code, dtype=np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    ef = (c >> 3) & 0xF
    m = c & 0x7
    val = np.where(ef == 0, m * SUB_QUANTUM, (1.0 + m / 8.0) * np.exp2(ef.astype(np.float64) - 7.0))
    val = np.where(((c & 0x7F) == 0x7F), np.nan, val)
    return sign * val


def e4m3_round(y):
    """Nearest E4M3 value to each real y (float64), ties to the even mantissa,
    magnitudes beyond 448 saturated to +-448; returns the codes (uint8).

    Normal range (|y| >= 2^-6): the spacing in the binade [2^E, 2^(E+1)) is
    2^(E-3); subnormal range: spacing 2^-9.  Rounding to a multiple of the
    spacing with ties to even is np.rint on the scaled value (round half to
    even), which also selects the even mantissa at a tie."""
    y = np.asarray(y, dtype=np.float64)
    a = np.abs(y)
    _, ex = np.frexp(a)                 # a = f * 2^ex, 0.5 <= f < 1, so E = ex - 1
    E = np.maximum(ex - 1, MIN_NORMAL_EXP)
    quantum = np.exp2(E.astype(np.float64) - 3.0)
    r = np.rint(a / quantum) * quantum  # may round up to 2^(E+1): still on the grid
    r = np.minimum(r, E4M3_MAX)
    return _encode_exact(np.copysign(r, y))


def _encode_exact(v):
    """Code of values that lie on the E4M3 grid (float64 array)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    sign = np.where(np.signbit(v), 0x80, 0)
    _, ex = np.frexp(a)
    E = ex - 1
    normal = a >= 2.0 ** MIN_NORMAL_EXP
    ef = np.where(normal, E + 7, 0)
    man = np.where(normal, a / np.exp2(E.astype(np.float64)) * 8.0 - 8.0, a / SUB_QUANTUM)
    man_i = np.rint(man).astype(np.int64)
    assert np.all(np.abs(man - man_i) == 0), "value not on the E4M3 grid"
    assert np.all((man_i >= 0) & (man_i <= 7)) and np.all((ef >= 0) & (ef <= 15)), "E4M3 field range"
    return (sign | (ef << 3) | man_i).astype(np.uint8)


def slab_shape(shape):
    """(number of slabs, rows, columns) of the last-two-mode slabs."""
    shape = tuple(int(s) for s in shape)
    assert len(shape) >= 2
    return int(np.prod(shape[:-2], dtype=np.int64)), shape[-2], shape[-1]


def slab_scale_exponent(amax):
    """e of the scale 2^(e-8): amax = f 2^e with 0.5 <= f < 1, e = 0 for amax = 0."""
    if amax == 0.0:
        return 0
    return int(np.frexp(amax)[1])


def quantize(X):
    """E4M3 codes (uint8, X's shape) and per-slab scales (float32, one per slab)
    of a float tensor X, by the rule in the module docstring."""
    X = np.asarray(X)
    S, n1, n2 = slab_shape(X.shape)
    Xs = X.astype(np.float64).reshape(S, n1, n2)
    codes = np.empty((S, n1, n2), dtype=np.uint8)
    scales = np.empty(S, dtype=np.float32)
    for s in range(S):
        amax = float(np.abs(Xs[s]).max()) if n1 * n2 else 0.0
        sigma = 2.0 ** (slab_scale_exponent(amax) - 8)
        scales[s] = sigma
        codes[s] = e4m3_round(Xs[s] / sigma)
    return codes.reshape(X.shape), scales


def dequantize(codes, scales):
    """The stored tensor: code value times its slab's scale, in float64 (exact)."""
    codes = np.asarray(codes)
    S, n1, n2 = slab_shape(codes.shape)
    v = e4m3_decode(codes.reshape(S, n1, n2)) * np.asarray(scales, dtype=np.float64)[:, None, None]
    return v.reshape(codes.shape)
