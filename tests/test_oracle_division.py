"""Pins for the oracle's division-type stencils (Table 4: j2d5pt, j2d9pt,
j2d9pt-gol, j3d27pt): the weighted sum of a star or box stencil divided by a
constant d at every step, either by one IEEE division or by a multiplication
with 1/d rounded once to the run's precision.

The checks do not come from the oracle: exact rational arithmetic (Python
Fractions, rounded to binary32/binary64 by a round-to-nearest-even helper
written from the format definition), an integer brute force through
scipy.ndimage.correlate with a power-of-two divisor, and constant-field
preservation with dyadic coefficients.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.ndimage

import oracle
from paper_2001_01473_gb300 import inputs

STAR, BOX = 0, 1
DIV, MUL = oracle.POST_DIV, oracle.POST_MUL_RCP
# (ndim, shape, R) of the division-type rows of Table 4
JSTENCILS = [(2, STAR, 1), (2, STAR, 2), (2, BOX, 1), (3, BOX, 1)]


def round_binary(q: Fraction, dtype: str) -> Fraction:
    """q rounded to the nearest binary32/binary64 value, ties to even
    (normal range only; the tests keep every value normal or zero)."""
    if q == 0:
        return Fraction(0)
    p = 24 if dtype == "f32" else 53
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # 2^e <= a < 2^(e+1): the unit in the last place is 2^(e-p+1)
    scaled = a / Fraction(2) ** (e - p + 1)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return sign * Fraction(m) * Fraction(2) ** (e - p + 1)


def _offsets(ndim, shape, R):
    return [tuple(int(v) for v in o) for o in oracle.offsets(ndim, shape, R)]


def exact_one_step(ndim, shape, R, c, d, post, u, dims, dtype):
    """One step at every interior point in exact arithmetic with one rounding
    per operation: the first product, each fma, then the division by d (or
    the product with the rounded reciprocal)."""
    offs = _offsets(ndim, shape, R)
    cq = [Fraction(float(v)) for v in c]
    dq = Fraction(float(d))
    rq = round_binary(1 / dq, dtype)
    out = u.astype(np.float64).copy()
    it = np.ndindex(*dims)
    for idx in it:
        p = tuple(i + R for i in idx)
        acc = None
        for k, (dz, dy, dx) in enumerate(offs):
            off = (dy, dx) if ndim == 2 else (dz, dy, dx)
            f = Fraction(float(u[tuple(a + b for a, b in zip(p, off))]))
            acc = round_binary(cq[k] * f if acc is None else cq[k] * f + acc, dtype)
        res = round_binary(acc / dq, dtype) if post == DIV else round_binary(acc * rq, dtype)
        out[p] = float(res)
    return out


@pytest.mark.parametrize("ndim,shape,R", JSTENCILS)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("post", [DIV, MUL])
def test_one_step_exact_rounding(ndim, shape, R, dtype, post):
    dims = (5, 6) if ndim == 2 else (3, 4, 5)
    n = inputs.coeff_count(ndim, shape, R)
    t = np.float32 if dtype == "f32" else np.float64
    d = 7.0                                  # 1/7 is not a dyadic number: DIV and MUL differ
    c = (inputs.uniform(31 + R, n, 24 if dtype == "f32" else 53) * 2.0 + 0.5).astype(t)
    shp = inputs.padded_shape(dims, R)
    u = (inputs.uniform(41 + n, int(np.prod(shp)), 24 if dtype == "f32" else 53)
         .reshape(shp) + 0.25).astype(t)
    ref = exact_one_step(ndim, shape, R, c, d, post, u, dims, dtype)
    got = oracle.run_div(dtype, ndim, shape, R, c, d, post, dims, u, 1)
    np.testing.assert_array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_division_and_reciprocal_differ(dtype):
    """With d = 7 the two forms must disagree somewhere (else one of them is
    not what it claims), and by at most two units in the last place (the
    reciprocal's and the product's roundings)."""
    dims = (40, 50)
    t = np.float32 if dtype == "f32" else np.float64
    c = inputs.normalised_coeffs(5, 0).astype(t) * t(7.0)
    u = inputs.field(dims, 1, 1, dtype)
    a = oracle.run_div(dtype, 2, STAR, 1, c, 7.0, DIV, dims, u, 1)
    b = oracle.run_div(dtype, 2, STAR, 1, c, 7.0, MUL, dims, u, 1)
    inner = (slice(1, -1), slice(1, -1))
    diff = np.abs(a[inner].astype(np.float64) - b[inner].astype(np.float64))
    ulp = np.spacing(np.abs(a[inner])).astype(np.float64)
    assert np.any(diff > 0)
    assert np.all(diff <= 2 * ulp)


def _correlate_div(ndim, shape, R, c, d, dims, u0, T):
    W = np.zeros((2 * R + 1,) * ndim)
    for k, (dz, dy, dx) in enumerate(_offsets(ndim, shape, R)):
        idx = (dy + R, dx + R) if ndim == 2 else (dz + R, dy + R, dx + R)
        W[idx] = c[k]
    u = u0.astype(np.float64).copy()
    inner = tuple(slice(R, R + n) for n in dims)
    for _ in range(T):
        full = scipy.ndimage.correlate(u, W, mode="constant", cval=0.0)
        nxt = u.copy()
        nxt[inner] = full[inner] / d
        u = nxt
    return u


@pytest.mark.parametrize("ndim,shape,R", JSTENCILS)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("post", [DIV, MUL])
def test_integer_bruteforce_power_of_two_divisor(ndim, shape, R, dtype, post):
    """Integer coefficients and fields with d = 4: every product, sum and
    division is exact while the values keep few enough bits, so both forms
    equal a library correlation followed by an exact division."""
    dims = (9, 12) if ndim == 2 else (4, 5, 6)
    n = inputs.coeff_count(ndim, shape, R)
    c = np.floor(inputs.uniform(7 + n, n, 53) * 3.0)
    shp = inputs.padded_shape(dims, R)
    u0 = np.floor(inputs.uniform(9 + n, int(np.prod(shp)), 53) * 4.0).reshape(shp)
    # each step multiplies the largest magnitude by at most sum(c)/4 and adds
    # two fraction bits; stay well inside 24 significant bits
    T = 3
    ref = _correlate_div(ndim, shape, R, c, 4.0, dims, u0, T)
    t = np.float32 if dtype == "f32" else np.float64
    got = oracle.run_div(dtype, ndim, shape, R, c.astype(t), 4.0, post, dims, u0.astype(t), T)
    np.testing.assert_array_equal(got.astype(np.float64), ref)


@pytest.mark.parametrize("ndim,shape,R", JSTENCILS)
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("post", [DIV, MUL])
def test_constant_field_preserved(ndim, shape, R, dtype, post):
    """Dyadic coefficients summing to d = 8 on the constant field 0.75: every
    partial sum is a multiple of 1/16 below 8, the weighted sum is exactly 6
    and 6/8 (or 6 * 0.125) is exactly 0.75."""
    dims = (6, 7) if ndim == 2 else (4, 5, 6)
    n = inputs.coeff_count(ndim, shape, R)
    c = np.full(n, 0.25)                     # products 0.1875 and partial sums stay exact
    c[0] = 8.0 - 0.25 * (n - 1)
    assert sum(Fraction(v) for v in c) == 8
    t = np.float32 if dtype == "f32" else np.float64
    u = np.full(inputs.padded_shape(dims, R), 0.75, dtype=t)
    got = oracle.run_div(dtype, ndim, shape, R, c.astype(t), 8.0, post, dims, u, 5)
    assert np.all(got == t(0.75))
