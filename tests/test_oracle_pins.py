"""Pins for the CPU oracle: checks against facts that do not come from the oracle.

Each test ties one oracle function to something fixed independently of its
code: the documented coefficient/offset convention, a hand-derived rounding
example, a library routine on an exactly representable special case, a
closed-form eigenvalue, an error bound from the literature, or an algebraic
identity (adjoint dot-product test, finite differences).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.ndimage

import oracle
from paper_2001_01473_gb300 import inputs

STAR, BOX = 0, 1
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "order_cases.txt")


def convention_offsets(ndim, shape, R):
    """The documented coefficient order, built here independently of the oracle."""
    if shape == STAR:
        offs = [(0, 0, 0)]
        for i in list(range(-R, 0)) + list(range(1, R + 1)):
            offs.append((0, 0, i))
            offs.append((0, i, 0))
            if ndim == 3:
                offs.append((i, 0, 0))
        return offs
    zr = R if ndim == 3 else 0
    return [(dz, dy, dx) for dz in range(-zr, zr + 1)
            for dy in range(-R, R + 1) for dx in range(-R, R + 1)]


STENCILS = [(2, STAR, r) for r in (1, 2, 3, 4)] + [(2, BOX, r) for r in (1, 2, 3, 4)] + \
           [(3, STAR, r) for r in (1, 2, 3, 4)] + [(3, BOX, r) for r in (1, 2)]


@pytest.mark.parametrize("ndim,shape,R", STENCILS)
def test_offsets_follow_convention(ndim, shape, R):
    got = [tuple(int(v) for v in row) for row in oracle.offsets(ndim, shape, R)]
    assert got == convention_offsets(ndim, shape, R)
    assert len(got) == inputs.coeff_count(ndim, shape, R)
    # FLOP/cell of Table 4 = one multiply + (n-1) fma = 2n - 1
    n = len(got)
    flops = {(2, STAR): 8 * R + 1, (2, BOX): 2 * (2 * R + 1) ** 2 - 1,
             (3, STAR): 12 * R + 1, (3, BOX): 2 * (2 * R + 1) ** 3 - 1}[(ndim, shape)]
    assert 2 * n - 1 == flops


def _dims_for(ndim):
    return (11, 13) if ndim == 2 else (5, 6, 7)


# ---------------------------------------------------------------------------
# Exact constant preservation: dyadic coefficients summing to 1 on a constant
# dyadic field keep every product and partial sum exact.

def dyadic_coeffs(n):
    m = 1 << max(1, math.ceil(math.log2(n)))
    c = np.full(n, 1.0 / m)
    c[0] = 1.0 - (n - 1) / m
    return c


@pytest.mark.parametrize("ndim,shape,R", STENCILS)
@pytest.mark.parametrize("dtype", ["f32", "f64", "f16", "dot2"])
def test_constant_field_exact(ndim, shape, R, dtype):
    dims = _dims_for(ndim)
    n = inputs.coeff_count(ndim, shape, R)
    c = dyadic_coeffs(n)
    assert sum(Fraction(v) for v in c) == 1
    shp = inputs.padded_shape(dims, R)
    T = 7
    if dtype == "f32":
        out = oracle.run_f32(ndim, shape, R, c.astype(np.float32), dims,
                             np.full(shp, 0.75, np.float32), T)
    elif dtype == "f64":
        out = oracle.run_f64(ndim, shape, R, c, dims, np.full(shp, 0.75), T)
    elif dtype == "dot2":
        out = oracle.run_dot2(ndim, shape, R, c.astype(np.float32), dims,
                              np.full(shp, 0.75, np.float32), T)
    else:
        out = oracle.run_f16s(ndim, shape, R, c.astype(np.float32), dims,
                              np.full(shp, 0.75, np.float16), T)
    assert np.all(out.astype(np.float64) == 0.75)


@pytest.mark.parametrize("ndim,shape,R", [(2, STAR, 1), (2, BOX, 2), (3, STAR, 1), (3, BOX, 1)])
def test_constant_field_normalised_bound(ndim, shape, R):
    """Seeded normalised coefficients: |u_T - 1| <= T * (|sum c - 1| + n u)."""
    dims = _dims_for(ndim)
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.normalised_coeffs(n, 0).astype(np.float32)
    s = abs(float(sum(Fraction(float(v)) for v in c)) - 1.0)
    T = 20
    out = oracle.run_f32(ndim, shape, R, c, dims,
                         np.ones(inputs.padded_shape(dims, R), np.float32), T)
    bound = T * (s + n * 2.0 ** -24)
    assert np.max(np.abs(out.astype(np.float64) - 1.0)) <= bound


# ---------------------------------------------------------------------------
# Exact integer brute force against scipy.ndimage.correlate (a library routine):
# small integer coefficients and fields keep every FP operation exact while
# all values stay below 2^24 (FP32), 2^11 (FP16) or 2^53 (FP64).

def correlate_reference(ndim, shape, R, c, dims, u0, T):
    offs = convention_offsets(ndim, shape, R)
    W = np.zeros((2 * R + 1,) * ndim)
    for k, (dz, dy, dx) in enumerate(offs):
        idx = (dy + R, dx + R) if ndim == 2 else (dz + R, dy + R, dx + R)
        W[idx] = c[k]
    u = u0.astype(np.float64).copy()
    inner = tuple(slice(R, R + d) for d in dims)
    for _ in range(T):
        full = scipy.ndimage.correlate(u, W, mode="constant", cval=0.0)
        nxt = u.copy()
        nxt[inner] = full[inner]
        u = nxt
    return u


def _int_case(ndim, shape, R, limit, seed):
    dims = (9, 12) if ndim == 2 else (4, 5, 6)
    n = inputs.coeff_count(ndim, shape, R)
    c = np.floor(inputs.uniform(seed, n, 53) * 3.0)           # {0,1,2}
    shp = inputs.padded_shape(dims, R)
    u0 = np.floor(inputs.uniform(seed + 1, int(np.prod(shp)), 53) * 4.0).reshape(shp)  # {0..3}
    growth = max(1.0, float(np.sum(c)))
    T = 1
    while 3.0 * growth ** (T + 1) < limit and T < 8:
        T += 1
    return dims, c, u0, T


@pytest.mark.parametrize("ndim,shape,R", STENCILS)
@pytest.mark.parametrize("dtype", ["f32", "f64", "dot2"])
def test_integer_bruteforce(ndim, shape, R, dtype):
    limit = 2.0 ** 53 if dtype == "f64" else 2.0 ** 24
    dims, c, u0, T = _int_case(ndim, shape, R, limit, 17 + R + 3 * shape + 7 * ndim)
    ref = correlate_reference(ndim, shape, R, c, dims, u0, T)
    if dtype == "f32":
        out = oracle.run_f32(ndim, shape, R, c.astype(np.float32), dims, u0.astype(np.float32), T)
    elif dtype == "dot2":
        out = oracle.run_dot2(ndim, shape, R, c.astype(np.float32), dims, u0.astype(np.float32), T)
    else:
        out = oracle.run_f64(ndim, shape, R, c, dims, u0, T)
    np.testing.assert_array_equal(out.astype(np.float64), ref)


@pytest.mark.parametrize("ndim,shape,R", [(2, STAR, 1), (2, BOX, 1), (3, STAR, 2), (3, BOX, 1)])
def test_integer_bruteforce_f16(ndim, shape, R):
    dims, c, u0, T = _int_case(ndim, shape, R, 2.0 ** 11, 5 + R)
    ref = correlate_reference(ndim, shape, R, c, dims, u0, T)
    out = oracle.run_f16s(ndim, shape, R, c.astype(np.float32), dims, u0.astype(np.float16), T)
    np.testing.assert_array_equal(out.astype(np.float64), ref)


def test_t0_identity_and_halo_untouched():
    dims = (10, 14)
    R = 2
    u0 = inputs.field(dims, R, 1, "f32")
    c = inputs.normalised_coeffs(9, 0).astype(np.float32)
    np.testing.assert_array_equal(oracle.run_f32(2, STAR, R, c, dims, u0, 0), u0)
    out = oracle.run_f32(2, STAR, R, c, dims, u0, 5)
    mask = np.ones_like(u0, dtype=bool)
    mask[R:-R, R:-R] = False
    np.testing.assert_array_equal(out[mask], u0[mask])


# ---------------------------------------------------------------------------
# Summation order: hand-derived worked examples (tests/golden/order_cases.txt).

def _load_cases():
    cases, cur = [], None
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = dict(name=tok[1], dtype=tok[2], ndim=int(tok[3]), shape=int(tok[4]),
                           R=int(tok[5]), v=[])
                cases.append(cur)
            elif tok[0] == "v":
                cur["v"].append((int(tok[1]), int(tok[2]), int(tok[3]), float.fromhex(tok[4])))
            elif tok[0] == "expect":
                cur["expect"] = float.fromhex(tok[1])
    return cases


@pytest.mark.parametrize("case", _load_cases(), ids=lambda c: c["name"])
def test_summation_order_golden(case):
    ndim, shape, R = case["ndim"], case["shape"], case["R"]
    dims = (7, 8) if ndim == 2 else (5, 6, 7)
    shp = inputs.padded_shape(dims, R)
    u = np.zeros(shp)
    probe = tuple(R + 2 for _ in range(ndim))
    for dz, dy, dx, val in case["v"]:
        off = (dy, dx) if ndim == 2 else (dz, dy, dx)
        u[tuple(p + o for p, o in zip(probe, off))] = val
    n = inputs.coeff_count(ndim, shape, R)
    c = np.ones(n)
    dt = case["dtype"]
    if dt == "f32":
        out = oracle.run_f32(ndim, shape, R, c.astype(np.float32), dims, u.astype(np.float32), 1)
    elif dt == "f64":
        out = oracle.run_f64(ndim, shape, R, c, dims, u, 1)
    else:
        out = oracle.run_f16s(ndim, shape, R, c.astype(np.float32), dims, u.astype(np.float16), 1)
    assert float(out[probe]) == case["expect"]


# ---------------------------------------------------------------------------
# Plane wave on a periodic grid: a Fourier mode is an eigenvector of the
# periodic stencil with eigenvalue lambda = sum_k c_k exp(i theta.o_k).

@pytest.mark.parametrize("ndim,shape,R", [(2, STAR, 1), (2, STAR, 3), (2, BOX, 2),
                                          (3, STAR, 2), (3, BOX, 1)])
def test_plane_wave_eigenvalue(ndim, shape, R):
    N = 16 if ndim == 2 else 8
    dims = (N,) * ndim
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.normalised_coeffs(n, 11 + R)           # asymmetric coefficients
    kvec = (1, 2) if ndim == 2 else (1, 1, 2)
    theta = [2 * math.pi * k / N for k in kvec]
    grids = np.meshgrid(*[np.arange(N, dtype=np.float64)] * ndim, indexing="ij")
    phase = sum(t * g for t, g in zip(theta, grids))
    u0 = np.cos(phase)
    lam = 0j
    for k, (dz, dy, dx) in enumerate(convention_offsets(ndim, shape, R)):
        o = (dy, dx) if ndim == 2 else (dz, dy, dx)
        lam += c[k] * np.exp(1j * sum(t * oo for t, oo in zip(theta, o)))
    T = 9
    while T > 1 and abs(lam) ** T < 1e-2:   # keep the mode's amplitude measurable
        T -= 1
    out = oracle.run_periodic_f64(ndim, shape, R, c, dims, u0, T)
    expect = np.real(lam ** T * np.exp(1j * phase))
    tol = 10 * T * n * 2.0 ** -53 * max(1.0, abs(lam) ** T)
    assert np.max(np.abs(out - expect)) <= tol
    # the mirrored stencil has the conjugate eigenvalue: a sign error is visible
    assert np.max(np.abs(np.real(np.conj(lam) ** T * np.exp(1j * phase)) - expect)) > 1e3 * tol


# ---------------------------------------------------------------------------
# Algebraic properties of the plain method.

def test_linearity_exact_integer_regime():
    ndim, shape, R = 2, BOX, 1
    dims, c, u0, T = _int_case(ndim, shape, R, 2.0 ** 20, 41)
    v0 = np.floor(inputs.uniform(99, u0.size, 53) * 4.0).reshape(u0.shape)
    a, b = 2.0, 3.0
    f = lambda u: oracle.run_f32(ndim, shape, R, c.astype(np.float32), dims, u.astype(np.float32), T)
    np.testing.assert_array_equal(f(a * u0 + b * v0), a * f(u0) + b * f(v0))


@pytest.mark.parametrize("ndim,shape,R", [(2, STAR, 2), (2, BOX, 1), (3, STAR, 1), (3, BOX, 1)])
def test_composition_bitwise(ndim, shape, R):
    """T steps at once equal T single steps, bit for bit (double buffering)."""
    dims = _dims_for(ndim)
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.normalised_coeffs(n, 0).astype(np.float32)
    u = inputs.field(dims, R, 1, "f32")
    T = 6
    whole = oracle.run_f32(ndim, shape, R, c, dims, u, T)
    step = u
    for _ in range(T):
        step = oracle.run_f32(ndim, shape, R, c, dims, step, 1)
    np.testing.assert_array_equal(whole, step)


# ---------------------------------------------------------------------------
# binary16 conversions against numpy's IEEE conversion (a library routine).

def test_f16_conversions_match_numpy():
    vals = [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.996, 65520.0, 1e6, -1e6,
            2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25,
            1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -11 + 2.0 ** -20,
            float("inf"), -float("inf"), 5.96e-8, 6.1e-5, 0.1, 1.0 / 3.0]
    rnd = inputs.uniform(7, 4000, 53)
    vals += list((rnd - 0.5) * 2.0 ** 17) + list(rnd * 2.0 ** -13) + list(rnd * 2.0 ** -23)
    for v in vals:
        f = np.float32(v)
        with np.errstate(over="ignore"):
            want = int(np.array([f], np.float32).astype(np.float16).view(np.uint16)[0])
        assert oracle.f32_to_f16_bits(float(f)) == want, v
    for h in range(0, 1 << 16, 7):
        want = np.array([h], np.uint16).view(np.float16).astype(np.float32)[0]
        got = np.float32(oracle.f16_bits_to_f32(h))
        if np.isnan(want):
            assert np.isnan(got)
        else:
            assert got == want, h


# ---------------------------------------------------------------------------
# Dot2 (Ogita, Rump, Oishi 2005): result error <= u|s| + gamma_n^2 sum|c_k f_k|,
# u = 2^-24, on ill-conditioned sums where the plain chain is far off.

def test_dot2_error_bound_ill_conditioned():
    ndim, shape, R = 2, BOX, 1
    dims = (6, 7)
    shp = inputs.padded_shape(dims, R)
    n = 9
    rnd = inputs.uniform(23, n, 53)
    c = np.array([(1.0 if k % 2 == 0 else -1.0) * (1.0 + rnd[k] * 2.0 ** -10) for k in range(n)],
                 np.float32)
    base = inputs.uniform(24, int(np.prod(shp)), 24).reshape(shp)
    u = (1.0 + base * 2.0 ** -12).astype(np.float32) * np.float32(2.0 ** 10)
    got = oracle.run_dot2(ndim, shape, R, c, dims, u, 1)
    plain = oracle.run_f32(ndim, shape, R, c, dims, u, 1)
    offs = convention_offsets(ndim, shape, R)
    uu = 2.0 ** -24
    gam = n * uu / (1 - n * uu)
    worst_plain = 0.0
    for y in range(R, R + dims[0]):
        for x in range(R, R + dims[1]):
            terms = [Fraction(float(c[k])) * Fraction(float(u[y + dy, x + dx]))
                     for k, (_, dy, dx) in enumerate(offs)]
            s = sum(terms)
            absum = sum(abs(t) for t in terms)
            err = abs(Fraction(float(got[y, x])) - s)
            assert err <= uu * abs(s) + gam * gam * absum
            worst_plain = max(worst_plain, float(abs(Fraction(float(plain[y, x])) - s) / absum))
    assert worst_plain > 1e3 * gam * gam   # the plain chain would fail the bound


# ---------------------------------------------------------------------------
# FP64 adjoint.

ADJ = [(2, STAR, 1), (2, BOX, 1), (2, STAR, 2), (3, STAR, 1), (3, BOX, 1)]


@pytest.mark.parametrize("ndim,shape,R", ADJ)
def test_adjoint_dot_product(ndim, shape, R):
    """<S^T u, v> = <u, (S^T)^T v> with a zero halo (linear part of the sweep)."""
    dims = (9, 11) if ndim == 2 else (4, 5, 6)
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.normalised_coeffs(n, 0) * 1.3 - 0.05
    shp = inputs.padded_shape(dims, R)
    inner = tuple(slice(R, R + d) for d in dims)
    u0 = np.zeros(shp)
    u0[inner] = inputs.uniform(1, int(np.prod(dims)), 53).reshape(dims) - 0.5
    v = np.zeros(shp)
    v[inner] = inputs.uniform(2, int(np.prod(dims)), 53).reshape(dims) - 0.5
    T = 5
    uT = oracle.run_f64(ndim, shape, R, c, dims, u0, T)
    _, g0, _ = oracle.adjoint_f64(ndim, shape, R, c, dims, u0, uT - v, T)   # g_T = v
    lhs = float(np.sum(uT[inner] * v[inner]))
    rhs = float(np.sum(u0[inner] * g0[inner]))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    halo = np.ones(shp, bool)
    halo[inner] = False
    assert np.all(g0[halo] == 0.0)


@pytest.mark.parametrize("ndim,shape,R", ADJ)
def test_adjoint_finite_differences(ndim, shape, R):
    dims = (7, 8) if ndim == 2 else (4, 4, 5)
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    u0 = inputs.field(dims, R, 1, "f64")
    tg = inputs.target_field(dims, R, 2, "f64")
    T = 4
    loss, gu, gc = oracle.adjoint_f64(ndim, shape, R, c, dims, u0, tg, T)
    inner = tuple(slice(R, R + d) for d in dims)

    def L(cc, uu):
        uT = oracle.run_f64(ndim, shape, R, cc, dims, uu, T)
        d = uT[inner] - tg[inner]
        return 0.5 * float(np.sum(d * d))

    assert abs(L(c, u0) - loss) <= 1e-12 * loss
    h = 1e-3
    for j in range(4):
        dc = inputs.uniform(50 + j, n, 53) - 0.5
        an = float(np.dot(gc, dc))
        # L is a polynomial of degree 2T in c: central differences converge as h^2
        e1 = abs((L(c + h * dc, u0) - L(c - h * dc, u0)) / (2 * h) - an)
        h2 = h / 4
        e2 = abs((L(c + h2 * dc, u0) - L(c - h2 * dc, u0)) / (2 * h2) - an)
        assert e1 <= 5e-2 * max(1.0, abs(an))
        assert e2 <= e1 / 10 + 1e-9 * max(1.0, abs(an))
        du = np.zeros_like(u0)
        du[inner] = (inputs.uniform(60 + j, int(np.prod(dims)), 53) - 0.5).reshape(dims)
        fd = (L(c, u0 + h * du) - L(c, u0 - h * du)) / (2 * h)
        an = float(np.sum(gu * du))
        assert abs(fd - an) <= 1e-9 * max(1.0, abs(an))      # L quadratic in u0: exact
