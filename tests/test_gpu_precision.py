"""Precision forms on the GPU: FP64 error norms, and the error of the FP32
plain, Dot2-compensated FP32 and binary16-storage forms against the FP64
oracle, each within a bound derived from its rounding model.

Bounds (u32 = 2^-24, u16 = 2^-11, n terms, sum |c_k| = 1 so one step does not
increase the max-norm of an error): one step of the plain chain errs by at
most gamma_n * max|u| (gamma_n = n u32 / (1 - n u32)); Dot2 by at most
(u32 + gamma_n^2) * max|u| (Ogita, Rump, Oishi 2005); binary16 storage adds
u16 * max|u| per level.  After T steps the error is at most T times that.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs
from _gpu_util import gpu_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX


def test_error_norms_match_numpy():
    import torch
    for ndim, dims, R, dt in [(2, (300, 517), 2, "f32"), (3, (20, 33, 70), 1, "f16"),
                              (2, (64, 64), 1, "f64")]:
        shp = inputs.padded_shape(dims, R)
        ref = inputs.uniform(5, int(np.prod(shp)), 53).reshape(shp)
        u = (ref + (inputs.uniform(6, ref.size, 53).reshape(shp) - 0.5) * 1e-3).astype(
            inputs.npdtype(dt))
        got = an5d.an5d_error_norms(ndim, R, dims, dt, torch.from_numpy(u).cuda(),
                                    torch.from_numpy(ref).cuda())
        inner = tuple(slice(R, R + d) for d in dims)
        d = u[inner].astype(np.float64) - ref[inner]
        assert got["max_abs"] == float(np.max(np.abs(d)))
        assert math.isclose(got["l2_diff"], float(np.sqrt(np.sum(d * d))), rel_tol=1e-12)
        assert math.isclose(got["l2_ref"], float(np.sqrt(np.sum(ref[inner] ** 2))), rel_tol=1e-12)


@pytest.mark.parametrize("ndim,shape,dims,T", [(3, STAR, (24, 30, 40), 200),
                                               (2, BOX, (120, 160), 300)])
def test_precision_forms_error_vs_fp64_oracle(ndim, shape, dims, T):
    import torch
    R = 1
    n = inputs.coeff_count(ndim, shape, R)
    c = inputs.heat_coeffs(ndim) if shape == STAR else inputs.normalised_coeffs(n, 0)
    c32 = c.astype(np.float32).astype(np.float64)       # the run's rounded coefficients
    u32 = inputs.gaussian_bump(dims, R, 1, "f32")
    u16 = u32.astype(np.float16)
    inner = tuple(slice(R, R + d) for d in dims)
    errs = {}
    for form, u0 in (("f32", u32), ("f32c", u32), ("f16", u16)):
        ref = oracle.run_f64(ndim, shape, R, c32, dims, u0.astype(np.float64), T)
        got = gpu_run(ndim, shape, R, c, form, dims, u0, T)
        d = got[inner].astype(np.float64) - ref[inner]
        norms = an5d.an5d_error_norms(ndim, R, dims, form, torch.from_numpy(got).cuda(),
                                      torch.from_numpy(ref).cuda())
        assert norms["max_abs"] == float(np.max(np.abs(d)))
        errs[form] = norms["max_abs"]
        umax = float(np.max(np.abs(u0.astype(np.float64))))
        u, g = 2.0 ** -24, n * 2.0 ** -24 / (1 - n * 2.0 ** -24)
        bound = {"f32": T * g, "f32c": T * (u + g * g), "f16": T * (2.0 ** -11 + g)}[form] * umax
        assert errs[form] <= bound, (form, errs[form], bound)
    # Dot2 is the more accurate form in this regime: small grids and runs of
    # a few hundred steps, where the error is the sum of per-step roundings
    # (one Dot2 step is correctly rounded).  On long runs over large smooth
    # fields the plain chain can end closer to FP64 (the benchmark reports it).
    assert errs["f32c"] < errs["f32"]
    assert errs["f16"] > errs["f32"]           # binary16 storage costs accuracy
