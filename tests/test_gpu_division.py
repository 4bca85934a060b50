"""GPU parity of the division-type stencils (Table 4: j2d5pt, j2d9pt,
j2d9pt-gol, j3d27pt) against the CPU oracle, through the C ABI, bit for bit,
in both forms of the per-step division (IEEE division, product with the
rounded reciprocal)."""
import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs
from paper_2001_01473_gb300.kernels import KERNELS_DIV_2D, KERNELS_DIV_3D
from _gpu_util import assert_bitwise, gpu_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX
DT = {"DT_F32": "f32", "DT_F64": "f64"}
SH = {"SH_STAR": STAR, "SH_BOX": BOX}
DIVISOR = 7.0        # not a power of two: the two forms differ in the last bit


def _built():
    out = {}
    for sh, r, bts, _s, dt in KERNELS_DIV_2D:
        out.setdefault((2, SH[sh], r, DT[dt]), []).extend(bts)
    for sh, r, bts, _s, dt, _nw in KERNELS_DIV_3D:
        out.setdefault((3, SH[sh], r, DT[dt]), []).extend(bts)
    return out


def _cases():
    cases = []
    for (ndim, shape, R, dt), bts in sorted(_built().items()):
        for bt in sorted(set(bts)):     # every compiled degree
            for post in ("div", "rcp"):
                cases.append((ndim, shape, R, dt, bt, post))
    return cases


def _coeffs(ndim, shape, R):
    # normalised coefficients scaled by the divisor: the quotient averages
    return inputs.normalised_coeffs(inputs.coeff_count(ndim, shape, R), 0) * DIVISOR


def _oracle(ndim, shape, R, c, dt, dims, u0, T, post):
    t = np.float32 if dt == "f32" else np.float64
    p = oracle.POST_DIV if post == "div" else oracle.POST_MUL_RCP
    return oracle.run_div(dt, ndim, shape, R, np.asarray(c).astype(t), DIVISOR, p, dims, u0, T)


@pytest.mark.parametrize("ndim,shape,R,dt,bt,post", _cases())
def test_division_parity_ragged(ndim, shape, R, dt, bt, post):
    dims = (61, 301) if ndim == 2 else (23, 45, 141)
    c = _coeffs(ndim, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    plan = an5d.Plan(ndim, shape, R, c, dt, dims, divisor=DIVISOR, post=post)
    try:
        for T in sorted({1, bt, bt + 1, 2 * bt + 3}):
            ref = _oracle(ndim, shape, R, c, dt, dims, u0, T, post)
            got = gpu_run(ndim, shape, R, c, dt, dims, u0, T, bT=bt, hsn=17 if ndim == 2 else 7,
                          plan=plan)
            assert_bitwise(got, ref, f"{ndim}d shape={shape} R={R} {dt} {post} bT={bt} T={T}")
    finally:
        plan.close()


@pytest.mark.parametrize("dims", [(1, 1), (3, 5), (9, 108), (40, 216)])
def test_division_degenerate_extents(dims):
    c = _coeffs(2, BOX, 1)
    u0 = inputs.field(dims, 1, 3, "f32")
    for post in ("div", "rcp"):
        ref = _oracle(2, BOX, 1, c, "f32", dims, u0, 9, post)
        plan = an5d.Plan(2, BOX, 1, c, "f32", dims, divisor=DIVISOR, post=post)
        try:
            for hsn in (0, 1, 3):
                got = gpu_run(2, BOX, 1, c, "f32", dims, u0, 9, bT=4, hsn=hsn, plan=plan)
                assert_bitwise(got, ref, f"dims={dims} {post} hsn={hsn}")
        finally:
            plan.close()


def test_division_forms_differ_and_plain_plan_unchanged():
    dims = (64, 200)
    c = _coeffs(2, STAR, 1)
    u0 = inputs.field(dims, 1, 1, "f32")
    res = {}
    for post in ("div", "rcp"):
        plan = an5d.Plan(2, STAR, 1, c, "f32", dims, divisor=DIVISOR, post=post)
        try:
            res[post] = gpu_run(2, STAR, 1, c, "f32", dims, u0, 5, plan=plan)
        finally:
            plan.close()
    assert np.any(res["div"] != res["rcp"])
    plain = gpu_run(2, STAR, 1, c / DIVISOR, "f32", dims, u0, 5)
    ref = oracle.run_f32(2, STAR, 1, (c / DIVISOR).astype(np.float32), dims, u0, 5)
    assert_bitwise(plain, ref, "plain plan next to division plans")


def test_division_plan_rejections():
    c = _coeffs(2, STAR, 1)
    with pytest.raises(an5d.An5dError) as e:
        an5d.Plan(2, STAR, 1, c, "f16", (8, 8), divisor=DIVISOR, post="div")
    assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    with pytest.raises(an5d.An5dError) as e:
        an5d.Plan(2, STAR, 3, _coeffs(2, STAR, 3), "f32", (8, 8), divisor=DIVISOR, post="div")
    assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    plan = an5d.Plan(2, STAR, 1, c, "f32", (16, 16), divisor=DIVISOR, post="rcp")
    try:
        import torch
        x = torch.zeros(18, 18, device="cuda")
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_run_adjoint(plan.handle, x, x, torch.zeros_like(x), 3)
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    finally:
        plan.close()
