"""GPU parity of the wider 2D tile variants (6 cells per lane) against the
CPU oracle, through the C ABI.  The variants compute the same per-cell fma
chains as the default kernels, so every comparison is bit for bit, including
runs whose remainder pass falls back to a default-width kernel."""
import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs
from paper_2001_01473_gb300.kernels import KERNELS_2D_WIDE, KERNELS_DIV_2D_WIDE
from _gpu_util import assert_bitwise, coeffs_for, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
STAR = inputs.STAR
SH = {"SH_STAR": inputs.STAR, "SH_BOX": inputs.BOX}
DT = {"DT_F32": "f32", "DT_F64": "f64", "DT_F16S": "f16"}

CASES = [(SH[sh], r, DT[dt], 32 * v, bt)
         for sh, r, bts, _s, _m, dt, v, _occ in KERNELS_2D_WIDE for bt in bts]
# each (stencil, tile) at its largest degree
TOP = sorted({(sh, r, dt, t, max(b for s2, r2, d2, t2, b in CASES if (s2, r2, d2, t2) == (sh, r, dt, t)))
              for sh, r, dt, t, _ in CASES})
DIV_CASES = [(SH[sh], r, DT[dt], 32 * v, bt, post)
             for sh, r, bts, _s, dt, v, _occ in KERNELS_DIV_2D_WIDE for bt in bts
             for post in ("div", "rcp")]


@pytest.mark.parametrize("shape,R,dt,tile,bt", CASES)
def test_wide_parity_several_tiles_ragged(shape, R, dt, tile, bt):
    dims = (47, 700)               # 3-4 tiles across x with a ragged last one
    c = coeffs_for(2, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    for T in sorted({1, max(1, bt - 1), bt, bt + 1, 2 * bt + 3}):
        ref = oracle_run(2, shape, R, c, dt, dims, u0, T)
        got = gpu_run(2, shape, R, c, dt, dims, u0, T, bT=bt, hsn=13, tile=tile)
        assert_bitwise(got, ref, f"tile={tile} bT={bt} T={T}")


@pytest.mark.parametrize("dims", [(1, 1), (3, 5), (2, 130), (9, 193), (5, 257), (40, 380), (1, 999)])
@pytest.mark.parametrize("shape,R,dt,tile,bt", TOP)
def test_wide_parity_degenerate_extents(dims, shape, R, dt, tile, bt):
    c = coeffs_for(2, shape, R, seed=5)
    u0 = inputs.field(dims, R, 3, dt)
    T = 2 * bt + 1
    ref = oracle_run(2, shape, R, c, dt, dims, u0, T)
    for hsn in (0, 1, 4):
        got = gpu_run(2, shape, R, c, dt, dims, u0, T, bT=bt, hsn=hsn, tile=tile)
        assert_bitwise(got, ref, f"dims={dims} tile={tile} hsn={hsn}")


@pytest.mark.parametrize("shape,R,dt,tile,bt,post", DIV_CASES)
def test_wide_division_parity(shape, R, dt, tile, bt, post):
    """Division-type stencils (Table 4, j2d5pt) on the wide tiles, both forms."""
    d = 7.0
    dims = (37, 650)
    c = inputs.normalised_coeffs(inputs.coeff_count(2, shape, R), 0) * d
    u0 = inputs.field(dims, R, 1, dt)
    t = np.float32 if dt == "f32" else np.float64
    form = oracle.POST_DIV if post == "div" else oracle.POST_MUL_RCP
    with an5d.Plan(2, shape, R, c, dt, dims, divisor=d, post=post) as plan:
        for T in sorted({1, bt, bt + 1, 2 * bt + 3}):
            ref = oracle.run_div(dt, 2, shape, R, np.asarray(c).astype(t), d, form, dims, u0, T)
            got = gpu_run(2, shape, R, c, dt, dims, u0, T, bT=bt, hsn=11, plan=plan, tile=tile)
            assert_bitwise(got, ref, f"{post} tile={tile} bT={bt} T={T}")


def test_tile_selection_and_fallback():
    dims = (64, 640)
    c = coeffs_for(2, STAR, 1)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        plan.set_config(5, 0)
        plan.set_tile(192)
        assert plan.config()["tile_x"] == 192
        plan.set_tile(0)
        assert plan.config()["tile_x"] == 128
        plan.set_tile(192)
        # a degree the variant does not build returns the plan to the default width
        plan.set_config(10, 0)
        assert plan.config()["tile_x"] == 128 and plan.config()["bT"] == 10
        with pytest.raises(an5d.An5dError) as e:
            plan.set_tile(192)      # no 192-wide kernel at bT = 10
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
        with pytest.raises(an5d.An5dError) as e:
            plan.set_tile(256)      # no such width
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
    with an5d.Plan(2, inputs.BOX, 1, coeffs_for(2, inputs.BOX, 1), "f32", dims) as plan:
        plan.set_config(10, 0)
        with pytest.raises(an5d.An5dError) as e:
            plan.set_tile(192)      # the wide box kernels stop at bT = 5
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED


def test_tuned_choice_is_exact():
    """Whatever variant the tuner keeps on a mid-size grid gives the oracle's bits."""
    dims = (512, 2000)
    c = coeffs_for(2, STAR, 1, seed=2)
    u0 = inputs.field(dims, 1, 4, "f32")
    T = 23
    ref = oracle_run(2, STAR, 1, c, "f32", dims, u0, T)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        plan.tune(topk=2, T_probe=10)
        got = gpu_run(2, STAR, 1, c, "f32", dims, u0, T, plan=plan)
    assert_bitwise(got, ref, "tuned")


@pytest.mark.parametrize("shape,R,bt", [(STAR, 1, 5), (STAR, 2, 3), (inputs.BOX, 1, 4)])
def test_adjoint_on_wide_tile_plan(shape, R, bt):
    """The adjoint recomputes the forward with the plan's own kernel and runs
    its transposed sweeps on default-width kernels: a plan on a wide tile
    variant gives exactly the gradients of the same plan on the default one."""
    import torch
    dims = (60, 420)
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = inputs.target_field(dims, R, 2, "f32")
    inner = tuple(slice(R, R + d) for d in dims)
    T = 2 * bt + 1
    out = {}
    for tile in (0, 192):
        with an5d.Plan(2, shape, R, c, "f32", dims) as plan:
            plan.set_config(bt, 19)
            plan.set_tile(tile)
            assert plan.config()["tile_x"] == (tile or 128)
            x = torch.from_numpy(u0).cuda()
            y = torch.empty_like(x)
            plan.run(x, y, T)
            gT = torch.zeros_like(x)
            gT[inner] = y[inner] - torch.from_numpy(tg).cuda()[inner]
            gu = torch.empty_like(x)
            gc = an5d.an5d_run_adjoint(plan.handle, x, gT, gu, T)[:n]
            torch.cuda.synchronize()
            out[tile] = (y.cpu().numpy(), gu.cpu().numpy(), gc.copy())
    assert_bitwise(out[192][0], out[0][0], "forward")
    assert_bitwise(out[192][1], out[0][1], "grad u0")
    assert_bitwise(out[192][2], out[0][2], "grad c")
