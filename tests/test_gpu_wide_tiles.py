"""GPU parity of the wider 2D tile variants (6 cells per lane) against the
CPU oracle, through the C ABI.  The variants compute the same per-cell fma
chains as the default kernels, so every comparison is bit for bit, including
runs whose remainder pass falls back to a default-width kernel."""
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from paper_2001_01473_gb300.kernels import KERNELS_2D_WIDE
from _gpu_util import assert_bitwise, coeffs_for, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
STAR = inputs.STAR
SH = {"SH_STAR": inputs.STAR, "SH_BOX": inputs.BOX}
DT = {"DT_F32": "f32", "DT_F64": "f64"}

CASES = [(SH[sh], r, DT[dt], 32 * v, bt)
         for sh, r, bts, _s, _m, dt, v in KERNELS_2D_WIDE for bt in bts]


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
@pytest.mark.parametrize("tile", sorted({t for _, _, _, t, _ in CASES}))
def test_wide_parity_degenerate_extents(dims, tile):
    bt = max(b for _, _, _, t, b in CASES if t == tile)
    c = coeffs_for(2, STAR, 1, seed=5)
    u0 = inputs.field(dims, 1, 3, "f32")
    T = 2 * bt + 1
    ref = oracle_run(2, STAR, 1, c, "f32", dims, u0, T)
    for hsn in (0, 1, 4):
        got = gpu_run(2, STAR, 1, c, "f32", dims, u0, T, bT=bt, hsn=hsn, tile=tile)
        assert_bitwise(got, ref, f"dims={dims} tile={tile} hsn={hsn}")


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
        with pytest.raises(an5d.An5dError) as e:
            plan.set_tile(192)      # built for the radius-1 star only
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
