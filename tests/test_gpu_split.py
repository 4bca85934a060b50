"""GPU parity of the halo-deepened domain split (an5d_run_split): the sweep
run as slabs of the slowest axis with bT R ghost planes and one exchange per
pass gives the single-grid bits, through the C ABI, against the oracle."""
import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from _gpu_util import assert_bitwise, coeffs_for, oracle_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX


@pytest.mark.parametrize("ndim,shape,R,dt,dims,bt,nsub,T", [
    (2, STAR, 1, "f32", (100, 300), 4, 2, 11),
    (2, STAR, 1, "f32", (100, 300), 4, 4, 9),
    (2, BOX, 2, "f32", (61, 140), 3, 3, 7),
    (2, STAR, 2, "f64", (50, 90), 2, 2, 5),
    (3, STAR, 1, "f32", (40, 30, 150), 3, 3, 8),
    (3, BOX, 1, "f32", (24, 20, 40), 2, 2, 5),
    (2, STAR, 1, "f16", (64, 200), 5, 3, 12),
])
def test_split_matches_single_grid(ndim, shape, R, dt, dims, bt, nsub, T):
    import torch
    c = coeffs_for(ndim, shape, R, seed=4)
    u0 = inputs.field(dims, R, 7, dt)
    ref = oracle_run(ndim, shape, R, c, dt, dims, u0, T)
    with an5d.Plan(ndim, shape, R, c, dt, dims) as plan:
        plan.set_config(bt, 0)
        x = torch.from_numpy(u0).cuda()
        y = torch.full_like(x, -1)
        an5d.an5d_run_split(plan.handle, nsub, x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert_bitwise(y.cpu().numpy(), ref, f"split {nsub} {dims} bT={bt} T={T}")
        y2 = torch.full_like(x, -1)
        an5d.an5d_run_split(plan.handle, nsub, x, y2, 0)      # T = 0 copies
        assert torch.equal(y2, x)


def test_split_rejects_thin_slabs():
    import torch
    c = coeffs_for(2, STAR, 1)
    dims = (12, 40)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        plan.set_config(4, 0)
        x = torch.zeros(inputs.padded_shape(dims, 1), device="cuda")
        y = torch.empty_like(x)
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_run_split(plan.handle, 3, x, y, 4)
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED
