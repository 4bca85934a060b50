"""GPU test of an5d_run_noalloc, the entry point for callers that cannot call
cudaMalloc (frameworks that give all device memory to their own pool, loops
that must not stall on an allocation).  It must give the same bits as the
plan-based an5d_run, call after call, although every call reuses one shared
device array for its ping-pong buffer and status word.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from _gpu_util import assert_bitwise, coeffs_for

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX

CASES = [
    # (ndim, shape, R, dtype, dims, T): several passes, so the shared array is used
    (2, STAR, 1, "f32", (200, 333), 37),
    (2, BOX, 2, "f64", (90, 150), 11),
    (2, STAR, 1, "f16", (64, 300), 25),
    (2, BOX, 1, "f32c", (70, 260), 9),
    (2, STAR, 3, "f32", (31, 129), 1),     # one pass
    (2, STAR, 1, "f32", (16, 16), 0),      # copy only
    # 3D: at every degree 1-3 of the radius-2 star a 136-wide grid is one
    # full 128-cell tile column plus a remainder that fits the narrow
    # last-column kernel, which the allocation-free call runs after the main
    # launch on the same stream
    (3, STAR, 2, "f32", (21, 40, 136), 7),
    (3, BOX, 1, "f64", (13, 30, 70), 4),   # 3D box, FP64
]


def _plan_run(ndim, shape, R, c, dt, dims, x, T):
    import torch
    y = torch.empty_like(x)
    with an5d.Plan(ndim, shape, R, c, dt, dims) as plan:
        plan.run(x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
    return y


def _noalloc_run(ndim, shape, R, c, dt, dims, x, T):
    import torch
    y = torch.full_like(x, float("nan"))
    an5d.an5d_run_noalloc(ndim, shape, R, c, dt, dims, x, y, T)
    torch.cuda.synchronize()
    return y


def test_noalloc_matches_plan_run_two_calls_in_a_row():
    import torch
    prepared = []
    for i, (ndim, shape, R, dt, dims, T) in enumerate(CASES):
        c = coeffs_for(ndim, shape, R, seed=i)
        if ndim == 3 and shape == STAR:
            # both calls pick the same configuration; it splits every pass
            with an5d.Plan(ndim, shape, R, c, dt, dims) as plan:
                assert plan.config()["launches_per_pass"] == 2, plan.config()
        u0 = inputs.field(dims, R, 10 + i, dt)
        x = torch.from_numpy(u0).cuda()
        prepared.append((ndim, shape, R, dt, dims, T, c, x,
                         _plan_run(ndim, shape, R, c, dt, dims, x, T).cpu().numpy()))
    for rep in range(2):                       # two calls in a row per case
        for ndim, shape, R, dt, dims, T, c, x, ref in prepared:
            got = _noalloc_run(ndim, shape, R, c, dt, dims, x, T).cpu().numpy()
            assert_bitwise(got, ref, f"call {rep} dims={dims} {dt} T={T}")
    # and back to back on the same case
    ndim, shape, R, dt, dims, T, c, x, ref = prepared[0]
    a = _noalloc_run(ndim, shape, R, c, dt, dims, x, T).cpu().numpy()
    b = _noalloc_run(ndim, shape, R, c, dt, dims, x, T).cpu().numpy()
    assert_bitwise(a, ref, "first of two")
    assert_bitwise(b, ref, "second of two")


def test_noalloc_rejects_grids_above_its_limit():
    import torch
    limit = 32 << 20
    dims = (3000, 3000)                          # 9,012,004 floats = 36 MB > limit
    assert (dims[0] + 2) * (dims[1] + 2) * 4 > limit
    x = torch.zeros(inputs.padded_shape(dims, 1), device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(an5d.An5dError) as e:
        an5d.an5d_run_noalloc(2, STAR, 1, np.ones(5) / 5, "f32", dims, x, y, 4)
    assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
    assert "limit" in str(e.value)
