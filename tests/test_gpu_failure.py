"""Failure path on the GPU without a fault: injected waits that can never
complete must give up (about one second), let the kernel return, report
AN5D_ERR_TIMEOUT through the status call, and leave the context usable."""
import time

import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from _gpu_util import assert_bitwise, coeffs_for, oracle_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX


def test_sweep_wait_timeout_reports_status_and_context_survives():
    import torch
    dims = (64, 300)
    c = coeffs_for(2, STAR, 1)
    u0 = inputs.field(dims, 1, 1, "f32")
    x = torch.from_numpy(u0).cuda()
    y = torch.empty_like(x)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        plan.set_config(4, 16)
        an5d.an5d_plan_inject_stall(plan.handle, True)
        t0 = time.time()
        plan.run(x, y, 4)                     # one pass
        st = plan.status()                    # synchronises
        dt = time.time() - t0
        assert st == an5d.AN5D_ERR_TIMEOUT
        assert 0.5 < dt < 30.0
        an5d.an5d_plan_inject_stall(plan.handle, False)
        plan.run(x, y, 9)                     # the context and the plan still work
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert_bitwise(y.cpu().numpy(), oracle_run(2, STAR, 1, c, "f32", dims, u0, 9), "after")


def test_batch_wait_timeout_reports_status():
    import torch
    descs = inputs.batch_descs(n=6, seed=9, side_lo=40, side_hi=200, t_lo=5, t_hi=20)
    grids = []
    for i, d in enumerate(descs):
        n = inputs.coeff_count(2, d.shape, d.radius)
        grids.append((d.shape, d.radius, inputs.normalised_coeffs(n, i), d.ny, d.nx, d.T))
    xs = [torch.from_numpy(inputs.field((g[3], g[4]), g[1], 30 + i, "f32")).cuda()
          for i, g in enumerate(grids)]
    ys = [torch.empty_like(x) for x in xs]
    with an5d.Batch(grids) as b:
        an5d.an5d_batch_inject_stall(b.handle, True)
        b.run(xs, ys)
        assert b.status() == an5d.AN5D_ERR_TIMEOUT
        an5d.an5d_batch_inject_stall(b.handle, False)
        b.run(xs, ys)
        torch.cuda.synchronize()
        assert b.status() == 0
        for i, g in enumerate(grids):
            ref = oracle_run(2, g[0], g[1], g[2], "f32", (g[3], g[4]), xs[i].cpu().numpy(), g[5])
            assert_bitwise(ys[i].cpu().numpy(), ref, f"grid {i}")
