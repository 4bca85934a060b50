"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the CPU oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_2001_01473_gb300 import an5d, inputs


def coeffs_for(ndim, shape, R, seed=0):
    return inputs.normalised_coeffs(inputs.coeff_count(ndim, shape, R), seed)


def oracle_run(ndim, shape, R, c, dtype, dims, u0, T):
    if dtype == "f64":
        return oracle.run_f64(ndim, shape, R, c, dims, u0, T)
    c32 = np.asarray(c, np.float64).astype(np.float32)
    if dtype == "f32":
        return oracle.run_f32(ndim, shape, R, c32, dims, u0, T)
    if dtype == "f16":
        return oracle.run_f16s(ndim, shape, R, c32, dims, u0, T)
    if dtype == "f32c":
        return oracle.run_dot2(ndim, shape, R, c32, dims, u0, T)
    raise ValueError(dtype)


def gpu_run(ndim, shape, R, c, dtype, dims, u0, T, bT=None, hsn=0, plan=None, tile=0):
    """Run through the C ABI.  With bT or hsn given, the plan is forced to that
    configuration on tile variant `tile` (0 = the default kernel width)."""
    import torch
    own = plan is None
    if own:
        plan = an5d.Plan(ndim, shape, R, c, dtype, dims)
    try:
        if bT is not None or hsn:
            plan.set_config(bT or 0, hsn)
            plan.set_tile(tile)
        x = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        torch.cuda.synchronize()
        st = plan.status()
        assert st == 0, f"plan status {st}: {an5d.an5d_last_error()}"
        return y.cpu().numpy()
    finally:
        if own:
            plan.close()


def assert_bitwise(got, ref, what=""):
    g = np.ascontiguousarray(got)
    r = np.ascontiguousarray(ref)
    assert g.shape == r.shape, (g.shape, r.shape)
    gb = g.view(np.uint8).reshape(-1, g.itemsize)
    rb = r.view(np.uint8).reshape(-1, r.itemsize)
    same = np.all(gb == rb, axis=1).reshape(g.shape)
    if not same.all():
        bad = np.argwhere(~same)
        i = tuple(bad[0])
        raise AssertionError(f"{what}: {len(bad)} of {g.size} cells differ; first at {i}: "
                             f"gpu={g[i]!r} oracle={r[i]!r}")
