"""GPU parity of the 2D plain method and precision forms against the CPU
oracle, through the C ABI.  FP32/FP64 plain, binary16 storage and Dot2 are
all deterministic definitions, so every comparison is bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs
from paper_2001_01473_gb300.kernels import KERNELS_2D
from _gpu_util import assert_bitwise, coeffs_for, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX
DT = {"DT_F32": "f32", "DT_F64": "f64", "DT_F16S": "f16", "DT_F32C": "f32c"}
SH = {"SH_STAR": STAR, "SH_BOX": BOX}

BUILT = {}
for _sh, _r, _bts, _s, _m, _dt in KERNELS_2D:
    BUILT[(SH[_sh], _r, DT[_dt])] = list(_bts)


def _cases():
    # every compiled degree of every (stencil, dtype): the tuner may pick any
    return [(shape, R, dt, bt) for (shape, R, dt), bts in sorted(BUILT.items()) for bt in bts]


@pytest.mark.parametrize("shape,R,dt,bt", _cases())
def test_parity_several_tiles_ragged(shape, R, dt, bt):
    dims = (61, 301)           # 3+ x-tiles, ragged tail in x and y
    c = coeffs_for(2, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    for T in sorted({1, max(1, bt - 1), bt, bt + 1, 2 * bt + 3}):
        ref = oracle_run(2, shape, R, c, dt, dims, u0, T)
        got = gpu_run(2, shape, R, c, dt, dims, u0, T, bT=bt, hsn=17)
        assert_bitwise(got, ref, f"shape={shape} R={R} {dt} bT={bt} T={T}")


@pytest.mark.parametrize("dims", [(1, 1), (1, 517), (433, 1), (3, 5), (2, 130), (9, 108),
                                  (9, 109), (40, 216), (5, 129)])
@pytest.mark.parametrize("shape,R,bt", [(STAR, 1, 10), (BOX, 2, 6), (STAR, 4, 4)])
def test_parity_degenerate_extents(dims, shape, R, bt):
    c = coeffs_for(2, shape, R, seed=5)
    u0 = inputs.field(dims, R, 3, "f32")
    T = 2 * bt + 1
    ref = oracle_run(2, shape, R, c, "f32", dims, u0, T)
    for hsn in (0, 1, 4):
        got = gpu_run(2, shape, R, c, "f32", dims, u0, T, bT=bt, hsn=hsn)
        assert_bitwise(got, ref, f"dims={dims} hsn={hsn}")


def test_t0_copies_and_halo_kept():
    dims = (33, 200)
    c = coeffs_for(2, STAR, 2)
    u0 = inputs.field(dims, 2, 1, "f32")
    assert_bitwise(gpu_run(2, STAR, 2, c, "f32", dims, u0, 0), u0, "T=0")
    got = gpu_run(2, STAR, 2, c, "f32", dims, u0, 9, bT=4)
    mask = np.ones_like(u0, bool)
    mask[2:-2, 2:-2] = False
    assert_bitwise(got[mask], u0[mask], "halo")


def test_bt_invariance_default_config():
    """The model-chosen and the tuned configuration give the same bits."""
    import torch
    dims = (257, 1031)
    c = coeffs_for(2, BOX, 1)
    u0 = inputs.field(dims, 1, 4, "f32")
    T = 23
    ref = oracle_run(2, BOX, 1, c, "f32", dims, u0, T)
    with an5d.Plan(2, BOX, 1, c, "f32", dims) as plan:
        assert_bitwise(gpu_run(2, BOX, 1, c, "f32", dims, u0, T, plan=plan), ref, "default")
        plan.tune(topk=3, T_probe=10)
        assert_bitwise(gpu_run(2, BOX, 1, c, "f32", dims, u0, T, plan=plan), ref, "tuned")
    torch.cuda.synchronize()


def test_run_errors():
    import torch
    dims = (16, 40)
    c = coeffs_for(2, STAR, 1)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        x = torch.zeros(inputs.padded_shape(dims, 1), device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(an5d.An5dError) as e:
            plan.run(x, x, 3)
        assert e.value.status == an5d.AN5D_ERR_ALIAS
        with pytest.raises(an5d.An5dError) as e:
            plan.run(x, y, -1)
        assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
        big = torch.zeros(x.numel() + 8, device="cuda")
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_run(plan.handle, big.data_ptr() + 4, y.data_ptr(), 3)
        assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
        with pytest.raises(an5d.An5dError) as e:
            plan.set_config(99, 0)
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED


def test_run_host_matches_device_run():
    dims = (100, 500)
    c = coeffs_for(2, STAR, 1)
    u0 = inputs.field(dims, 1, 1, "f32")
    ref = oracle_run(2, STAR, 1, c, "f32", dims, u0, 21)
    with an5d.Plan(2, STAR, 1, c, "f32", dims) as plan:
        out = np.empty_like(u0)
        plan.run_host(u0, out, 21)
        assert_bitwise(out, ref, "run_host")


# ---------------------------------------------------------------------------
# Full-size (16384^2) checks in the benchmark's launch configuration.

def _window_reference(shape, R, c, dt, u0, T, y, x):
    """Oracle value of cell (y, x) after T steps from the light-cone window.

    A cell depends only on cells within T*R per axis; a window whose own
    R-wide border is at least that far away (or is the true halo) evolves
    that cell exactly as the full grid does."""
    ny, nx = u0.shape
    h = T * R + R
    y0, y1 = max(0, y - h), min(ny, y + h + 1)
    x0, x1 = max(0, x - h), min(nx, x + h + 1)
    win = np.ascontiguousarray(u0[y0:y1, x0:x1])
    wd = (win.shape[0] - 2 * R, win.shape[1] - 2 * R)
    out = oracle_run(2, shape, R, c, dt, wd, win, T)
    return out[y - y0, x - x0]


@pytest.mark.parametrize("shape,R,dt", [(STAR, 1, "f32"), (BOX, 2, "f32"), (STAR, 2, "f64")])
def test_full_size_sampled(shape, R, dt):
    import torch
    n = 16384
    dims = (n, n)
    c = coeffs_for(2, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    T = 50
    with an5d.Plan(2, shape, R, c, dt, dims) as plan:
        plan.tune(topk=3, T_probe=20)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
        cfg = plan.config()
    tile = cfg["tile_x"] - 2 * cfg["bT"] * R
    rng = np.random.default_rng(7)
    pts = [(R, R), (R, n + R - 1), (n + R - 1, R), (n + R - 1, n + R - 1),
           (n // 2, R + tile - 1), (n // 2, R + tile), (R + cfg["hsn"], n // 3),
           (R + cfg["hsn"] - 1, R + 2 * tile)]
    pts += [tuple(int(v) for v in rng.integers(R, n + R, 2)) for _ in range(24)]
    for (yy, xx) in pts:
        want = _window_reference(shape, R, c, dt, u0, T, yy, xx)
        got = y[yy, xx].item()
        assert got == want or (np.isnan(got) and np.isnan(want)), (yy, xx, got, want, cfg)


def test_full_size_constant_field_T1000():
    """Dyadic coefficients summing to 1 keep a dyadic constant exactly, at the
    benchmark's size and length (16384^2, T = 1000)."""
    import torch
    n = 16384
    c = np.array([0.5, 0.125, 0.125, 0.125, 0.125])
    with an5d.Plan(2, STAR, 1, c, "f32", (n, n)) as plan:
        plan.tune(topk=3, T_probe=20)
        x = torch.full(inputs.padded_shape((n, n), 1), 0.75, device="cuda")
        y = torch.empty_like(x)
        plan.run(x, y, 1000)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert bool((y == 0.75).all())


@pytest.mark.parametrize("shape,R,dt", [(BOX, 1, "f32c"), (BOX, 1, "f16")])
def test_full_size_precision_forms_sampled(shape, R, dt):
    """The precision-form kernels at 16384^2 in their tuned configuration,
    checked cell by cell against the oracle's Dot2 / binary16 forms."""
    import torch
    n = 16384
    dims = (n, n)
    c = coeffs_for(2, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    T = 30
    with an5d.Plan(2, shape, R, c, dt, dims) as plan:
        plan.tune(topk=3, T_probe=10)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
        cfg = plan.config()
    rng = np.random.default_rng(3)
    pts = [(R, R), (n + R - 1, n // 2), (R + cfg["hsn"], R + 100)]
    pts += [tuple(int(v) for v in rng.integers(R, n + R, 2)) for _ in range(12)]
    for (yy, xx) in pts:
        want = _window_reference(shape, R, c, dt, u0, T, yy, xx)
        got = y[yy, xx].item()
        assert got == float(want), (yy, xx, got, want, cfg)
