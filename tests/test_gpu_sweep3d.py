"""GPU parity of the 3D (2.5D-blocked) sweeps against the CPU oracle, through
the C ABI, bit for bit."""
import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from paper_2001_01473_gb300.kernels import (KERNELS_3D, KERNELS_3D_BOX1, KERNELS_3D_STAR, KERNELS_3D_STAR_NARROW,
                                            KERNELS_3D_VARIANTS)
from _gpu_util import assert_bitwise, coeffs_for, gpu_run, oracle_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX
DT = {"DT_F32": "f32", "DT_F64": "f64", "DT_F16S": "f16", "DT_F32C": "f32c"}
SH = {"SH_STAR": STAR, "SH_BOX": BOX}

BUILT = {}
for _sh, _r, _bts, _s, _m, _dt, _nw in KERNELS_3D:
    BUILT.setdefault((SH[_sh], _r, DT[_dt]), []).extend(list(_bts))
for _r, _bts, _nw, _rw in KERNELS_3D_STAR:
    BUILT.setdefault((STAR, _r, "f32"), []).extend(list(_bts))
for _r, _s, _dt, _nw, _rw in KERNELS_3D_BOX1:
    BUILT.setdefault((BOX, _r, DT[_dt]), []).append(1)
CASES = [(shape, R, dt, bt) for (shape, R, dt), bts in sorted(BUILT.items()) for bt in bts]


@pytest.mark.parametrize("shape,R,dt,bt", CASES)
def test_parity_3d_several_tiles_ragged(shape, R, dt, bt):
    dims = (23, 45, 141)       # ragged tails on every axis, several tiles in x and y
    c = coeffs_for(3, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    for T in sorted({1, bt, bt + 1, 2 * bt + 1}):
        ref = oracle_run(3, shape, R, c, dt, dims, u0, T)
        got = gpu_run(3, shape, R, c, dt, dims, u0, T, bT=bt, hsn=7)
        assert_bitwise(got, ref, f"3d shape={shape} R={R} {dt} bT={bt} T={T}")


VARIANT_CASES = ([(STAR, r, "f32", 32 * v, bt) for r, bts, _nw, _rw, v in KERNELS_3D_STAR_NARROW for bt in bts] +
                 [(SH[sh], r, DT[dt], 32 * v, bt) for sh, r, bts, _s, _m, dt, _nw, v, _rw, posts in KERNELS_3D_VARIANTS
                  if "POST_NONE" in posts for bt in bts])


@pytest.mark.parametrize("shape,R,dt,tile,bt", VARIANT_CASES)
def test_parity_3d_tile_variant(shape, R, dt, tile, bt):
    # the 64-cell-wide tiles: several tiles in x and y with ragged tails,
    # stream blocks of 5 planes, and a degenerate thin grid
    c = coeffs_for(3, shape, R, seed=7)
    for dims in [(21, 150, 131), (4, 3, 61)]:
        u0 = inputs.field(dims, R, 2, dt)
        for T in sorted({1, bt, bt + 1, 2 * bt + 1}):
            ref = oracle_run(3, shape, R, c, dt, dims, u0, T)
            got = gpu_run(3, shape, R, c, dt, dims, u0, T, bT=bt, hsn=5, tile=tile)
            assert_bitwise(got, ref, f"3d shape={shape} R={R} tile={tile} bT={bt} T={T} dims={dims}")


@pytest.mark.parametrize("dims", [(1, 1, 1), (1, 5, 300), (40, 1, 1), (3, 40, 7), (9, 33, 129),
                                  (6, 26, 122)])
@pytest.mark.parametrize("shape,R,bt", [(STAR, 1, 3), (BOX, 1, 2), (STAR, 4, 1), (STAR, 1, 4)])
def test_parity_3d_degenerate_extents(dims, shape, R, bt):
    c = coeffs_for(3, shape, R, seed=5)
    u0 = inputs.field(dims, R, 3, "f32")
    T = 2 * bt + 1
    ref = oracle_run(3, shape, R, c, "f32", dims, u0, T)
    for hsn in (0, 1, 3):
        got = gpu_run(3, shape, R, c, "f32", dims, u0, T, bT=bt, hsn=hsn)
        assert_bitwise(got, ref, f"dims={dims} hsn={hsn}")


def _window_reference_3d(shape, R, c, dt, u0, T, p):
    h = T * R + R
    lo = [max(0, q - h) for q in p]
    hi = [min(n, q + h + 1) for q, n in zip(p, u0.shape)]
    win = np.ascontiguousarray(u0[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
    wd = tuple(s - 2 * R for s in win.shape)
    out = oracle_run(3, shape, R, c, dt, wd, win, T)
    return out[p[0] - lo[0], p[1] - lo[1], p[2] - lo[2]]


@pytest.mark.parametrize("shape,R,dt", [(STAR, 1, "f32"), (BOX, 1, "f32"), (STAR, 2, "f64")])
def test_full_size_3d_sampled(shape, R, dt):
    import torch
    n = 512
    dims = (n, n, n)
    c = coeffs_for(3, shape, R)
    u0 = inputs.field(dims, R, 1, dt)
    T = 10
    with an5d.Plan(3, shape, R, c, dt, dims) as plan:
        plan.tune(topk=3, T_probe=6)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
        cfg = plan.config()
        got_all = None
    rng = np.random.default_rng(11)
    tsx = cfg["tile_x"] - 2 * cfg["bT"] * R
    tsy = cfg["tile_y"] - 2 * cfg["bT"] * R
    pts = [(R, R, R), (n + R - 1, n + R - 1, n + R - 1), (R + cfg["hsn"], R + tsy, R + tsx),
           (R + cfg["hsn"] - 1, R + tsy - 1, R + tsx - 1), (n // 2, R, n + R - 1)]
    pts += [tuple(int(v) for v in rng.integers(R, n + R, 3)) for _ in range(16)]
    for p in pts:
        want = _window_reference_3d(shape, R, c, dt, u0, T, p)
        got = y[p].item()
        assert got == want, (p, got, want, cfg)
    del got_all


def test_full_size_3d_constant_field_T200():
    import torch
    n = 512
    c = np.array([0.25] + [0.125] * 6)   # dyadic, sums to 1
    with an5d.Plan(3, STAR, 1, c, "f32", (n, n, n)) as plan:
        plan.tune(topk=3, T_probe=6)
        x = torch.full(inputs.padded_shape((n, n, n), 1), 0.75, device="cuda")
        y = torch.empty_like(x)
        plan.run(x, y, 200)
        torch.cuda.synchronize()
        assert plan.status() == 0
        assert bool((y == 0.75).all())


@pytest.mark.parametrize("dt", ["f32c", "f16"])
def test_full_size_3d_heat_precision_forms_sampled(dt):
    import torch
    n = 512
    dims = (n, n, n)
    c = inputs.heat_coeffs(3)
    u0 = inputs.gaussian_bump(dims, 1, 1, dt if dt != "f32c" else "f32")
    T = 8
    with an5d.Plan(3, STAR, 1, c, dt, dims) as plan:
        plan.tune(topk=3, T_probe=4)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        torch.cuda.synchronize()
        assert plan.status() == 0
    rng = np.random.default_rng(5)
    pts = [(1, 1, 1), (n // 2, n // 2, n // 2)] + \
          [tuple(int(v) for v in rng.integers(1, n + 1, 3)) for _ in range(8)]
    for p in pts:
        want = _window_reference_3d(STAR, 1, c, dt, u0, T, p)
        got = y[p].item()
        assert got == float(want), (p, got, want)


@pytest.mark.parametrize("shape,R,bt", [(STAR, 1, 3), (STAR, 1, 1), (BOX, 1, 3), (STAR, 1, 4),
                                        (STAR, 2, 1), (STAR, 2, 2)])
@pytest.mark.parametrize("rest", ["narrow", "narrow+1", "one", "none"])
def test_narrow_last_column(shape, R, bt, rest):
    """A ragged remainder of at most one narrow tile's compute width runs on
    the narrow kernel (R cells per lane: 32 or 64 cells wide; two launches
    per pass); one cell wider, or none at all, stays on full tiles.
    Bit-exact either way."""
    tsx, ts_narrow = 128 - 2 * bt * R, 32 * R - 2 * bt * R
    # two full columns plus the remainder; tiles start on even columns, so
    # when R (bT - 1) is odd the first compute region starts one column early
    # (on the halo column) and the tiles cover one column more than the
    # interior
    early = (R * (bt - 1)) & 1
    rest = {"narrow": ts_narrow, "narrow+1": ts_narrow + 1, "one": 1, "none": 0}[rest]
    nx = 2 * tsx + rest - early
    dims = (9, 30, nx)
    c = coeffs_for(3, shape, R, seed=3)
    u0 = inputs.field(dims, R, 2, "f32")
    T = 2 * bt + 1
    with an5d.Plan(3, shape, R, c, "f32", dims) as plan:
        plan.set_config(bt, 4)
        plan.set_tile(0)  # the default 128-cell tile (the narrow column belongs to it)
        cfg = plan.config()
        assert cfg["launches_per_pass"] == (2 if 0 < rest <= ts_narrow else 1), (cfg, rest)
        # 2 halo copies + 3 passes (2 of bT, 1 of 1 step), a narrow launch more where split
        n = plan.launches(T)
        assert 5 + 2 * (cfg["launches_per_pass"] - 1) <= n <= 8, n
        assert cfg["ctas"] > 0
        got = gpu_run(3, shape, R, c, "f32", dims, u0, T, plan=plan)
    ref = oracle_run(3, shape, R, c, "f32", dims, u0, T)
    assert_bitwise(got, ref, f"nx={nx} bT={bt}")


def test_narrow_column_runs_in_a_captured_graph():
    """A split pass forks its narrow launch onto the plan's second stream and
    joins it back; captured into a CUDA graph (torch's capture on the
    caller's stream) and replayed on new contents of the captured input, it
    still gives the oracle's bits, and a run on the legacy default stream
    does too."""
    import torch
    R, bt = 1, 3
    dims = (11, 28, 2 * (128 - 2 * bt * R) + 20)
    c = coeffs_for(3, STAR, R, seed=6)
    T = 2 * bt + 2
    with an5d.Plan(3, STAR, R, c, "f32", dims) as plan:
        plan.set_config(bt, 5)
        plan.set_tile(0)  # the default 128-cell tile and its narrow last column
        assert plan.config()["launches_per_pass"] == 2
        x = torch.empty(inputs.padded_shape(dims, R), dtype=torch.float32, device="cuda")
        y = torch.empty_like(x)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            x.copy_(torch.from_numpy(inputs.field(dims, R, 1, "f32")))
            plan.run(x, y, T)                       # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            plan.run(x, y, T)
        for seed in (2, 3):
            u0 = inputs.field(dims, R, seed, "f32")
            x.copy_(torch.from_numpy(u0))
            g.replay()
            torch.cuda.synchronize()
            assert plan.status() == 0
            assert_bitwise(y.cpu().numpy(), oracle_run(3, STAR, R, c, "f32", dims, u0, T), f"replay {seed}")
        u0 = inputs.field(dims, R, 4, "f32")
        x.copy_(torch.from_numpy(u0))
        torch.cuda.synchronize()
        plan.run(x, y, T, stream=0)                 # legacy default stream
        torch.cuda.synchronize()
        assert_bitwise(y.cpu().numpy(), oracle_run(3, STAR, R, c, "f32", dims, u0, T), "default stream")
