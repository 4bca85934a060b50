"""GPU parity of the batched form: every grid of a batch gets the bits of
the single-grid method (the CPU oracle for small batches, the oracle-exact
single-grid GPU path for the full 512-grid batch)."""
import numpy as np
import pytest

from paper_2001_01473_gb300 import an5d, inputs
from _gpu_util import assert_bitwise, oracle_run

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX


def _grids_from(descs, seed0=100):
    grids = []
    for i, d in enumerate(descs):
        n = inputs.coeff_count(2, d.shape, d.radius)
        grids.append((d.shape, d.radius, inputs.normalised_coeffs(n, seed0 + i), d.ny, d.nx, d.T))
    return grids


def _inputs(grids, seed0=500):
    import torch
    xs = [torch.from_numpy(inputs.field((g[3], g[4]), g[1], seed0 + i, "f32")).cuda()
          for i, g in enumerate(grids)]
    return xs, [torch.empty_like(x) for x in xs]


def _check_vs_oracle(grids, xs, ys):
    for i, g in enumerate(grids):
        shape, R, c, ny, nx, T = g
        ref = oracle_run(2, shape, R, c, "f32", (ny, nx), xs[i].cpu().numpy(), T)
        assert_bitwise(ys[i].cpu().numpy(), ref, f"grid {i} {g[:2]} {ny}x{nx} T={T}")


SMALL = inputs.batch_descs(n=24, seed=7, side_lo=20, side_hi=400, t_lo=0, t_hi=40)


@pytest.mark.parametrize("degrees", [None, (1, 1, 1, 1), (4, 2, 4, 2), (8, 4, 8, 4)])
def test_batch_small_vs_oracle(degrees):
    import torch
    grids = _grids_from(SMALL)
    with an5d.Batch(grids) as b:
        if degrees:
            b.set_degrees(degrees)
        xs, ys = _inputs(grids)
        b.run(xs, ys)
        torch.cuda.synchronize()
        assert b.status() == 0, an5d.an5d_batch_last_error()
        _check_vs_oracle(grids, xs, ys)


@pytest.mark.parametrize("tiles", [(192, 192, 192, 192), (192, 128, 128, 192)])
def test_batch_wide_tiles_vs_oracle(tiles):
    """192-cell tiles at each class's wide degree (4 for radius 1, 2 for
    radius 2; the remaining steps at degree 1 on the same tiles) give the
    oracle's bits; the info reports the width in force per class."""
    import torch
    grids = _grids_from(SMALL)
    with an5d.Batch(grids) as b:
        b.set_degrees((4, 2, 4, 2))
        b.set_tiles(tiles)
        assert b.info()["class_tile_x"] == list(tiles)
        xs, ys = _inputs(grids)
        b.run(xs, ys)
        torch.cuda.synchronize()
        assert b.status() == 0, an5d.an5d_batch_last_error()
        _check_vs_oracle(grids, xs, ys)
        b.set_degrees((8, 4, 1, 1))          # not the wide degrees: 128-cell tiles
        assert b.info()["class_tile_x"] == [128, 128, 128, 128]
        with pytest.raises(an5d.An5dError) as e:
            b.set_tiles((256, 128, 128, 128))
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED


def test_batch_graph_replay_and_new_buffers():
    import torch
    grids = _grids_from(SMALL[:10])
    with an5d.Batch(grids) as b:
        xs, ys = _inputs(grids)
        b.run(xs, ys)
        b.run(xs, ys)                        # graph replay, same buffers
        torch.cuda.synchronize()
        assert b.status() == 0
        _check_vs_oracle(grids, xs, ys)
        xs2, ys2 = _inputs(grids, seed0=900)  # new buffers: table rebuilt
        b.run(xs2, ys2)
        torch.cuda.synchronize()
        assert b.status() == 0
        _check_vs_oracle(grids, xs2, ys2)


def test_batch_rejects_bad_input():
    with pytest.raises(an5d.An5dError):
        an5d.Batch([(STAR, 3, np.ones(13), 10, 10, 5)])
    import torch
    grids = _grids_from(SMALL[:2])
    with an5d.Batch(grids) as b:
        xs, ys = _inputs(grids)
        with pytest.raises(an5d.An5dError) as e:
            b.run(xs, [xs[0], ys[1]])
        assert e.value.status == an5d.AN5D_ERR_ALIAS


def test_batch_full_config_vs_single_grid_path():
    """512 grids, sides log-uniform in [128, 4096], star/box R1-2, T in [10, 500]:
    every grid equal to the single-grid method's result, bit for bit."""
    import torch
    grids = _grids_from(inputs.batch_descs())
    with an5d.Batch(grids) as b:
        info = b.tune()
        xs, ys = _inputs(grids)
        b.run(xs, ys)
        torch.cuda.synchronize()
        assert b.status() == 0, an5d.an5d_batch_last_error()
    bad = []
    for i, g in enumerate(grids):
        shape, R, c, ny, nx, T = g
        with an5d.Plan(2, shape, R, c, "f32", (ny, nx)) as p:
            ref = torch.empty_like(xs[i])
            p.run(xs[i], ref, T)
            torch.cuda.synchronize()
        if not torch.equal(ref, ys[i]):
            bad.append(i)
    assert not bad, (bad[:10], info)


def test_batch_tune_on_caller_buffers_then_oracle():
    """Tuning on the caller's buffers (whole-batch timing) leaves a plan whose
    result is still every grid's oracle result; remainders T mod bT are split
    over the built degrees."""
    import torch
    grids = _grids_from(SMALL, seed0=300)
    with an5d.Batch(grids) as b:
        xs, ys = _inputs(grids, seed0=900)
        info = b.tune(None, xs, ys)
        assert all(d in (1, 2, 4, 8) for d in info["class_bt"])
        b.run(xs, ys)
        torch.cuda.synchronize()
        assert b.status() == 0, an5d.an5d_batch_last_error()
    _check_vs_oracle(grids, xs, ys)
