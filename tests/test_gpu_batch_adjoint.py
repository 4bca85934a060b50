"""GPU batched adjoint (an5d_adjoint_batch_*): every grid's dL/du_0 and
dL/dc against the FP64 oracle adjoint (relative L2 1e-4, as for the
single-grid adjoint), the halo of dL/du_0 zero, a split into several waves
bit-identical to one wave, repeated runs bit-identical (deterministic sums),
and dL/du_0 bit-identical to the single-grid adjoint's."""
import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX

# (shape, R, ny, nx, T): every class, T = 0, T below, at and off the block
# degree, ragged extents, several x tiles and stream blocks
GRIDS = [(STAR, 1, 70, 300, 11), (STAR, 2, 90, 140, 7), (BOX, 1, 40, 260, 4), (BOX, 2, 300, 130, 5),
         (STAR, 1, 33, 17, 1), (BOX, 1, 5, 9, 9), (STAR, 2, 21, 333, 0), (BOX, 2, 12, 40, 3),
         (STAR, 1, 260, 129, 16), (BOX, 1, 129, 64, 2)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _setup(seed=0):
    import torch
    grids, u0s, gTs, refs = [], [], [], []
    for i, (shape, R, ny, nx, T) in enumerate(GRIDS):
        n = inputs.coeff_count(2, shape, R)
        c = inputs.normalised_coeffs(n, seed + i)
        dims = (ny, nx)
        u0 = inputs.field(dims, R, 100 + i, "f32")
        tg = inputs.target_field(dims, R, 200 + i, "f32")
        grids.append((shape, R, c, ny, nx, T))
        # dL/du_T of 0.5 ||u_T - target||^2 from the FP64 oracle forward
        c32 = c.astype(np.float32).astype(np.float64)
        _loss, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, c32, dims, u0.astype(np.float64),
                                                   tg.astype(np.float64), T)
        uT = oracle.run_f64(2, shape, R, c32, dims, u0.astype(np.float64), T)
        inner = (slice(R, R + ny), slice(R, R + nx))
        gT = np.zeros_like(u0)
        gT[inner] = (uT[inner] - tg[inner].astype(np.float64)).astype(np.float32)
        u0s.append(torch.from_numpy(u0).cuda())
        gTs.append(torch.from_numpy(gT).cuda())
        refs.append((ref_gu, ref_gc, inner, n))
    return grids, u0s, gTs, refs


def test_batch_adjoint_vs_fp64_oracle_and_waves():
    import torch
    grids, u0s, gTs, refs = _setup()
    outs = [torch.full_like(x, 7.0) for x in u0s]
    with an5d.AdjointBatch(grids) as ab:
        assert ab.info()["waves"] == 1
        dc = ab.run(u0s, gTs, outs)
        dc2 = ab.run(u0s, gTs, outs)              # replay of the captured graph
        assert np.array_equal(dc, dc2)
    for i, (ref_gu, ref_gc, inner, n) in enumerate(refs):
        gu = outs[i].cpu().numpy()
        halo = np.ones(gu.shape, bool)
        halo[inner] = False
        assert np.all(gu[halo] == 0.0), i
        assert _rel(gu[inner].astype(np.float64), ref_gu[inner]) < 1e-4, (i, grids[i][:2], grids[i][3:])
        if grids[i][5] == 0:
            assert np.all(dc[i] == 0.0)
        else:
            assert _rel(dc[i][:n], ref_gc) < 1e-4, (i, dc[i][:n], ref_gc)
        assert np.all(dc[i][n:] == 0.0)
    # a budget that forces several waves gives the same bits
    outs_w = [torch.full_like(x, -3.0) for x in u0s]
    with an5d.AdjointBatch(grids, budget_bytes=1 << 20) as ab:
        assert ab.info()["waves"] > 1
        dcw = ab.run(u0s, gTs, outs_w)
    assert np.array_equal(dcw, dc)
    for a, b in zip(outs_w, outs):
        assert torch.equal(a, b)


def test_batch_adjoint_matches_single_grid_adjoint():
    """The single-grid adjoint (another schedule: level-storing passes and a
    separate reduction) gives the same dL/du_0 bit for bit (the same FP32
    chains in the same order; any split into passes gives the same bits) and
    dL/dc within FP32 summation-order rounding."""
    import torch
    grids, u0s, gTs, refs = _setup(seed=3)
    outs = [torch.empty_like(x) for x in u0s]
    with an5d.AdjointBatch(grids) as ab:
        dc = ab.run(u0s, gTs, outs)
    for i, (shape, R, c, ny, nx, T) in enumerate(grids):
        with an5d.Plan(2, shape, R, c, "f32", (ny, nx)) as plan:
            gu = torch.empty_like(u0s[i])
            gc = an5d.an5d_run_adjoint(plan.handle, u0s[i], gTs[i], gu, T)
        n = refs[i][3]
        assert np.array_equal(outs[i].cpu().numpy(), gu.cpu().numpy()), i
        if T:
            assert _rel(dc[i][:n], gc[:n]) < 1e-5


def test_batch_adjoint_rejects_bad_buffers():
    grids, u0s, gTs, _ = _setup()
    with an5d.AdjointBatch(grids) as ab:
        with pytest.raises(an5d.An5dError) as e:
            ab.run(u0s, gTs, u0s)                     # grad_u0 overlapping u0
        assert e.value.status == an5d.AN5D_ERR_ALIAS
    with pytest.raises(an5d.An5dError) as e:
        an5d.AdjointBatch([(STAR, 3, np.ones(13) / 13, 20, 20, 5)])
    assert e.value.status == an5d.AN5D_ERR_INVALID_ARG
