"""GPU adjoint (checkpointed, temporally blocked transposed sweep) against the
FP64 oracle adjoint, which the CPU pins tie to central finite differences and
the adjoint dot-product identity.  Tolerance: relative L2 error 1e-4 (FP32
forward and backward over up to a few dozen steps; the FP64 oracle starts
from the same FP32 inputs and the run's FP32-rounded coefficients)."""
import numpy as np
import pytest

import oracle
from paper_2001_01473_gb300 import an5d, inputs

pytestmark = pytest.mark.gpu
STAR, BOX = inputs.STAR, inputs.BOX


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("shape,R", [(STAR, 1), (STAR, 2), (BOX, 1), (BOX, 2)])
@pytest.mark.parametrize("bt,T", [(1, 5), (2, 7), (3, 11), (4, 11), (4, 16)])
def test_adjoint_vs_fp64_oracle(shape, R, bt, T):
    import torch
    dims = (70, 300)
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    c32 = c.astype(np.float32).astype(np.float64)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = inputs.target_field(dims, R, 2, "f32")
    inner = tuple(slice(R, R + d) for d in dims)
    with an5d.Plan(2, shape, R, c, "f32", dims) as plan:
        plan.set_config(bt, 23)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        gT = torch.zeros_like(x)
        gT[inner] = y[inner] - torch.from_numpy(tg).cuda()[inner]
        gu = torch.empty_like(x)
        gc = an5d.an5d_run_adjoint(plan.handle, x, gT, gu, T)[:n]
        gu = gu.cpu().numpy()
    loss, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, c32, dims, u0.astype(np.float64),
                                              tg.astype(np.float64), T)
    halo = np.ones(gu.shape, bool)
    halo[inner] = False
    assert np.all(gu[halo] == 0.0)
    assert _rel(gu[inner].astype(np.float64), ref_gu[inner]) < 1e-4
    assert _rel(gc, ref_gc) < 1e-4, (gc, ref_gc)


def test_adjoint_dot_product_gpu():
    """<S^T x, y> = <x, (S^T)^T y> for zero-halo x, in the GPU's own arithmetic."""
    import torch
    dims = (90, 260)
    R, shape = 1, BOX
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 4) * 1.2 - 0.02
    inner = tuple(slice(R, R + d) for d in dims)
    xs = np.zeros(inputs.padded_shape(dims, R), np.float32)
    xs[inner] = inputs.uniform(7, int(np.prod(dims)), 24).reshape(dims) - 0.5
    ys = np.zeros_like(xs)
    ys[inner] = inputs.uniform(8, int(np.prod(dims)), 24).reshape(dims) - 0.5
    T = 10
    with an5d.Plan(2, shape, R, c, "f32", dims) as plan:
        x = torch.from_numpy(xs).cuda()
        sx = torch.empty_like(x)
        plan.run(x, sx, T)
        gu = torch.empty_like(x)
        an5d.an5d_run_adjoint(plan.handle, x, torch.from_numpy(ys).cuda(), gu, T)
    lhs = float(np.sum(sx.cpu().numpy()[inner].astype(np.float64) * ys[inner]))
    rhs = float(np.sum(xs[inner].astype(np.float64) * gu.cpu().numpy()[inner]))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1.0)


def test_autograd_function_matches_oracle():
    import torch
    from paper_2001_01473_gb300.autograd import stencil_sweep
    dims = (64, 200)
    shape, R, T = STAR, 2, 9
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = inputs.target_field(dims, R, 2, "f32")
    inner = tuple(slice(R, R + d) for d in dims)
    x = torch.from_numpy(u0).cuda().requires_grad_(True)
    ct = torch.tensor(c.astype(np.float32).astype(np.float64), requires_grad=True)
    uT = stencil_sweep(x, ct, T, shape, R)
    loss = 0.5 * ((uT[inner] - torch.from_numpy(tg).cuda()[inner]) ** 2).double().sum()
    loss.backward()
    ref_loss, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, ct.detach().numpy(), dims,
                                                  u0.astype(np.float64), tg.astype(np.float64), T)
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    assert _rel(x.grad.cpu().numpy()[inner].astype(np.float64), ref_gu[inner]) < 1e-4
    assert _rel(ct.grad.numpy(), ref_gc) < 1e-4


def test_adjoint_rejects_unsupported():
    import torch
    with an5d.Plan(2, STAR, 3, np.ones(13) / 13, "f32", (16, 16)) as plan:
        x = torch.zeros(inputs.padded_shape((16, 16), 3), device="cuda")
        with pytest.raises(an5d.An5dError) as e:
            an5d.an5d_run_adjoint(plan.handle, x, x, torch.empty_like(x), 3)
        assert e.value.status == an5d.AN5D_ERR_UNSUPPORTED


def test_adjoint_vs_central_differences_gpu():
    """dL/dc along random directions vs central differences (h = 1e-3) of the
    GPU forward.  L is a polynomial of degree 2T in c, so a central difference
    at h = 1e-3 carries an O(h^2) truncation error; it is measured on the FP64
    oracle at the same h and direction and allowed for, plus 1e-3 relative
    for the FP32 forward runs inside the difference quotient."""
    import torch
    dims = (80, 140)
    shape, R, T = BOX, 1, 12
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = inputs.target_field(dims, R, 2, "f32")
    inner = tuple(slice(R, R + d) for d in dims)
    x = torch.from_numpy(u0).cuda()
    t = torch.from_numpy(tg).cuda()

    def loss_gpu(cc):
        with an5d.Plan(2, shape, R, cc, "f32", dims) as p:
            y = torch.empty_like(x)
            p.run(x, y, T)
            d = (y[inner] - t[inner]).double()
            return 0.5 * float((d * d).sum()), y

    def loss_f64(cc):
        uT = oracle.run_f64(2, shape, R, cc, dims, u0.astype(np.float64), T)
        d = uT[inner] - tg[inner].astype(np.float64)
        return 0.5 * float(np.sum(d * d))

    _, y = loss_gpu(c)
    gT = torch.zeros_like(x)
    gT[inner] = y[inner] - t[inner]
    with an5d.Plan(2, shape, R, c, "f32", dims) as p:
        gc = an5d.an5d_run_adjoint(p.handle, x, gT, torch.empty_like(x), T)[:n]
    c32 = c.astype(np.float32).astype(np.float64)
    _, _, gc64 = oracle.adjoint_f64(2, shape, R, c32, dims, u0.astype(np.float64),
                                    tg.astype(np.float64), T)
    h = 1e-3
    for j in range(3):
        dcv = inputs.uniform(70 + j, n, 53) - 0.5
        fd = (loss_gpu(c + h * dcv)[0] - loss_gpu(c - h * dcv)[0]) / (2 * h)
        an = float(np.dot(gc, dcv))
        trunc = abs((loss_f64(c32 + h * dcv) - loss_f64(c32 - h * dcv)) / (2 * h)
                    - float(np.dot(gc64, dcv)))
        assert abs(fd - an) <= 1.5 * trunc + 1e-3 * abs(an), (fd, an, trunc)


@pytest.mark.parametrize("shape,R,dims,T,bt", [(BOX, 2, (2000, 1500), 60, 4),
                                               (STAR, 1, (3000, 1200), 100, 4),
                                               (STAR, 2, (1100, 4096), 40, 3)])
def test_adjoint_at_batch_grid_scale(shape, R, dims, T, bt):
    """The batched workload's grids reach sides of 4096 and hundreds of steps:
    the coefficient gradient sums g_{t+1}(p) u_t(p + o_k) over every cell and
    step (FP32 products, FP64 partial sums), so its error is checked at that
    scale, against the FP64 oracle adjoint.  Measured relative L2 errors are
    printed; the bound is the same 1e-4 as on the small grids."""
    import torch
    n = inputs.coeff_count(2, shape, R)
    c = inputs.normalised_coeffs(n, 0)
    c32 = c.astype(np.float32).astype(np.float64)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = inputs.target_field(dims, R, 2, "f32")
    inner = tuple(slice(R, R + d) for d in dims)
    with an5d.Plan(2, shape, R, c, "f32", dims) as plan:
        plan.set_config(bt, 0)
        x = torch.from_numpy(u0).cuda()
        y = torch.empty_like(x)
        plan.run(x, y, T)
        gT = torch.zeros_like(x)
        gT[inner] = y[inner] - torch.from_numpy(tg).cuda()[inner]
        gu = torch.empty_like(x)
        gc = an5d.an5d_run_adjoint(plan.handle, x, gT, gu, T)[:n]
        gu = gu.cpu().numpy()
    _, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, c32, dims, u0.astype(np.float64),
                                           tg.astype(np.float64), T)
    e_u = _rel(gu[inner].astype(np.float64), ref_gu[inner])
    e_c = _rel(gc, ref_gc)
    print(f"adjoint {dims} shape={shape} R={R} T={T}: rel L2 dL/du0 {e_u:.2e}, dL/dc {e_c:.2e}")
    assert e_u < 1e-4
    assert e_c < 1e-4, (gc, ref_gc)


def test_autograd_training_loop_keeps_one_plan():
    """A loop that updates the coefficients every step reuses one cached plan
    (coefficients replaced in place): device memory stays constant over 50
    backward steps, and the last step's gradients still match the oracle."""
    import torch
    from paper_2001_01473_gb300 import autograd
    dims = (96, 300)
    shape, R, T = BOX, 1, 7
    n = inputs.coeff_count(2, shape, R)
    u0 = inputs.field(dims, R, 1, "f32")
    tg = torch.from_numpy(inputs.target_field(dims, R, 2, "f32")).cuda()
    inner = tuple(slice(R, R + d) for d in dims)
    x = torch.from_numpy(u0).cuda().requires_grad_(True)
    ct = torch.tensor(inputs.normalised_coeffs(n, 0).astype(np.float32).astype(np.float64),
                      requires_grad=True)
    free = []
    for step in range(50):
        x.grad = None
        ct.grad = None
        uT = autograd.stencil_sweep(x, ct, T, shape, R)
        loss = 0.5 * ((uT[inner] - tg[inner]) ** 2).double().sum()
        loss.backward()
        with torch.no_grad():
            ct -= 1e-6 * ct.grad      # the coefficients change every step
            ct.copy_(ct.float().double())
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert sum(1 for k in autograd._plans if k[1:] == (shape, R, dims)) == 1
    assert max(free[5:]) - min(free[5:]) <= 4 << 20, (min(free[5:]), max(free[5:]))
    # gradients of the final coefficients
    x.grad = None
    ct.grad = None
    uT = autograd.stencil_sweep(x, ct, T, shape, R)
    (0.5 * ((uT[inner] - tg[inner]) ** 2).double().sum()).backward()
    _, ref_gu, ref_gc = oracle.adjoint_f64(2, shape, R, ct.detach().numpy(), dims,
                                           u0.astype(np.float64),
                                           tg.cpu().numpy().astype(np.float64), T)
    assert _rel(x.grad.cpu().numpy()[inner].astype(np.float64), ref_gu[inner]) < 1e-4
    assert _rel(ct.grad.numpy(), ref_gc) < 1e-4
