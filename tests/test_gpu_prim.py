"""The primitive carry between time steps (fv_time_step_prim, and
fv_run_steps which uses it): bitwise equal to plain fv_time_step chains on
periodic, outflow and wall meshes, in FP64 and FP32, under every schedule of
an uneven batch; the carried block holds the primitives of the new state;
bad arguments are refused."""
import numpy as np
import pytest

from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu

GAMMA = 1.4


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def prim_buffers(b, n, prec, count=2):
    torch = fvtest.torch_cuda()
    dt = torch.float64 if prec == 0 else torch.float32
    return [torch.full((n * b.prim_stride(),), float("nan"), dtype=dt, device="cuda")
            for _ in range(count)]


def run_plain(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, lam=None):
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    b.halo_fill(x, toff, tsz, tnbr)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    for k in range(steps):
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl, lambda_patch=lam if k == steps - 1 else None)
        x, y = y, x
    return x


def run_carry(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, prec, lam=None):
    n = toff.numel()
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    pa, pb = prim_buffers(b, n, prec)
    b.halo_fill(x, toff, tsz, tnbr)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    pin = None
    for k in range(steps):
        pout = None if k == steps - 1 else (pa if k % 2 == 0 else pb)
        b.time_step_prim(x, y, pin, pout, toff, tsz, tnbr, dx, cfl,
                         lambda_patch=lam if k == steps - 1 else None)
        x, y = y, x
        pin = pout
    return x


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,p,grid,periodic,bnd", [
    (3, 5, (6, 5, 4), True, -1), (2, 3, (8, 8), True, -1), (2, 5, (5, 4), False, -1),
    (3, 3, (3, 4, 3), False, -2), (2, 8, (3, 3), False, -2), (1, 4, (9,), True, -1),
    (1, 6, (5,), False, -2), (3, 4, (3, 3, 3), True, -1), (3, 8, (2, 3, 2), True, -1),
    (2, 17, (3, 2), False, -2)])
def test_carry_equals_plain_time_steps_bitwise(fv, prec, d, p, grid, periodic, bnd):
    torch = fvtest.torch_cuda()
    dtype = np.float32 if prec else np.float64
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, p, d, 61, dtype)
    nbr = inputs.grid_neighbours(grid, periodic=periodic, boundary=bnd)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl, steps = 1.0 / (grid[0] * p), 0.4, 4
    outs, lams, dts = [], [], []
    for carry in (False, True):
        b = fv.Batch(d, precision=prec, max_patch_size=p)
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        if carry:
            x = run_carry(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, prec, lam)
        else:
            x = run_plain(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, lam)
        assert b.status() == fv.FV_OK
        outs.append(x.cpu().numpy())
        lams.append(lam.cpu().numpy())
        dts.append(fv.fv_read_dt(b.h))
        b.close()
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert np.array_equal(outs[0][mask], outs[1][mask])
    assert np.array_equal(lams[0], lams[1])
    assert dts[0] == dts[1]


@pytest.mark.parametrize("prec", [0, 1])
def test_carried_block_holds_the_primitives_of_the_new_state(fv, prec):
    d, p, grid = 3, 5, (3, 4, 2)
    dtype = np.float32 if prec else np.float64
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, p, d, 62, dtype)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    (pa,) = prim_buffers(b, n, prec, 1)
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    b.halo_fill(x, toff, tsz, tnbr)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    b.time_step_prim(x, y, None, pa, toff, tsz, tnbr, dx, cfl)
    assert b.status() == fv.FV_OK
    stride = b.prim_stride()
    assert stride == -(-(d + 3) * p ** d // (2 if prec == 0 else 4)) * (2 if prec == 0 else 4)
    out = y.cpu().numpy().astype(np.float64)
    prim = pa.cpu().numpy().astype(np.float64)
    tol = 1e-14 if prec == 0 else 2e-6
    for i in range(n):
        blk = out[off[i]:off[i] + (p + 2) ** d * (d + 2)].reshape((p + 2,) * d + (d + 2,))
        Q = blk[1:-1, 1:-1, 1:-1].reshape(-1, d + 2)  # interior, z-major: x fastest
        rho, j, E = Q[:, 0], Q[:, 1:1 + d], Q[:, -1]
        u = j / rho[:, None]
        pr = (GAMMA - 1.0) * (E - 0.5 * np.sum(j * u, axis=1))
        c = np.sqrt(GAMMA * pr / rho)
        want = np.concatenate([u.T, pr[None], c[None], (E + pr)[None]])
        got = prim[i * stride:i * stride + (d + 3) * p ** d].reshape(d + 3, p ** d)
        scale = np.max(np.abs(want), axis=1, keepdims=True)
        assert np.all(np.abs(got - want) <= tol * scale), i
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_carry_under_every_schedule_of_an_uneven_batch(fv, prec):
    torch = fvtest.torch_cuda()
    n = 1200
    sizes = inputs.uneven_sizes(n, seed=63, mix=((3, 0.4), (5, 0.3), (7, 0.2), (4, 0.1)))
    dtype = np.float32 if prec else np.float64
    q, off, sz = inputs.random_batch(n, sizes, 3, seed=63, dtype=dtype)
    nbr = inputs.self_periodic_neighbours(n, 3)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl, steps = 0.01, 0.4, 3
    b0 = fv.Batch(3, precision=prec, max_patch_size=7)
    ref = run_plain(fv, b0, q, toff, tsz, tnbr, dx, cfl, steps).cpu().numpy()
    assert b0.status() == fv.FV_OK
    b0.close()
    mask = fvtest.interior_mask(off, sz, 3, 5, len(q))
    for sched in (fv.FV_SCHED_STRIDE, fv.FV_SCHED_LPT, fv.FV_SCHED_CLASSES):
        b = fv.Batch(3, precision=prec, max_patch_size=7)
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, sched)
        got = run_carry(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, prec).cpu().numpy()
        assert b.status() == fv.FV_OK
        assert np.array_equal(got[mask], ref[mask]), sched
        b.close()


def test_run_steps_carry_equals_plain_chain(fv):
    """fv_run_steps carries the primitives between its steps (eager and as a
    graph) and still equals a chain of plain time steps."""
    torch = fvtest.torch_cuda()
    d, p, grid, steps = 3, 5, (4, 3, 5), 6
    q, off, sz = fvtest.random_batch(int(np.prod(grid)), p, d, 64)
    nbr = inputs.grid_neighbours(grid, periodic=False, boundary=-2)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    b0 = fv.Batch(d, max_patch_size=p)
    ref = run_plain(fv, b0, q, toff, tsz, tnbr, dx, cfl, steps).cpu().numpy()
    b0.close()
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    for use_graph in (False, True):
        stream = torch.cuda.Stream()
        b = fv.Batch(d, max_patch_size=p, stream=stream)
        q0, q1 = fvtest.to_dev(q), fvtest.to_dev(q)
        torch.cuda.synchronize()
        b.run_steps(q0, q1, toff, tsz, tnbr, dx, cfl, steps, use_graph)
        assert b.status() == fv.FV_OK
        assert np.array_equal(q0.cpu().numpy()[mask], ref[mask])
        b.close()


def test_carry_arguments_are_checked(fv):
    torch = fvtest.torch_cuda()
    d, p, grid = 2, 4, (3, 3)
    q, off, sz = fvtest.random_batch(9, p, d, 65)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    b = fv.Batch(d, max_patch_size=p)
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    pa, pb = prim_buffers(b, 9, 0)
    with pytest.raises(fv.FvError) as e:
        b.time_step_prim(x, y, pa, pa, toff, tsz, tnbr, 0.1, 0.4)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError) as e:
        b.time_step_prim(x, y, pa[1:], pb, toff, tsz, tnbr, 0.1, 0.4)
    assert e.value.status == fv.FV_ERR_ALIGNMENT
    with pytest.raises(fv.FvError) as e:
        b.time_step_prim(x, y, None, pb[1:], toff, tsz, tnbr, 0.1, 0.4)
    assert e.value.status == fv.FV_ERR_ALIGNMENT
    assert b.status() == fv.FV_OK
    b.close()
