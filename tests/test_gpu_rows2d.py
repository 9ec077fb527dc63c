"""The FP32 kernel for launches of one 2D patch size (csrc/fv_rows2d.cu, p x p
patches for p = 3 .. 6, a lane per row of cells, four patches a warp): it runs
(launch counter) for planned batches under every schedule and for its classes
of uneven batches, and its results
are bitwise those of the general kernel -- time steps on periodic, outflow
and wall meshes (with per-patch wave speeds, the time step and the
primitives of the new state), update mode with more patches than resident
warps -- and within the FP32 tolerance of the FP64 oracle.  Bad patches and
non-physical states are flagged as by the general kernel."""
import numpy as np
import pytest

import oracle
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu

D = 2


@pytest.fixture(params=[5, 3, 4, 6], ids=["p5", "p3", "p4", "p6"])
def P(request):
    return request.param


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def batch(fv, planned, tsz, n, sched=0, p=5):
    b = fv.Batch(D, precision=fv.FV_FP32, max_patch_size=p)
    if planned:
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, sched)
    return b


def time_steps(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, lam=None):
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    b.halo_fill(x, toff, tsz, tnbr)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    for k in range(steps):
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl, lambda_patch=lam if k == steps - 1 else None)
        x, y = y, x
    return x


@pytest.mark.parametrize("sched", [0, 1, 2])
@pytest.mark.parametrize("grid,periodic,bnd", [
    ((12, 10), True, -1), ((3, 3), False, -1), ((4, 7), False, -2), ((1, 1), True, -1),
    ((80, 60), True, -1), ((200, 100), False, -2)])
def test_time_steps_bitwise_equal_general_kernel(fv, sched, grid, periodic, bnd, P):
    torch = fvtest.torch_cuda()
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 91, np.float32)
    nbr = inputs.grid_neighbours(grid, periodic=periodic, boundary=bnd)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl, steps = 1.0 / (grid[0] * P), 0.4, 3
    outs, lams, dts, launches = [], [], [], []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, sched, p=P)
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        x = time_steps(fv, b, q, toff, tsz, tnbr, dx, cfl, steps, lam)
        assert b.status() == fv.FV_OK
        outs.append(x.cpu().numpy())
        lams.append(lam.cpu().numpy())
        dts.append(fv.fv_read_dt(b.h))
        launches.append(fv.fv_batch_pairs_launches(b.h))
        b.close()
    assert launches == [0, steps]
    mask = fvtest.interior_mask(off, sz, D, D + 2, len(q))
    assert np.array_equal(outs[0][mask], outs[1][mask])
    assert np.array_equal(lams[0], lams[1])
    assert dts[0] == dts[1]


def test_primitives_of_the_new_state_bitwise(fv, P):
    torch = fvtest.torch_cuda()
    grid = (7, 5)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 92, np.float32)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * P), 0.4
    res = []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, p=P)
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        pa = torch.full((n * b.prim_stride(),), float("nan"), dtype=torch.float32, device="cuda")
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
        b.time_step_prim(x, y, None, pa, toff, tsz, tnbr, dx, cfl)
        assert b.status() == fv.FV_OK
        stride = b.prim_stride()
        prim = pa.cpu().numpy().reshape(n, stride)[:, :5 * P ** 2]  # (u, p, c, E+p) blocks
        res.append((y.cpu().numpy(), prim, fv.fv_batch_pairs_launches(b.h)))
        b.close()
    assert res[0][2] == 0 and res[1][2] == 1
    mask = fvtest.interior_mask(off, sz, D, D + 2, len(q))
    assert np.array_equal(res[0][0][mask], res[1][0][mask])
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("device_dt,n", [(False, 9000), (True, 9000), (False, 40000)])
def test_update_mode_bitwise_equal_general_kernel(fv, device_dt, n, P):
    torch = fvtest.torch_cuda()
    # more patches than resident warps: several per CTA (40,000: about 11)
    q, off, sz = fvtest.random_batch(n, P, D, 93, np.float32)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    dx = 0.01
    res = []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, 2, p=P)
        x = fvtest.to_dev(q)
        y = x.clone()
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        if device_dt:
            b.max_eigenvalue(x, toff, tsz, 0.4, dx)
            b.update(x, y, toff, tsz, dx, -1.0, lambda_patch=lam)
        else:
            b.update(x, y, toff, tsz, dx, 0.001, lambda_patch=lam)
        assert b.status() == fv.FV_OK
        res.append((y.cpu().numpy(), lam.cpu().numpy(), fv.fv_batch_pairs_launches(b.h)))
        b.close()
    assert res[0][2] == 0 and res[1][2] == 1
    assert np.array_equal(res[0][0], res[1][0])  # halos untouched as well
    assert np.array_equal(res[0][1], res[1][1])


def test_time_step_matches_oracle(fv, P):
    grid = (6, 5)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 94)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * P), 0.4
    b = batch(fv, True, tsz, n, p=P)
    x = time_steps(fv, b, q.astype(np.float32), toff, tsz, tnbr, dx, cfl, 1)
    assert b.status() == fv.FV_OK and fv.fv_batch_pairs_launches(b.h) == 1
    ref, dt = oracle.step(q, off, sz, nbr, D, dx, cfl)
    assert fv.fv_read_dt(b.h) == pytest.approx(dt, rel=1e-6)
    mask = fvtest.interior_mask(off, sz, D, D + 2, len(q))
    err = fvtest.per_unknown_rel_err(x.cpu().numpy(), ref, mask, D + 2)
    assert np.all(err <= 1e-5), err
    b.close()


def test_uneven_batch_uses_it_for_its_classes(fv):
    n = 900
    sizes = inputs.uneven_sizes(n, seed=95, mix=((3, 0.4), (5, 0.4), (8, 0.2)))
    q, off, sz = inputs.random_batch(n, sizes, D, seed=95, dtype=np.float32)
    nbr = inputs.self_periodic_neighbours(n, D)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl, steps = 0.01, 0.4, 2
    b0 = batch(fv, False, tsz, n, p=8)
    ref = time_steps(fv, b0, q, toff, tsz, tnbr, dx, cfl, steps).cpu().numpy()
    b0.close()
    b = batch(fv, True, tsz, n, 2, p=8)
    got = time_steps(fv, b, q, toff, tsz, tnbr, dx, cfl, steps).cpu().numpy()
    assert b.status() == fv.FV_OK
    assert fv.fv_batch_pairs_launches(b.h) == 2 * steps  # 3x3 and 5x5, not 8x8
    mask = fvtest.interior_mask(off, sz, D, D + 2, len(q))
    assert np.array_equal(got[mask], ref[mask])
    b.close()


def test_nonphysical_state_is_reported(fv, P):
    n = 8
    q, off, sz = fvtest.random_batch(n, P, D, 96, np.float32)
    ne = P + 2
    q[off[3] + (2 + ne * 3) * (D + 2)] = -1.0  # negative density, interior cell
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    b = batch(fv, True, tsz, n, p=P)
    x = fvtest.to_dev(q)
    b.update(x, x.clone(), toff, tsz, 0.01, 0.001)
    assert fv.fv_batch_pairs_launches(b.h) == 1
    assert b.status() == fv.FV_ERR_NONPHYSICAL
    b.close()


def test_graph_of_steps_on_a_fresh_handle(fv, P):
    """fv_run_steps captured into a CUDA graph on a fresh, planned handle (the
    kernel's first launch happens inside the capture) equals the general
    kernel's eager steps bitwise."""
    torch = fvtest.torch_cuda()
    grid = (9, 8)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 97, np.float32)
    nbr = inputs.grid_neighbours(grid, periodic=False, boundary=-2)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl, steps = 1.0 / (grid[0] * P), 0.4, 4
    b0 = batch(fv, False, tsz, n, p=P)
    ref = time_steps(fv, b0, q, toff, tsz, tnbr, dx, cfl, steps).cpu().numpy()
    b0.close()
    stream = torch.cuda.Stream()
    b = fv.Batch(D, precision=fv.FV_FP32, max_patch_size=P, stream=stream)
    fv.fv_batch_plan(b.h, tsz, n)
    q0, q1 = fvtest.to_dev(q), fvtest.to_dev(q)
    torch.cuda.synchronize()
    b.run_steps(q0, q1, toff, tsz, tnbr, dx, cfl, steps, use_graph=True)
    assert b.status() == fv.FV_OK
    assert fv.fv_batch_pairs_launches(b.h) >= steps
    mask = fvtest.interior_mask(off, sz, D, D + 2, len(q))
    got = (q0 if steps % 2 == 0 else q1).cpu().numpy()
    assert np.array_equal(got[mask], ref[mask])
    b.close()


def test_patch_beyond_the_buffer_is_flagged_and_skipped(fv, P):
    n = 40
    q, off, sz = fvtest.random_batch(n, P, D, 98, np.float32)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    n_elems = int(off[-1]) + 10  # the last patch does not fit
    res = []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, p=P)
        x = fvtest.to_dev(q)
        y = x.clone()
        b.update(x, y, toff, tsz, 0.01, 0.001, n_elems=n_elems)
        res.append((b.status(), y.cpu().numpy(), fv.fv_batch_pairs_launches(b.h)))
        b.close()
    assert res[0][0] == fv.FV_ERR_BAD_PATCH and res[1][0] == fv.FV_ERR_BAD_PATCH
    assert res[0][2] == 0 and res[1][2] == 1
    assert np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[1][1][off[-1]:], q[off[-1]:])


@pytest.mark.parametrize("step", [False, True])
def test_invalid_patches_inside_the_sequence(fv, step, P):
    """Patches with a misaligned offset scattered through a long sequence (many
    patches per CTA): both kernels report FV_ERR_BAD_PATCH, skip them (and,
    in a time step, treat them as absent neighbours the same way) and agree
    bitwise on everything else."""
    torch = fvtest.torch_cuda()
    grid = (200, 100)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 99, np.float32)
    bad = np.arange(17, n, 1511)
    off = off.copy()
    off[bad] += 1  # not a multiple of 16 bytes
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx = 1.0 / (grid[0] * P)
    res = []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, 2, p=P)
        x = fvtest.to_dev(q)
        y = x.clone()
        if step:
            b.max_eigenvalue(x, toff, tsz, 0.4, dx)
            b.time_step(x, y, toff, tsz, tnbr, dx, 0.4)
        else:
            b.update(x, y, toff, tsz, dx, 0.001)
        res.append((b.status(), y.cpu().numpy(), fv.fv_batch_pairs_launches(b.h)))
        b.close()
    assert res[0][0] == fv.FV_ERR_BAD_PATCH and res[1][0] == fv.FV_ERR_BAD_PATCH
    assert res[0][2] == 0 and res[1][2] == 1
    assert np.array_equal(res[0][1], res[1][1])


def test_bad_neighbour_entries_flagged_like_the_general_kernel(fv, P):
    """Neighbour-table entries that name no patch (an index past the batch, an
    unknown boundary code): both kernels report FV_ERR_BAD_PATCH, take those
    faces as outflow and agree bitwise on the new state."""
    torch = fvtest.torch_cuda()
    grid = (40, 30)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, P, D, 98, np.float32)
    nbr = inputs.grid_neighbours(grid).copy()
    nbr[7, 1] = n + 2
    nbr[300, 2] = -7
    nbr[901, 3] = n
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx = 1.0 / (grid[0] * P)
    res = []
    for planned in (False, True):
        b = batch(fv, planned, tsz, n, 2, p=P)
        x = fvtest.to_dev(q)
        y = x.clone()
        b.max_eigenvalue(x, toff, tsz, 0.4, dx)
        b.time_step(x, y, toff, tsz, tnbr, dx, 0.4)
        res.append((b.status(), y.cpu().numpy(), fv.fv_batch_pairs_launches(b.h)))
        b.close()
    assert res[0][0] == fv.FV_ERR_BAD_PATCH and res[1][0] == fv.FV_ERR_BAD_PATCH
    assert res[0][2] == 0 and res[1][2] == 1
    assert np.array_equal(res[0][1], res[1][1])
