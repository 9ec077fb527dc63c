"""fv_time_step (halo gather + update + next-step CFL maximum in one kernel)
and fv_run_steps (multi-step driver, optionally one CUDA graph): bitwise
equal to the separate halo fill -> reduce -> update path, and within the
FP64 tolerance of the oracle's own steps."""
import numpy as np
import pytest

import oracle
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def mesh(d, p, grid, prec, seed, periodic=True, bnd=-1):
    dtype = np.float32 if prec else np.float64
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, p, d, seed, dtype)
    nbr = inputs.grid_neighbours(grid, periodic=periodic, boundary=bnd)
    return q, off, sz, nbr


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,p,grid,periodic,bnd", [
    (3, 5, (6, 5, 4), True, -1), (2, 3, (8, 8), True, -1), (2, 5, (5, 4), False, -1),
    (3, 3, (3, 4, 3), False, -2), (2, 8, (3, 3), False, -2), (1, 4, (9,), True, -1),
    (3, 4, (3, 3, 3), True, -1)])
def test_time_step_equals_separate_kernels_bitwise(fv, prec, d, p, grid, periodic, bnd):
    torch = fvtest.torch_cuda()
    q, off, sz, nbr = mesh(d, p, grid, prec, 41, periodic, bnd)
    n = len(off)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    # separate kernels, two steps
    ba = fv.Batch(d, precision=prec, max_patch_size=p)
    xa, ya = fvtest.to_dev(q), fvtest.to_dev(q)
    lam_a = torch.zeros(n, dtype=torch.float64, device="cuda")
    for step in range(2):
        ba.halo_fill(xa, toff, tsz, tnbr)
        ba.max_eigenvalue(xa, toff, tsz, cfl, dx)
        ba.update(xa, ya, toff, tsz, dx, -1.0, lambda_patch=lam_a if step == 1 else None)
        xa, ya = ya, xa
    assert ba.status() == fv.FV_OK
    # fused: seed lambda with one reduce after a halo fill, then two time steps
    bb = fv.Batch(d, precision=prec, max_patch_size=p)
    xb, yb = fvtest.to_dev(q), fvtest.to_dev(q)
    lam_b = torch.zeros(n, dtype=torch.float64, device="cuda")
    bb.halo_fill(xb, toff, tsz, tnbr)
    bb.max_eigenvalue(xb, toff, tsz, cfl, dx)
    for step in range(2):
        bb.time_step(xb, yb, toff, tsz, tnbr, dx, cfl, lambda_patch=lam_b if step == 1 else None)
        xb, yb = yb, xb
    assert bb.status() == fv.FV_OK
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    ga, gb = xa.cpu().numpy(), xb.cpu().numpy()
    assert np.array_equal(ga[mask], gb[mask])
    assert torch.equal(lam_a, lam_b)
    # the dt of the last step agrees bitwise too
    assert fv.fv_read_dt(ba.h) == fv.fv_read_dt(bb.h)
    ba.close()
    bb.close()


def test_time_steps_match_oracle_steps(fv):
    """Five fused steps on a periodic 3D mesh vs five oracle steps."""
    d, p, grid = 3, 5, (4, 4, 3)
    q, off, sz, nbr = mesh(d, p, grid, 0, 42)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    b = fv.Batch(d, max_patch_size=p)
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    b.halo_fill(x, toff, tsz, tnbr)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    ref = q.copy()
    for _ in range(5):
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
        x, y = y, x
        ref, _ = oracle.step(ref, off, sz, nbr, d, dx, cfl)
    assert b.status() == fv.FV_OK
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    err = fvtest.per_unknown_rel_err(x.cpu().numpy(), ref, mask, d + 2)
    assert np.all(err <= 1e-11), err
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("n_steps", [1, 4, 5])
def test_run_steps_graph_equals_eager(fv, prec, n_steps):
    torch = fvtest.torch_cuda()
    d, p, grid = 3, 3, (5, 4, 6)
    q, off, sz, nbr = mesh(d, p, grid, prec, 43)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    res = []
    for use_graph in (False, True):  # the graph is captured, run, then replayed
        stream = torch.cuda.Stream()
        b = fv.Batch(d, precision=prec, max_patch_size=p, stream=stream)
        q0, q1 = fvtest.to_dev(q), fvtest.to_dev(q)
        torch.cuda.synchronize()
        b.run_steps(q0, q1, toff, tsz, tnbr, dx, cfl, n_steps, use_graph)
        if use_graph:  # replay the cached graph from the same start
            stream.synchronize()  # the first run is done with q0 before it is reset
            q0.copy_(fvtest.to_dev(q))
            torch.cuda.synchronize()
            b.run_steps(q0, q1, toff, tsz, tnbr, dx, cfl, n_steps, use_graph)
        assert b.status() == fv.FV_OK
        out = (q0 if n_steps % 2 == 0 else q1).cpu().numpy()
        res.append(out)
        b.close()
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert np.array_equal(res[0][mask], res[1][mask])


def test_fp32_path_conserves_and_tracks_fp64(fv):
    """Precision workload in small: a periodic 2D Fourier-perturbed state in
    5x5 patches, 20 fused steps in FP64 and in FP32.  FP64 conserves the
    totals to roundoff; the FP32 path (FP32 fluxes and update, FP64 sums
    and dt) drifts by FP32 roundoff only and stays within 1e-5 (relative L1)
    of the FP64 state."""
    torch = fvtest.torch_cuda()
    N, p, steps = 255, 5, 20
    U = inputs.fourier_perturbation(N, seed=3)
    q64, off, sz, grid = inputs.domain_to_patches(U, p, align_bytes=32)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 1.0 / N, 0.4
    res = {}
    for prec in (0, 1):
        q = q64 if prec == 0 else q64.astype(np.float32)
        b = fv.Batch(2, precision=prec, max_patch_size=p)
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        t0 = torch.zeros(4, dtype=torch.float64, device="cuda")
        t1 = torch.zeros(4, dtype=torch.float64, device="cuda")
        b.totals(x, toff, tsz, t0)
        b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, steps)
        out = x if steps % 2 == 0 else y
        b.totals(out, toff, tsz, t1)
        assert b.status() == fv.FV_OK
        res[prec] = (inputs.patches_to_domain(out.cpu().numpy(), off, p, grid, 4),
                     t0.cpu().numpy(), t1.cpu().numpy())
        b.close()
    d64, a64, b64 = res[0]
    d32, a32, b32 = res[1]
    scale = np.abs(a64)
    assert np.all(np.abs(b64 - a64) <= 1e-13 * np.maximum(scale, 1.0))
    assert np.all(np.abs(b32 - a32) <= 1e-5 * np.maximum(scale, 1.0))
    rel_l1 = np.abs(d32 - d64).sum(axis=(0, 1)) / np.abs(d64).sum(axis=(0, 1))
    assert np.all(rel_l1 <= 1e-5), rel_l1
    # and the FP64 run matches the oracle
    ref = q64.copy()
    for _ in range(steps):
        ref, _ = oracle.step(ref, off, sz, nbr, 2, dx, cfl)
    dref = inputs.patches_to_domain(ref, off, p, grid, 4)
    err = np.abs(d64 - dref).max(axis=(0, 1)) / np.abs(dref).max(axis=(0, 1))
    assert np.all(err <= 1e-11), err
