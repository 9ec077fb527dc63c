"""CUDA path vs the FP64 CPU oracle, through the C ABI (libfv.so).

Tolerances (from the rounding of each precision over the few tens of
operations per cell of one step):
  * FP64 update: per unknown, max|Q_gpu - Q_ref| / max|Q_ref| <= 1e-12.
  * FP32 update: the same measure <= 1e-5 against the oracle run on the
    FP32-rounded input.
  * Maxima (per-patch and global wave speed): relative 1e-14 against the
    oracle; bitwise between the GPU's own update epilogue and its reduce.
  * Halo fill: bitwise (a copy).
  * Bitwise invariants: a uniform state is preserved exactly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5
TOL_MAX = 1e-14


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def run_update(fv, q, off, sz, d, dx, dt, *, prec=0, pmax=0, want_lambda=False, dt_dev=False):
    torch = fvtest.torch_cuda()
    tdt = torch.float64 if prec == 0 else torch.float32
    qin = fvtest.to_dev(q, tdt)
    qout = qin.clone()
    toff = fvtest.to_dev(off)
    tsz = fvtest.to_dev(sz)
    b = fv.Batch(d, precision=prec, max_patch_size=pmax)
    lam = torch.zeros(len(off), dtype=torch.float64, device="cuda") if want_lambda else None
    b.update(qin, qout, toff, tsz, dx, dt, lambda_patch=lam, n_elems=qin.numel())
    st = b.status()
    assert st == fv.FV_OK, fv.fv_last_error(b.h)
    res = qout.cpu().numpy()
    lam_np = lam.cpu().numpy() if want_lambda else None
    b.close()
    return res, lam_np


@pytest.mark.parametrize("d,p,n,seed", [(2, 3, 64, 0), (3, 5, 200, 1), (2, 5, 150, 2),
                                        (2, 8, 60, 3), (3, 3, 300, 4), (3, 7, 40, 5),
                                        (2, 17, 12, 6), (2, 4, 33, 7), (3, 4, 17, 8),
                                        (1, 6, 40, 9), (3, 1, 50, 10), (2, 1, 9, 11),
                                        (3, 8, 12, 12), (2, 16, 10, 13)])
def test_update_fp64_matches_oracle(fv, d, p, n, seed):
    s = d + 2
    q, off, sz = fvtest.random_batch(n, p, d, seed)
    dx, dt = 1.0 / 64, 0.002
    got, lam = run_update(fv, q, off, sz, d, dx, dt, want_lambda=True)
    ref, lam_ref = oracle.patch_update(q, off, sz, d, dx, dt, want_lambda=True)
    mask = fvtest.interior_mask(off, sz, d, s, len(q))
    err = fvtest.per_unknown_rel_err(got, ref, mask, s)
    assert np.all(err <= TOL64), err
    # halo and padding of out are untouched
    assert np.array_equal(got[~mask], q[~mask])
    assert np.allclose(lam, lam_ref, rtol=TOL_MAX, atol=0)


def test_update_ragged_sizes_one_launch(fv):
    """Uneven sizes (compiled 3/5/7 and runtime-size 2/4/6) in one launch."""
    d, s = 3, 5
    rng = np.random.default_rng(3)
    sizes = rng.choice([2, 3, 4, 5, 6, 7], size=257)
    q, off, sz = inputs.random_batch(len(sizes), sizes, d, seed=12)
    dx, dt = 0.01, 0.001
    got, lam = run_update(fv, q, off, sz, d, dx, dt, pmax=7, want_lambda=True)
    ref, lam_ref = oracle.patch_update(q, off, sz, d, dx, dt, want_lambda=True)
    mask = fvtest.interior_mask(off, sz, d, s, len(q))
    assert np.all(fvtest.per_unknown_rel_err(got, ref, mask, s) <= TOL64)
    assert np.allclose(lam, lam_ref, rtol=TOL_MAX, atol=0)


@pytest.mark.parametrize("d,p,n", [(2, 3, 64), (3, 5, 100), (2, 5, 80), (3, 8, 12), (2, 17, 9)])
def test_update_fp32_within_1e5(fv, d, p, n):
    s = d + 2
    q32, off, sz = fvtest.random_batch(n, p, d, 13, np.float32)
    dx, dt = 1.0 / 64, 0.002
    got, lam = run_update(fv, q32, off, sz, d, dx, dt, prec=1, want_lambda=True)
    ref, lam_ref = oracle.patch_update(q32.astype(np.float64), off, sz, d, dx, dt,
                                       want_lambda=True)
    mask = fvtest.interior_mask(off, sz, d, s, len(q32))
    err = fvtest.per_unknown_rel_err(got, ref, mask, s)
    assert np.all(err <= TOL32), err
    assert np.allclose(lam, lam_ref, rtol=1e-6, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,p", [(2, 3), (3, 5), (3, 4)])
def test_uniform_state_bitwise(fv, prec, d, p):
    s = d + 2
    n = 20
    q, off, sz = fvtest.random_batch(n, p, d, 14)
    rng = np.random.default_rng(5)
    for i in range(n):
        ne = (p + 2) ** d
        q[off[i]:off[i] + ne * s] = np.tile(inputs.random_cells(rng, 1, d)[0], ne)
    qq = q if prec == 0 else q.astype(np.float32)
    if prec:  # FP32 layout: offsets in multiples of 4 elements
        qq, off, sz = fvtest.random_batch(n, p, d, 14, np.float32)
        for i in range(n):
            ne = (p + 2) ** d
            qq[off[i]:off[i] + ne * s] = np.tile(q[0:s].astype(np.float32), ne)
    got, _ = run_update(fv, qq, off, sz, d, 0.01, 0.003, prec=prec)
    assert np.array_equal(got, qq)


def test_eigen_reduce_and_device_dt(fv):
    """Per-patch maxima equal the update's epilogue bitwise and the oracle to
    1e-14; dt = cfl dx / (d lambda) lands in the device slot, and an update
    with dt <= 0 reads it."""
    torch = fvtest.torch_cuda()
    d, p, n = 3, 5, 300
    q, off, sz = fvtest.random_batch(n, p, d, 15)
    qin = fvtest.to_dev(q)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    b = fv.Batch(d, max_patch_size=5)
    per = torch.zeros(n, dtype=torch.float64, device="cuda")
    glob = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    dx, cfl = 1.0 / 64, 0.4
    b.max_eigenvalue(qin, toff, tsz, cfl, dx, per, glob, dt_out)
    lam_u = torch.zeros(n, dtype=torch.float64, device="cuda")
    q1 = qin.clone()
    b.update(qin, q1, toff, tsz, dx, -1.0, lambda_patch=lam_u)
    q2 = qin.clone()
    b.update(qin, q2, toff, tsz, dx, float(dt_out.item()))
    assert b.status() == fv.FV_OK
    lam_ref, g_ref = oracle.max_eigenvalue(q, off, sz, d)
    assert torch.equal(per, lam_u)
    assert np.allclose(per.cpu().numpy(), lam_ref, rtol=TOL_MAX, atol=0)
    assert glob.item() == pytest.approx(g_ref, rel=TOL_MAX)
    assert glob.item() == per.max().item()
    dt_ref = oracle.cfl_dt(glob.item(), cfl, dx, d)
    assert dt_out.item() == dt_ref  # same formula, same operand, correctly rounded
    assert torch.equal(q1, q2)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,p,grid,periodic,bnd", [
    (2, 5, (7, 5), True, -1), (3, 3, (4, 3, 5), True, -1), (2, 4, (3, 3), False, -1),
    (2, 4, (3, 2), False, -2), (3, 2, (2, 2, 3), False, -2), (1, 5, (6,), True, -1)])
def test_halo_fill_bitwise(fv, prec, d, p, grid, periodic, bnd):
    torch = fvtest.torch_cuda()
    s = d + 2
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, p, d, 16, np.float32 if prec else np.float64)
    nbr = inputs.grid_neighbours(grid, periodic=periodic, boundary=bnd)
    ref = q.astype(np.float64).copy()
    oracle.halo_fill(ref, off, sz, nbr, d, s)
    tq = fvtest.to_dev(q)
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    b.halo_fill(tq, fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr))
    assert b.status() == fv.FV_OK
    got = tq.cpu().numpy().astype(np.float64)
    assert np.array_equal(got, ref)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_conserved_totals_deterministic(fv, prec):
    torch = fvtest.torch_cuda()
    d, p, n = 3, 5, 2500  # spans three sum chunks, ragged last chunk
    s = d + 2
    q, off, sz = fvtest.random_batch(n, p, d, 17, np.float32 if prec else np.float64)
    tq = fvtest.to_dev(q)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    b = fv.Batch(d, precision=prec, max_patch_size=5)
    t1 = torch.zeros(s, dtype=torch.float64, device="cuda")
    t2 = torch.zeros(s, dtype=torch.float64, device="cuda")
    b.totals(tq, toff, tsz, t1)
    b.totals(tq, toff, tsz, t2)
    assert b.status() == fv.FV_OK
    assert torch.equal(t1, t2)
    ps = oracle.patch_sums(q.astype(np.float64), off, sz, d, s)
    for v in range(s):
        exact = math.fsum(ps[:, v])
        scale = math.fsum(np.abs(ps[:, v]))
        assert abs(t1[v].item() - exact) <= 1e-14 * scale
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_patch_sums_match_oracle_and_make_up_the_totals(fv, prec):
    """fv_patch_sums: every valid patch's FP64 sums within 1e-14 of the
    oracle's (relative to the sum of magnitudes), the totals it writes
    bitwise those of fv_conserved_totals, the row of an invalid patch left
    alone and reported."""
    torch = fvtest.torch_cuda()
    d, p, n = 2, 8, 2100  # three sum chunks, the last ragged
    s = d + 2
    q, off, sz = fvtest.random_batch(n, p, d, 19, np.float32 if prec else np.float64)
    tq = fvtest.to_dev(q)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    per = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    t1 = torch.zeros(s, dtype=torch.float64, device="cuda")
    t2 = torch.zeros(s, dtype=torch.float64, device="cuda")
    fv.fv_patch_sums(b.h, tq, toff, tsz, n, per, t1)
    b.totals(tq, toff, tsz, t2)
    assert b.status() == fv.FV_OK
    assert torch.equal(t1, t2)
    q64 = q.astype(np.float64)
    ps = oracle.patch_sums(q64, off, sz, d, s)
    pa = oracle.patch_sums(np.abs(q64), off, sz, d, s)
    got = per.cpu().numpy()
    assert np.all(np.abs(got - ps) <= 2e-14 * pa)  # both sums of <= 64 terms
    for v in range(s):
        assert abs(t1[v].item() - math.fsum(got[:, v])) <= 1e-14 * math.fsum(pa[:, v])
    # an invalid patch: reported, its row untouched; totals may be omitted
    bad = sz.copy()
    bad[7] = 0
    per2 = torch.full((n, s), float("nan"), dtype=torch.float64, device="cuda")
    fv.fv_patch_sums(b.h, tq, toff, fvtest.to_dev(bad), n, per2)
    assert b.status() == fv.FV_ERR_BAD_PATCH
    got2 = per2.cpu().numpy()
    assert np.all(np.isnan(got2[7])) and np.array_equal(np.delete(got2, 7, 0), np.delete(got, 7, 0))
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_sums(b.h, tq, toff, tsz, n, None)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    b.close()


def test_multistep_periodic_matches_oracle_and_conserves(fv):
    """Ten steps of halo fill -> CFL reduce -> update with the device dt on a
    periodic 2D patch mesh: parity with the oracle's own steps, and the
    conserved totals drift only by roundoff."""
    torch = fvtest.torch_cuda()
    d, p, grid = 2, 5, (8, 6)
    s = d + 2
    N = [g * p for g in grid]
    rng = np.random.default_rng(18)
    U = inputs.random_cells(rng, N[0] * N[1], d).reshape(N[1], N[0], s)
    q, off, sz, _ = inputs.domain_to_patches(U, p)
    nbr = inputs.grid_neighbours(grid)
    dx, cfl = 1.0 / N[0], 0.4
    b = fv.Batch(d, max_patch_size=p)
    qa, qb = fvtest.to_dev(q), fvtest.to_dev(q)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    tot0 = torch.zeros(s, dtype=torch.float64, device="cuda")
    tot1 = torch.zeros(s, dtype=torch.float64, device="cuda")
    ref = q.copy()
    for _ in range(10):
        b.halo_fill(qa, toff, tsz, tnbr)
        b.max_eigenvalue(qa, toff, tsz, cfl, dx)
        b.update(qa, qb, toff, tsz, dx, -1.0)
        qa, qb = qb, qa
        ref, _dt = oracle.step(ref, off, sz, nbr, d, dx, cfl)
    b.totals(fvtest.to_dev(q), toff, tsz, tot0)
    b.totals(qa, toff, tsz, tot1)
    assert b.status() == fv.FV_OK
    mask = fvtest.interior_mask(off, sz, d, s, len(q))
    err = fvtest.per_unknown_rel_err(qa.cpu().numpy(), ref, mask, s)
    assert np.all(err <= 1e-11), err
    drift = (tot1 - tot0).abs().cpu().numpy()
    assert np.all(drift <= 1e-12 * np.abs(tot0.cpu().numpy()) + 1e-13)
    b.close()
