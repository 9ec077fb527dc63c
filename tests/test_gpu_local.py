"""Per-patch cell size and time step (fv_patch_update_local): each patch
advances with its own dx_i and dt_i, given or from its own CFL condition,
and matches the oracle run patch by patch with those values; with one dx and
dt for all it is bitwise fv_patch_update_batch."""
import numpy as np
import pytest

import oracle
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def oracle_per_patch(q, off, sz, d, dx, dt):
    out = q.astype(np.float64).copy()
    for i in range(len(off)):
        out = oracle.patch_update(q, off[i:i + 1], sz[i:i + 1], d, float(dx[i]), float(dt[i]),
                                  q_out=out)
    return out


@pytest.mark.parametrize("d,p,n", [(3, 5, 40), (2, 8, 50), (3, 3, 60), (1, 6, 30)])
def test_given_dx_dt_per_patch_match_oracle(fv, d, p, n):
    torch = fvtest.torch_cuda()
    rng = np.random.default_rng(70 + d)
    q, off, sz = fvtest.random_batch(n, p, d, 71)
    dx = rng.uniform(0.005, 0.02, n)
    dt = 0.1 * dx
    b = fv.Batch(d, max_patch_size=p)
    x = fvtest.to_dev(q)
    y = x.clone()
    tdx, tdt = fvtest.to_dev(dx), fvtest.to_dev(dt)
    fv.fv_patch_update_local(b.h, x, y, fvtest.to_dev(off), fvtest.to_dev(sz), n, tdx, tdt)
    assert b.status() == fv.FV_OK
    assert np.array_equal(tdt.cpu().numpy(), dt)  # an input here: untouched
    ref = oracle_per_patch(q, off, sz, d, dx, dt)
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    err = fvtest.per_unknown_rel_err(y.cpu().numpy(), ref, mask, d + 2)
    assert np.all(err <= 1e-12), err
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_local_cfl_steps(fv, prec):
    """cfl > 0: dt_i = cfl dx_i / (d lambda_i) from the patch's own maximum
    wave speed, bitwise the formula on fv_max_eigenvalue_reduce's per-patch
    value; the FP64 update matches the oracle with those dt_i."""
    torch = fvtest.torch_cuda()
    d, p, n, cfl = 3, 5, 80, 0.4
    rng = np.random.default_rng(72)
    dtype = np.float32 if prec else np.float64
    q, off, sz = fvtest.random_batch(n, p, d, 73, dtype)
    dx = rng.uniform(0.005, 0.02, n)
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    x = fvtest.to_dev(q)
    y = x.clone()
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    tdx = fvtest.to_dev(dx)
    tdt = torch.zeros(n, dtype=torch.float64, device="cuda")
    lam = torch.zeros(n, dtype=torch.float64, device="cuda")
    fv.fv_patch_update_local(b.h, x, y, toff, tsz, n, tdx, tdt, cfl, lam)
    per = torch.zeros(n, dtype=torch.float64, device="cuda")
    glob = torch.zeros(1, dtype=torch.float64, device="cuda")
    b.max_eigenvalue(x, toff, tsz, cfl, 1.0, per, glob)
    assert b.status() == fv.FV_OK
    lam_np, dt_np = lam.cpu().numpy(), tdt.cpu().numpy()
    assert np.array_equal(lam_np, per.cpu().numpy())
    assert np.array_equal(dt_np, (cfl * dx) / (d * lam_np))
    if prec == 0:
        ref = oracle_per_patch(q, off, sz, d, dx, dt_np)
        mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
        err = fvtest.per_unknown_rel_err(y.cpu().numpy(), ref, mask, d + 2)
        assert np.all(err <= 1e-12), err
        lam_ref, _ = oracle.max_eigenvalue(q, off, sz, d)
        assert np.allclose(lam_np, lam_ref, rtol=1e-14, atol=0)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_uniform_dx_dt_equal_batch_update_bitwise(fv, prec):
    torch = fvtest.torch_cuda()
    d, p, n = 2, 8, 64
    dtype = np.float32 if prec else np.float64
    q, off, sz = fvtest.random_batch(n, p, d, 74, dtype)
    dx, dt = 1.0 / 64, 0.002
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    x = fvtest.to_dev(q)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    y0, y1 = x.clone(), x.clone()
    b.update(x, y0, toff, tsz, dx, dt)
    tdx = torch.full((n,), dx, dtype=torch.float64, device="cuda")
    tdt = torch.full((n,), dt, dtype=torch.float64, device="cuda")
    fv.fv_patch_update_local(b.h, x, y1, toff, tsz, n, tdx, tdt)
    assert b.status() == fv.FV_OK
    assert torch.equal(y0, y1)
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_local(b.h, x, y1, toff, tsz, n, None, tdt)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    b.close()
