"""The batched update on patches in host memory (fv_patch_update_host): the
chunked copy-in / update / copy-out pipeline gives bitwise the device
update's result for any chunk size, mixed patch sizes and both precisions;
halo cells come back as they went in; bad layouts are refused."""
import numpy as np
import pytest

from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("chunk", [0, 1, 7, 1000])
def test_host_pipeline_equals_device_update_bitwise(fv, prec, chunk):
    torch = fvtest.torch_cuda()
    n = 301
    sizes = inputs.uneven_sizes(n, seed=80, mix=((3, 0.5), (5, 0.3), (4, 0.2)))
    dtype = np.float32 if prec else np.float64
    q, off, sz = inputs.random_batch(n, sizes, 3, seed=80, dtype=dtype)
    dx, dt = 0.01, 0.001
    b = fv.Batch(3, precision=prec, max_patch_size=5)
    x = fvtest.to_dev(q)
    y = x.clone()
    b.update(x, y, fvtest.to_dev(off), fvtest.to_dev(sz), dx, dt)
    ref = y.cpu().numpy()
    hin = torch.from_numpy(q).pin_memory()
    hout = torch.full_like(hin, float("nan")).pin_memory()
    fv.fv_patch_update_host(b.h, hin, hout, off, sz, n, dx, dt, chunk)
    assert b.status() == fv.FV_OK
    got = hout.numpy()
    mask = fvtest.interior_mask(off, sz, 3, 5, len(q))
    assert np.array_equal(got[mask], ref[mask])
    covered = np.zeros(len(q), dtype=bool)
    for o, p in zip(off, sz):
        covered[int(o):int(o) + (int(p) + 2) ** 3 * 5] = True
    halo = covered & ~mask
    assert np.array_equal(got[halo], q[halo])
    # a second call reuses the staging
    fv.fv_patch_update_host(b.h, hin, hout, off, sz, n, dx, dt, chunk)
    assert np.array_equal(hout.numpy()[mask], ref[mask])
    b.close()


def test_host_pipeline_device_dt_and_pageable_buffers(fv):
    torch = fvtest.torch_cuda()
    d, p, n = 2, 8, 200
    q, off, sz = fvtest.random_batch(n, p, d, 81)
    dx, cfl = 1.0 / 128, 0.4
    b = fv.Batch(d, max_patch_size=p)
    x = fvtest.to_dev(q)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    b.max_eigenvalue(x, toff, tsz, cfl, dx)
    y = x.clone()
    b.update(x, y, toff, tsz, dx, -1.0)  # the device dt
    out = np.full_like(q, np.nan)
    fv.fv_patch_update_host(b.h, q, out, off, sz, n, dx, -1.0, 33)  # numpy (pageable)
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert np.array_equal(out[mask], y.cpu().numpy()[mask])
    assert b.status() == fv.FV_OK
    b.close()


def test_host_pipeline_refuses_bad_layouts(fv):
    d, p, n = 2, 4, 10
    q, off, sz = fvtest.random_batch(n, p, d, 82)
    out = np.zeros_like(q)
    b = fv.Batch(d, max_patch_size=p)
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_host(b.h, q, out, off[::-1].copy(), sz, n, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    bad = sz.copy()
    bad[3] = 9
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_host(b.h, q, out, off, bad, n, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_BAD_PATCH
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_host(b.h, q, out, off + 1, sz, n, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_ALIGNMENT
    b.close()
