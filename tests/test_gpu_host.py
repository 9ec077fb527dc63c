"""The batched update on patches in host memory (fv_patch_update_host): the
chunked copy-in / update / copy-out pipeline gives bitwise the device
update's result for any chunk size, mixed patch sizes and both precisions;
halo cells come back as they went in; in place (host_in == host_out, where
equally spaced patches of one size copy back only their interior spans) the
whole buffer ends as out of place, also when the device staging still holds
another batch's values; the results match the oracle's update (1e-12 in
FP64; 1e-5 in FP32 against the oracle on the FP32-rounded input); bad
layouts are refused."""
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
    oref = oracle.patch_update(q.astype(np.float64), off, sz, 3, dx, dt)
    tol = 1e-5 if prec else 1e-12
    assert np.all(fvtest.per_unknown_rel_err(got, oref, mask, 5) <= tol)
    covered = np.zeros(len(q), dtype=bool)
    for o, p in zip(off, sz):
        covered[int(o):int(o) + (int(p) + 2) ** 3 * 5] = True
    halo = covered & ~mask
    assert np.array_equal(got[halo], q[halo])
    # a second call reuses the staging
    fv.fv_patch_update_host(b.h, hin, hout, off, sz, n, dx, dt, chunk)
    assert np.array_equal(hout.numpy()[mask], ref[mask])
    b.close()


def spaced_batch(q, off, sz, d, gap_every):
    """The boxes of a batch moved apart by 8 extra elements after every
    gap_every-th patch (equal sizes, unequal spacing)."""
    box = (int(sz[0]) + 2) ** d * (d + 2)
    off2 = off + 8 * (np.arange(len(off)) // gap_every)
    q2 = np.zeros(int(off2[-1]) + box + 8, dtype=q.dtype)
    for o, o2 in zip(off, off2):
        q2[int(o2):int(o2) + box] = q[int(o):int(o) + box]
    return q2, off2


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case,chunk", [("uniform3d", 0), ("uniform3d", 7), ("uniform2d", 0),
                                        ("uneven", 5), ("spaced", 4), ("one", 0)])
def test_in_place_equals_out_of_place_bitwise(fv, prec, case, chunk):
    torch = fvtest.torch_cuda()
    dtype = np.float32 if prec else np.float64
    d, p = (2, 8) if case == "uniform2d" else (3, 5)
    n = 1 if case == "one" else 157
    if case == "uneven":
        sizes = inputs.uneven_sizes(n, seed=83, mix=((3, 0.5), (5, 0.5)))
        q, off, sz = inputs.random_batch(n, sizes, d, seed=83, dtype=dtype)
    else:
        q, off, sz = fvtest.random_batch(n, p, d, 83, dtype)
        if case == "spaced":
            q, off = spaced_batch(q, off, sz, d, 3)
    dx, dt = 0.01, 0.001
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    hin = torch.from_numpy(q).pin_memory()
    hout = torch.from_numpy(q.copy()).pin_memory()  # halos and gaps as the input's
    fv.fv_patch_update_host(b.h, hin, hout, off, sz, n, dx, dt, chunk)
    hbuf = torch.from_numpy(q.copy()).pin_memory()
    fv.fv_patch_update_host(b.h, hbuf, hbuf, off, sz, n, dx, dt, chunk)
    assert b.status() == fv.FV_OK
    assert np.array_equal(hbuf.numpy(), hout.numpy())
    x = fvtest.to_dev(q)
    y = x.clone()
    b.update(x, y, fvtest.to_dev(off), fvtest.to_dev(sz), dx, dt)
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert np.array_equal(hbuf.numpy()[mask], y.cpu().numpy()[mask])
    assert not np.array_equal(hbuf.numpy()[mask], q[mask])
    oref = oracle.patch_update(q.astype(np.float64), off, sz, d, dx, dt)
    tol = 1e-5 if prec else 1e-12
    assert np.all(fvtest.per_unknown_rel_err(hbuf.numpy(), oref, mask, d + 2) <= tol)
    b.close()


@pytest.mark.parametrize("prec,d,p", [(0, 3, 5), (1, 3, 5), (0, 3, 3), (1, 3, 7), (1, 2, 5),
                                        (0, 2, 8)])
def test_in_place_after_poisoned_staging(fv, prec, d, p):
    """In place, the span upload leaves the cells of a box outside the span
    (leading and trailing edge / corner cells) as the staging slot last held
    them, and 3D boxes come back plane by plane (each z-plane's interior
    span).  Fill every slot with NaN boxes first (an out-of-place call on a
    NaN batch of the same layout, whose non-physical status is read and
    cleared), then run the in-place call: no NaN may reach the update (status
    FV_OK), the interiors match the oracle, and every halo and gap element of
    the host buffer stays as it was."""
    torch = fvtest.torch_cuda()
    dtype = np.float32 if prec else np.float64
    n, chunk = 157, 16
    q, off, sz = fvtest.random_batch(n, p, d, 85 + d, dtype)
    dx, dt = 0.01, 0.001
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    poison = torch.full((len(q),), float("nan"), dtype=torch.from_numpy(q).dtype).pin_memory()
    sink = torch.zeros_like(poison).pin_memory()
    fv.fv_patch_update_host(b.h, poison, sink, off, sz, n, dx, dt, chunk)
    assert b.status() == fv.FV_ERR_NONPHYSICAL  # the slots now hold NaN boxes
    hbuf = torch.from_numpy(q.copy()).pin_memory()
    fv.fv_patch_update_host(b.h, hbuf, hbuf, off, sz, n, dx, dt, chunk)
    assert b.status() == fv.FV_OK
    got = hbuf.numpy()
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert not np.isnan(got).any()
    assert np.array_equal(got[~mask], q[~mask])
    oref = oracle.patch_update(q.astype(np.float64), off, sz, d, dx, dt)
    tol = 1e-5 if prec else 1e-12
    assert np.all(fvtest.per_unknown_rel_err(got, oref, mask, d + 2) <= tol)
    x = fvtest.to_dev(q)
    y = x.clone()
    b.update(x, y, fvtest.to_dev(off), fvtest.to_dev(sz), dx, dt)
    assert np.array_equal(got[mask], y.cpu().numpy()[mask])
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
