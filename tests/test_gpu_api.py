"""Edge cases of the C ABI on the GPU: empty batches, argument errors
answered on the host, bad per-patch metadata and non-physical states
reported through the device status word (never a trap), the largest patch
size, and two handles on two streams at once."""
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


def setup_batch(n=8, p=3, d=3, seed=0, dtype=np.float64):
    q, off, sz = fvtest.random_batch(n, p, d, seed, dtype)
    return q, off, sz, fvtest.to_dev(q), fvtest.to_dev(off), fvtest.to_dev(sz)


def test_empty_batch_is_a_noop(fv):
    torch = fvtest.torch_cuda()
    b = fv.Batch(3, max_patch_size=5)
    q = torch.ones(64, dtype=torch.float64, device="cuda")
    o = q.clone()
    off = torch.zeros(0, dtype=torch.int64, device="cuda")
    sz = torch.zeros(0, dtype=torch.int32, device="cuda")
    b.update(q, o, off, sz, 0.1, 0.01)
    b.halo_fill(q, off, sz, torch.zeros(0, dtype=torch.int32, device="cuda"))
    g = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    b.max_eigenvalue(q, off, sz, 0.4, 0.1, None, g)
    tot = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    b.totals(q, off, sz, tot)
    assert b.status() == fv.FV_OK
    assert torch.equal(q, o)
    assert g.item() == 0.0
    assert torch.all(tot == 0.0)
    b.close()


def test_host_side_argument_errors(fv):
    q, off, sz, tq, toff, tsz = setup_batch()
    b = fv.Batch(3, max_patch_size=5)
    out = tq.clone()
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_batch(b.h, tq, out, toff, tsz, len(off), 2, 4, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_batch(b.h, tq, None, toff, tsz, len(off), 3, 5, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_batch(b.h, tq, tq, toff, tsz, len(off), 3, 5, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError) as e:  # 8-byte shifted buffer
        fv.fv_patch_update_batch(b.h, tq[1:], out, toff, tsz, len(off) - 1, 3, 5, 0.1, 0.01)
    assert e.value.status == fv.FV_ERR_ALIGNMENT
    with pytest.raises(fv.FvError) as e:
        fv.fv_patch_update_batch(b.h, tq, out, toff, tsz, len(off), 3, 5, 0.0, 0.01)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError) as e:
        fv.fv_max_eigenvalue_reduce(b.h, tq, toff, tsz, len(off), cfl=-1.0, dx=0.1)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    with pytest.raises(fv.FvError):
        fv.Batch(3, max_patch_size=40)  # does not fit in shared memory
    assert b.status() == fv.FV_OK
    b.close()


def test_bad_patch_metadata_is_flagged_and_skipped(fv):
    torch = fvtest.torch_cuda()
    d, p, n = 3, 3, 10
    q, off, sz = fvtest.random_batch(n, p, d, 1)
    bad_sz = sz.copy()
    bad_sz[2] = 0      # empty patch
    bad_sz[5] = 9      # above max_patch_size
    bad_off = off.copy()
    bad_off[7] += 1    # not 16-byte aligned
    tq = fvtest.to_dev(q)
    out = tq.clone()
    b = fv.Batch(d, max_patch_size=5)
    b.update(tq, out, fvtest.to_dev(bad_off), fvtest.to_dev(bad_sz), 0.1, 0.01,
             n_elems=tq.numel())
    assert b.status() == fv.FV_ERR_BAD_PATCH
    assert b.status() == fv.FV_OK  # reading clears the word
    ref = oracle.patch_update(q, off, sz, d, 0.1, 0.01)
    got = out.cpu().numpy()
    s = d + 2
    ne = (p + 2) ** d * s
    for i in range(n):
        blk = slice(off[i], off[i] + ne)
        if i in (2, 5, 7):
            assert np.array_equal(got[blk], q[blk])  # skipped, untouched
        else:
            assert np.allclose(got[blk], ref[blk], rtol=1e-12, atol=1e-12)
    # a patch that would run past n_elems is skipped as well
    out2 = tq.clone()
    b.update(tq, out2, fvtest.to_dev(off), fvtest.to_dev(sz), 0.1, 0.01,
             n_elems=int(off[-1]) + 10)
    assert b.status() == fv.FV_ERR_BAD_PATCH
    assert torch.equal(out2[off[-1]:], tq[off[-1]:])
    # a neighbour index outside the batch
    nbr = inputs.self_periodic_neighbours(n, d)
    nbr[4, 1] = n + 3
    b.halo_fill(tq, fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr))
    assert b.status() == fv.FV_ERR_BAD_PATCH
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_nonphysical_state_is_reported(fv, prec):
    q, off, sz = fvtest.random_batch(6, 3, 2, 2, np.float32 if prec else np.float64)
    q[off[3] + 4 * 5] = -1.0  # negative density in a face-halo cell
    q[off[1] + 4 * 6 + 3] = np.nan  # NaN energy in an interior cell
    tq = fvtest.to_dev(q)
    b = fv.Batch(2, precision=prec, max_patch_size=3)
    b.update(tq, tq.clone(), fvtest.to_dev(off), fvtest.to_dev(sz), 0.1, 0.01)
    assert b.status() == fv.FV_ERR_NONPHYSICAL
    b.max_eigenvalue(tq, fvtest.to_dev(off), fvtest.to_dev(sz), 0.4, 0.1)
    assert b.status() == fv.FV_ERR_NONPHYSICAL
    b.close()


def test_largest_patch_size(fv):
    """p = max_patch_size at its shared-memory limit (3D FP64 p = 8)."""
    d, p, n = 3, 8, 30
    q, off, sz = fvtest.random_batch(n, p, d, 3)
    tq = fvtest.to_dev(q)
    out = tq.clone()
    b = fv.Batch(d, max_patch_size=8)
    b.update(tq, out, fvtest.to_dev(off), fvtest.to_dev(sz), 0.02, 0.002)
    assert b.status() == fv.FV_OK
    ref = oracle.patch_update(q, off, sz, d, 0.02, 0.002)
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    assert np.all(fvtest.per_unknown_rel_err(out.cpu().numpy(), ref, mask, d + 2) <= 1e-12)
    b.close()


def test_two_handles_two_streams(fv):
    """Concurrent offload from two handles on two streams (each its own
    workspace) gives the same results as one at a time."""
    torch = fvtest.torch_cuda()
    d, p, n = 3, 5, 500
    q, off, sz = fvtest.random_batch(n, p, d, 4)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    b1 = fv.Batch(d, max_patch_size=5, stream=s1)
    b2 = fv.Batch(d, max_patch_size=5, stream=s2)
    qa, qb = fvtest.to_dev(q), fvtest.to_dev(q)
    oa, ob = qa.clone(), qb.clone()
    torch.cuda.synchronize()
    for _ in range(3):
        b1.max_eigenvalue(qa, toff, tsz, 0.4, 0.02)
        b1.update(qa, oa, toff, tsz, 0.02, -1.0)
        b2.max_eigenvalue(qb, toff, tsz, 0.4, 0.02)
        b2.update(qb, ob, toff, tsz, 0.02, -1.0)
    assert b1.status() == fv.FV_OK and b2.status() == fv.FV_OK
    assert torch.equal(oa, ob)
    # and both equal the oracle's step (CFL dt from the batch maximum, Eq. 3-5)
    _, lam = oracle.max_eigenvalue(q, off, sz, d)
    ref = oracle.patch_update(q, off, sz, d, 0.02, oracle.cfl_dt(lam, 0.4, 0.02, d))
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    for o in (oa, ob):
        assert np.all(fvtest.per_unknown_rel_err(o.cpu().numpy(), ref, mask, d + 2) <= 1e-12)
    b1.close()
    b2.close()


def test_concurrent_offload_from_host_threads(fv):
    """Four host threads, each with its own handle and stream, offload at the
    same time: the host pipeline and device time steps, FP64 and FP32, 2D and
    3D, patch sizes whose kernels raise their shared-memory limits
    concurrently.  Every result equals the same calls made alone, bitwise,
    and the oracle (one update; three full time steps) within 1e-12 (FP64)
    or 1e-5 (FP32, against the oracle on the FP32-rounded input)."""
    import threading
    torch = fvtest.torch_cuda()
    cases = [(3, 5, 0, 300, 11), (3, 7, 1, 200, 12), (2, 17, 0, 400, 13), (3, 3, 1, 500, 14)]

    def run(case):
        d, p, prec, n, seed = case
        q, off, sz = fvtest.random_batch(n, p, d, seed, np.float32 if prec else np.float64)
        nbr = inputs.self_periodic_neighbours(n, d)
        stream = torch.cuda.Stream()
        b = fv.Batch(d, precision=prec, max_patch_size=p, stream=stream)
        hin = torch.from_numpy(q).pin_memory()
        hout = torch.from_numpy(q.copy()).pin_memory()  # the padding between boxes is not written
        for _ in range(3):
            fv.fv_patch_update_host(b.h, hin, hout, off, sz, n, 0.01, 1e-4, 64)
        with torch.cuda.stream(stream):
            x = hin.to("cuda", non_blocking=True)
            y = x.clone()
            toff = torch.from_numpy(off).to("cuda", non_blocking=True)
            tsz = torch.from_numpy(sz).to("cuda", non_blocking=True)
            tnbr = torch.from_numpy(nbr).to("cuda", non_blocking=True)
            b.halo_fill(x, toff, tsz, tnbr)
            b.max_eigenvalue(x, toff, tsz, 0.4, 0.01)
            for _ in range(3):
                b.time_step(x, y, toff, tsz, tnbr, 0.01, 0.4)
                x, y = y, x
        stream.synchronize()
        st = b.status()
        b.close()
        return st, hout.numpy().copy(), x.cpu().numpy()

    alone = [run(c) for c in cases]
    results, errors = [None] * len(cases), []

    def worker(i):
        try:
            results[i] = run(cases[i])
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for a_, r in zip(alone, results):
        assert a_[0] == fv.FV_OK and r[0] == fv.FV_OK
        assert np.array_equal(a_[1], r[1])
        assert np.array_equal(a_[2], r[2])
    for case, r in zip(cases, results):
        d, p, prec, n, seed = case
        q, off, sz = fvtest.random_batch(n, p, d, seed, np.float32 if prec else np.float64)
        q = q.astype(np.float64)
        nbr = inputs.self_periodic_neighbours(n, d)
        tol = 1e-5 if prec else 1e-12
        mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
        ref_host = oracle.patch_update(q, off, sz, d, 0.01, 1e-4)
        assert np.all(fvtest.per_unknown_rel_err(r[1], ref_host, mask, d + 2) <= tol), case
        ref = q
        for _ in range(3):
            ref, _ = oracle.step(ref, off, sz, nbr, d, 0.01, 0.4)
        assert np.all(fvtest.per_unknown_rel_err(r[2], ref, mask, d + 2) <= tol), case


@pytest.mark.parametrize("mode", ["update", "time_step"])
def test_copy_wait_that_runs_out_reports_timeout(fv, mode):
    """Every device wait is bounded.  With the step kernel's copy-wait limit
    set to one clock cycle, CTAs give up on the bulk copies of their patches:
    the status word reports FV_ERR_TIMEOUT (no trap, no hang), and after the
    default limit is restored the same handle computes the step again,
    bitwise equal to a handle that never timed out and to the oracle."""
    torch = fvtest.torch_cuda()
    d, p = 3, 5
    grid = (32, 32, 32)
    n = int(np.prod(grid))
    q, off, sz = fvtest.random_batch(n, p, d, 21)
    nbr = inputs.grid_neighbours(grid)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, dt = 1.0 / 160, 2e-4

    def run(b):
        x = fvtest.to_dev(q)
        y = torch.zeros_like(x)
        if mode == "update":
            b.update(x, y, toff, tsz, dx, dt)
        else:
            b.halo_fill(x, toff, tsz, tnbr)
            b.max_eigenvalue(x, toff, tsz, 0.4, dx)
            b.time_step(x, y, toff, tsz, tnbr, dx, 0.4)
        return y

    b = fv.Batch(d, max_patch_size=p)
    fv.fv_batch_set_wait_limit(b.h, 1)
    run(b)
    assert b.status() == fv.FV_ERR_TIMEOUT
    fv.fv_batch_set_wait_limit(b.h, 0)  # back to the default
    y = run(b)
    assert b.status() == fv.FV_OK
    ref_b = fv.Batch(d, max_patch_size=p)
    y_ref = run(ref_b)
    assert ref_b.status() == fv.FV_OK
    assert torch.equal(y, y_ref)
    with pytest.raises(fv.FvError):
        fv.fv_batch_set_wait_limit(b.h, 10 ** 12)
    b.close()
    ref_b.close()
    # the first 64 patches against the oracle
    k = 64
    got = y.cpu().numpy()
    if mode == "update":
        ref = oracle.patch_update(q, off, sz, d, dx, dt)
    else:
        ref, _ = oracle.step(q, off, sz, nbr, d, dx, 0.4)
    mask = fvtest.interior_mask(off[:k], sz[:k], d, d + 2, len(q))
    assert np.all(fvtest.per_unknown_rel_err(got, ref, mask, d + 2) <= 1e-12)


def test_fp64_reciprocal_and_sqrt_within_two_ulp(fv):
    """The FP64 kernels' Newton-refined reciprocal and square root stay
    within 2 ulp of the IEEE results over the range of physical states."""
    torch = fvtest.torch_cuda()
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(0.05, 20.0, 200000), np.exp(rng.uniform(-30, 30, 100000)),
                        np.array([1.0, 2.0, 0.5, 1e-300, 1e300])])
    tx = fvtest.to_dev(x)
    out = torch.empty_like(tx)
    for which, ref in ((0, 1.0 / x), (1, np.sqrt(x))):
        fv.fv_selftest_math(tx, out, which)
        got = out.cpu().numpy()
        ulp = np.spacing(ref)
        assert np.max(np.abs(got - ref) / ulp) <= 2.0, which
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    o = torch.empty_like(z)
    fv.fv_selftest_math(z, o, 1)
    assert torch.all(o == 0.0)
