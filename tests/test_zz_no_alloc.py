"""fv_conserved_totals_noalloc, the allocation-free conservation sums.

Callers that own the whole GPU through their own memory pool, or that run
latency-critical loops where cudaMalloc/cudaFree would synchronise the
device, cannot create a handle (its workspace is allocated).  The
allocation-free entry point keeps its scratch in a static device array of
the library.  These checks call it through the C ABI and compare it with the
handle-based fv_conserved_totals on two consecutive calls with different
inputs: the results must agree bitwise (the tests' tolerance for the
fixed-order sums, which are deterministic), so the second call cannot pass
on the first call's leftover scratch.  This file is collected last.
"""
import numpy as np
import pytest

from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def _handle_totals(fv, d, prec, tq, toff, tsz):
    torch = fvtest.torch_cuda()
    b = fv.Batch(d, precision=prec, max_patch_size=7)
    out = torch.zeros(d + 2, dtype=torch.float64, device="cuda")
    b.totals(tq, toff, tsz, out)
    assert b.status() == fv.FV_OK
    b.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_totals_match_handle_totals_twice(fv, prec):
    torch = fvtest.torch_cuda()
    dtype = np.float32 if prec else np.float64
    calls = [(3, 5, 2500, 31), (2, 7, 1500, 32)]  # two calls, different data and shapes
    for d, p, n, seed in calls:
        q, off, sz = fvtest.random_batch(n, p, d, seed, dtype)
        tq, toff, tsz = fvtest.to_dev(q), fvtest.to_dev(off), fvtest.to_dev(sz)
        ref = _handle_totals(fv, d, prec, tq, toff, tsz)
        got = torch.full((d + 2,), -7.0, dtype=torch.float64, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        fv.fv_conserved_totals_noalloc(d, d + 2, prec, tq, toff, tsz, n, got, status)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (got, ref)
        assert status.item() == 0


def test_noalloc_rejects_batches_beyond_its_scratch(fv):
    torch = fvtest.torch_cuda()
    q = torch.zeros(64, dtype=torch.float64, device="cuda")
    off = torch.zeros(1, dtype=torch.int64, device="cuda")
    sz = torch.ones(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(fv.FvError) as e:
        fv.fv_conserved_totals_noalloc(3, 5, 0, q, off, sz, 4096 * 1024 + 1, out, status)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    fv.fv_conserved_totals_noalloc(3, 5, 0, q, off, sz, 0, out, status)  # empty batch: zeros
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)


def test_noalloc_needs_a_status_word(fv):
    """Without a status word of the caller's the bad-patch bit would have
    nowhere to go: the call is refused and enqueues nothing."""
    torch = fvtest.torch_cuda()
    q, off, sz = fvtest.random_batch(10, 3, 2, 33)
    tq, toff, tsz = fvtest.to_dev(q), fvtest.to_dev(off), fvtest.to_dev(sz)
    out = torch.full((4,), -7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(fv.FvError) as e:
        fv.fv_conserved_totals_noalloc(2, 4, 0, tq, toff, tsz, 10, out, None)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    torch.cuda.synchronize()
    assert torch.all(out == -7.0)


def test_noalloc_reports_a_bad_patch_in_the_callers_word(fv):
    """A patch of size 65 (beyond 1..64) is skipped and bit 1 (bad patch) is
    OR-ed into the caller's status word; the other patches' totals equal the
    handle path's on the same batch, bitwise."""
    torch = fvtest.torch_cuda()
    d, p, n = 3, 4, 600
    q, off, sz = fvtest.random_batch(n, p, d, 34)
    bad = sz.copy()
    bad[17] = 65
    tq, toff, tbad = fvtest.to_dev(q), fvtest.to_dev(off), fvtest.to_dev(bad)
    b = fv.Batch(d, max_patch_size=7)
    ref = torch.zeros(d + 2, dtype=torch.float64, device="cuda")
    b.totals(tq, toff, tbad, ref)
    assert b.status() == fv.FV_ERR_BAD_PATCH
    b.close()
    got = torch.zeros(d + 2, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    fv.fv_conserved_totals_noalloc(d, d + 2, 0, tq, toff, tbad, n, got, status)
    torch.cuda.synchronize()
    assert status.item() == 1
    assert torch.equal(got, ref)
    # the same batch without the bad patch's contribution, summed in numpy
    keep = np.ones(n, dtype=bool)
    keep[17] = False
    mask = fvtest.interior_mask(off[keep], sz[keep], d, d + 2, len(q))
    exp = q[mask].reshape(-1, d + 2).sum(axis=0)
    assert np.allclose(got.cpu().numpy(), exp, rtol=1e-13, atol=0)
