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
    with pytest.raises(fv.FvError) as e:
        fv.fv_conserved_totals_noalloc(3, 5, 0, q, off, sz, 4096 * 1024 + 1, out)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    fv.fv_conserved_totals_noalloc(3, 5, 0, q, off, sz, 0, out)  # empty batch: zeros
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)
