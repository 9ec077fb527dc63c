"""Schedules of batches with uneven patch sizes: one persistent launch in
index order, one over the size-sorted order (LPT), one launch per size
class.  All give bitwise the same state, per-patch maxima and dt, which match
the oracle; the autotuner keeps the caller's wave speed and time step."""
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


def uneven(n, seed, prec, mix=((3, 0.5), (5, 0.3), (7, 0.2))):
    sizes = inputs.uneven_sizes(n, seed=seed, mix=mix)
    dtype = np.float32 if prec else np.float64
    q, off, sz = inputs.random_batch(n, sizes, 3, seed=seed, dtype=dtype)
    return q, off, sz, inputs.self_periodic_neighbours(n, 3)


@pytest.mark.parametrize("prec", [0, 1])
def test_schedules_bitwise_equal_time_step(fv, prec):
    torch = fvtest.torch_cuda()
    n = 1500
    q, off, sz, nbr = uneven(n, 51, prec, mix=((3, 0.4), (5, 0.3), (7, 0.2), (4, 0.05),
                                               (6, 0.05)))
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 0.01, 0.4
    outs, lams, dts = [], [], []
    for sched in (fv.FV_SCHED_STRIDE, fv.FV_SCHED_LPT, fv.FV_SCHED_CLASSES, fv.FV_SCHED_QUEUE):
        b = fv.Batch(3, precision=prec, max_patch_size=7)
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, sched)
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
        b.time_step(y, x, toff, tsz, tnbr, dx, cfl, lambda_patch=lam)
        assert b.status() == fv.FV_OK
        outs.append(x.cpu().numpy())
        lams.append(lam.cpu().numpy())
        dts.append(fv.fv_read_dt(b.h))
        b.close()
    mask = fvtest.interior_mask(off, sz, 3, 5, len(q))
    for o, l, t in zip(outs[1:], lams[1:], dts[1:]):
        assert np.array_equal(o[mask], outs[0][mask])
        assert np.array_equal(l, lams[0])
        assert t == dts[0]
    if prec == 0:  # two oracle steps with self-periodic halos
        ref = q.copy()
        for _ in range(2):
            ref, _ = oracle.step(ref, off, sz, nbr, 3, dx, cfl)
        err = fvtest.per_unknown_rel_err(outs[0], ref, mask, 5)
        assert np.all(err <= 1e-11), err


def test_schedules_bitwise_equal_update_mode(fv):
    torch = fvtest.torch_cuda()
    n = 900
    q, off, sz, _ = uneven(n, 52, 0)
    toff, tsz = fvtest.to_dev(off), fvtest.to_dev(sz)
    res = []
    for sched in (0, 1, 2, 3):
        b = fv.Batch(3, max_patch_size=7)
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, sched)
        x = fvtest.to_dev(q)
        y = x.clone()
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        b.update(x, y, toff, tsz, 0.02, 0.001, lambda_patch=lam)
        assert b.status() == fv.FV_OK
        res.append((y.cpu().numpy(), lam.cpu().numpy()))
        b.close()
    for y, lam in res[1:]:
        assert np.array_equal(y, res[0][0])
        assert np.array_equal(lam, res[0][1])
    ref, lam_ref = oracle.patch_update(q, off, sz, 3, 0.02, 0.001, want_lambda=True)
    mask = fvtest.interior_mask(off, sz, 3, 5, len(q))
    assert np.all(fvtest.per_unknown_rel_err(res[0][0], ref, mask, 5) <= 1e-12)
    assert np.allclose(res[0][1], lam_ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("prec", [0, 1])
def test_queue_schedule_in_a_graph_of_steps(fv, prec):
    """The work queue's counter is zeroed by a one-thread kernel before every
    launch, a kernel node of the captured graph: ten graph-replayed steps under
    FV_SCHED_QUEUE equal ten eager steps under FV_SCHED_STRIDE, bitwise."""
    torch = fvtest.torch_cuda()
    n = 2000
    q, off, sz, nbr = uneven(n, 57, prec)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    out = []
    for sched, graph in ((fv.FV_SCHED_STRIDE, False), (fv.FV_SCHED_QUEUE, True)):
        st = torch.cuda.Stream()  # graph capture needs a stream of its own
        b = fv.Batch(3, precision=prec, max_patch_size=7, stream=st)
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, sched)
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        torch.cuda.synchronize()
        b.run_steps(x, y, toff, tsz, tnbr, 0.01, 0.4, 10, use_graph=graph)
        assert b.status() == fv.FV_OK
        out.append((x.cpu().numpy(), y.cpu().numpy(), fv.fv_read_dt(b.h)))
        b.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_autotune_keeps_state_and_picks_a_schedule(fv):
    n = 2000
    q, off, sz, nbr = uneven(n, 53, 0)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 0.01, 0.4

    def run(autotune):
        b = fv.Batch(3, max_patch_size=7)
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
        chosen, ms = None, None
        if autotune:
            scratch = x.clone()
            chosen, ms = fv.fv_batch_autotune(b.h, x, scratch, toff, tsz, tnbr, n, dx, cfl)
        b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
        assert b.status() == fv.FV_OK
        out = (y.cpu().numpy(), fv.fv_read_dt(b.h))
        b.close()
        return out, chosen, ms

    (y0, dt0), _, _ = run(False)
    (y1, dt1), chosen, ms = run(True)
    assert chosen in (0, 1, 2)
    assert all(m > 0 for m in ms) and ms[chosen] == min(ms)
    mask = fvtest.interior_mask(off, sz, 3, 5, len(q))
    assert np.array_equal(y0[mask], y1[mask])
    assert dt0 == dt1


def test_classes_schedule_flags_rejected_sizes(fv):
    n = 300
    q, off, sz, _ = uneven(n, 54, 0)
    bad = sz.copy()
    bad[7] = 0
    tq = fvtest.to_dev(q)
    tbad = fvtest.to_dev(bad)
    b = fv.Batch(3, max_patch_size=7)
    fv.fv_batch_plan(b.h, tbad, n)
    fv.fv_batch_set_schedule(b.h, fv.FV_SCHED_CLASSES)
    out = tq.clone()
    b.update(tq, out, fvtest.to_dev(off), tbad, 0.02, 0.001)
    assert b.status() == fv.FV_ERR_BAD_PATCH
    ne = (sz[7] + 2) ** 3 * 5
    assert np.array_equal(out[off[7]:off[7] + ne].cpu().numpy(), q[off[7]:off[7] + ne])
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d", [2, 3])
def test_class_thread_mappings_bitwise_equal(fv, prec, d):
    """Every CTA size of the size-class launches (a warp per patch up to
    eight warps per patch) gives bitwise the same steps, in all three kernel
    modes (update, time step, time step with the primitive carry)."""
    torch = fvtest.torch_cuda()
    n = 700
    mix = ((3, 0.4), (5, 0.3), (7, 0.2), (4, 0.1)) if d == 3 else \
        ((3, 0.3), (5, 0.3), (8, 0.2), (17, 0.1), (6, 0.1))
    pmax = 7 if d == 3 else 17
    sizes = inputs.uneven_sizes(n, seed=55, mix=mix)
    dtype = np.float32 if prec else np.float64
    q, off, sz = inputs.random_batch(n, sizes, d, seed=55, dtype=dtype)
    nbr = inputs.self_periodic_neighbours(n, d)
    toff, tsz, tnbr = fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr)
    dx, cfl = 0.01, 0.4
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    ref = None
    for nt in (128, 32, 64, 256):
        b = fv.Batch(d, precision=prec, max_patch_size=pmax)
        fv.fv_batch_plan(b.h, tsz, n)
        fv.fv_batch_set_schedule(b.h, fv.FV_SCHED_CLASSES)
        for p, _ in mix:
            fv.fv_batch_set_class_threads(b.h, p, nt)
            assert fv.fv_batch_class_threads(b.h, p) == nt
        x, y = fvtest.to_dev(q), fvtest.to_dev(q)
        pa = torch.empty(n * b.prim_stride(), dtype=x.dtype, device="cuda")
        pb = torch.empty_like(pa)
        lam = torch.zeros(n, dtype=torch.float64, device="cuda")
        u = x.clone()
        b.update(x, u, toff, tsz, dx, 0.001, lambda_patch=lam)
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
        b.time_step_prim(x, y, None, pa, toff, tsz, tnbr, dx, cfl)
        b.time_step_prim(y, x, pa, pb, toff, tsz, tnbr, dx, cfl)
        assert b.status() == fv.FV_OK
        got = (u.cpu().numpy()[mask], lam.cpu().numpy(), x.cpu().numpy()[mask],
               fv.fv_read_dt(b.h))
        b.close()
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0]), nt
        assert np.array_equal(got[1], ref[1]), nt
        assert np.array_equal(got[2], ref[2]), nt
        assert got[3] == ref[3]


def test_class_threads_arguments_are_checked(fv):
    b = fv.Batch(3, max_patch_size=7)
    for p, nt, status in ((0, 128, fv.FV_ERR_INVALID_ARG), (8, 128, fv.FV_ERR_INVALID_ARG),
                          (5, 96, fv.FV_ERR_INVALID_ARG)):
        with pytest.raises(fv.FvError) as e:
            fv.fv_batch_set_class_threads(b.h, p, nt)
        assert e.value.status == status
    b.close()
    b1 = fv.Batch(1, max_patch_size=8)
    with pytest.raises(fv.FvError) as e:
        fv.fv_batch_set_class_threads(b1.h, 4, 32)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    b1.close()


def test_default_cta_size_follows_the_patch_size(fv):
    """Untuned launches and classes: a warp for up to 64 interior cells, eight
    warps for 3D patches above 200 cells, else four; d = 1 stays at 128."""
    for d, pmax, expect in ((2, 8, {5: 32, 8: 32}), (2, 17, {9: 128, 17: 128}),
                            (3, 7, {3: 32, 4: 32, 5: 128, 6: 256, 7: 256}), (1, 8, {8: 128})):
        b = fv.Batch(d, max_patch_size=pmax)
        for p, nt in expect.items():
            assert fv.fv_batch_class_threads(b.h, p) == nt, (d, p)
        b.close()
