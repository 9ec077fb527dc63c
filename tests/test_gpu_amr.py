"""Halos of 3:1 refined meshes on the GPU (fv_amr_plan_create /
fv_amr_halo_fill) against the oracle (oracle/amr.py): same-level copies,
constant prolongation from coarser neighbours, restriction from finer ones,
periodic / outflow / wall edges, FP64 and FP32; a time step of a refined mesh
(AMR halos + per-patch cell sizes) against the oracle patch by patch; and the
refusal of meshes the plan cannot serve."""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def face_halo_mask(off, p, d, s, total):
    m = np.zeros(total, dtype=bool)
    ne = p + 2
    for o in off:
        blk = np.zeros((ne,) * d + (s,), dtype=bool)
        for k in range(d):
            for c in (0, ne - 1):
                sl = [slice(1, ne - 1)] * d
                sl[d - 1 - k] = c
                blk[tuple(sl)] = True
        m[int(o):int(o) + blk.size] = blk.reshape(-1)
    return m


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("d,p,lev,refine,boundary", [
    (2, 4, 1, [(1, 1)], 0), (2, 3, 1, [(0, 0), (2, 1)], -1), (2, 6, 1, [(1, 0), (1, 1)], -2),
    (3, 3, 1, [(1, 1, 1)], 0), (3, 4, 1, [(0, 2, 1)], -2), (1, 5, 2, [(4,), (0,)], 0),
    (2, 5, 2, [(4, 4), (0, 8)], 0)])
def test_amr_halos_match_oracle(fv, prec, d, p, lev, refine, boundary):
    s = d + 2
    dtype = np.float32 if prec else np.float64
    q, off, sz, level, coord = inputs.amr_mesh(d, p, lev, refine, seed=5, dtype=dtype)
    ref = amr.amr_halo_fill(q.astype(np.float64), off, p, d, level, coord, boundary)
    b = fv.Batch(d, precision=prec, max_patch_size=p)
    plan = fv.AmrPlan(b.h, level, coord, off, p, boundary)
    x = fvtest.to_dev(q)
    plan.fill(x)
    assert b.status() == fv.FV_OK
    got = x.cpu().numpy().astype(np.float64)
    mask = face_halo_mask(off, p, d, s, len(q))
    tol = 1e-14 if prec == 0 else 1e-6
    assert np.allclose(got[mask], ref[mask], rtol=tol, atol=tol)
    assert np.array_equal(got[~mask], q[~mask].astype(np.float64))  # nothing else written
    plan.close()
    b.close()


@pytest.mark.parametrize("boundary", [0, -1, -2])
def test_single_level_equals_uniform_halo_fill_bitwise(fv, boundary):
    d, p, lev = 3, 4, 1
    q, off, sz, level, coord = inputs.amr_mesh(d, p, lev, (), seed=6)
    nbr = inputs.grid_neighbours((3,) * d, periodic=boundary == 0,
                                 boundary=boundary if boundary else -1)
    b = fv.Batch(d, max_patch_size=p)
    plan = fv.AmrPlan(b.h, level, coord, off, p, boundary)
    x, y = fvtest.to_dev(q), fvtest.to_dev(q)
    plan.fill(x)
    b.halo_fill(y, fvtest.to_dev(off), fvtest.to_dev(sz), fvtest.to_dev(nbr))
    assert b.status() == fv.FV_OK
    assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
    plan.close()
    b.close()


def test_refined_mesh_time_step_matches_oracle(fv):
    """AMR halos, then each patch advances with its own cell size and one dt
    (fv_patch_update_local); the oracle does the same patch by patch."""
    torch = fvtest.torch_cuda()
    d, p, lev, refine = 2, 6, 1, [(1, 1), (2, 2)]
    q, off, sz, level, coord = inputs.amr_mesh(d, p, lev, refine, seed=7)
    n = len(off)
    dx = 1.0 / (3.0 ** level * p)
    dt = np.full(n, 0.1 * dx.min())
    b = fv.Batch(d, max_patch_size=p)
    plan = fv.AmrPlan(b.h, level, coord, off, p, 0)
    x = fvtest.to_dev(q)
    y = x.clone()
    plan.fill(x)
    fv.fv_patch_update_local(b.h, x, y, fvtest.to_dev(off), fvtest.to_dev(sz), n,
                             fvtest.to_dev(dx), fvtest.to_dev(dt))
    assert b.status() == fv.FV_OK
    qh = amr.amr_halo_fill(q, off, p, d, level, coord, 0)
    ref = qh.copy()
    for i in range(n):
        ref = oracle.patch_update(qh, off[i:i + 1], sz[i:i + 1], d, float(dx[i]), float(dt[i]),
                                  q_out=ref)
    mask = fvtest.interior_mask(off, sz, d, d + 2, len(q))
    err = fvtest.per_unknown_rel_err(y.cpu().numpy(), ref, mask, d + 2)
    assert np.all(err <= 1e-12), err
    plan.close()
    b.close()


def test_plans_the_mesh_cannot_serve_are_refused(fv):
    d = 2
    b = fv.Batch(d, max_patch_size=8)
    # a hole: one child of a refined cell missing
    q, off, sz, level, coord = inputs.amr_mesh(d, 4, 1, [(1, 1)], seed=8)
    with pytest.raises(fv.FvError) as e:
        fv.AmrPlan(b.h, level[:-1], coord[:-1], off[:-1], 4, 0)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    # two patches on one tree cell
    with pytest.raises(fv.FvError) as e:
        fv.AmrPlan(b.h, np.r_[level, level[:1]], np.r_[coord, coord[:1]], np.r_[off, off[:1]],
                   4, 0)
    assert e.value.status == fv.FV_ERR_INVALID_ARG
    # refined meshes with p < 3
    q, off, sz, level, coord = inputs.amr_mesh(d, 2, 1, [(1, 1)], seed=8)
    with pytest.raises(fv.FvError) as e:
        fv.AmrPlan(b.h, level, coord, off, 2, 0)
    assert e.value.status == fv.FV_ERR_UNSUPPORTED
    b.close()
