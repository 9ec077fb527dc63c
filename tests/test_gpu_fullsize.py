"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times, on sampled patches (and faces) the oracle computes one by one.

* 3D Euler FP64, 262,144 patches of 5^3 on a 64^3 periodic patch mesh: the
  time step with the primitive carry, two steps (the second reads carried
  primitives); each step against an oracle step from the same state.  The
  same mesh in FP32, the batch planned (the one-size 5^3 kernel), two steps.
* Uneven batch, 200,000 patches (50/30/20 % of 3^3/5^3/7^3, self-periodic),
  FP64 and FP32: per-size-class launches with autotuned CTA sizes, one step
  of the multi-step graph driver.
* Precision workload, 2D periodic 4095^2 in 5x5 patches, FP32 and FP64: one
  step of the graph driver.
* Learned correction on the 1024^2 shear layer: sampled faces of the
  tensor-core correction against the network evaluated by the oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import learned as olearned
from oracle import mlp as omlp
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def interior(q, off, p, d, s, i):
    ne = p + 2
    blk = q[int(off[i]):int(off[i]) + ne ** d * s].reshape((ne,) * d + (s,))
    return blk[(slice(1, p + 1),) * d]


def oracle_step_sampled(q, off, sz, nbr, d, dx, cfl, ids):
    """Oracle step of the sampled patches: halo fill and CFL maximum over the
    whole batch, the update of the sampled patches only.  Returns (per-id
    interiors, dt)."""
    s = d + 2
    qh = q.astype(np.float64)  # a copy
    oracle.halo_fill(qh, off, sz, nbr, d, s)
    _, lam = oracle.max_eigenvalue(qh, off, sz, d)
    dt = oracle.cfl_dt(lam, cfl, dx, d)
    # the sampled patches (halos filled) as a batch of their own
    lens = [(int(sz[i]) + 2) ** d * s for i in ids]
    coff = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    cq = np.concatenate([qh[int(off[i]):int(off[i]) + ln] for i, ln in zip(ids, lens)])
    csz = sz[ids].astype(np.int32)
    cout = oracle.patch_update(cq, coff, csz, d, dx, dt)
    res = {i: interior(cout, coff, int(csz[c]), d, s, c).copy() for c, i in enumerate(ids)}
    return res, dt


def check_sampled(got_q, ref, off, sz, d, tol):
    s = d + 2
    worst = np.zeros(s)
    for i, want in ref.items():
        worst = np.maximum(worst, np.abs(interior(got_q, off, int(sz[i]), d, s, i) - want)
                           .reshape(-1, s).max(axis=0))
    scale = np.max(np.abs(np.concatenate([w.reshape(-1, s) for w in ref.values()])), axis=0)
    err = worst / scale
    assert np.all(err <= tol), err


def test_config2_fp64_carry_steps_full_size(fv):
    torch = fvtest.torch_cuda()
    d, p, grid = 3, 5, (64, 64, 64)
    n = int(np.prod(grid))
    q, off, sz = inputs.random_batch(n, p, d, seed=0)
    nbr = inputs.grid_neighbours(grid)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    ids = np.sort(np.random.default_rng(1).choice(n, 48, replace=False))
    stream = torch.cuda.Stream()
    b = fv.Batch(d, max_patch_size=p, stream=stream)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    prims = [torch.empty(n * b.prim_stride(), dtype=torch.float64, device="cuda")
             for _ in range(2)]
    state = q
    with torch.cuda.stream(stream):
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
    for step, (pin, pout) in enumerate(((None, prims[0]), (prims[0], prims[1]))):
        with torch.cuda.stream(stream):
            b.time_step_prim(x, y, pin, pout, toff, tsz, tnbr, dx, cfl)
        stream.synchronize()
        assert b.status() == fv.FV_OK
        got = y.cpu().numpy()
        ref, dt_ref = oracle_step_sampled(state, off, sz, nbr, d, dx, cfl, ids)
        assert fv.fv_read_dt(b.h) == pytest.approx(dt_ref, rel=1e-14)
        check_sampled(got, ref, off, sz, d, TOL64)
        state = got
        x, y = y, x
    b.close()


def test_config2_fp32_planned_steps_full_size(fv):
    """The same mesh in FP32 as bench.py's FP32 variant times it: the batch
    planned, so the one-size kernel for 5^3 runs; two time steps, sampled
    patches against the oracle (FP64 from the FP32 state) at 1e-5."""
    torch = fvtest.torch_cuda()
    d, p, grid = 3, 5, (64, 64, 64)
    n = int(np.prod(grid))
    q, off, sz = inputs.random_batch(n, p, d, seed=0, dtype=np.float32)
    nbr = inputs.grid_neighbours(grid)
    dx, cfl = 1.0 / (grid[0] * p), 0.4
    ids = np.sort(np.random.default_rng(2).choice(n, 48, replace=False))
    stream = torch.cuda.Stream()
    b = fv.Batch(d, precision=fv.FV_FP32, max_patch_size=p, stream=stream)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    fv.fv_batch_plan(b.h, tsz, n)
    state = q
    with torch.cuda.stream(stream):
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
    for step in range(2):
        with torch.cuda.stream(stream):
            b.time_step(x, y, toff, tsz, tnbr, dx, cfl)
        stream.synchronize()
        assert b.status() == fv.FV_OK
        got = y.cpu().numpy()
        ref, dt_ref = oracle_step_sampled(state.astype(np.float64), off, sz, nbr, d, dx, cfl, ids)
        assert fv.fv_read_dt(b.h) == pytest.approx(dt_ref, rel=1e-6)
        check_sampled(got.astype(np.float64), ref, off, sz, d, TOL32)
        state = got
        x, y = y, x
    assert fv.fv_batch_pairs_launches(b.h) == 2
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_config3_uneven_classes_graph_step_full_size(fv, prec):
    torch = fvtest.torch_cuda()
    n, d = 200000, 3
    sizes = inputs.uneven_sizes(n, seed=0)
    q64, off, sz = inputs.random_batch(n, sizes, d, seed=0, align_bytes=32)
    q = q64 if prec == 0 else q64.astype(np.float32)
    nbr = inputs.self_periodic_neighbours(n, d)
    dx, cfl = 1.0 / 64, 0.4
    stream = torch.cuda.Stream()
    b = fv.Batch(d, precision=prec, max_patch_size=7, stream=stream)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    with torch.cuda.stream(stream):
        b.halo_fill(x, toff, tsz, tnbr)
        b.max_eigenvalue(x, toff, tsz, cfl, dx)
    fv.fv_batch_autotune(b.h, x, y, toff, tsz, tnbr, n, dx, cfl)
    x.copy_(torch.from_numpy(q))
    with torch.cuda.stream(stream):
        b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, 1, use_graph=True)
    stream.synchronize()
    assert b.status() == fv.FV_OK
    got = y.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2)
    ids = np.sort(np.concatenate([rng.choice(np.nonzero(sz == pp)[0], 16, replace=False)
                                  for pp in (3, 5, 7)]))
    ref, _ = oracle_step_sampled(q.astype(np.float64), off, sz, nbr, d, dx, cfl, ids)
    check_sampled(got, ref, off, sz, d, TOL64 if prec == 0 else TOL32)
    b.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_config4_precision_graph_step_full_size(fv, prec):
    torch = fvtest.torch_cuda()
    N, p = 4095, 5
    U = inputs.fourier_perturbation(N, seed=0)
    q64, off, sz, grid = inputs.domain_to_patches(U, p, align_bytes=32)
    del U
    q = q64 if prec == 0 else q64.astype(np.float32)
    nbr = inputs.grid_neighbours(grid)
    n = len(off)
    dx, cfl = 1.0 / N, 0.4
    stream = torch.cuda.Stream()
    b = fv.Batch(2, precision=prec, max_patch_size=p, stream=stream)
    x = torch.from_numpy(q).cuda()
    y = x.clone()
    toff, tsz, tnbr = (torch.from_numpy(a).cuda() for a in (off, sz, nbr))
    with torch.cuda.stream(stream):
        b.run_steps(x, y, toff, tsz, tnbr, dx, cfl, 1, use_graph=True)
    stream.synchronize()
    assert b.status() == fv.FV_OK
    got = y.cpu().numpy().astype(np.float64)
    ids = np.sort(np.random.default_rng(3).choice(n, 64, replace=False))
    ref, _ = oracle_step_sampled(q.astype(np.float64), off, sz, nbr, 2, dx, cfl, ids)
    check_sampled(got, ref, off, sz, 2, TOL64 if prec == 0 else TOL32)
    b.close()


def test_config5_correction_sampled_faces_full_size(fv):
    torch = fvtest.torch_cuda()
    from paper_2302_09005_gb300 import learned
    N, p = 1024, 8
    U = inputs.shear_layer(N, seed=3)
    stream = torch.cuda.current_stream()
    m = learned.Mesh2D(N, p, fv.FV_FP64, stream, U=U)
    rng = np.random.default_rng(4)
    theta = omlp.init_params(5) + 0.05 * rng.standard_normal(omlp.N_PARAM)
    theta = theta.astype(np.float32).astype(np.float64)
    mu = rng.uniform(-0.2, 1.2, 16)
    sd = rng.uniform(0.3, 1.0, 16)
    sdy = rng.uniform(0.01, 0.05, 4)
    pv = fvtest.to_dev(theta, torch.float32)
    nv = fvtest.to_dev(np.concatenate([mu, sd, sdy]), torch.float32)
    stride = fv.fv_corr_stride(m.b.h)
    corr = torch.zeros(m.n * stride, dtype=torch.float32, device="cuda")
    fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, pv, nv, corr)
    assert m.b.status() == fv.FV_OK
    got = corr.cpu().numpy().astype(np.float64)
    nf1 = (p + 1) * p
    grid = (N // p, N // p)
    r = omlp.bf16_round
    prm = omlp.unpack(theta)
    worst, scale = 0.0, 0.0
    for axis, k in ((1, 0), (0, 1)):  # x faces (normal along axis 1 of U), y faces
        S = ((olearned.stencils(U, axis) - mu) / sd).astype(np.float32).astype(np.float64)
        for _ in range(256):  # sampled faces: patch, face index
            pid = int(rng.integers(m.n))
            j = int(rng.integers(nf1))
            a, bb = pid % grid[0], pid // grid[0]
            b_, tr = j // p, j % p
            if k == 0:
                J, I = bb * p + tr, (a * p + b_) % N
            else:
                J, I = (bb * p + b_) % N, a * p + tr
            xb = r(S[J, I].reshape(1, 16))
            h1 = r(omlp.gelu(xb @ r(prm["W1"]).T + prm["b1"]))
            h2 = r(omlp.gelu(h1 @ r(prm["W2"]).T + prm["b2"]))
            y = (h2 @ r(prm["W3"]).T + prm["b3"])[0] * sdy
            want = olearned.to_normal(y, axis)  # physical frame
            base = pid * stride + k * 4 * nf1
            have = np.array([got[base + v * nf1 + j] for v in range(4)])
            worst = max(worst, float(np.max(np.abs(have - want))))
            scale = max(scale, float(np.max(np.abs(want))))
    assert worst <= 2e-2 * scale, (worst, scale)
    m.close()
