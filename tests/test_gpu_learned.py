"""The learned conservative face-flux correction on the GPU against the FP64
oracle (oracle/learned.py, oracle/mlp.py): the tensor-core correction kernel,
the corrected update, the training targets, and the gain of a trained
network over the plain Rusanov method."""
import numpy as np
import pytest

from oracle import learned as olearned
from oracle import mlp as omlp
from paper_2302_09005_gb300 import inputs
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def gpu_faces_to_domain(arr, n_per_patch_stride, grid, p, comps=4):
    """Per-patch face array [patch][k][v][j] -> domain face arrays (Fx, Fy)
    of shape (N, N, comps) (x-face (J, I) between cells I-1 and I)."""
    N = grid[0] * p
    nf1 = (p + 1) * p
    Fx = np.full((N, N, comps), np.nan)
    Fy = np.full((N, N, comps), np.nan)
    for pid in range(grid[0] * grid[1]):
        a, b = pid % grid[0], pid // grid[0]
        base = pid * n_per_patch_stride
        for k, F in ((0, Fx), (1, Fy)):
            blk = arr[base + k * comps * nf1: base + (k + 1) * comps * nf1].reshape(comps, nf1)
            for j in range(nf1):
                bb, tr = j // p, j % p
                if k == 0:
                    J, I = b * p + tr, (a * p + bb) % N
                else:
                    J, I = (b * p + bb) % N, a * p + tr
                F[J, I] = blk[:, j]
    return Fx, Fy


def bf16_correction(U, axis, theta, norm):
    """Oracle correction with the GPU's BF16 rounding points."""
    mu, sd, sdy = norm
    r = omlp.bf16_round
    X = ((olearned.stencils(U, axis) - mu) / sd).astype(np.float32).astype(np.float64)
    p = omlp.unpack(theta)
    Xb = r(X.reshape(-1, 16))
    h1 = r(omlp.gelu(Xb @ r(p["W1"]).T + p["b1"]))
    h2 = r(omlp.gelu(h1 @ r(p["W2"]).T + p["b2"]))
    y = (h2 @ r(p["W3"]).T + p["b3"]).reshape(U.shape[:2] + (4,))
    return olearned.to_normal(y * sdy, axis)


def random_net(seed):
    rng = np.random.default_rng(seed)
    theta = omlp.init_params(seed) + 0.05 * rng.standard_normal(omlp.N_PARAM)
    theta = theta.astype(np.float32).astype(np.float64)
    mu = rng.uniform(-0.2, 1.2, 16)
    sd = rng.uniform(0.3, 1.0, 16)
    sdy = rng.uniform(0.01, 0.05, 4)
    return theta, (mu, sd, sdy)


def net_to_dev(theta, norm):
    torch = fvtest.torch_cuda()
    pv = fvtest.to_dev(theta, torch.float32)
    nv = fvtest.to_dev(np.concatenate(norm), torch.float32)
    return pv, nv


def mesh(fv, N, p, prec, U):
    from paper_2302_09005_gb300 import learned
    torch = fvtest.torch_cuda()
    return learned.Mesh2D(N, p, prec, torch.cuda.current_stream(), U=U)


@pytest.mark.parametrize("prec", [0, 1])
def test_correction_kernel_matches_oracle(fv, prec):
    torch = fvtest.torch_cuda()
    N, p = 32, 8
    rng = np.random.default_rng(1)
    U = inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)
    m = mesh(fv, N, p, prec, U)
    theta, norm = random_net(2)
    pv, nv = net_to_dev(theta, norm)
    stride = fv.fv_corr_stride(m.b.h)
    corr = torch.zeros(m.n * stride, dtype=torch.float32, device="cuda")
    fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, pv, nv, corr)
    assert m.b.status() == fv.FV_OK
    Gx, Gy = gpu_faces_to_domain(corr.cpu().numpy().astype(np.float64), stride, m.grid, p)
    Uq = U if prec == 0 else U.astype(np.float32).astype(np.float64)
    Cx = bf16_correction(Uq, 1, theta, norm)
    Cy = bf16_correction(Uq, 0, theta, norm)
    scale = max(np.abs(Cx).max(), np.abs(Cy).max())
    assert np.max(np.abs(Gx - Cx)) <= 2e-2 * scale
    assert np.max(np.abs(Gy - Cy)) <= 2e-2 * scale
    m.close()


def bf16_net(X, theta, norm):
    """The network on normalised-frame stencils X (..., 16) with the GPU's
    BF16 rounding points; outputs in the normal frame times sd_y."""
    mu, sd, sdy = norm
    r = omlp.bf16_round
    Xn = ((X - mu) / sd).astype(np.float32).astype(np.float64)
    p = omlp.unpack(theta)
    h1 = r(omlp.gelu(r(Xn.reshape(-1, 16)) @ r(p["W1"]).T + p["b1"]))
    h2 = r(omlp.gelu(h1 @ r(p["W2"]).T + p["b2"]))
    return ((h2 @ r(p["W3"]).T + p["b3"]) * sdy).reshape(X.shape[:-1] + (4,))


def test_correction_faces_once_with_walls(fv):
    """Walls on the x boundaries (mirror cells, x momentum negated), periodic
    in y.  Each face is evaluated once: a shared face has bitwise the same
    correction in both patches' slots, and the faces on the walls (the low
    wall by the first patch's face b = 0, the high wall by the last patch's
    own face b = p) match the network on stencils with mirrored ghost cells."""
    torch = fvtest.torch_cuda()
    N, p = 32, 8
    g = N // p
    rng = np.random.default_rng(5)
    U = inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)
    m = mesh(fv, N, p, 0, U)
    nbr = inputs.grid_neighbours((g, g))
    for pid in range(g * g):
        a = pid % g
        if a == 0:
            nbr[pid, 0] = -2
        if a == g - 1:
            nbr[pid, 1] = -2
    m.nbr = fvtest.to_dev(nbr)
    theta, norm = random_net(6)
    pv, nv = net_to_dev(theta, norm)
    stride = fv.fv_corr_stride(m.b.h)
    corr = torch.full((m.n * stride,), float("nan"), dtype=torch.float32, device="cuda")
    fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, pv, nv, corr)
    assert m.b.status() == fv.FV_OK
    c = corr.cpu().numpy().reshape(m.n, 2, 4, (p + 1) * p)
    assert not np.isnan(c).any()
    nf = p * p  # offset of the high faces b = p in a direction's block
    for pid in range(g * g):
        for k in range(2):
            hi = nbr[pid, 2 * k + 1]
            if hi >= 0:  # the high face is the high neighbour's low face, bitwise
                assert np.array_equal(c[pid, k, :, nf:], c[hi, k, :, :p]), (pid, k)
    # x faces i = 0..N against the network on mirrored stencils
    mir = np.array([1.0, -1.0, 1.0, 1.0])
    Ue = np.concatenate([U[:, 1:2] * mir, U[:, 0:1] * mir, U, U[:, N - 1:N] * mir,
                         U[:, N - 2:N - 1] * mir], axis=1)  # columns -2 .. N + 1
    X = np.concatenate([olearned.to_normal(Ue[:, s:s + N + 1], 1) for s in range(4)], axis=-1)
    Cx = olearned.to_normal(bf16_net(X, theta, norm), 1)  # (N, N + 1, 4), physical frame
    Gx = np.full((N, N + 1, 4), np.nan)
    for pid in range(g * g):
        a, b = pid % g, pid // g
        for j in range((p + 1) * p):
            bb, tr = j // p, j % p
            Gx[b * p + tr, a * p + bb] = c[pid, 0, :, j]
    scale = np.abs(Cx).max()
    assert np.max(np.abs(Gx - Cx)) <= 2e-2 * scale
    m.close()


def test_corrected_update_matches_oracle_and_conserves(fv):
    """Given the corrections, the GPU update is the oracle's update with
    F + C to FP64 roundoff, and the totals are conserved."""
    torch = fvtest.torch_cuda()
    N, p = 32, 8
    rng = np.random.default_rng(3)
    U = inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)
    m = mesh(fv, N, p, 0, U)
    theta, norm = random_net(4)
    pv, nv = net_to_dev(theta, norm)
    stride = fv.fv_corr_stride(m.b.h)
    corr = torch.zeros(m.n * stride, dtype=torch.float32, device="cuda")
    fv.fv_flux_correction(m.b.h, m.x, m.off, m.sizes, m.nbr, m.n, pv, nv, corr)
    dt = 0.002
    m.step(dt, corr)
    got = m.domain()
    Cx, Cy = gpu_faces_to_domain(corr.cpu().numpy().astype(np.float64), stride, m.grid, p)
    ref = olearned.step(U, dt, 1.0 / N, Cx, Cy)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    for v in range(4):
        assert abs(got[..., v].sum() - U[..., v].sum()) <= 1e-12 * np.abs(U[..., v]).sum()
    assert np.max(np.abs(got - olearned.step(U, dt, 1.0 / N))) > 1e-7  # the network acts
    m.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_learned_step_with_side_stream_halo_fill(fv, prec):
    """Mesh2D.step_learned (the halo fill on a second stream beside the
    correction kernel, then the update) gives bitwise the state of the same
    kernels run in sequence on one stream, over several steps, and its last
    step is the oracle's update with F + C (the GPU's corrections) to FP64
    roundoff, or within 1e-5 for an FP32 state."""
    torch = fvtest.torch_cuda()
    N, p = 64, 8
    rng = np.random.default_rng(11)
    U = inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)
    a, b = mesh(fv, N, p, prec, U), mesh(fv, N, p, prec, U)
    theta, norm = random_net(12)
    pv, nv = net_to_dev(theta, norm)
    stride = fv.fv_corr_stride(a.b.h)
    ca = torch.zeros(a.n * stride, dtype=torch.float32, device="cuda")
    cb = torch.zeros_like(ca)
    dt = 0.001
    for _ in range(3):
        Ua = a.domain()
        a.step_learned(dt, pv, nv, ca)
        fv.fv_flux_correction(b.b.h, b.x, b.off, b.sizes, b.nbr, b.n, pv, nv, cb)
        b.step(dt, cb)
    torch.cuda.synchronize()
    assert a.status() == fv.FV_OK and b.status() == fv.FV_OK
    got = a.domain()
    assert np.array_equal(got, b.domain())
    Cx, Cy = gpu_faces_to_domain(ca.cpu().numpy().astype(np.float64), stride, a.grid, p)
    ref = olearned.step(Ua, dt, 1.0 / N, Cx, Cy)
    tol = 1e-12 if prec == fv.FV_FP64 else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    a.close()
    b.close()


def test_zero_network_equals_plain_time_step(fv):
    torch = fvtest.torch_cuda()
    N, p = 24, 8
    rng = np.random.default_rng(5)
    U = inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)
    a, b = mesh(fv, N, p, 0, U), mesh(fv, N, p, 0, U)
    pv = torch.zeros(omlp.N_PARAM, dtype=torch.float32, device="cuda")
    nv = fvtest.to_dev(np.concatenate([np.zeros(16), np.ones(16), np.ones(4)]), torch.float32)
    corr = torch.zeros(b.n * fv.fv_corr_stride(b.b.h), dtype=torch.float32, device="cuda")
    for m in (a, b):
        m.cfl_dt(0.4)
    a.b.time_step(a.x, a.y, a.off, a.sizes, a.nbr, a.dx, 0.4)
    fv.fv_flux_correction(b.b.h, b.x, b.off, b.sizes, b.nbr, b.n, pv, nv, corr)
    fv.fv_time_step_corrected(b.b.h, b.x, b.y, b.off, b.sizes, b.nbr, b.n, b.dx, 0.4, corr)
    assert a.b.status() == fv.FV_OK and b.b.status() == fv.FV_OK
    mask = fvtest.interior_mask(a.off_np, np.full(a.n, p), 2, 4, a.y.numel())
    assert np.array_equal(a.y.cpu().numpy()[mask], b.y.cpu().numpy()[mask])
    a.close()
    b.close()


def test_training_targets_match_oracle_and_close_the_gap(fv):
    """The GPU's stencils and ideal corrections equal the oracle's, and the
    coarse update with C* reproduces the restricted fine state."""
    torch = fvtest.torch_cuda()
    from paper_2302_09005_gb300 import learned
    Nc, pc, pf, r = 16, 8, 8, 4
    Uf = inputs.shear_layer(Nc * r, seed=4)
    X, T, dts, refs = learned.generate(Uf, Nc, pc, pf, r, 1, 0.4, torch.cuda.current_stream())
    Uc0, Uc1, Cx, Cy, _ = olearned.ideal_correction(Uf, r, dts[0], 1.0 / (Nc * r))
    assert np.allclose(refs[0], Uc0, rtol=0, atol=1e-14)
    assert np.allclose(refs[1], Uc1, rtol=0, atol=1e-13)
    # samples back onto domain faces (normal frame -> physical frame)
    nf1 = (pc + 1) * pc
    grid = (Nc // pc, Nc // pc)
    Xn, Tn = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    per = np.zeros(grid[0] * grid[1] * 8 * nf1)
    for pid in range(grid[0] * grid[1]):
        for k in range(2):
            s = Tn[pid * 2 * nf1 + k * nf1: pid * 2 * nf1 + (k + 1) * nf1]  # (nf1, 4) normal
            phys = s[:, [0, 2, 1, 3]] if k == 1 else s
            per[pid * 8 * nf1 + k * 4 * nf1: pid * 8 * nf1 + (k + 1) * 4 * nf1] = phys.T.reshape(-1)
    Gx, Gy = gpu_faces_to_domain(per, 8 * nf1, grid, pc)
    sc = max(np.abs(Cx).max(), np.abs(Cy).max())
    assert np.max(np.abs(Gx - Cx)) <= 1e-6 * sc
    assert np.max(np.abs(Gy - Cy)) <= 1e-6 * sc
    Sx = olearned.stencils(Uc0, 1)
    xs = Xn.reshape(grid[1], grid[0], 2, nf1, 16)
    # spot-check stencils of the x faces of patch 0
    for j in range(nf1):
        bb, tr = j // pc, j % pc
        assert np.allclose(xs[0, 0, 0, j], Sx[tr, bb % Nc], rtol=1e-6, atol=1e-6)
    # the corrected coarse step with C* lands on the restricted fine state
    m = mesh(fv, Nc, pc, 0, Uc0)
    corr = fvtest.to_dev(per, torch.float32)
    m.step(dts[0], corr)
    got = m.domain()
    assert np.max(np.abs(got - Uc1)) <= 1e-6 * np.max(np.abs(Uc1))
    assert np.max(np.abs(olearned.step(Uc0, dts[0], 1.0 / Nc) - Uc1)) > 1e-4
    m.close()


def test_trained_network_beats_plain_rusanov_on_unseen_data(fv):
    """Train on two shear layers (seeds 1, 2), evaluate on a third (seed 3):
    the learned coarse run is closer to the restricted fine run than the
    plain coarse run (relative L1, mean over the unknowns, after 8 steps)."""
    torch = fvtest.torch_cuda()
    from paper_2302_09005_gb300 import learned
    Nc, pc, pf, r, steps = 64, 8, 8, 4, 8
    st = torch.cuda.current_stream()
    Xs, Ts = [], []
    for seed in (1, 2):
        X, T, _, _ = learned.generate(inputs.shear_layer(Nc * r, seed=seed), Nc, pc, pf, r,
                                      steps, 0.4, st)
        Xs.append(X)
        Ts.append(T)
    X, T = torch.cat(Xs), torch.cat(Ts)
    norm = learned.normalisation(X, T, st)
    params, losses = learned.train(X, T, norm, steps=1500, batch=8192, lr=2e-3, seed=0, stream=st)
    assert losses[-1][1] < 0.5 * losses[0][1], losses
    Uf = inputs.shear_layer(Nc * r, seed=3)
    _, _, dts, refs = learned.generate(Uf, Nc, pc, pf, r, steps, 0.4, st)
    l1_plain, l1_learned, _ = learned.evaluate(refs[0], refs, dts, pc, params, norm, st)
    plain = float(np.mean(l1_plain[-1]))
    lrn = float(np.mean(l1_learned[-1]))
    assert lrn < 0.85 * plain, (plain, lrn, losses)
