"""BF16 tensor-core network kernels (tcgen05) against the FP64 oracle
(oracle/mlp.py).

The GPU rounds weights, inputs and hidden activations to BF16 before every
product and accumulates in FP32; the oracle is run in FP64 on the same
BF16-rounded weights and inputs, with the hidden activations rounded to BF16
at the same points.  Tolerances follow from BF16's 8-bit significand
(relative rounding error 2^-9 ~ 2e-3 per operand): outputs within 1% of their
scale, gradients within 5% in relative L2 norm."""
import numpy as np
import pytest

from oracle import mlp
from tests import fvtest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fv():
    fvtest.ensure_built()
    fvtest.torch_cuda()
    from paper_2302_09005_gb300 import fv as fvmod
    return fvmod


def bf16_forward(theta, X):
    """FP64 forward with the GPU's BF16 rounding points."""
    p = mlp.unpack(theta)
    r = mlp.bf16_round
    Xb = r(X)
    z1 = Xb @ r(p["W1"]).T + p["b1"]
    h1 = r(mlp.gelu(z1))
    z2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(mlp.gelu(z2))
    return h2 @ r(p["W3"]).T + p["b3"]


def data(B, seed):
    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed) + 0.05 * rng.standard_normal(mlp.N_PARAM)
    X = rng.standard_normal((B, 16))
    T = 0.3 * rng.standard_normal((B, 4))
    return theta, X, T


@pytest.mark.parametrize("B", [1, 37, 4096, 70000])
def test_forward_matches_oracle(fv, B):
    torch = fvtest.torch_cuda()
    theta, X, _ = data(B, 1)
    tr = fv.MlpTrainer(max(B, 16))
    y = torch.empty((B, 4), dtype=torch.float32, device="cuda")
    tr.forward(fvtest.to_dev(theta, torch.float32), fvtest.to_dev(X, torch.float32), y)
    torch.cuda.synchronize()
    ref = bf16_forward(theta.astype(np.float32).astype(np.float64),
                       X.astype(np.float32).astype(np.float64))
    got = y.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-2 * max(1.0, np.max(np.abs(ref)))
    tr.close()


@pytest.mark.parametrize("B", [64, 5000, 50000])
def test_gradient_matches_oracle(fv, B):
    """B = 50000 is 391 tiles of 128 samples: more than the kernel's CTAs, so
    the weight gradients accumulate over several tiles in tensor memory."""
    torch = fvtest.torch_cuda()
    theta, X, T = data(B, 2)
    tr = fv.MlpTrainer(B)
    g = torch.empty(mlp.N_PARAM, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    tr.grad(fvtest.to_dev(theta, torch.float32), fvtest.to_dev(X, torch.float32),
            fvtest.to_dev(T, torch.float32), g, loss)
    torch.cuda.synchronize()
    th32 = theta.astype(np.float32).astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    lref, gref = mlp.loss_and_grad(mlp.bf16_round(th32), mlp.bf16_round(X32),
                                   T.astype(np.float32).astype(np.float64))
    got = g.cpu().numpy().astype(np.float64)
    assert loss.item() == pytest.approx(lref, rel=2e-2)
    blocks = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    for (name, _), a, b in zip(mlp.SHAPES, blocks[:-1], blocks[1:]):
        err = np.linalg.norm(got[a:b] - gref[a:b]) / max(np.linalg.norm(gref[a:b]), 1e-12)
        assert err <= 5e-2, (name, err)
    # deterministic
    g2 = torch.empty_like(g)
    tr.grad(fvtest.to_dev(theta, torch.float32), fvtest.to_dev(X, torch.float32),
            fvtest.to_dev(T, torch.float32), g2, loss)
    torch.cuda.synchronize()
    assert torch.equal(g, g2)
    tr.close()


def test_adam_training_reduces_the_loss(fv):
    """Fitting a smooth target with the GPU Adam loop lowers the loss ten-fold."""
    torch = fvtest.torch_cuda()
    rng = np.random.default_rng(3)
    B = 8192
    X = rng.standard_normal((B, 16))
    A = rng.standard_normal((16, 4)) / 4.0
    T = np.tanh(X @ A)
    tr = fv.MlpTrainer(B)
    theta = fvtest.to_dev(mlp.init_params(3), torch.float32)
    x, t = fvtest.to_dev(X, torch.float32), fvtest.to_dev(T, torch.float32)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    losses = []
    for step in range(1, 401):
        tr.train_step(theta, x, t, 3e-3, step, loss)
        if step in (1, 400):
            losses.append(loss.item())
    assert losses[-1] < 0.1 * losses[0], losses
    assert tr.status() == fv.FV_OK
    tr.close()


def test_train_steps_equal_single_steps_bitwise(fv):
    """fv_mlp_train_steps (many steps per call, losses on the device) gives
    bitwise the parameters and losses of the same steps taken one call at a
    time; the minibatches cycle through the sample set, the last partial
    batch unused."""
    torch = fvtest.torch_cuda()
    rng = np.random.default_rng(4)
    n, B, steps = 5000, 1024, 11
    X = fvtest.to_dev(rng.standard_normal((n, 16)), torch.float32)
    T = fvtest.to_dev(0.3 * rng.standard_normal((n, 4)), torch.float32)
    th0 = fvtest.to_dev(mlp.init_params(4), torch.float32)
    ta, tb = fv.MlpTrainer(B), fv.MlpTrainer(B)
    pa, pb = th0.clone(), th0.clone()
    la = torch.zeros(steps, dtype=torch.float32, device="cuda")
    ta.train_steps(pa, X, T, B, 1, 6, 2e-3, la[:6])
    ta.train_steps(pa, X, T, B, 7, steps - 6, 2e-4, la[6:])
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lb = []
    nb = n // B
    for it in range(1, steps + 1):
        i0 = ((it - 1) % nb) * B
        tb.train_step(pb, X[i0:i0 + B], T[i0:i0 + B], 2e-3 if it <= 6 else 2e-4, it, loss)
        lb.append(loss.clone())
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)
    assert torch.equal(la, torch.cat(lb))
    assert ta.status() == fv.FV_OK and tb.status() == fv.FV_OK
    ta.close()
    tb.close()
