"""BF16 tensor-core network kernels against the FP64 oracle (oracle/mlp.py).

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


@pytest.mark.parametrize("B", [64, 5000])
def test_gradient_matches_oracle(fv, B):
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
    tr.close()
