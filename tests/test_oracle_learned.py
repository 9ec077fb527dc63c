"""Pins of the learned-correction oracle (oracle/mlp.py, oracle/learned.py)
against facts that do not come from the oracle itself."""
import math

import numpy as np
import pytest

import oracle
from oracle import learned, mlp
from paper_2302_09005_gb300 import inputs


def test_gelu_textbook_values():
    """gelu(z) = z Phi(z): Phi(1) = 0.841344746068543, Phi(-1) = 1 - Phi(1);
    gelu'(0) = Phi(0) = 1/2; gelu'(z) -> 1 for large z."""
    z = np.array([0.0, 1.0, -1.0, 2.0])
    g = mlp.gelu(z)
    assert g[0] == 0.0
    assert g[1] == pytest.approx(0.8413447460685429, rel=1e-15)
    assert g[2] == pytest.approx(-0.15865525393145707, rel=1e-14)
    assert g[3] == pytest.approx(2 * 0.9772498680518208, rel=1e-15)
    assert mlp.gelu_prime(np.array([0.0]))[0] == 0.5
    assert mlp.gelu_prime(np.array([12.0]))[0] == pytest.approx(1.0, abs=1e-12)


def test_mlp_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(1) + 0.1 * rng.standard_normal(mlp.N_PARAM)
    X = rng.standard_normal((7, 16))
    T = rng.standard_normal((7, 4))
    loss, g = mlp.loss_and_grad(theta, X, T)
    idx = rng.choice(mlp.N_PARAM, 60, replace=False)
    idx = np.concatenate([idx, [0, 1023, 1024, 1087, 5183, 5503, 5507]])  # every block
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, T)[0] - mlp.loss_and_grad(tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_mlp_forward_by_hand_for_one_hidden_unit():
    """With only W1[0, 0], W2[0, 0], W3[0, 0] nonzero the network is a chain
    of scalars: y0 = w3 gelu(w2 gelu(w1 x0 + b1) + b2) + b3."""
    theta = np.zeros(mlp.N_PARAM)
    p = mlp.unpack(theta)
    p["W1"][0, 0], p["b1"][0] = 0.7, -0.2
    p["W2"][0, 0], p["b2"][0] = -1.3, 0.4
    p["W3"][0, 0], p["b3"][:] = 2.0, [0.1, 0.2, 0.3, 0.4]
    theta = mlp.pack(p)
    x0 = 1.5
    X = np.zeros((1, 16))
    X[0, 0] = x0
    y, _ = mlp.forward(theta, X)

    def Phi(z):
        return 0.5 * (1 + math.erf(z / math.sqrt(2)))
    z1 = 0.7 * x0 - 0.2
    h1 = z1 * Phi(z1)
    z2 = -1.3 * h1 + 0.4
    h2 = z2 * Phi(z2)
    # every other hidden unit has z = 0 and gelu(0) = 0
    assert y[0, 0] == pytest.approx(2.0 * h2 + 0.1, rel=1e-14)
    assert np.allclose(y[0, 1:], [0.2, 0.3, 0.4], rtol=0, atol=1e-15)


def test_adam_first_step_closed_form():
    """At step 1 from zero moments the Adam update is lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    th, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_bf16_round_ties_and_exact_values():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.0, 0.0])
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway, ties to even (mantissa 0)
    assert r[2] == 1.0 + 2 ** -7  # above halfway rounds up
    assert r[3] == -3.0 and r[4] == 0.0


def _periodic_state(N, seed):
    rng = np.random.default_rng(seed)
    return inputs.random_cells(rng, N * N, 2).reshape(N, N, 4)


def test_numpy_step_matches_c_oracle():
    """The vectorised domain update equals the C oracle's patch update on
    the same periodic domain (cut into patches, halos filled)."""
    N, p = 12, 4
    U = _periodic_state(N, 2)
    dx, dt = 1.0 / N, 0.003
    q, off, sz, grid = inputs.domain_to_patches(U, p)
    nbr = inputs.grid_neighbours(grid)
    oracle.halo_fill(q, off, sz, nbr, 2, 4)
    ref = inputs.patches_to_domain(oracle.patch_update(q, off, sz, 2, dx, dt), off, p, grid, 4)
    got = learned.step(U, dt, dx)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_learned_step_conserves_by_construction():
    N = 16
    U = _periodic_state(N, 3)
    theta = mlp.init_params(4) * 5.0
    norm = (np.zeros(16), np.ones(16), np.full(4, 0.1))
    U1 = learned.learned_step(U, 0.002, 1.0 / N, theta, norm)
    for v in range(4):
        assert abs(math.fsum(U1[..., v].ravel()) - math.fsum(U[..., v].ravel())) <= \
            1e-13 * math.fsum(np.abs(U[..., v]).ravel())
    assert np.max(np.abs(U1 - learned.step(U, 0.002, 1.0 / N))) > 1e-6  # it does act


def test_learned_step_is_rotation_equivariant():
    """Transposing x and y (and swapping the momenta) commutes with the
    learned step, because the network sees normal-frame stencils."""
    N = 10
    U = _periodic_state(N, 5)
    theta = mlp.init_params(6)
    norm = (np.zeros(16), np.ones(16), np.full(4, 0.05))
    A = learned.learned_step(U, 0.002, 0.1, theta, norm)
    Ut = np.swapaxes(U, 0, 1)[..., [0, 2, 1, 3]]
    B = learned.learned_step(Ut, 0.002, 0.1, theta, norm)
    assert np.array_equal(np.swapaxes(B, 0, 1)[..., [0, 2, 1, 3]], A)


def test_ideal_correction_reproduces_restricted_fine_state():
    """The coarse update with F + C* equals the restricted fine solution to
    roundoff (telescoping sum of the fine fluxes)."""
    Nc, r = 8, 4
    Uf = inputs.shear_layer(Nc * r, seed=1)
    dx_c = 1.0 / Nc
    dt = 0.2 * dx_c / learned.max_wave_speed(Uf)
    Uc0, Uc1, Cx, Cy, _ = learned.ideal_correction(Uf, r, dt, dx_c / r)
    got = learned.step(Uc0, dt, dx_c, Cx, Cy)
    assert np.max(np.abs(got - Uc1)) <= 1e-13 * np.max(np.abs(Uc1))
    plain = learned.step(Uc0, dt, dx_c)
    assert np.max(np.abs(plain - Uc1)) > 1e-5  # the correction is not trivial
