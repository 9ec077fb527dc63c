"""Pins of the FP64 CPU oracle against facts fixed by the paper's equations and
by mathematics, independent of the oracle itself (no GPU).

Each test names what it pins and which equation of arXiv 2302.09005 it
exercises.  A plausible slip in the oracle -- a dropped term, a wrong sign,
a swapped index, a transposed operand -- fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle.riemann import sample, star_state
from paper_2302_09005_gb300 import inputs

G = 1.4


def patch_view(q, off, i, p, d, s, halo=1):
    ne = p + 2 * halo
    return q[off[i]:off[i] + ne ** d * s].reshape((ne,) * d + (s,))


def interior(view, p, d, halo=1):
    return view[(slice(halo, halo + p),) * d]


def random_states(rng, n, d):
    return inputs.random_cells(rng, n, d, G)


# ---------------------------------------------------------------- Eq. 4 --

@pytest.mark.parametrize("d", [1, 2, 3])
def test_flux_consistency_bitwise(d):
    """F(q, q) = f(q) exactly: (f+f)/2 is exact and a (q - q) = 0 (Eq. 4)."""
    rng = np.random.default_rng(1)
    for q in random_states(rng, 50, d):
        for j in range(d):
            F, a = oracle.rusanov_flux(q, q, d, j, G)
            f = oracle.euler_flux(q, d, j, G)
            assert np.array_equal(F, f)
            assert a == oracle.euler_wave_speed(q, d, j, G)


def test_closed_form_sod_face():
    """Rusanov flux between the two Sod states, worked by hand:
    f(qL) = (0, 1, 0), f(qR) = (0, 0.1, 0), a = max(sqrt(1.4), sqrt(1.12)) =
    sqrt(1.4), F = 1/2 (fL + fR - a (qR - qL)) with qR - qL =
    (-0.875, 0, 0.25 - 2.5)."""
    qL = np.array([1.0, 0.0, 2.5])
    qR = np.array([0.125, 0.0, 0.25])
    F, a = oracle.rusanov_flux(qL, qR, 1, 0, G)
    sq = math.sqrt(1.4)
    assert a == pytest.approx(sq, rel=1e-15)
    assert F[0] == pytest.approx(0.5 * sq * 0.875, rel=1e-15)
    assert F[1] == pytest.approx(0.55, rel=1e-15)
    assert F[2] == pytest.approx(0.5 * sq * 2.25, rel=1e-15)
    # a moving state: u = 2, rho = 1, p = 1 -> E = 2.5 + 2 = 4.5,
    # f = (2, 2*2 + 1, (4.5 + 1) * 2) = (2, 5, 11), |u| + c = 2 + sqrt(1.4)
    q = np.array([1.0, 2.0, 4.5])
    assert np.allclose(oracle.euler_flux(q, 1, 0, G), [2.0, 5.0, 11.0], rtol=1e-15)
    assert oracle.euler_wave_speed(q, 1, 0, G) == pytest.approx(2.0 + sq, rel=1e-15)


def test_transverse_flux_2d_by_hand():
    """y-flux of a 2D state, worked by hand: rho = 2, (u, v) = (0.5, -1),
    p = 0.8 -> j = (1, -2), E = 0.8/0.4 + 0.5*2*1.25 = 3.25;
    f^y = (-2, j_x v, j_y v + p, (E + p) v) = (-2, -1, 2.8, -4.05)."""
    q = np.array([2.0, 1.0, -2.0, 3.25])
    assert np.allclose(oracle.euler_flux(q, 2, 1, G), [-2.0, -1.0, 2.8, -4.05], rtol=1e-14)
    c = math.sqrt(1.4 * 0.8 / 2.0)
    assert oracle.euler_wave_speed(q, 2, 1, G) == pytest.approx(1.0 + c, rel=1e-15)
    assert oracle.euler_wave_speed(q, 2, 0, G) == pytest.approx(0.5 + c, rel=1e-15)


# --------------------------------------------------------- Eq. 3, Alg. 1 --

@pytest.mark.parametrize("d,p", [(1, 4), (2, 3), (2, 5), (3, 3), (3, 5)])
def test_uniform_state_preserved_bitwise(d, p):
    """A uniform state has equal fluxes on every face, so Q^{n+1} = Q^n exactly."""
    s = d + 2
    rng = np.random.default_rng(2)
    n = 3
    q, off, sz = inputs.random_batch(n, p, d, seed=3)
    for i in range(n):
        v = patch_view(q, off, i, p, d, s)
        v[...] = random_states(rng, 1, d)[0]
    out, lam = oracle.patch_update(q, off, sz, d, 0.01, 0.002, want_lambda=True)
    assert np.array_equal(out, q)
    for i in range(n):
        v = patch_view(q, off, i, p, d, s)
        q0 = v.reshape(-1, s)[0]
        assert lam[i] == max(oracle.euler_wave_speed(q0, d, j, G) for j in range(d))


def _periodic_domain(d, p, grid, seed):
    rng = np.random.default_rng(seed)
    N = [g * p for g in grid]
    U = random_states(rng, int(np.prod(N)), d).reshape(tuple(N[::-1]) + (d + 2,))
    q, off, sz, g = inputs.domain_to_patches(U, p)
    assert tuple(g) == tuple(grid)
    nbr = inputs.grid_neighbours(grid)
    return U, q, off, sz, nbr


@pytest.mark.parametrize("d,p,grid", [(1, 5, (6,)), (2, 4, (3, 2)), (3, 3, (2, 3, 2))])
def test_periodic_conservation(d, p, grid):
    """Sum of each conserved quantity over a periodic domain is unchanged up
    to roundoff: every interior face flux enters two cells with opposite
    signs (Eq. 3)."""
    s = d + 2
    _, q, off, sz, nbr = _periodic_domain(d, p, grid, 4)
    oracle.halo_fill(q, off, sz, nbr, d, s)
    _, lam = oracle.max_eigenvalue(q, off, sz, d)
    dx = 1.0 / (grid[0] * p)
    dt = oracle.cfl_dt(lam, 0.4, dx, d)
    out = oracle.patch_update(q, off, sz, d, dx, dt)
    before = oracle.patch_sums(q, off, sz, d, s)
    after = oracle.patch_sums(out, off, sz, d, s)
    for v in range(s):
        b = math.fsum(before[:, v])
        a = math.fsum(after[:, v])
        scale = math.fsum(np.abs(before[:, v]))
        assert abs(a - b) <= 1e-13 * scale, (v, a, b)
    # and the update did change the state (the pin is not vacuous)
    assert np.abs(out - q).max() > 1e-3


@pytest.mark.parametrize("d,halo", [(1, 1), (2, 1), (3, 1), (2, 2)])
def test_patch_sums_are_interior_sums(d, halo):
    """The per-patch conservation sums (the FP64 epilogue of Eq. 3) cover the
    p^d interior cells of each patch and nothing else.  Expected values come
    from numpy slicing of each patch's box, not from the oracle: every cell
    holds a small integer state, so every sum is exact in FP64 and any order
    gives the same bits.  The halo cells hold values far from the interior's
    (1000 + ...), so a sum over the whole box, or an interior read at the
    wrong stride, is off by hundreds."""
    s = d + 2
    rng = np.random.default_rng(40 + d)
    sizes = rng.integers(1, 7, 9).astype(np.int32)
    off, total = inputs.layout(sizes, d, s, halo, 8, 16)
    q = np.zeros(total)
    expected = np.zeros((len(sizes), s))
    for i, p in enumerate(sizes):
        ne = int(p) + 2 * halo
        box = 1000.0 + rng.integers(0, 50, (ne,) * d + (s,)).astype(np.float64)
        inner = (slice(halo, halo + int(p)),) * d
        box[inner] = rng.integers(-20, 20, (int(p),) * d + (s,))
        q[off[i]:off[i] + ne ** d * s] = box.reshape(-1)
        expected[i] = box[inner].reshape(-1, s).sum(axis=0)
    got = oracle.patch_sums(q, off, sizes, d, s, halo=halo)
    assert np.array_equal(got, expected)


@pytest.mark.parametrize("d,p,grid", [(1, 5, (4,)), (2, 3, (4, 3)), (3, 2, (2, 3, 2))])
def test_patch_sums_add_up_to_the_domain_totals(d, p, grid):
    """On a patch mesh cut from a domain (halos then filled from the
    neighbours, so they differ from the interior), the per-patch sums of
    each patch equal the sum of that patch's block of the domain, and
    together the domain total (integer states: exact)."""
    s = d + 2
    rng = np.random.default_rng(50 + d)
    N = [g * p for g in grid]
    U = rng.integers(-30, 30, tuple(N[::-1]) + (s,)).astype(np.float64)
    q, off, sz, g = inputs.domain_to_patches(U, p)
    oracle.halo_fill(q, off, sz, inputs.grid_neighbours(grid), d, s)
    got = oracle.patch_sums(q, off, sz, d, s)
    D = inputs.patches_to_domain(q, off, p, grid, s)
    assert np.array_equal(D, U)
    idx = 0
    for blk in np.ndindex(*grid[::-1]):  # slowest axis first; patch index x fastest
        sl = tuple(slice(b * p, (b + 1) * p) for b in blk)
        assert np.array_equal(got[idx], U[sl].reshape(-1, s).sum(axis=0)), idx
        idx += 1
    assert np.array_equal(got.sum(axis=0), U.reshape(-1, s).sum(axis=0))


@pytest.mark.parametrize("d,p,grid", [(2, 4, (3, 3)), (3, 3, (2, 2, 2))])
def test_patch_decomposition_invariance_bitwise(d, p, grid):
    """Cutting a periodic domain into patches does not change the result:
    the same faces see the same two states (Eq. 3-4 are local)."""
    s = d + 2
    U, q, off, sz, nbr = _periodic_domain(d, p, grid, 5)
    oracle.halo_fill(q, off, sz, nbr, d, s)
    dx, dt = 0.02, 0.001
    out = oracle.patch_update(q, off, sz, d, dx, dt)
    res_patches = inputs.patches_to_domain(out, off, p, grid, s)
    # the whole domain as one self-periodic patch
    N = U.shape[0]
    assert all(n == N for n in U.shape[:-1])
    q1, off1, sz1, _ = inputs.domain_to_patches(U, N)
    oracle.halo_fill(q1, off1, sz1, inputs.self_periodic_neighbours(1, d), d, s)
    out1 = oracle.patch_update(q1, off1, sz1, d, dx, dt)
    res_one = inputs.patches_to_domain(out1, off1, N, (1,) * d, s)
    assert np.array_equal(res_patches, res_one)


@pytest.mark.parametrize("d,axis", [(1, 0), (2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
def test_mirror_symmetry_bitwise(d, axis):
    """Reflecting the data along an axis and negating that momentum component
    reflects the result exactly (negation is exact; +, max commute)."""
    s = d + 2
    p = 4
    q, off, sz = inputs.random_batch(2, p, d, seed=6)
    out = oracle.patch_update(q, off, sz, d, 0.01, 0.001)
    qm = q.copy()
    ax = d - 1 - axis  # axis of the (z, y, x, s) view
    for i in range(2):
        v = patch_view(qm, off, i, p, d, s)
        v[...] = np.flip(patch_view(q, off, i, p, d, s), axis=ax)
        v[..., 1 + axis] *= -1.0
    outm = oracle.patch_update(qm, off, sz, d, 0.01, 0.001)
    for i in range(2):
        got = np.flip(interior(patch_view(outm, off, i, p, d, s), p, d), axis=ax).copy()
        got[..., 1 + axis] *= -1.0
        assert np.array_equal(got, interior(patch_view(out, off, i, p, d, s), p, d))


@pytest.mark.parametrize("d,a,b,exact", [(2, 0, 1, True), (3, 0, 1, True), (3, 0, 2, False),
                                         (3, 1, 2, False)])
def test_axis_permutation(d, a, b, exact):
    """Swapping two axes together with their momentum components swaps the
    result: bitwise when the swap keeps the order of the sums (x <-> y),
    to roundoff otherwise."""
    s = d + 2
    p = 4
    q, off, sz = inputs.random_batch(2, p, d, seed=7)
    out = oracle.patch_update(q, off, sz, d, 0.01, 0.001)
    qs = q.copy()
    A, B = d - 1 - a, d - 1 - b
    perm = list(range(d + 2))
    perm[1 + a], perm[1 + b] = perm[1 + b], perm[1 + a]
    for i in range(2):
        v = patch_view(qs, off, i, p, d, s)
        v[...] = np.swapaxes(patch_view(q, off, i, p, d, s), A, B)[..., perm]
    outs = oracle.patch_update(qs, off, sz, d, 0.01, 0.001)
    for i in range(2):
        got = np.swapaxes(interior(patch_view(outs, off, i, p, d, s), p, d), A, B)[..., perm]
        ref = interior(patch_view(out, off, i, p, d, s), p, d)
        if exact:
            assert np.array_equal(got, ref)
        else:
            assert np.max(np.abs(got - ref)) <= 4e-16 * np.max(np.abs(ref))


@pytest.mark.parametrize("d", [2, 3])
def test_dimensional_reduction_bitwise(d):
    """Data constant along y (and z) with zero transverse velocity: the
    transverse flux differences vanish exactly, so every row evolves as the
    1D scheme."""
    p = 5
    s = d + 2
    rng = np.random.default_rng(8)
    ne = p + 2
    row = inputs.random_cells(rng, ne, 1, G)  # (ne, 3): rho, jx, E
    q1, off1, sz1 = inputs.random_batch(1, p, 1, seed=0)
    q1[off1[0]:off1[0] + ne * 3] = row.reshape(-1)
    out1 = oracle.patch_update(q1, off1, sz1, 1, 0.01, 0.002)
    qd, offd, szd = inputs.random_batch(1, p, d, seed=0)
    v = patch_view(qd, offd, 0, p, d, s)
    v[...] = 0.0
    v[..., 0] = row[:, 0]
    v[..., 1] = row[:, 1]
    v[..., d + 1] = row[:, 2]
    outd = oracle.patch_update(qd, offd, szd, d, 0.01, 0.002)
    r1 = patch_view(out1, off1, 0, p, 1, 3)[1:1 + p]
    vd = interior(patch_view(outd, offd, 0, p, d, s), p, d)
    for idx in np.ndindex(*(p,) * (d - 1)):
        rowd = vd[idx]
        assert np.array_equal(rowd[:, 0], r1[:, 0])
        assert np.array_equal(rowd[:, 1], r1[:, 1])
        assert np.array_equal(rowd[:, d + 1], r1[:, 2])
        assert np.all(rowd[:, 2:d + 1] == 0.0)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_linear_advection_is_upwind(d):
    """For f^j(q) = c_j q the Rusanov flux with a = |c_j| is the upwind flux,
    so the update is the textbook first-order upwind scheme
    Q_i - sum_j c_j dt/dx (Q_i - Q_{i - sign(c_j) e_j})."""
    p, s = 4, 3
    rng = np.random.default_rng(9)
    adv = np.array([0.7, -1.3, 0.4])[:d]
    ne = p + 2
    n = 2
    q = rng.standard_normal(n * ne ** d * s)
    off = np.arange(n, dtype=np.int64) * ne ** d * s
    sz = np.full(n, p, dtype=np.int32)
    dx, dt = 0.1, 0.01
    out = oracle.patch_update(q, off, sz, d, dx, dt, s=s, pde=oracle.core.PDE_ADVECTION,
                              adv=np.pad(adv, (0, 3 - d)))
    for i in range(n):
        V = patch_view(q, off, i, p, d, s)
        exp = V.copy()
        for j in range(d):
            ax = d - 1 - j
            c = adv[j]
            if c > 0:  # upwind neighbour is i - e_j
                exp = exp - c * dt / dx * (V - np.roll(V, 1, axis=ax))
            else:  # upwind neighbour is i + e_j
                exp = exp - c * dt / dx * (np.roll(V, -1, axis=ax) - V)
        got = interior(patch_view(out, off, i, p, d, s), p, d)
        ref = interior(exp, p, d)
        assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))


# --------------------------------------------------------------- Eq. 5 --

def test_max_eigenvalue_matches_update_and_brute_force():
    """The per-patch maximum eigenvalue is the maximum over the faces that
    bound interior cells; the update's epilogue reports the same value
    (Algorithm 1, step 10), and a brute force over all cells of the patch
    that enter a face agrees."""
    d, p, s = 3, 3, 5
    q, off, sz = inputs.random_batch(4, p, d, seed=10)
    lam, g = oracle.max_eigenvalue(q, off, sz, d)
    _, lam_u = oracle.patch_update(q, off, sz, d, 0.01, 0.001, want_lambda=True)
    assert np.array_equal(lam, lam_u)
    assert g == lam.max()
    for i in range(4):
        V = patch_view(q, off, i, p, d, s)
        best = 0.0
        for idx in np.ndindex(*(p + 2,) * d):
            outside = [k for k in range(d) if idx[d - 1 - k] in (0, p + 1)]
            if len(outside) > 1:
                continue  # edge / corner halo cells enter no face
            dirs = outside if outside else range(d)
            for j in dirs:
                best = max(best, oracle.euler_wave_speed(V[idx], d, j, G))
        assert best == lam[i]


def test_cfl_dt():
    assert oracle.cfl_dt(2.0, 0.4, 0.1, 2) == pytest.approx(0.4 * 0.1 / 4.0, rel=1e-16)


# ------------------------------------------------------------ halo fill --

@pytest.mark.parametrize("d,p,grid", [(1, 3, (4,)), (2, 3, (3, 4)), (3, 2, (2, 3, 2))])
def test_halo_fill_periodic_matches_rolled_domain(d, p, grid):
    """Face halos of a periodic patch mesh are the neighbouring domain cells,
    i.e. the domain array rolled by one cell; edges/corners stay untouched."""
    s = d + 2
    U, q, off, sz, nbr = _periodic_domain(d, p, grid, 11)
    q0 = q.copy()
    oracle.halo_fill(q, off, sz, nbr, d, s)
    N = [g * p for g in grid]
    for i in range(len(off)):
        rem, pc = i, []
        for k in range(d):
            pc.append(rem % grid[k])
            rem //= grid[k]
        V = patch_view(q, off, i, p, d, s)
        V0 = patch_view(q0, off, i, p, d, s)
        for idx in np.ndindex(*(p + 2,) * d):
            cx = [idx[d - 1 - k] for k in range(d)]  # x, y, z
            outside = [k for k in range(d) if cx[k] in (0, p + 1)]
            if len(outside) == 0:
                continue
            if len(outside) > 1:
                assert np.array_equal(V[idx], V0[idx])
                continue
            g = [(pc[k] * p + cx[k] - 1) % N[k] for k in range(d)]
            assert np.array_equal(V[idx], U[tuple(g[::-1])])


def test_halo_fill_outflow_and_wall():
    """-1 copies the nearest interior cell; -2 mirrors it and negates the
    normal momentum."""
    d, p, s = 2, 3, 4
    q, off, sz = inputs.random_batch(1, p, d, seed=12)
    nbr = np.array([[-1, -2, -2, -1]], dtype=np.int32)
    oracle.halo_fill(q, off, sz, nbr, d, s)
    V = patch_view(q, off, 0, p, d, s)
    for y in range(1, p + 1):
        assert np.array_equal(V[y, 0], V[y, 1])  # -x outflow
        exp = V[y, p].copy()
        exp[1] = -exp[1]
        assert np.array_equal(V[y, p + 1], exp)  # +x wall
    for x in range(1, p + 1):
        exp = V[1, x].copy()
        exp[2] = -exp[2]
        assert np.array_equal(V[0, x], exp)  # -y wall
        assert np.array_equal(V[p + 1, x], V[p, x])  # +y outflow


def test_oracle_rejects_bad_arguments():
    q, off, sz = inputs.random_batch(2, 3, 2, seed=0)
    with pytest.raises(ValueError):
        oracle.halo_fill(q, off, sz, np.array([[5, 0, 0, 0], [0, 0, 0, 0]], np.int32), 2, 4)
    with pytest.raises(ValueError):
        oracle.patch_update(q, off, np.array([0, 3], np.int32), 2, 0.1, 0.01)


# -------------------------------------------- exact solutions / order --

def test_exact_riemann_star_state_golden(golden_dir):
    """The exact solver reproduces the textbook Sod star state."""
    with open(os.path.join(golden_dir, "sod_star_toro.json")) as f:
        g = json.load(f)
    L, R = g["left"], g["right"]
    ps, us, rl, rr = star_state(L["rho"], L["u"], L["p"], R["rho"], R["u"], R["p"], g["gamma"])
    st = g["star"]
    for got, exp in ((ps, st["p"]), (us, st["u"]), (rl, st["rho_left"]), (rr, st["rho_right"])):
        assert got == pytest.approx(exp, abs=0.6e-5)


def _run_1d(U0, p, T, cfl=0.4, periodic=True):
    N = U0.shape[0]
    q, off, sz, grid = inputs.domain_to_patches(U0, p)
    nbr = inputs.grid_neighbours(grid, periodic=periodic, boundary=-1)
    dx = 1.0 / N
    t = 0.0
    while t < T - 1e-14:
        qh = q.copy()
        oracle.halo_fill(qh, off, sz, nbr, 1, 3)
        _, lam = oracle.max_eigenvalue(qh, off, sz, 1)
        dt = min(oracle.cfl_dt(lam, cfl, dx, 1), T - t)
        q = oracle.patch_update(qh, off, sz, 1, dx, dt)
        t += dt
    return inputs.patches_to_domain(q, off, p, grid, 3)


def test_density_wave_first_order_convergence():
    """A density wave in uniform flow (u = 1, p = 1) is translated exactly by
    the Euler equations; the first-order Rusanov scheme converges with L1
    order close to 1."""
    T = 0.25
    errs = []
    Ns = [64, 128, 256, 512]
    for N in Ns:
        U = _run_1d(inputs.density_wave(N, 1), 8, T)
        x = inputs.cell_centres(N)
        # exact cell averages of 1 + 0.2 sin(2 pi (x - T))
        h = 1.0 / N
        exact = 1.0 + 0.2 * (np.cos(2 * np.pi * (x - h / 2 - T)) -
                             np.cos(2 * np.pi * (x + h / 2 - T))) / (2 * np.pi * h)
        errs.append(np.mean(np.abs(U[:, 0] - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(0.8 <= o <= 1.2 for o in orders), (errs, orders)
    # velocity and pressure stay uniform up to roundoff
    assert np.max(np.abs(U[:, 1] / U[:, 0] - 1.0)) < 1e-12


def test_sod_converges_to_exact_riemann_solution():
    """Sod's shock tube: L1 distance to the exact solution shrinks with N,
    at an order between 0.5 and 1 (discontinuities limit it)."""
    T = 0.2
    errs = []
    for N in (100, 200, 400):
        U = _run_1d(inputs.sod(N, 1), 10, T, periodic=False)
        x = inputs.cell_centres(N)
        rho_e, u_e, p_e = sample((x - 0.5) / T, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1)
        errs.append(np.mean(np.abs(U[:, 0] - rho_e)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 0.02
    assert all(0.4 <= o <= 1.1 for o in orders), (errs, orders)


@pytest.mark.parametrize("d,axis", [(2, 0), (2, 1), (3, 2)])
def test_sod_embedded_along_axis_matches_1d(d, axis):
    """A Sod tube along any axis of a 2D/3D patch mesh reproduces the 1D run
    (dimensional reduction + axis permutation; to roundoff, bitwise for the
    orders of summation that agree)."""
    N, p, T = 40, 10, 0.05
    U1 = _run_1d(inputs.sod(N, 1), p, T, periodic=False)
    U = inputs.sod(N, d, axis)
    q, off, sz, grid = inputs.domain_to_patches(U, p)
    nbr = inputs.grid_neighbours(grid, periodic=False, boundary=-1)
    s = d + 2
    t, dx = 0.0, 1.0 / N
    while t < T - 1e-14:
        qh = q.copy()
        oracle.halo_fill(qh, off, sz, nbr, d, s)
        _, lam = oracle.max_eigenvalue(qh, off, sz, d)
        # the 1D run uses d = 1 in the CFL factor; match its time steps
        dt = min(oracle.cfl_dt(lam, 0.4, dx, 1), T - t)
        q = oracle.patch_update(qh, off, sz, d, dx, dt)
        t += dt
    Ud = inputs.patches_to_domain(q, off, p, grid, s)
    ax = d - 1 - axis
    line = np.moveaxis(Ud, ax, -2)  # (..., N, s) along the tube
    line = line.reshape(-1, N, s)
    for l in line:
        assert np.allclose(l[:, 0], U1[:, 0], rtol=0, atol=1e-13)
        assert np.allclose(l[:, 1 + axis], U1[:, 1], rtol=0, atol=1e-13)
        assert np.allclose(l[:, d + 1], U1[:, 2], rtol=0, atol=1e-13)
