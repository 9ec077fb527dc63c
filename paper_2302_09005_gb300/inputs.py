"""Seeded synthetic inputs shaped like the patch workloads of arXiv 2302.09005.

This module is shared by the CUDA path's tests and benchmarks and by the CPU
oracle's tests.  It holds no arithmetic of the finite-volume method: it only
draws states, lays patches out in a flat buffer and builds neighbour tables.
Initial conditions are given in primitive variables (rho, u, p) and turned
into the conserved state (rho, rho u, E) with E = p/(gamma-1) + rho |u|^2/2.

Layout of a batch (the library's convention): patch i occupies elements
[off[i], off[i] + (p_i + 2h)^d * s) of one flat buffer; cells run x fastest,
then y, then z, the s unknowns of a cell innermost.  Every offset is a
multiple of ``align_bytes / itemsize`` elements.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def patch_elems(p: int, d: int, s: int, halo: int = 1) -> int:
    """Number of elements of one halo-inclusive patch."""
    return (p + 2 * halo) ** d * s


def layout(sizes, d: int, s: int, halo: int = 1, itemsize: int = 8, align_bytes: int = 16):
    """Offsets of consecutive patches, each rounded up to the alignment.

    Returns (offsets int64[n], total_elements)."""
    sizes = np.asarray(sizes, dtype=np.int64)
    a = max(1, align_bytes // itemsize)
    lens = (sizes + 2 * halo) ** d * s
    lens = (lens + a - 1) // a * a
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        off[1:] = np.cumsum(lens[:-1])
    total = int(lens.sum()) if len(sizes) else 0
    return off, total


def conserved_from_primitive(rho, vel, p, gamma: float = GAMMA):
    """(rho, u_1..u_d, p) -> (rho, rho u_1..rho u_d, E); vel has shape (..., d)."""
    vel = np.asarray(vel, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    p = np.asarray(p, dtype=np.float64)
    d = vel.shape[-1]
    q = np.empty(rho.shape + (d + 2,), dtype=np.float64)
    q[..., 0] = rho
    for k in range(d):
        q[..., 1 + k] = rho * vel[..., k]
    q[..., d + 1] = p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel, axis=-1)
    return q


def random_cells(rng: np.random.Generator, ncell: int, d: int, gamma: float = GAMMA):
    """Per-cell random states: rho ~ U[0.5,1.5], u_j ~ U[-0.5,0.5], p ~ U[0.5,1.5]."""
    rho = rng.uniform(0.5, 1.5, ncell)
    vel = rng.uniform(-0.5, 0.5, (ncell, d))
    p = rng.uniform(0.5, 1.5, ncell)
    return conserved_from_primitive(rho, vel, p, gamma)


def random_batch(n: int, p, d: int, *, seed: int = 0, halo: int = 1, dtype=np.float64,
                 align_bytes: int = 16, gamma: float = GAMMA):
    """A batch of n independent patches whose every cell (interior and the
    whole halo) holds an i.i.d. random state.

    ``p`` is one size for all patches or an array of n sizes.
    Returns (q flat array of ``dtype``, offsets int64[n], sizes int32[n]).
    Padding elements between patches are 0."""
    s = d + 2
    sizes = np.full(n, p, dtype=np.int32) if np.isscalar(p) else np.asarray(p, dtype=np.int32)
    itemsize = np.dtype(dtype).itemsize
    off, total = layout(sizes, d, s, halo, itemsize, align_bytes)
    rng = np.random.default_rng(seed)
    q = np.zeros(total, dtype=np.float64)
    if n:
        if np.all(sizes == sizes[0]):
            ne = patch_elems(int(sizes[0]), d, s, halo)
            stride = int(off[1] - off[0]) if n > 1 else ne
            view = q[:n * stride].reshape(n, stride)
            chunk = 1 << 14
            for c0 in range(0, n, chunk):
                c1 = min(n, c0 + chunk)
                view[c0:c1, :ne] = random_cells(rng, (c1 - c0) * ne // s, d,
                                                gamma).reshape(c1 - c0, ne)
        else:
            # one draw for all cells, written over every element that is not
            # alignment padding (patches are consecutive in the buffer)
            lens = (sizes.astype(np.int64) + 2 * halo) ** d * s
            padded = np.diff(np.append(off, total))
            npad = padded - lens
            mask = np.ones(total, dtype=bool)
            if npad.sum():
                ends = np.cumsum(npad)
                pos = (np.arange(ends[-1]) - np.repeat(ends - npad, npad)
                       + np.repeat(off + lens, npad))
                mask[pos] = False
            q[mask] = random_cells(rng, int(lens.sum()) // s, d, gamma).reshape(-1)
    return q.astype(dtype), off, sizes


def uneven_sizes(n: int, *, seed: int = 0, mix=((3, 0.5), (5, 0.3), (7, 0.2))):
    """n patch sizes in the stated proportions, shuffled (seeded)."""
    rng = np.random.default_rng(seed + 1000)
    counts = [int(round(frac * n)) for _, frac in mix]
    counts[0] += n - sum(counts)
    sizes = np.concatenate([np.full(c, p, dtype=np.int32) for (p, _), c in zip(mix, counts)])
    rng.shuffle(sizes)
    return sizes


def grid_neighbours(shape, periodic=True, boundary: int = -1):
    """Neighbour table of a Cartesian arrangement of patches.

    shape = (Px,) / (Px, Py) / (Px, Py, Pz) patches along each axis; patch
    index = a + Px*(b + Py*c).  Entries per patch in the order -x,+x,-y,+y,
    -z,+z; a missing neighbour gets ``boundary`` (-1 outflow, -2 wall)."""
    shape = tuple(int(x) for x in shape)
    d = len(shape)
    n = int(np.prod(shape))
    nbr = np.empty((n, 2 * d), dtype=np.int32)
    idx = np.arange(n)
    coords = []
    rem = idx.copy()
    for k in range(d):
        coords.append(rem % shape[k])
        rem //= shape[k]
    strides = [int(np.prod(shape[:k])) for k in range(d)]
    for k in range(d):
        for side, step in ((0, -1), (1, 1)):
            c = coords[k] + step
            inside = (c >= 0) & (c < shape[k])
            cw = c % shape[k]
            nb = idx + (cw - coords[k]) * strides[k]
            if not periodic:
                nb = np.where(inside, nb, boundary)
            nbr[:, 2 * k + side] = nb
    return nbr


def self_periodic_neighbours(n: int, d: int):
    """Every patch is its own neighbour on all faces (periodic per patch)."""
    return np.repeat(np.arange(n, dtype=np.int32)[:, None], 2 * d, axis=1)


def domain_to_patches(U, p: int, *, halo: int = 1, dtype=np.float64, align_bytes: int = 16):
    """Cut a domain array U of shape (Nz, Ny, Nx, s) / (Ny, Nx, s) / (Nx, s)
    (x fastest) into patches of p^d cells, patch index x fastest.

    Halo cells are set to 0; fill them with the library's or the oracle's
    halo fill.  Returns (q, offsets, sizes, patch_grid_shape)."""
    U = np.asarray(U, dtype=np.float64)
    d = U.ndim - 1
    s = U.shape[-1]
    ncell_axes = U.shape[:-1][::-1]  # (Nx, Ny, Nz)
    for N in ncell_axes:
        if N % p:
            raise ValueError("domain not divisible by the patch size")
    grid = tuple(N // p for N in ncell_axes)
    n = int(np.prod(grid))
    sizes = np.full(n, p, dtype=np.int32)
    off, total = layout(sizes, d, s, halo, np.dtype(dtype).itemsize, align_bytes)
    q = np.zeros(total, dtype=np.float64)
    ne = p + 2 * halo
    # reshape the domain into (patch coords..., cell coords...) with x fastest
    if d == 1:
        blocks = U.reshape(grid[0], p, s)
        for a in range(grid[0]):
            P = q[off[a]:off[a] + ne * s].reshape(ne, s)
            P[halo:halo + p] = blocks[a]
    elif d == 2:
        blocks = U.reshape(grid[1], p, grid[0], p, s).transpose(0, 2, 1, 3, 4)
        view = np.zeros((n, ne, ne, s))
        view[:, halo:halo + p, halo:halo + p] = blocks.reshape(n, p, p, s)
        idx = off[:, None] + np.arange(ne * ne * s)[None, :]
        q[idx] = view.reshape(n, -1)
    else:
        blocks = U.reshape(grid[2], p, grid[1], p, grid[0], p, s).transpose(0, 2, 4, 1, 3, 5, 6)
        view = np.zeros((n, ne, ne, ne, s))
        view[:, halo:halo + p, halo:halo + p, halo:halo + p] = blocks.reshape(n, p, p, p, s)
        idx = off[:, None] + np.arange(ne ** 3 * s)[None, :]
        q[idx] = view.reshape(n, -1)
    return q.astype(dtype), off, sizes, grid


def patches_to_domain(q, off, p: int, grid, s: int, *, halo: int = 1):
    """Inverse of ``domain_to_patches`` for the interior cells."""
    q = np.asarray(q, dtype=np.float64)
    d = len(grid)
    ne = p + 2 * halo
    n = int(np.prod(grid))
    idx = np.asarray(off)[:, None] + np.arange(ne ** d * s)[None, :]
    P = q[idx].reshape((n,) + (ne,) * d + (s,))
    sl = (slice(None),) + (slice(halo, halo + p),) * d
    P = P[sl]
    if d == 1:
        return P.reshape(grid[0] * p, s)
    if d == 2:
        return P.reshape(grid[1], grid[0], p, p, s).transpose(0, 2, 1, 3, 4).reshape(
            grid[1] * p, grid[0] * p, s)
    return P.reshape(grid[2], grid[1], grid[0], p, p, p, s).transpose(0, 3, 1, 4, 2, 5, 6).reshape(
        grid[2] * p, grid[1] * p, grid[0] * p, s)


def cell_centres(N: int):
    """Cell centres of N cells on [0, 1)."""
    return (np.arange(N) + 0.5) / N


def density_wave(N: int, d: int = 1, *, amp: float = 0.2, u: float = 1.0, pres: float = 1.0,
                 gamma: float = GAMMA):
    """rho = 1 + amp sin(2 pi x), velocity (u, 0, ..), p = const on N^d cells
    (domain array, x fastest)."""
    x = cell_centres(N)
    shape = (N,) * d
    rho = np.broadcast_to(1.0 + amp * np.sin(2 * np.pi * x), shape).copy()
    vel = np.zeros(shape + (d,))
    vel[..., 0] = u
    return conserved_from_primitive(rho, vel, np.full(shape, pres), gamma)


def sod(N: int, d: int = 1, axis: int = 0, *, gamma: float = GAMMA, x0: float = 0.5):
    """Sod shock tube (rho, u, p) = (1, 0, 1) | (0.125, 0, 0.1) split at x0
    along ``axis`` (0 = x), constant along the other axes; domain array."""
    x = cell_centres(N)
    shape = (N,) * d
    left = x < x0
    rho1 = np.where(left, 1.0, 0.125)
    p1 = np.where(left, 1.0, 0.1)
    # the domain array has axes (z, y, x); x is the last spatial axis
    ax = d - 1 - axis
    bshape = [1] * d
    bshape[ax] = N
    rho = np.broadcast_to(rho1.reshape(bshape), shape).copy()
    p = np.broadcast_to(p1.reshape(bshape), shape).copy()
    return conserved_from_primitive(rho, np.zeros(shape + (d,)), p, gamma)


def fourier_perturbation(N: int, *, seed: int = 0, amp: float = 0.1, modes: int = 16,
                         nwaves: int = 16, gamma: float = GAMMA):
    """2D periodic state rho = 1 + drho, (u, v) = (du, dv), p = 1, each
    perturbation a sum of ``nwaves`` random Fourier modes (k_x, k_y) with
    max(|k_x|, |k_y|) in [1, modes] and random phases, scaled to max |.| = amp."""
    rng = np.random.default_rng(seed)
    x = cell_centres(N)
    fields = []
    for _ in range(3):
        f = np.zeros((N, N))  # (y, x)
        for _w in range(nwaves):
            while True:
                kx, ky = rng.integers(-modes, modes + 1, size=2)
                if max(abs(kx), abs(ky)) >= 1:
                    break
            phi = rng.uniform(0, 2 * np.pi)
            # sin(a + b) = sin a cos b + cos a sin b, a = 2 pi kx x + phi, b = 2 pi ky y
            a = 2 * np.pi * kx * x + phi
            b = 2 * np.pi * ky * x
            f += np.sin(b)[:, None] * np.cos(a)[None, :]
            f += np.cos(b)[:, None] * np.sin(a)[None, :]
        f *= amp / np.max(np.abs(f))
        fields.append(f)
    rho = 1.0 + fields[0]
    vel = np.stack([fields[1], fields[2]], axis=-1)
    return conserved_from_primitive(rho, vel, np.ones((N, N)), gamma)


def shear_layer(N: int, *, seed: int = 0, amp: float = 0.01, gamma: float = GAMMA):
    """2D periodic shear layer: rho = 2, u = -0.5 for |y - 1/2| < 1/4, else
    rho = 1, u = +0.5; p = 2.5; v = sum_{k=1..4} a_k sin(2 pi k x + phi_k)
    scaled to max |v| = amp (seeded a_k, phi_k)."""
    rng = np.random.default_rng(seed)
    x = cell_centres(N)
    X, Y = np.meshgrid(x, x, indexing="xy")
    band = np.abs(Y - 0.5) < 0.25
    rho = np.where(band, 2.0, 1.0)
    u = np.where(band, -0.5, 0.5)
    a = rng.uniform(0, 1, 4)
    phi = rng.uniform(0, 2 * np.pi, 4)
    v1 = sum(a[k] * np.sin(2 * np.pi * (k + 1) * x + phi[k]) for k in range(4))
    v1 *= amp / np.max(np.abs(v1))
    v = np.broadcast_to(v1[None, :], (N, N))
    vel = np.stack([u, v], axis=-1)
    return conserved_from_primitive(rho, vel, np.full((N, N), 2.5), gamma)


def amr_mesh(d: int, p: int, base_level: int, refine=(), *, seed: int = 0, dtype=np.float64,
             align_bytes: int = 16, halo: int = 1):
    """A 3:1 refined patch mesh on the unit domain [0, 1]^d.

    The domain is a tree: a tree cell of level l has edge 3^-l and splits into
    3^d children of level l + 1.  Every tree cell of ``base_level`` (3^l per
    axis, integer coordinates c) carries a patch of p^d cells, except the
    cells listed in ``refine`` (coordinates at ``base_level``), which are
    replaced by their 3^d children (coordinates 3 c + a, a in {0, 1, 2}^d).
    Every cell, halo included, holds a random state (``random_cells``).

    Returns (q, off, sizes, level int32[n], coord int32[n, d]); patches are the
    unrefined base cells in index order (x fastest), then the children of each
    refined cell."""
    refine = {tuple(int(v) for v in c) for c in refine}
    nb = 3 ** base_level
    levels, coords = [], []
    for idx in np.ndindex(*(nb,) * d):
        c = tuple(reversed(idx))  # x fastest
        if c not in refine:
            levels.append(base_level)
            coords.append(c)
    for c in sorted(refine, key=lambda t: tuple(reversed(t))):
        for a in np.ndindex(*(3,) * d):
            child = tuple(3 * c[m] + a[d - 1 - m] for m in range(d))
            levels.append(base_level + 1)
            coords.append(child)
    n = len(levels)
    q, off, sizes = random_batch(n, p, d, seed=seed, dtype=dtype, align_bytes=align_bytes,
                                 halo=halo)
    return (q, off, sizes, np.asarray(levels, dtype=np.int32),
            np.asarray(coords, dtype=np.int32).reshape(n, d))
