"""Pins of the oracle of halos on 3:1 refined meshes (oracle/amr.py).

* On a mesh of one level it is the uniform halo fill (itself pinned), bitwise,
  for periodic, outflow and wall edges.
* Cell averages of a linear field: a halo cell next to a coarser patch holds
  the field at the centre of the coarse cell that contains it; one next to
  finer patches (or the same level) holds the field at its own centre (the
  mean of a linear field over 3^d sub-cells is its centre value).  The
  expected values come from point location, not from overlap integrals.
"""
import numpy as np
import pytest

import oracle
from oracle import amr
from paper_2302_09005_gb300 import inputs


@pytest.mark.parametrize("d,p,lev,boundary", [(2, 4, 1, 0), (2, 3, 2, -1), (3, 3, 1, -2),
                                               (1, 5, 2, 0), (3, 2, 1, 0)])
def test_single_level_equals_uniform_halo_fill(d, p, lev, boundary):
    q, off, sz, level, coord = inputs.amr_mesh(d, p, lev, (), seed=1)
    nbr = inputs.grid_neighbours((3 ** lev,) * d, periodic=boundary == 0,
                                 boundary=boundary if boundary else -1)
    ref = q.copy()
    oracle.halo_fill(ref, off, sz, nbr, d, d + 2)
    got = amr.amr_halo_fill(q, off, p, d, level, coord, boundary)
    mask = np.zeros(len(q), dtype=bool)  # face halos only (corners untouched by both)
    for o in off:
        ne = p + 2
        blk = np.zeros((ne,) * d + (d + 2,), dtype=bool)
        for k in range(d):
            for c in (0, ne - 1):
                sl = [slice(1, ne - 1)] * d
                sl[d - 1 - k] = c
                blk[tuple(sl)] = True
        mask[int(o):int(o) + blk.size] = blk.reshape(-1)
    assert np.array_equal(got[mask], ref[mask])


def linear_mesh(d, p, lev, refine, a, b):
    """Interior cells hold the exact cell averages of f_v(x) = a_v + b_v . x."""
    q, off, sz, level, coord = inputs.amr_mesh(d, p, lev, refine, seed=2)
    q = q.copy()
    s = d + 2
    for i in range(len(off)):
        h = 1.0 / (3 ** int(level[i]) * p)
        ne = p + 2
        blk = q[int(off[i]):int(off[i]) + ne ** d * s].reshape((ne,) * d + (s,))
        for loc in np.ndindex(*(p,) * d):
            xc = (coord[i] * p + np.array(loc[::-1]) + 0.5) * h  # x first
            blk[tuple(np.array(loc) + 1)] = a + b @ xc
    return q, off, level, coord


def leaf_at(point, level, coord):
    """Index of the patch whose tree cell contains the point (interior point)."""
    for i in range(len(level)):
        e = 3.0 ** -int(level[i])
        lo = coord[i] * e
        if np.all(point >= lo) and np.all(point < lo + e):
            return i
    raise AssertionError("no leaf")


@pytest.mark.parametrize("d,p,lev,refine", [
    (2, 4, 1, [(1, 1)]), (2, 3, 1, [(0, 0), (2, 1)]), (3, 3, 1, [(1, 1, 1)]),
    (1, 5, 1, [(1,)]), (2, 6, 1, [(1, 0), (1, 1)])])
def test_linear_field_prolongation_and_restriction(d, p, lev, refine):
    rng = np.random.default_rng(3)
    s = d + 2
    a = rng.uniform(-1, 1, s)
    b = rng.uniform(-1, 1, (s, d))
    q, off, level, coord = linear_mesh(d, p, lev, refine, a, b)
    got = amr.amr_halo_fill(q, off, p, d, level, coord, boundary=-1)
    checked = {"coarser": 0, "finer": 0, "same": 0}
    for i in range(len(off)):
        h = 1.0 / (3 ** int(level[i]) * p)
        ne = p + 2
        blk = got[int(off[i]):int(off[i]) + ne ** d * s].reshape((ne,) * d + (s,))
        for k in range(d):
            for side in (0, 1):
                for tr in np.ndindex(*(p,) * (d - 1)):
                    loc = np.zeros(d, dtype=np.int64)
                    trans = [m for m in range(d) if m != k]
                    for m, t in zip(trans, tr):
                        loc[m] = t
                    loc[k] = p if side else -1
                    xc = (coord[i] * p + loc + 0.5) * h
                    if np.any(xc < 0) or np.any(xc > 1):
                        continue  # domain edge: outflow copy, pinned above
                    j = leaf_at(xc, level, coord)
                    if level[j] < level[i]:  # coarser: centre of the containing coarse cell
                        H = 1.0 / (3 ** int(level[j]) * p)
                        xcc = (np.floor(xc / H) + 0.5) * H
                        want = a + b @ xcc
                        checked["coarser"] += 1
                    else:
                        want = a + b @ xc
                        checked["finer" if level[j] > level[i] else "same"] += 1
                    assert np.allclose(blk[tuple((loc + 1)[::-1])], want, rtol=0, atol=1e-14)
    assert checked["coarser"] > 0 and checked["finer"] > 0
