"""Halo cells of patches on a 3:1 refined mesh (FP64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's meshes come from spacetrees that split a cube into three parts
along every axis (Sec. 2, "block-structured mesh"); each cube carries a patch
of p^d cells and a halo layer whose consistency the engine maintains (Sec.
2).  The paper does not state the transfer between levels; the reading taken
here (one definition for every case): a halo cell holds the mean of the
piecewise-constant solution of the neighbouring patches over the halo cell's
region.  For a neighbour of the same level that is one cell (a copy); for a
coarser neighbour, the one coarse cell containing the halo cell (constant
prolongation); for finer neighbours, the mean of the 3^d fine cells it covers
(restriction by averaging).  Cells beyond a non-periodic domain edge follow
the rules of the uniform halo fill (-1 outflow: copy of the own adjacent
interior cell; -2 wall: its mirror image, normal momentum negated).

Geometry is integer: with L the finest level present, a level-l cell spans
3^(L-l) units of 1 / (3^L p).
"""
from __future__ import annotations

import numpy as np


def _interior(q, off, p, d, s, i, halo=1):
    """Interior cells of patch i as an array indexed [z][y][x][v] (d = 3)."""
    ne = p + 2 * halo
    blk = q[int(off[i]):int(off[i]) + ne ** d * s].reshape((ne,) * d + (s,))
    return blk[(slice(halo, halo + p),) * d]


def amr_halo_fill(q, off, p: int, d: int, level, coord, boundary: int = 0, halo: int = 1):
    """Fill the face halos of every patch (returns a copy of q as float64).

    level: int[n]; coord: int[n, d] tree-cell coordinates (x first) at each
    patch's level; boundary: 0 periodic, -1 outflow, -2 wall."""
    q = np.asarray(q, dtype=np.float64)
    out = q.copy()
    s = d + 2
    n = len(off)
    level = np.asarray(level)
    coord = np.asarray(coord)
    L = int(level.max())
    span = 3 ** (L - level)            # units per cell of each patch
    org = coord * p * span[:, None]    # patch origin in units (x first)
    dom = 3 ** L * p                   # domain edge in units
    ne = p + 2 * halo
    interiors = [_interior(q, off, p, d, s, j, halo) for j in range(n)]

    def mean_over(lo, hi):
        """Mean of the piecewise-constant solution over the box [lo, hi)
        (inside the domain: a periodic image is wrapped in first)."""
        vol = np.prod(hi - lo)
        parts = []  # (value, overlap volume)
        olo = np.maximum(lo[None, :], org)
        ohi = np.minimum(hi[None, :], org + p * span[:, None])
        for j in np.nonzero(np.all(ohi > olo, axis=1))[0]:
            a0 = (olo[j] - org[j]) // span[j]
            a1 = (ohi[j] - org[j] + span[j] - 1) // span[j]
            for loc in np.ndindex(*[int(a1[m] - a0[m]) for m in range(d)]):
                cl = np.array([a0[m] + loc[m] for m in range(d)])
                clo = org[j] + cl * span[j]
                w = np.prod(np.minimum(clo + span[j], hi) - np.maximum(clo, lo))
                if w > 0:
                    parts.append((interiors[j][tuple(cl[::-1])], w))
        if len(parts) == 1 and parts[0][1] == vol:  # one cell covers it: its value
            return parts[0][0].copy()
        acc = np.zeros(s)
        for v, w in parts:
            acc += v * w
        return acc / vol

    for i in range(n):
        blk = out[int(off[i]):int(off[i]) + ne ** d * s].reshape((ne,) * d + (s,))
        h = span[i]
        for k in range(d):
            for side in (0, 1):
                trans = [m for m in range(d) if m != k]
                for tr in np.ndindex(*(p,) * (d - 1)):
                    loc = np.zeros(d, dtype=np.int64)
                    for m, t in zip(trans, tr[::-1] if d > 1 else ()):
                        loc[m] = t
                    loc[k] = p if side else -1
                    lo = org[i] + loc * h
                    hi = lo + h
                    outside = lo[k] < 0 or hi[k] > dom
                    hidx = loc + halo
                    if outside and boundary == 0:  # periodic image inside the domain
                        lo = lo.copy()
                        lo[k] %= dom
                        hi = lo + h
                        outside = False
                    if outside:
                        src = loc.copy()
                        src[k] = p - 1 if side else 0
                        v = interiors[i][tuple(src[::-1])].copy()
                        if boundary == -2:
                            v[1 + k] = -v[1 + k]
                    else:
                        v = mean_over(lo, hi)
                    blk[tuple(hidx[::-1])] = v
    return out
