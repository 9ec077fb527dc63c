"""FP64 oracle of the learned conservative face-flux correction on periodic 2D
domains (numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Domain arrays have shape (Ny, Nx, 4), unknowns (rho, j_x, j_y, E), periodic
on both axes.  The x-face (J, I) lies between cells (J, I-1) and (J, I); the
y-face (J, I) between (J-1, I) and (J, I).

* Rusanov flux of Eq. 4 with a = max(|u_n|+c) of the two cells (Eq. 5), the
  Euler flux of Eq. 2, and the update of Eq. 3 -- here vectorised over a
  domain; tests check it against the C oracle (fv_oracle.c).
* The correction C is added to the face flux F (so both cells of a face see
  the same F + C and the totals are conserved by construction).  It is an
  MLP (oracle/mlp.py) of the normalised 4-cell stencil Q_{i-2..i+1} normal to
  the face, written in the face's normal frame (rho, j_n, j_t, E); its output
  (normal frame, scaled by sd_y) is rotated back.
* Training targets: the fine solution at r-times the resolution, advanced by
  r substeps of dt/r, restricted by block averages, evolves exactly by the
  time-and-face averages of the fine fluxes through the coarse faces
  (telescoping of Eq. 3).  The ideal correction is that average minus the
  coarse Rusanov flux of the restricted state.
"""
from __future__ import annotations

import numpy as np

from . import mlp

GAMMA = 1.4


def _prims(U, gamma=GAMMA):
    rho = U[..., 0]
    u = U[..., 1] / rho
    v = U[..., 2] / rho
    p = (gamma - 1.0) * (U[..., 3] - 0.5 * (U[..., 1] * U[..., 1] + U[..., 2] * U[..., 2]) / rho)
    c = np.sqrt(gamma * p / rho)
    return u, v, p, c


def euler_flux(U, axis, gamma=GAMMA):
    """f^axis(U) of Eq. 2 (axis 1 = x, axis 0 = y) and |u_axis| + c."""
    u, v, p, c = _prims(U, gamma)
    un = u if axis == 1 else v
    f = np.empty_like(U)
    f[..., 0] = U[..., 1] if axis == 1 else U[..., 2]
    f[..., 1] = U[..., 1] * un + (p if axis == 1 else 0.0)
    f[..., 2] = U[..., 2] * un + (p if axis == 0 else 0.0)
    f[..., 3] = (U[..., 3] + p) * un
    return f, np.abs(un) + c


def face_fluxes(U, axis, gamma=GAMMA):
    """Rusanov flux (Eq. 4) on every face normal to `axis`; index = right cell."""
    f, lam = euler_flux(U, axis, gamma)
    fl = np.roll(f, 1, axis=axis)
    ll = np.roll(lam, 1, axis=axis)
    UL = np.roll(U, 1, axis=axis)
    a = np.maximum(ll, lam)[..., None]
    return 0.5 * ((fl + f) - a * (U - UL))


def to_normal(A, axis):
    """Physical (rho, j_x, j_y, E) -> normal frame (rho, j_n, j_t, E) for faces
    normal to `axis` (a swap of the momenta for y faces; its own inverse)."""
    if axis == 1:
        return A
    B = A.copy()
    B[..., 1], B[..., 2] = A[..., 2], A[..., 1]
    return B


def stencils(U, axis):
    """(Ny, Nx, 16): Q_{i-2}, Q_{i-1}, Q_i, Q_{i+1} along `axis` for the face
    left of cell i, each in the normal frame."""
    parts = [to_normal(np.roll(U, s, axis=axis), axis) for s in (2, 1, 0, -1)]
    return np.concatenate(parts, axis=-1)


def correction(U, axis, theta, norm):
    """MLP correction on every face normal to `axis`, physical frame.
    norm = (mu_x (16), sd_x (16), sd_y (4))."""
    mu_x, sd_x, sd_y = norm
    X = (stencils(U, axis) - mu_x) / sd_x
    y, _ = mlp.forward(theta, X.reshape(-1, 16))
    return to_normal(y.reshape(U.shape[:2] + (4,)) * sd_y, axis)


def step(U, dt, dx, corr_x=None, corr_y=None, gamma=GAMMA):
    """One explicit step (Eq. 3) with face fluxes F + C."""
    Fx = face_fluxes(U, 1, gamma)
    Fy = face_fluxes(U, 0, gamma)
    if corr_x is not None:
        Fx = Fx + corr_x
    if corr_y is not None:
        Fy = Fy + corr_y
    div = (np.roll(Fx, -1, axis=1) - Fx) + (np.roll(Fy, -1, axis=0) - Fy)
    return U - (dt / dx) * div


def learned_step(U, dt, dx, theta, norm, gamma=GAMMA):
    return step(U, dt, dx, correction(U, 1, theta, norm), correction(U, 0, theta, norm), gamma)


def max_wave_speed(U, gamma=GAMMA):
    _, _, _, c = _prims(U, gamma)
    u, v, _, _ = _prims(U, gamma)
    return float(max(np.max(np.abs(u) + c), np.max(np.abs(v) + c)))


def restrict(Uf, r):
    """Block average of r x r fine cells."""
    Ny, Nx, s = Uf.shape
    return Uf.reshape(Ny // r, r, Nx // r, r, s).mean(axis=(1, 3))


def coarse_face_average(F, r, axis):
    """Average of the r fine face fluxes on each coarse face normal to `axis`."""
    Ny, Nx, s = F.shape
    if axis == 1:  # x faces at fine x = r I; rows J r .. J r + r - 1
        return F[:, ::r].reshape(Ny // r, r, Nx // r, s).mean(axis=1)
    return F[::r, :].reshape(Ny // r, Nx // r, r, s).mean(axis=2)


def ideal_correction(Uf, r, dt, dx_f, gamma=GAMMA):
    """Advance the fine state by r substeps of dt / r; return (restricted
    start, restricted end, Cx*, Cy*, fine end) with C* = time-and-face
    averaged fine flux - coarse Rusanov flux of the restricted start."""
    Uc0 = restrict(Uf, r)
    Ax = np.zeros_like(Uc0)
    Ay = np.zeros_like(Uc0)
    U = Uf
    for _ in range(r):
        Ax += coarse_face_average(face_fluxes(U, 1, gamma), r, 1) / r
        Ay += coarse_face_average(face_fluxes(U, 0, gamma), r, 0) / r
        U = step(U, dt / r, dx_f, gamma=gamma)
    Cx = Ax - face_fluxes(Uc0, 1, gamma)
    Cy = Ay - face_fluxes(Uc0, 0, gamma)
    return Uc0, restrict(U, r), Cx, Cy, U
