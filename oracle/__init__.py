"""FP64 CPU oracle for the batched Rusanov finite-volume patch update.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (``paper_2302_09005_gb300``) never imports it
and shares no code with it.

Contents:
  * ``fv_oracle.c`` -- Eq. 2-5 and Algorithm 1 of arXiv 2302.09005 written out
    in plain C (FP64, no FMA contraction), loaded here through ctypes.
  * ``riemann.py`` -- exact Riemann solver for the Euler equations (Toro,
    "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4), used
    only to verify the oracle.
  * ``mlp.py`` -- FP64 forward/backward of the learned face-flux correction.
  * ``amr.py`` -- halos of patches on 3:1 refined meshes (mean of the
    neighbouring solution over each halo cell).

Every function cites the passage of the paper it follows.  Functions without
an independent pin say "parity unpinned" in their docstring.
"""
from .core import (  # noqa: F401
    ORACLE_SO,
    build,
    lib,
    euler_flux,
    euler_wave_speed,
    rusanov_flux,
    patch_update,
    max_eigenvalue,
    cfl_dt,
    halo_fill,
    patch_sums,
    step,
)
