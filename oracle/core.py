"""ctypes front end of the C oracle (``fv_oracle.c``).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Arrays are numpy
float64 / int64 / int32 on the host.  Each wrapper names the equation or
algorithm step of arXiv 2302.09005 that the C function implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(_HERE, "fv_oracle.c")
ORACLE_SO = os.path.join(_HERE, "_build", "libfv_oracle.so")
# A test that plants a mistake in a copy of the oracle points this at the
# mutated library (tests/test_oracle_mutations.py); it is then used as is.
_SO_OVERRIDE = os.environ.get("FV_ORACLE_SO_OVERRIDE")

_lock = threading.Lock()
_lib = None

PDE_EULER = 0
PDE_ADVECTION = 1


def build(force: bool = False) -> str:
    """Compile ``fv_oracle.c`` with gcc (-O2, no FMA contraction)."""
    os.makedirs(os.path.dirname(ORACLE_SO), exist_ok=True)
    if (not force and os.path.exists(ORACLE_SO)
            and os.path.getmtime(ORACLE_SO) >= os.path.getmtime(ORACLE_SRC)):
        return ORACLE_SO
    tmp = ORACLE_SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99", "-fPIC",
           "-shared", "-o", tmp, ORACLE_SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, ORACLE_SO)
    return ORACLE_SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if _SO_OVERRIDE:
                L = ctypes.CDLL(_SO_OVERRIDE)
            else:
                build()
                L = ctypes.CDLL(ORACLE_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            c_int, c_dbl, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
            L.orc_euler_flux.argtypes = [dp, c_int, c_int, c_dbl, dp]
            L.orc_euler_flux.restype = None
            L.orc_euler_wave_speed.argtypes = [dp, c_int, c_int, c_dbl]
            L.orc_euler_wave_speed.restype = c_dbl
            L.orc_rusanov_flux.argtypes = [dp, dp, c_int, c_int, c_dbl, dp, dp]
            L.orc_rusanov_flux.restype = None
            L.orc_patch_update_pde.argtypes = [c_int, dp, dp, dp, i64p, i32p, c_i64, c_int,
                                               c_int, c_int, c_dbl, c_dbl, c_dbl, dp]
            L.orc_patch_update_pde.restype = c_int
            L.orc_max_eigenvalue.argtypes = [dp, i64p, i32p, c_i64, c_int, c_int, c_dbl, dp,
                                             dp]
            L.orc_max_eigenvalue.restype = c_int
            L.orc_cfl_dt.argtypes = [c_dbl, c_dbl, c_dbl, c_int]
            L.orc_cfl_dt.restype = c_dbl
            L.orc_halo_fill.argtypes = [dp, i64p, i32p, i32p, c_i64, c_int, c_int, c_int]
            L.orc_halo_fill.restype = c_int
            L.orc_patch_sums.argtypes = [dp, i64p, i32p, c_i64, c_int, c_int, c_int, dp]
            L.orc_patch_sums.restype = c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _meta(off, sizes):
    off = np.ascontiguousarray(off, dtype=np.int64)
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    return off, sizes, off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), \
        sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def euler_flux(q, d: int, direction: int, gamma: float = 1.4) -> np.ndarray:
    """Euler flux f^j(q) of Eq. 2 (energy flux (E+p) j_j / rho)."""
    q = _f64(q)
    f = np.empty(d + 2)
    lib().orc_euler_flux(_dp(q), d, direction, gamma, _dp(f))
    return f


def euler_wave_speed(q, d: int, direction: int, gamma: float = 1.4) -> float:
    """|u_j| + c, the largest |eigenvalue| of the flux Jacobian (Eq. 5)."""
    q = _f64(q)
    return lib().orc_euler_wave_speed(_dp(q), d, direction, gamma)


def rusanov_flux(qL, qR, d: int, direction: int, gamma: float = 1.4):
    """Rusanov face flux of Eq. 4; returns (F, a)."""
    qL, qR = _f64(qL), _f64(qR)
    F = np.empty(d + 2)
    a = ctypes.c_double()
    lib().orc_rusanov_flux(_dp(qL), _dp(qR), d, direction, gamma, _dp(F), ctypes.byref(a))
    return F, a.value


def patch_update(q_in, off, sizes, d: int, dx: float, dt: float, *, halo: int = 1,
                 gamma: float = 1.4, s: int | None = None, pde: int = PDE_EULER,
                 adv=None, q_out=None, want_lambda: bool = False):
    """One explicit step of every patch (Eq. 3 with Eq. 4 fluxes; Algorithm 1).

    Returns the output buffer (a copy of q_in whose interior cells are
    replaced), and, with ``want_lambda``, the per-patch maximum eigenvalue
    over the faces used (Algorithm 1, step 10).
    """
    q_in = _f64(q_in)
    s = d + 2 if s is None else s
    out = q_in.copy() if q_out is None else q_out
    off, sizes, offp, szp = _meta(off, sizes)
    lam = np.zeros(len(off)) if want_lambda else None
    advv = _f64(np.zeros(3) if adv is None else np.asarray(adv, dtype=np.float64))
    rc = lib().orc_patch_update_pde(pde, _dp(advv), _dp(q_in), _dp(out), offp, szp,
                                    len(off), d, s, halo, gamma, dx, dt,
                                    _dp(lam) if lam is not None else None)
    if rc != 0:
        raise ValueError("oracle patch_update: invalid arguments")
    return (out, lam) if want_lambda else out


def max_eigenvalue(q, off, sizes, d: int, *, halo: int = 1, gamma: float = 1.4):
    """Per-patch and batch maximum of a over the faces bounding interior cells
    (Eq. 5; Algorithm 1, step 10).  Returns (per_patch, global)."""
    q = _f64(q)
    off, sizes, offp, szp = _meta(off, sizes)
    lam = np.zeros(len(off))
    g = ctypes.c_double()
    rc = lib().orc_max_eigenvalue(_dp(q), offp, szp, len(off), d, halo, gamma, _dp(lam),
                                  ctypes.byref(g))
    if rc != 0:
        raise ValueError("oracle max_eigenvalue: invalid arguments")
    return lam, g.value


def cfl_dt(lam_max: float, cfl: float, dx: float, d: int) -> float:
    """dt = cfl * dx / (d * lambda_max) (the CFL reading used throughout)."""
    return lib().orc_cfl_dt(lam_max, cfl, dx, d)


def halo_fill(q, off, sizes, nbr, d: int, s: int, *, halo: int = 1) -> np.ndarray:
    """Fill face halos from neighbours (-1 outflow, -2 reflecting wall), in place."""
    assert q.dtype == np.float64 and q.flags.c_contiguous
    off, sizes, offp, szp = _meta(off, sizes)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    rc = lib().orc_halo_fill(_dp(q), offp, szp, nbr.ctypes.data_as(
        ctypes.POINTER(ctypes.c_int32)), len(off), d, s, halo)
    if rc != 0:
        raise ValueError("oracle halo_fill: invalid arguments")
    return q


def patch_sums(q, off, sizes, d: int, s: int, *, halo: int = 1) -> np.ndarray:
    """Per-patch interior sums of each unknown, shape (n, s)."""
    q = _f64(q)
    off, sizes, offp, szp = _meta(off, sizes)
    out = np.zeros((len(off), s))
    rc = lib().orc_patch_sums(_dp(q), offp, szp, len(off), d, s, halo, _dp(out))
    if rc != 0:
        raise ValueError("oracle patch_sums: invalid arguments")
    return out


def step(q, off, sizes, nbr, d: int, dx: float, cfl: float, *, halo: int = 1,
         gamma: float = 1.4, dt: float | None = None):
    """One full time step of a patch mesh: halo fill, CFL time step from the
    batch maximum eigenvalue, then the update of Eq. 3.  Returns (q_new, dt)."""
    s = d + 2
    q = _f64(q).copy()
    halo_fill(q, off, sizes, nbr, d, s, halo=halo)
    if dt is None:
        _, lam = max_eigenvalue(q, off, sizes, d, halo=halo, gamma=gamma)
        dt = cfl_dt(lam, cfl, dx, d)
    q_new = patch_update(q, off, sizes, d, dx, dt, halo=halo, gamma=gamma)
    return q_new, dt
