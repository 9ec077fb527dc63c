"""Builds libfv.so, the CUDA library behind include/fv.h, for sm_103a.

Each translation unit under csrc/ compiles in its own nvcc process (in
parallel); the objects link into one shared library inside the package
(``_build/libfv.so``), which the ctypes binding loads.
"""
from __future__ import annotations

import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libfv.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")) + \
        [os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=(), out: str | None = None) -> str:
    """Compile every csrc/*.cu for sm_103a and link libfv.so; returns its path.
    ``out`` builds a variant (with ``extra_flags``) elsewhere instead."""
    lib = LIB if out is None else out
    build_dir = BUILD if out is None else os.path.dirname(os.path.abspath(out))
    if out is None and not force and up_to_date():
        return LIB
    os.makedirs(build_dir, exist_ok=True)
    procs = []
    objs = []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra_flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                            stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed.append((src, out))
        elif verbose and out.strip():
            print(out)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart=static"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def source_hash() -> str:
    """Hash of every source that goes into libfv.so (kernels, headers)."""
    import hashlib
    hsh = hashlib.sha256()
    for f in sorted(_deps()):
        if f.endswith("_build.py"):
            continue
        with open(f, "rb") as fh:
            hsh.update(os.path.basename(f).encode())
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


# Sources of each update / time-step kernel (device code and the headers it
# includes); host-side API changes leave its counters valid.
_STEP_CORE = ("fv_step.cuh", "fv_device.cuh", "fv_ptx.cuh")
KERNEL_SOURCES = {
    "step": _STEP_CORE + ("fv_update.cu", "fv_update_f32.cu", "fv_update_nt.cu",
                          "fv_update_nt_f32.cu"),
    "march3d": _STEP_CORE + ("fv_march3d.cu", "fv_cell3.cuh", "fv_meta.cuh"),
    "rows2d": _STEP_CORE + ("fv_rows2d.cu", "fv_meta.cuh"),
    "corr": ("fv_learned.cu", "fv_device.cuh", "fv_mma.cuh", "fv_ptx.cuh", "fv_tc.cuh",
             "fv_x2.cuh"),
}


def kernel_hash(kind: str = "step") -> str:
    """Hash of one kernel's sources (keys the committed ncu traffic)."""
    import hashlib
    hsh = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(CSRC, name), "rb") as fh:
            hsh.update(name.encode())
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]
