"""Thin ctypes binding of libfv (include/fv.h), with the C names.

Argument marshalling only: every step of the path runs in the CUDA kernels
of libfv.so.  Buffers are CUDA tensors (or raw device addresses as ints);
the library enqueues work on the handle's stream and returns a status that
this module turns into an exception.  If the library cannot be loaded the
import of this module fails: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

FV_OK = 0
FV_ERR_INVALID_ARG = 1
FV_ERR_ALIGNMENT = 2
FV_ERR_UNSUPPORTED = 3
FV_ERR_CUDA = 4
FV_ERR_NONPHYSICAL = 5
FV_ERR_TIMEOUT = 6
FV_ERR_BAD_PATCH = 7

FV_FP64 = 0
FV_FP32 = 1


class FvError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = _lib().fv_status_string(status).decode() if _LIB is not None else str(status)
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


class fv_options(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("halo", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_patch_size", ctypes.c_int)]


class fv_update_extras(ctypes.Structure):
    _fields_ = [("lambda_patch", ctypes.c_void_p), ("n_elems", ctypes.c_int64),
                ("corr", ctypes.c_void_p)]


_LIB = None


def lib_path() -> str:
    return _build.LIB


def _lib() -> ctypes.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libfv.so is not built ({_build.LIB}); run "
                              "paper_2302_09005_gb300._build.build() or __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        vp, i64, i32, dbl, c_int = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_double, ctypes.c_int)
        L.fv_options_default.argtypes = [ctypes.POINTER(fv_options)]
        L.fv_options_default.restype = None
        L.fv_status_string.argtypes = [c_int]
        L.fv_status_string.restype = ctypes.c_char_p
        L.fv_batch_create.argtypes = [ctypes.POINTER(vp), c_int, c_int,
                                      ctypes.POINTER(fv_options), vp]
        L.fv_batch_destroy.argtypes = [vp]
        L.fv_batch_set_stream.argtypes = [vp, vp]
        L.fv_patch_update_batch.argtypes = [vp, vp, vp, vp, vp, i64, c_int, c_int, dbl, dbl]
        L.fv_patch_update_batch_ex.argtypes = [vp, vp, vp, vp, vp, i64, c_int, c_int, dbl, dbl,
                                               ctypes.POINTER(fv_update_extras)]
        L.fv_halo_fill.argtypes = [vp, vp, vp, vp, vp, i64]
        L.fv_patch_update_host.argtypes = [vp, vp, vp, vp, vp, i64, dbl, dbl, i64]
        L.fv_patch_update_host.restype = c_int
        L.fv_patch_update_local.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, dbl, vp]
        L.fv_patch_update_local.restype = c_int
        L.fv_amr_plan_create.argtypes = [vp, ctypes.POINTER(vp), i64, vp, vp, vp, c_int, c_int]
        L.fv_amr_plan_create.restype = c_int
        L.fv_amr_halo_fill.argtypes = [vp, vp, vp]
        L.fv_amr_halo_fill.restype = c_int
        L.fv_amr_plan_destroy.argtypes = [vp]
        L.fv_amr_plan_destroy.restype = c_int
        L.fv_max_eigenvalue_reduce.argtypes = [vp, vp, vp, vp, i64, vp, vp, dbl, dbl, vp]
        L.fv_conserved_totals.argtypes = [vp, vp, vp, vp, i64, vp]
        L.fv_patch_sums.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.fv_get_dt_ptr.argtypes = [vp, ctypes.POINTER(vp)]
        L.fv_get_status.argtypes = [vp]
        L.fv_selftest_math.argtypes = [vp, vp, i64, c_int]
        L.fv_selftest_math.restype = c_int
        L.fv_conserved_totals_noalloc.argtypes = [c_int, c_int, c_int, vp, vp, vp, i64, vp, vp,
                                                  vp]
        L.fv_conserved_totals_noalloc.restype = c_int
        L.fv_time_step.argtypes = [vp, vp, vp, vp, vp, vp, i64, dbl, dbl, vp]
        L.fv_time_step.restype = c_int
        L.fv_time_step_prim.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i64, dbl, dbl, vp]
        L.fv_time_step_prim.restype = c_int
        L.fv_prim_stride.argtypes = [vp, ctypes.POINTER(i64)]
        L.fv_prim_stride.restype = c_int
        L.fv_run_steps.argtypes = [vp, vp, vp, vp, vp, vp, i64, dbl, dbl, c_int, c_int]
        L.fv_run_steps.restype = c_int
        L.fv_read_dt.argtypes = [vp, ctypes.POINTER(dbl)]
        L.fv_read_dt.restype = c_int
        L.fv_batch_plan.argtypes = [vp, vp, i64]
        L.fv_batch_plan.restype = c_int
        L.fv_batch_set_schedule.argtypes = [vp, c_int]
        L.fv_batch_set_schedule.restype = c_int
        L.fv_batch_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
        L.fv_batch_set_wait_limit.restype = c_int
        L.fv_batch_set_class_threads.argtypes = [vp, c_int, c_int]
        L.fv_batch_set_class_threads.restype = c_int
        L.fv_batch_class_threads.argtypes = [vp, c_int, ctypes.POINTER(c_int)]
        L.fv_batch_class_threads.restype = c_int
        L.fv_batch_pairs_launches.argtypes = [vp, ctypes.POINTER(i64)]
        L.fv_batch_pairs_launches.restype = c_int
        L.fv_batch_autotune.argtypes = [vp, vp, vp, vp, vp, vp, i64, dbl, dbl,
                                        ctypes.POINTER(c_int), ctypes.POINTER(dbl)]
        L.fv_batch_autotune.restype = c_int
        L.fv_mlp_trainer_create.argtypes = [ctypes.POINTER(vp), i64, vp]
        L.fv_mlp_trainer_destroy.argtypes = [vp]
        L.fv_mlp_forward.argtypes = [vp, vp, vp, i64, vp]
        L.fv_mlp_grad.argtypes = [vp, vp, vp, vp, i64, vp, vp]
        L.fv_mlp_train_step.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, c_int, vp]
        L.fv_mlp_train_steps.argtypes = [vp, vp, vp, vp, i64, i64, c_int, c_int, ctypes.c_float,
                                         vp]
        L.fv_mlp_trainer_status.argtypes = [vp]
        for name in ("fv_mlp_trainer_create", "fv_mlp_trainer_destroy", "fv_mlp_forward",
                     "fv_mlp_grad", "fv_mlp_train_step", "fv_mlp_train_steps",
                     "fv_mlp_trainer_status"):
            getattr(L, name).restype = c_int
        L.fv_corr_stride.argtypes = [vp]
        L.fv_corr_stride.restype = i64
        L.fv_flux_correction.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.fv_time_step_corrected.argtypes = [vp, vp, vp, vp, vp, vp, i64, dbl, dbl, vp]
        L.fv_restrict_mesh.argtypes = [vp, vp, vp, c_int, c_int, vp, vp, vp, c_int, c_int, c_int]
        L.fv_accumulate_face_flux.argtypes = [vp, vp, vp, c_int, c_int, vp, c_int, c_int, c_int,
                                              dbl, vp]
        L.fv_correction_samples.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp]
        L.fv_column_moments.argtypes = [vp, i64, c_int, vp, vp, vp, vp]
        L.fv_normalize_columns.argtypes = [vp, i64, c_int, vp, vp, vp]
        for name in ("fv_flux_correction", "fv_time_step_corrected", "fv_restrict_mesh",
                     "fv_accumulate_face_flux", "fv_correction_samples", "fv_column_moments",
                     "fv_normalize_columns"):
            getattr(L, name).restype = c_int
        L.fv_last_error.argtypes = [vp]
        L.fv_last_error.restype = ctypes.c_char_p
        for name in ("fv_batch_create", "fv_batch_destroy", "fv_batch_set_stream",
                     "fv_patch_update_batch", "fv_patch_update_batch_ex", "fv_halo_fill",
                     "fv_max_eigenvalue_reduce", "fv_conserved_totals", "fv_get_dt_ptr",
                     "fv_get_status"):
            getattr(L, name).restype = c_int
        _LIB = L
    return _LIB


def _ptr(x) -> int | None:
    """Device address of a tensor / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(h, status: int, where: str):
    if status != FV_OK:
        detail = ""
        if h is not None:
            detail = (_lib().fv_last_error(h) or b"").decode()
        raise FvError(status, where, detail)


def fv_options_default() -> fv_options:
    o = fv_options()
    _lib().fv_options_default(ctypes.byref(o))
    return o


def fv_batch_create(d: int, s: int, options: fv_options | None = None, stream=None) -> int:
    """Create a handle; ``stream`` is a torch.cuda.Stream, a raw cudaStream_t
    int or None (the current torch stream)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    sp = stream if isinstance(stream, int) else stream.cuda_stream
    h = ctypes.c_void_p()
    st = _lib().fv_batch_create(ctypes.byref(h), d, s,
                                ctypes.byref(options) if options is not None else None, sp)
    _check(None, st, "fv_batch_create")
    return h.value


def fv_batch_destroy(h: int):
    _check(None, _lib().fv_batch_destroy(h), "fv_batch_destroy")


def fv_batch_set_stream(h: int, stream):
    sp = stream if isinstance(stream, int) else stream.cuda_stream
    _check(h, _lib().fv_batch_set_stream(h, sp), "fv_batch_set_stream")


def fv_patch_update_batch(h, in_with_halo, out, patch_offsets, patch_sizes, n_patches: int,
                          d: int, s: int, dx: float, dt: float):
    st = _lib().fv_patch_update_batch(h, _ptr(in_with_halo), _ptr(out), _ptr(patch_offsets),
                                      _ptr(patch_sizes), n_patches, d, s, dx, dt)
    _check(h, st, "fv_patch_update_batch")


def fv_patch_update_batch_ex(h, in_with_halo, out, patch_offsets, patch_sizes, n_patches: int,
                             d: int, s: int, dx: float, dt: float, lambda_patch=None,
                             n_elems: int = 0, corr=None):
    ex = fv_update_extras(_ptr(lambda_patch), n_elems, _ptr(corr))
    st = _lib().fv_patch_update_batch_ex(h, _ptr(in_with_halo), _ptr(out), _ptr(patch_offsets),
                                         _ptr(patch_sizes), n_patches, d, s, dx, dt,
                                         ctypes.byref(ex))
    _check(h, st, "fv_patch_update_batch_ex")


def fv_patch_update_host(h, host_in, host_out, patch_offsets, patch_sizes, n_patches: int,
                         dx: float, dt: float, chunk_patches: int = 0):
    """host_in / host_out: host tensors (pinned for overlap) or numpy arrays;
    patch_offsets / patch_sizes: host int64 / int32 arrays."""
    import numpy as np
    off = np.ascontiguousarray(np.asarray(patch_offsets), dtype=np.int64)
    sz = np.ascontiguousarray(np.asarray(patch_sizes), dtype=np.int32)
    def hptr(x):
        return x.data_ptr() if hasattr(x, "data_ptr") else x.ctypes.data
    st = _lib().fv_patch_update_host(h, hptr(host_in), hptr(host_out), off.ctypes.data,
                                     sz.ctypes.data, n_patches, dx, dt, chunk_patches)
    _check(h, st, "fv_patch_update_host")


def fv_patch_update_local(h, in_with_halo, out, patch_offsets, patch_sizes, n_patches: int,
                          dx_patch, dt_patch, cfl: float = 0.0, lambda_patch=None):
    st = _lib().fv_patch_update_local(h, _ptr(in_with_halo), _ptr(out), _ptr(patch_offsets),
                                      _ptr(patch_sizes), n_patches, _ptr(dx_patch),
                                      _ptr(dt_patch), cfl, _ptr(lambda_patch))
    _check(h, st, "fv_patch_update_local")


class AmrPlan:
    """Owns an fv_amr_plan: halos of a 3:1 refined mesh (host level / coord /
    offset arrays, numpy)."""

    def __init__(self, h, level, coord, patch_offsets, p: int, boundary: int = 0):
        import numpy as np
        self._level = np.ascontiguousarray(level, dtype=np.int32)
        self._coord = np.ascontiguousarray(coord, dtype=np.int32)
        self._off = np.ascontiguousarray(patch_offsets, dtype=np.int64)
        self.h = h
        self.plan = ctypes.c_void_p()
        st = _lib().fv_amr_plan_create(h, ctypes.byref(self.plan), len(self._off),
                                       self._level.ctypes.data, self._coord.ctypes.data,
                                       self._off.ctypes.data, p, boundary)
        _check(h, st, "fv_amr_plan_create")

    def fill(self, q_with_halo):
        _check(self.h, _lib().fv_amr_halo_fill(self.h, self.plan, _ptr(q_with_halo)),
               "fv_amr_halo_fill")

    def close(self):
        if self.plan:
            _lib().fv_amr_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fv_halo_fill(h, q_with_halo, patch_offsets, patch_sizes, neighbours, n_patches: int):
    st = _lib().fv_halo_fill(h, _ptr(q_with_halo), _ptr(patch_offsets), _ptr(patch_sizes),
                             _ptr(neighbours), n_patches)
    _check(h, st, "fv_halo_fill")


def fv_max_eigenvalue_reduce(h, q_with_halo, patch_offsets, patch_sizes, n_patches: int,
                             per_patch_max=None, global_max=None, cfl: float = 0.4,
                             dx: float = 1.0, dt_out=None):
    st = _lib().fv_max_eigenvalue_reduce(h, _ptr(q_with_halo), _ptr(patch_offsets),
                                         _ptr(patch_sizes), n_patches, _ptr(per_patch_max),
                                         _ptr(global_max), cfl, dx, _ptr(dt_out))
    _check(h, st, "fv_max_eigenvalue_reduce")


def fv_time_step(h, in_with_halo, out, patch_offsets, patch_sizes, neighbours, n_patches: int,
                 dx: float, cfl: float, lambda_patch=None):
    st = _lib().fv_time_step(h, _ptr(in_with_halo), _ptr(out), _ptr(patch_offsets),
                             _ptr(patch_sizes), _ptr(neighbours), n_patches, dx, cfl,
                             _ptr(lambda_patch))
    _check(h, st, "fv_time_step")


def fv_prim_stride(h) -> int:
    out = ctypes.c_int64(0)
    _check(h, _lib().fv_prim_stride(h, ctypes.byref(out)), "fv_prim_stride")
    return int(out.value)


def fv_time_step_prim(h, in_with_halo, out, prim_in, prim_out, patch_offsets, patch_sizes,
                      neighbours, n_patches: int, dx: float, cfl: float, lambda_patch=None):
    st = _lib().fv_time_step_prim(h, _ptr(in_with_halo), _ptr(out), _ptr(prim_in),
                                  _ptr(prim_out), _ptr(patch_offsets), _ptr(patch_sizes),
                                  _ptr(neighbours), n_patches, dx, cfl, _ptr(lambda_patch))
    _check(h, st, "fv_time_step_prim")


def fv_run_steps(h, q0, q1, patch_offsets, patch_sizes, neighbours, n_patches: int, dx: float,
                 cfl: float, n_steps: int, use_graph: bool = False):
    st = _lib().fv_run_steps(h, _ptr(q0), _ptr(q1), _ptr(patch_offsets), _ptr(patch_sizes),
                             _ptr(neighbours), n_patches, dx, cfl, n_steps, int(use_graph))
    _check(h, st, "fv_run_steps")


def fv_conserved_totals(h, q_with_halo, patch_offsets, patch_sizes, n_patches: int, totals):
    st = _lib().fv_conserved_totals(h, _ptr(q_with_halo), _ptr(patch_offsets),
                                    _ptr(patch_sizes), n_patches, _ptr(totals))
    _check(h, st, "fv_conserved_totals")


def fv_patch_sums(h, q_with_halo, patch_offsets, patch_sizes, n_patches: int, per_patch,
                  totals=None):
    st = _lib().fv_patch_sums(h, _ptr(q_with_halo), _ptr(patch_offsets), _ptr(patch_sizes),
                              n_patches, _ptr(per_patch), _ptr(totals))
    _check(h, st, "fv_patch_sums")


def fv_conserved_totals_noalloc(d: int, s: int, precision: int, q_with_halo, patch_offsets,
                                patch_sizes, n_patches: int, totals, status_word=None,
                                stream=None):
    """Conservation sums without a handle and without device allocation
    (scratch in the library's static device memory); see include/fv.h."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    sp = stream if isinstance(stream, int) else stream.cuda_stream
    st = _lib().fv_conserved_totals_noalloc(d, s, precision, _ptr(q_with_halo),
                                            _ptr(patch_offsets), _ptr(patch_sizes), n_patches,
                                            _ptr(totals), _ptr(status_word), sp)
    _check(None, st, "fv_conserved_totals_noalloc")


def fv_get_dt_ptr(h) -> int:
    p = ctypes.c_void_p()
    _check(h, _lib().fv_get_dt_ptr(h, ctypes.byref(p)), "fv_get_dt_ptr")
    return p.value


FV_SCHED_STRIDE = 0
FV_SCHED_LPT = 1
FV_SCHED_CLASSES = 2
FV_SCHED_QUEUE = 3


def fv_batch_plan(h, patch_sizes, n_patches: int):
    _check(h, _lib().fv_batch_plan(h, _ptr(patch_sizes), n_patches), "fv_batch_plan")


def fv_batch_set_schedule(h, schedule: int):
    _check(h, _lib().fv_batch_set_schedule(h, schedule), "fv_batch_set_schedule")


def fv_batch_set_wait_limit(h, cycles: int):
    _check(h, _lib().fv_batch_set_wait_limit(h, cycles), "fv_batch_set_wait_limit")


def fv_batch_set_class_threads(h, p: int, threads: int):
    _check(h, _lib().fv_batch_set_class_threads(h, p, threads), "fv_batch_set_class_threads")


def fv_batch_class_threads(h, p: int) -> int:
    out = ctypes.c_int(0)
    _check(h, _lib().fv_batch_class_threads(h, p, ctypes.byref(out)), "fv_batch_class_threads")
    return int(out.value)


def fv_batch_pairs_launches(h) -> int:
    """Launches of the handle that ran on the FP32 kernel for one patch size."""
    out = ctypes.c_int64(0)
    _check(h, _lib().fv_batch_pairs_launches(h, ctypes.byref(out)), "fv_batch_pairs_launches")
    return int(out.value)


def fv_batch_autotune(h, in_with_halo, scratch_out, patch_offsets, patch_sizes, neighbours,
                      n_patches: int, dx: float, cfl: float):
    """Returns (chosen schedule, [ms of STRIDE, LPT, CLASSES])."""
    chosen = ctypes.c_int()
    ms = (ctypes.c_double * 3)()
    st = _lib().fv_batch_autotune(h, _ptr(in_with_halo), _ptr(scratch_out), _ptr(patch_offsets),
                                  _ptr(patch_sizes), _ptr(neighbours), n_patches, dx, cfl,
                                  ctypes.byref(chosen), ms)
    _check(h, st, "fv_batch_autotune")
    return chosen.value, list(ms)


FV_MLP_NPARAM = 5508
FV_MLP_NNORM = 36


class MlpTrainer:
    """Owns an fv_mlp_trainer (workspace for batches up to max_batch)."""

    def __init__(self, max_batch: int, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream()
        sp = stream if isinstance(stream, int) else stream.cuda_stream
        h = ctypes.c_void_p()
        _check(None, _lib().fv_mlp_trainer_create(ctypes.byref(h), max_batch, sp),
               "fv_mlp_trainer_create")
        self.h = h.value
        self.max_batch = max_batch

    def close(self):
        if self.h:
            _check(None, _lib().fv_mlp_trainer_destroy(self.h), "fv_mlp_trainer_destroy")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def forward(self, params, x, y):
        _check(None, _lib().fv_mlp_forward(self.h, _ptr(params), _ptr(x), x.shape[0], _ptr(y)),
               "fv_mlp_forward")

    def grad(self, params, x, target, grad, loss):
        _check(None, _lib().fv_mlp_grad(self.h, _ptr(params), _ptr(x), _ptr(target), x.shape[0],
                                        _ptr(grad), _ptr(loss)), "fv_mlp_grad")

    def train_step(self, params, x, target, lr: float, step: int, loss):
        _check(None, _lib().fv_mlp_train_step(self.h, _ptr(params), _ptr(x), _ptr(target),
                                              x.shape[0], lr, step, _ptr(loss)),
               "fv_mlp_train_step")

    def train_steps(self, params, x, target, batch: int, first_step: int, n_steps: int,
                    lr: float, losses=None):
        """n_steps Adam steps on consecutive minibatches of (x, target)."""
        _check(None, _lib().fv_mlp_train_steps(self.h, _ptr(params), _ptr(x), _ptr(target),
                                               x.shape[0], batch, first_step, n_steps, lr,
                                               _ptr(losses)), "fv_mlp_train_steps")

    def status(self) -> int:
        return _lib().fv_mlp_trainer_status(self.h)


def _sp(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream if isinstance(stream, int) else stream.cuda_stream


def fv_corr_stride(h) -> int:
    return _lib().fv_corr_stride(h)


def fv_flux_correction(h, q, patch_offsets, patch_sizes, neighbours, n_patches: int, params,
                       norm, corr):
    st = _lib().fv_flux_correction(h, _ptr(q), _ptr(patch_offsets), _ptr(patch_sizes),
                                   _ptr(neighbours), n_patches, _ptr(params), _ptr(norm),
                                   _ptr(corr))
    _check(h, st, "fv_flux_correction")


def fv_time_step_corrected(h, in_with_halo, out, patch_offsets, patch_sizes, neighbours,
                           n_patches: int, dx: float, cfl: float, corr):
    st = _lib().fv_time_step_corrected(h, _ptr(in_with_halo), _ptr(out), _ptr(patch_offsets),
                                       _ptr(patch_sizes), _ptr(neighbours), n_patches, dx, cfl,
                                       _ptr(corr))
    _check(h, st, "fv_time_step_corrected")


def fv_restrict_mesh(hf, qf, off_f, pfx: int, pfy: int, hc, qc, off_c, pcx: int, pcy: int,
                     ratio: int):
    st = _lib().fv_restrict_mesh(hf, _ptr(qf), _ptr(off_f), pfx, pfy, hc, _ptr(qc), _ptr(off_c),
                                 pcx, pcy, ratio)
    _check(hc, st, "fv_restrict_mesh")


def fv_accumulate_face_flux(hf, qf, off_f, pfx: int, pfy: int, hc, pcx: int, pcy: int,
                            ratio: int, weight: float, acc):
    st = _lib().fv_accumulate_face_flux(hf, _ptr(qf), _ptr(off_f), pfx, pfy, hc, pcx, pcy, ratio,
                                        weight, _ptr(acc))
    _check(hc, st, "fv_accumulate_face_flux")


def fv_correction_samples(hc, qc, patch_offsets, patch_sizes, neighbours, n_patches: int, acc,
                          x_raw, t_raw):
    st = _lib().fv_correction_samples(hc, _ptr(qc), _ptr(patch_offsets), _ptr(patch_sizes),
                                      _ptr(neighbours), n_patches, _ptr(acc), _ptr(x_raw),
                                      _ptr(t_raw))
    _check(hc, st, "fv_correction_samples")


def fv_column_moments(x, s, s2, scratch, stream=None):
    st = _lib().fv_column_moments(_ptr(x), x.shape[0], x.shape[1], _ptr(s), _ptr(s2),
                                  _ptr(scratch), _sp(stream))
    _check(None, st, "fv_column_moments")


def fv_normalize_columns(x, mu, sd, stream=None):
    st = _lib().fv_normalize_columns(_ptr(x), x.shape[0], x.shape[1], _ptr(mu), _ptr(sd),
                                     _sp(stream))
    _check(None, st, "fv_normalize_columns")


def fv_read_dt(h) -> float:
    """Synchronise and return the handle's device time step."""
    x = ctypes.c_double()
    _check(h, _lib().fv_read_dt(h, ctypes.byref(x)), "fv_read_dt")
    return x.value


def fv_get_status(h) -> int:
    """Synchronise and return the device status (does not raise)."""
    return _lib().fv_get_status(h)


def fv_selftest_math(x, out, which: int):
    """Device FP64 reciprocal (which=0) / square root (which=1) of x into out."""
    _check(None, _lib().fv_selftest_math(_ptr(x), _ptr(out), x.numel(), which),
           "fv_selftest_math")


def fv_last_error(h) -> str:
    return (_lib().fv_last_error(h) or b"").decode()


class Batch:
    """Owns one handle; methods forward to the C entry points."""

    def __init__(self, d: int, *, precision: int = FV_FP64, gamma: float = 1.4,
                 max_patch_size: int = 0, stream=None):
        o = fv_options_default()
        o.gamma = gamma
        o.precision = precision
        o.max_patch_size = max_patch_size
        self.d, self.s = d, d + 2
        self.precision = precision
        self.h = fv_batch_create(d, d + 2, o, stream)

    def close(self):
        if self.h:
            fv_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, q_in, q_out, off, sizes, dx, dt, lambda_patch=None, n_elems=None,
               corr=None):
        n = off.numel()
        if lambda_patch is None and n_elems is None and corr is None:
            fv_patch_update_batch(self.h, q_in, q_out, off, sizes, n, self.d, self.s, dx, dt)
        else:
            fv_patch_update_batch_ex(self.h, q_in, q_out, off, sizes, n, self.d, self.s, dx, dt,
                                     lambda_patch, n_elems or 0, corr)

    def halo_fill(self, q, off, sizes, nbr):
        fv_halo_fill(self.h, q, off, sizes, nbr, off.numel())

    def time_step(self, q_in, q_out, off, sizes, nbr, dx, cfl, lambda_patch=None):
        fv_time_step(self.h, q_in, q_out, off, sizes, nbr, off.numel(), dx, cfl, lambda_patch)

    def time_step_prim(self, q_in, q_out, prim_in, prim_out, off, sizes, nbr, dx, cfl,
                       lambda_patch=None):
        fv_time_step_prim(self.h, q_in, q_out, prim_in, prim_out, off, sizes, nbr, off.numel(),
                          dx, cfl, lambda_patch)

    def prim_stride(self) -> int:
        return fv_prim_stride(self.h)

    def run_steps(self, q0, q1, off, sizes, nbr, dx, cfl, n_steps, use_graph=False):
        fv_run_steps(self.h, q0, q1, off, sizes, nbr, off.numel(), dx, cfl, n_steps, use_graph)

    def max_eigenvalue(self, q, off, sizes, cfl, dx, per_patch=None, global_max=None,
                       dt_out=None):
        fv_max_eigenvalue_reduce(self.h, q, off, sizes, off.numel(), per_patch, global_max, cfl,
                                 dx, dt_out)

    def totals(self, q, off, sizes, out):
        fv_conserved_totals(self.h, q, off, sizes, off.numel(), out)

    def status(self) -> int:
        return fv_get_status(self.h)

    def dt_ptr(self) -> int:
        return fv_get_dt_ptr(self.h)
