"""Training and evaluation of the learned conservative face-flux correction
on regular periodic 2D patch meshes.

Orchestration only: every arithmetic step runs in libfv's kernels (fine and
coarse Rusanov steps, restriction, face-flux accumulation, target
computation, normalisation statistics, BF16 tensor-core training and
inference).  PyTorch provides the device buffers and the one shuffle of the
training set.

Data (per coarse step of length dt, dt from the CFL condition on the
restricted state): the fine mesh (ratio r times finer, FP64) takes r
substeps of dt / r; the time-and-face averages of its Rusanov fluxes through
the coarse faces, minus the coarse Rusanov flux of the restricted state,
are the ideal corrections C*; the network learns C* from the coarse 4-cell
stencils.
"""
from __future__ import annotations

import numpy as np

from . import fv, inputs


class Mesh2D:
    """A regular periodic 2D patch mesh on the device (patch a + px b)."""

    def __init__(self, N: int, p: int, precision: int, stream, U=None, align_bytes: int = 32):
        import torch
        assert N % p == 0
        self.N, self.p, self.precision = N, p, precision
        self.grid = (N // p, N // p)
        self.n = self.grid[0] * self.grid[1]
        dtype = np.float64 if precision == fv.FV_FP64 else np.float32
        if U is None:
            sizes = np.full(self.n, p, dtype=np.int32)
            off, total = inputs.layout(sizes, 2, 4, 1, np.dtype(dtype).itemsize, align_bytes)
            q = np.zeros(total, dtype=dtype)
        else:
            q, off, sizes, grid = inputs.domain_to_patches(U, p, dtype=dtype,
                                                           align_bytes=align_bytes)
            assert tuple(grid) == self.grid
        nbr = inputs.grid_neighbours(self.grid)
        self.off_np = off
        self.x = torch.from_numpy(q).cuda()
        self.y = self.x.clone()
        self.off = torch.from_numpy(off).cuda()
        self.sizes = torch.from_numpy(sizes).cuda()
        self.nbr = torch.from_numpy(nbr).cuda()
        self.stream = stream
        self.b = fv.Batch(2, precision=precision, max_patch_size=p, stream=stream)
        self.dx = 1.0 / N
        self._side = None  # halo fills beside the correction kernel (step_learned)

    def halo_fill(self):
        self.b.halo_fill(self.x, self.off, self.sizes, self.nbr)

    def cfl_dt(self, cfl: float) -> float:
        self.halo_fill()
        self.b.max_eigenvalue(self.x, self.off, self.sizes, cfl, self.dx)
        return fv.fv_read_dt(self.b.h)

    def step(self, dt: float, corr=None):
        """Halo fill + one update with an explicit dt (and optional C)."""
        self.halo_fill()
        self.b.update(self.x, self.y, self.off, self.sizes, self.dx, dt, corr=corr)
        self.x, self.y = self.y, self.x

    def step_learned(self, dt: float, params, norm, corr):
        """One learned step: C = net(stencils) on the mesh's stream while the
        halo fill runs on a second stream, then the update with F + C.  The
        two overlap safely: the correction kernel reads interior cells only
        (a patch's and its neighbours'), the halo fill writes halo cells only;
        the update waits for both."""
        import torch
        if self._side is None:
            side = torch.cuda.Stream()
            self._side = (side, fv.Batch(2, precision=self.precision, max_patch_size=self.p,
                                         stream=side),
                          torch.cuda.Event(), torch.cuda.Event())
        side, hb, ready, filled = self._side
        ready.record(self.stream)  # the previous update has written x
        side.wait_event(ready)
        hb.halo_fill(self.x, self.off, self.sizes, self.nbr)
        filled.record(side)
        fv.fv_flux_correction(self.b.h, self.x, self.off, self.sizes, self.nbr, self.n, params,
                              norm, corr)
        self.stream.wait_event(filled)
        self.b.update(self.x, self.y, self.off, self.sizes, self.dx, dt, corr=corr)
        self.x, self.y = self.y, self.x

    def status(self) -> int:
        """The first non-OK status of the mesh's handles (the side handle's
        halo fills included)."""
        st = self.b.status()
        if st == fv.FV_OK and self._side is not None:
            st = self._side[1].status()
        return st

    def domain(self) -> np.ndarray:
        return inputs.patches_to_domain(self.x.double().cpu().numpy(), self.off_np, self.p,
                                        self.grid, 4)

    def close(self):
        if self._side is not None:
            self._side[0].synchronize()
            self._side[1].close()
            self._side = None
        self.b.close()


def generate(U_fine, Nc: int, pc: int, pf: int, r: int, n_steps: int, cfl: float, stream):
    """Fine run and training samples.  Returns (X_raw, T_raw, dts, coarse
    reference domains at steps 0..n_steps)."""
    import torch
    Nf = Nc * r
    fine = Mesh2D(Nf, pf, fv.FV_FP64, stream, U=U_fine)
    coarse = Mesh2D(Nc, pc, fv.FV_FP64, stream)
    stride = fv.fv_corr_stride(coarse.b.h)
    nsamp = coarse.n * 2 * (pc + 1) * pc
    acc = torch.zeros(coarse.n * stride, dtype=torch.float64, device="cuda")
    X = torch.empty((n_steps, nsamp, 16), dtype=torch.float32, device="cuda")
    T = torch.empty((n_steps, nsamp, 4), dtype=torch.float32, device="cuda")
    dts, refs = [], []
    with torch.cuda.stream(stream):
        for step in range(n_steps + 1):
            fv.fv_restrict_mesh(fine.b.h, fine.x, fine.off, *fine.grid, coarse.b.h, coarse.x,
                                coarse.off, *coarse.grid, r)
            refs.append(coarse.domain())
            if step == n_steps:
                break
            dt = coarse.cfl_dt(cfl)
            dts.append(dt)
            acc.zero_()
            for _ in range(r):
                fine.halo_fill()
                fv.fv_accumulate_face_flux(fine.b.h, fine.x, fine.off, *fine.grid, coarse.b.h,
                                           *coarse.grid, r, 1.0 / r, acc)
                fine.b.update(fine.x, fine.y, fine.off, fine.sizes, fine.dx, dt / r)
                fine.x, fine.y = fine.y, fine.x
            fv.fv_correction_samples(coarse.b.h, coarse.x, coarse.off, coarse.sizes, coarse.nbr,
                                     coarse.n, acc, X[step], T[step])
    stream.synchronize()
    st = coarse.b.status() or fine.b.status()
    fine.close()
    coarse.close()
    if st != fv.FV_OK:
        raise RuntimeError(f"data generation status {st}")
    return X.reshape(-1, 16), T.reshape(-1, 4), dts, refs


def normalisation(X, T, stream):
    """mu_x, sd_x (16) and sd_y (4) from FP64 column moments (kernels)."""
    import torch
    norm = torch.empty(fv.FV_MLP_NNORM, dtype=torch.float32, device="cuda")
    rows = X.shape[0]
    scratch = torch.empty(2 * 16 * ((rows + 65535) // 65536), dtype=torch.float64,
                          device="cuda")
    s = torch.empty(16, dtype=torch.float64, device="cuda")
    s2 = torch.empty(16, dtype=torch.float64, device="cuda")
    fv.fv_column_moments(X, s, s2, scratch, stream)
    ts = torch.empty(4, dtype=torch.float64, device="cuda")
    ts2 = torch.empty(4, dtype=torch.float64, device="cuda")
    fv.fv_column_moments(T, ts, ts2, scratch, stream)
    stream.synchronize()
    mu = s.cpu().numpy() / rows
    var = np.maximum(s2.cpu().numpy() / rows - mu * mu, 0.0)
    sd = np.sqrt(var) + 1e-6
    sdy = np.sqrt(ts2.cpu().numpy() / rows) + 1e-12  # targets: root mean square
    vals = np.concatenate([mu, sd, sdy]).astype(np.float32)
    norm.copy_(torch.from_numpy(vals))
    return norm


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters (FP32 vector of FV_MLP_NPARAM): weights
    ~ N(0, 1/fan_in), biases 0, last layer scaled by 0.1."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in ((64, 16), (64,), (64, 64), (64,), (4, 64), (4,)):
        if len(shape) == 1:
            parts.append(np.zeros(shape))
        else:
            w = rng.standard_normal(shape) / np.sqrt(shape[1])
            parts.append(w * (0.1 if shape[0] == 4 else 1.0))
    return np.concatenate([a.reshape(-1) for a in parts]).astype(np.float32)


def train(X, T, norm, *, steps: int, batch: int, lr: float, seed: int, stream):
    """Normalise the samples in place, shuffle once, and run `steps` Adam
    steps on contiguous minibatches (the BF16 tensor-core trainer; the last
    tenth of the steps at lr / 10).  Returns (params, losses); train.last_ms
    holds the device time of the Adam steps alone (CUDA events on `stream`)."""
    import torch
    fv.fv_normalize_columns(X, norm[0:16], norm[16:32], stream)
    fv.fv_normalize_columns(T, None, norm[32:36], stream)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    perm = torch.randperm(X.shape[0], device="cuda", generator=g)
    Xs, Ts = X[perm].contiguous(), T[perm].contiguous()
    params = torch.from_numpy(init_params(seed)).cuda()
    trainer = fv.MlpTrainer(batch, stream)
    step_loss = torch.zeros(steps, dtype=torch.float32, device="cuda")
    n1 = int(0.9 * steps)  # steps 1..n1 at lr, the rest at lr / 10
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        if n1 > 0:
            trainer.train_steps(params, Xs, Ts, batch, 1, n1, lr, step_loss[:n1])
        if steps > n1:
            trainer.train_steps(params, Xs, Ts, batch, n1 + 1, steps - n1, lr * 0.1,
                                step_loss[n1:])
        e1.record(stream)
    stream.synchronize()
    train.last_ms = e0.elapsed_time(e1)
    st = trainer.status()
    trainer.close()
    if st != fv.FV_OK:
        raise RuntimeError(f"training status {st}")
    sl = step_loss.cpu().numpy()
    losses = [(it, float(sl[it - 1])) for it in range(1, steps + 1)
              if it == 1 or it % max(1, steps // 20) == 0 or it == steps]
    return params, losses


def evaluate(U_coarse0, refs, dts, pc: int, params, norm, stream, precision=fv.FV_FP64):
    """Plain and learned coarse runs from the restricted initial state with
    the reference time steps; relative L1 distance to the restricted fine
    run after every step, per unknown.  Returns (l1_plain, l1_learned, ms)."""
    import torch
    Nc = U_coarse0.shape[0]
    out = {}
    times = {}
    for learned in (False, True):
        m = Mesh2D(Nc, pc, precision, stream, U=U_coarse0)
        corr = torch.zeros(m.n * fv.fv_corr_stride(m.b.h), dtype=torch.float32, device="cuda")
        errs = []
        ms_total = 0.0
        for n, dt in enumerate(dts):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                if learned:
                    m.step_learned(dt, params, norm, corr)
                else:
                    m.step(dt)
                e1.record(stream)
            stream.synchronize()
            ms_total += e0.elapsed_time(e1)
            D = m.domain()
            ref = refs[n + 1]
            errs.append((np.abs(D - ref).sum(axis=(0, 1)) / np.abs(ref).sum(axis=(0, 1))).tolist())
        if m.status() != fv.FV_OK:
            raise RuntimeError("evaluation run failed")
        m.close()
        out[learned] = errs
        times[learned] = ms_total / len(dts)
    return out[False], out[True], times
