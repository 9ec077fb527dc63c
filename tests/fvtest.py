"""Helpers shared by the GPU tests: build/load libfv, move batches between
numpy and CUDA tensors, and compare against the oracle per unknown."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2302_09005_gb300 import inputs

_BUILT = False


def ensure_built():
    global _BUILT
    if not _BUILT:
        from paper_2302_09005_gb300 import _build
        _build.build()
        oracle.build()
        _BUILT = True


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def to_dev(a, dtype=None):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def interior_mask(off, sizes, d, s, total, halo=1):
    """Boolean mask of the interior elements of every patch."""
    m = np.zeros(total, dtype=bool)
    for o, p in zip(off, sizes):
        ne = int(p) + 2 * halo
        blk = np.zeros((ne,) * d + (s,), dtype=bool)
        blk[(slice(halo, halo + int(p)),) * d] = True
        m[int(o):int(o) + blk.size] = blk.reshape(-1)
    return m


def per_unknown_rel_err(got, ref, mask, s):
    """max |got - ref| / max |ref| for each unknown over the masked cells."""
    g = got[mask].reshape(-1, s).astype(np.float64)
    r = ref[mask].reshape(-1, s).astype(np.float64)
    return np.max(np.abs(g - r), axis=0) / np.max(np.abs(r), axis=0)


def random_batch(n, p, d, seed, dtype=np.float64):
    return inputs.random_batch(n, p, d, seed=seed, dtype=dtype)
