"""The sharded form of the method on two host ranks (gloo): the patches of a
periodic 2D mesh are split by patch columns; every step each rank exchanges
the patches on its partition boundary, fills its halos, takes the global
maximum wave speed with an all-reduce (MAX), and updates its own patches.
The gathered result equals the single-domain run bitwise -- the exchange
and the reduction the multi-GPU form of the path needs (one halo exchange
and one max all-reduce per step) reproduce it exactly.

Runs the FP64 oracle on CPU ranks; no GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2302_09005_gb300 import inputs

PX, PY, P, STEPS, CFL = 4, 3, 4, 5, 0.4


def _initial():
    rng = np.random.default_rng(7)
    N = (PX * P, PY * P)
    U = inputs.random_cells(rng, N[0] * N[1], 2).reshape(N[1], N[0], 4)
    return inputs.domain_to_patches(U, P)


def _single_domain():
    q, off, sz, grid = _initial()
    nbr = inputs.grid_neighbours(grid)
    dx = 1.0 / (PX * P)
    for _ in range(STEPS):
        q, _ = oracle.step(q, off, sz, nbr, 2, dx, CFL)
    return inputs.patches_to_domain(q, off, P, grid, 4)


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q_all, off_all, sz_all, grid = _initial()
    nbr_all = inputs.grid_neighbours(grid)
    pe = int(off_all[1] - off_all[0])  # elements per patch (uniform layout)
    cols = [c for c in range(PX) if c * world // PX == rank]
    owned = [a + PX * b for b in range(PY) for a in cols]
    edge_cols = {cols[0], cols[-1]}
    send = [i for i in owned if i % PX in edge_cols]  # patches others may need
    # local buffer: owned patches, then ghost slots for every patch index
    local_index = {g: k for k, g in enumerate(owned)}
    n_local = len(owned)
    q = np.zeros((n_local + PX * PY) * pe)
    for g, k in local_index.items():
        q[k * pe:(k + 1) * pe] = q_all[g * pe:(g + 1) * pe]
    off = np.arange(n_local + PX * PY, dtype=np.int64) * pe
    sz = np.full(n_local + PX * PY, P, dtype=np.int32)
    nbr = np.full((n_local + PX * PY, 4), -1, dtype=np.int32)
    for g, k in local_index.items():
        for f in range(4):
            nb = int(nbr_all[g, f])
            nbr[k, f] = local_index.get(nb, n_local + nb)  # ghost slot of a remote patch
    ghost_needed = sorted({int(nbr_all[g, f]) for g in owned for f in range(4)} - set(owned))
    dx = 1.0 / (PX * P)
    counts = [None] * world
    dist.all_gather_object(counts, len(send))
    for _ in range(STEPS):
        # exchange the partition-boundary patches (index + interior data)
        mine = torch.tensor(np.concatenate([[g] + list(q[local_index[g] * pe:
                                                        (local_index[g] + 1) * pe])
                                            for g in send]) if send else np.zeros(0))
        width = pe + 1
        bufs = [torch.zeros(c * width, dtype=torch.float64) for c in counts]
        dist.all_gather(bufs, mine.to(torch.float64))
        for r, buf in enumerate(bufs):
            if r == rank:
                continue
            arr = buf.numpy().reshape(-1, width)
            for row in arr:
                g = int(row[0])
                if g in ghost_needed:
                    s = n_local + g
                    q[s * pe:(s + 1) * pe] = row[1:]
        own_off, own_sz, own_nbr = off[:n_local], sz[:n_local], nbr[:n_local]
        # halo fill of the owned patches (sources: owned or ghost slots)
        qh = q.copy()
        full_nbr = np.full((len(off), 4), -1, dtype=np.int32)
        full_nbr[:n_local] = own_nbr
        full_nbr[n_local:] = np.arange(n_local, len(off))[:, None]  # ghosts: self, unused
        oracle.halo_fill(qh, off, sz, full_nbr, 2, 4)
        lam_local, lam = oracle.max_eigenvalue(qh, own_off, own_sz, 2)
        t = torch.tensor([lam], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dt = oracle.cfl_dt(float(t.item()), CFL, dx, 2)
        q = oracle.patch_update(qh, own_off, own_sz, 2, dx, dt, q_out=qh.copy())
    # gather owned patches at rank 0
    mine = torch.tensor(np.concatenate([[g] + list(q[local_index[g] * pe:
                                                    (local_index[g] + 1) * pe])
                                        for g in owned]))
    sizes = [None] * world
    dist.all_gather_object(sizes, mine.numel())
    bufs = [torch.zeros(s, dtype=torch.float64) for s in sizes]
    dist.all_gather(bufs, mine)
    if rank == 0:
        out = np.zeros_like(q_all)
        for buf in bufs:
            for row in buf.numpy().reshape(-1, pe + 1):
                g = int(row[0])
                out[g * pe:(g + 1) * pe] = row[1:]
        np.save(out_path, inputs.patches_to_domain(out, off_all, P, grid, 4))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2])
def test_two_rank_sharded_steps_equal_single_domain(tmp_path, world):
    oracle.build()
    out = str(tmp_path / "sharded.npy")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(out)
    ref = _single_domain()
    assert np.array_equal(got, ref)
