"""x-slab decomposition of a box: the host logic around ns_slab_* (section "Numerical
methods": the paper's solver splits its domain over MPI ranks).

A box of NX columns is cut at column boundaries into slabs; slab k covers columns
[a_k, b_k) and is stored as a padded box of b_k - a_k + 2 columns whose first and last
columns (the ghosts) hold the neighbouring slabs' boundary columns, periodic in x as a
whole.  Within one process a SlabGroup (api.py) steps all slabs and exchanges their
ghosts with device copies.  With one slab per process, exchange_ghosts below moves the
ghost columns between ranks with torch.distributed point-to-point calls (NCCL for CUDA
tensors, gloo for CPU ones), halo_exchange_fn turns it into the library's host exchange
hook, and allreduce_sum adds the per-slab reductions (the objective's plane sums, the
adjoint energy, dot products) in FP64.  No arithmetic of the method happens here.
"""
from __future__ import annotations

import numpy as np


def cuts_even(nx: int, n: int):
    """n slabs of nearly equal width: [(a_0, b_0), ...]."""
    edges = [nx * k // n for k in range(n + 1)]
    return [(edges[k], edges[k + 1]) for k in range(n)]


def padded_columns(nx: int, a: int, b: int):
    """Box columns of the padded slab [a, b): the left ghost, the interior, the right ghost."""
    return [(a - 1) % nx] + list(range(a, b)) + [b % nx]


def split(w, cuts):
    """Padded slabs of a field whose last axis is x (numpy array or torch tensor)."""
    nx = w.shape[-1]
    out = []
    for a, b in cuts:
        cols = padded_columns(nx, a, b)
        out.append(w[..., cols])
    return out


def join(slabs):
    """The box from the interiors of its padded slabs (numpy arrays or torch tensors)."""
    parts = [s[..., 1:-1] for s in slabs]
    if isinstance(parts[0], np.ndarray):
        return np.concatenate(parts, axis=-1)
    import torch
    return torch.cat(parts, dim=-1)


def exchange_ghosts(t, rank: int, world: int, group=None):
    """Fill the ghost columns (first and last along the last axis) of this rank's padded
    slab t from its neighbours' boundary columns: the left neighbour's last interior
    column and the right neighbour's first.  Every rank calls this at the same point.
    The four messages are posted in one order on every rank (send right, send left,
    receive from left, receive from right), with tags, so that they pair up under gloo
    (which matches tags) and NCCL (which matches posting order) even when the left and
    right neighbours are the same rank."""
    import torch
    import torch.distributed as dist
    if world == 1:
        t[..., 0] = t[..., -2]
        t[..., -1] = t[..., 1]
        return
    left, right = (rank - 1) % world, (rank + 1) % world
    to_right = t[..., -2].contiguous()
    to_left = t[..., 1].contiguous()
    from_left = torch.empty_like(to_right)
    from_right = torch.empty_like(to_left)
    ops = [dist.P2POp(dist.isend, to_right, right, group, tag=0),
           dist.P2POp(dist.isend, to_left, left, group, tag=1),
           dist.P2POp(dist.irecv, from_left, left, group, tag=0),
           dist.P2POp(dist.irecv, from_right, right, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    t[..., 0] = from_left
    t[..., -1] = from_right


def allreduce_sum(values, group=None):
    """Sum of per-slab partial reductions over the ranks, in FP64 (a tensor, in place)."""
    import torch
    import torch.distributed as dist
    if values.dtype != torch.float64:
        raise ValueError("per-slab reductions are summed in FP64")
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(values, op=dist.ReduceOp.SUM, group=group)
    return values


class _DeviceView:
    """A raw device field seen as a torch tensor (CUDA array interface, no copy)."""

    def __init__(self, ptr: int, shape, elem_bytes: int):
        self.__cuda_array_interface__ = {
            "shape": tuple(shape), "typestr": "<f8" if elem_bytes == 8 else "<f4",
            "data": (int(ptr), False), "version": 3, "strides": None, "stream": None}


def halo_exchange_fn(solver, rank: int, world: int, group=None):
    """The host exchange hook (ns_slab_set_exchange, via api.SlabGroup(exchange=...)) of a
    one-slab group whose neighbours are other ranks: the field the library passes is
    viewed as a tensor of the slab's shape and its ghost columns are exchanged on the
    current stream, which must be the slab context's."""
    import torch

    def fn(ptr, elem_bytes, ncomp):
        shape = (solver.batch, ncomp) + tuple(solver.shape[2:])
        t = torch.as_tensor(_DeviceView(ptr, shape, elem_bytes), device="cuda")
        exchange_ghosts(t, rank, world, group)
        return 0

    return fn
