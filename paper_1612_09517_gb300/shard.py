"""Sharding of the samples over ranks (one process per GPU) and the one
collective of the path.

The stochastic estimate (Eq. 18) averages independent samples, so ranks take
disjoint contiguous sample ranges (``sample_offset`` of ``rp_yields``; the
counter-based sampler gives sample s the same directions on every rank) and
never exchange data while they propagate.  The per-field results are then
combined with one FP64 all-reduce of five sums per field:

    sum phi_S, sum phi_S^2, sum phi_T, sum phi_T^2, sum survival,

from which the global mean and standard error (Eq. 23, sample variance with
M - 1) follow exactly.  Each rank's sums come from its own ``rp_yields``
output (mean and standard error over its M_r samples) through
``rp_field_sums``, and the combined block through ``rp_combine_sums``, both in
the library; no per-sample data crosses ranks.

Argument marshalling around ``torch.distributed`` only; the arithmetic runs in
the library.
"""
from __future__ import annotations

import numpy as np


def sample_range(M: int, world: int, rank: int):
    """(offset, count) of rank's contiguous share of samples 0 .. M-1; the
    first M % world ranks take one sample more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    if M < 0:
        raise ValueError("M must be >= 0")
    base, extra = divmod(int(M), int(world))
    count = base + (1 if rank < extra else 0)
    offset = rank * base + min(rank, extra)
    return offset, count


def field_sums(out, M: int):
    """Per-field sums (n_fields, 5) from an rp_yields output block (n_fields, 5)
    = (Phi_S, Phi_T, SE_S, SE_T, mean survival) over M >= 2 samples
    (rp_field_sums)."""
    from . import rp
    if M < 2:
        raise ValueError("each rank needs M >= 2 samples (the standard error needs it)")
    return rp.rp_field_sums(out, M)


def combine(sums, M: int):
    """The rp_yields output block over all M samples from summed field_sums
    (rp_combine_sums)."""
    from . import rp
    if M < 2:
        raise ValueError("M must be >= 2")
    return rp.rp_combine_sums(sums, M)


def allreduce_yields(out, M_local: int, group=None):
    """Combine per-rank rp_yields outputs over the process group: one FP64
    all-reduce of (5 n_fields + 1) numbers.  Returns (out_global, M_global).
    Works with the gloo (CPU tensor) and nccl (CUDA tensor) backends."""
    import torch
    import torch.distributed as dist

    s = field_sums(out, M_local)
    flat = np.concatenate([s.ravel(), [float(M_local)]])
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(flat, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    r = t.cpu().numpy()
    M = int(round(r[-1]))
    return combine(r[:-1], M), M


def max_over_ranks(values, group=None):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time)."""
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor(np.asarray(values, dtype=np.float64), device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.cpu().numpy()
