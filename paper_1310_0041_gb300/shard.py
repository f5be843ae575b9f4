"""Splitting the method across GPUs: one process per GPU, each with its own
libgd stack, torch.distributed for the few exchanges.

* **Screened Poisson** (paper Sec. 3.1, Eq. screened_poisson) has no z term,
  so every slice is an independent problem (the paper solves it slice by
  slice, Sec. 4.1).  Ranks take disjoint sets of slices -- contiguous
  z-ranges of a stack (:func:`slabs`), or size-balanced bins of a batch of
  slices of different sizes (:func:`balanced_bins`) -- solve them with no
  exchange on the data path, and combine only their residual norms and cycle
  counts (:func:`combine_reports`, two all-reduces).
* **Anisotropic diffusion** couples the slices.  Its split is by z-slabs with
  even boundaries (so the z-pairs of the first coarsenings stay on one rank),
  a one-plane halo exchanged after every red-black half-sweep, all-reduces of
  the residual norm and of the iterate's sum (the mean fix), and the coarse
  levels gathered on one rank; the protocol is exercised by a CPU-rank
  emulation in the tests (each box here has one GPU).

Only sequencing and host logic live here; the solves are libgd calls.
"""
from __future__ import annotations

import math


def slabs(n: int, nranks: int, align: int = 1) -> list:
    """Contiguous near-equal ranges [(z0, z1), ...] of range(n), one per rank,
    with every inner boundary a multiple of `align` (empty ranges when n is
    too small)."""
    if nranks < 1 or align < 1:
        raise ValueError("nranks and align must be >= 1")
    units = -(-n // align)
    out, u0 = [], 0
    for r in range(nranks):
        u1 = u0 + units // nranks + (1 if r < units % nranks else 0)
        out.append((min(n, u0 * align), min(n, u1 * align)))
        u0 = u1
    return out


def balanced_bins(costs, nranks: int) -> list:
    """Greedy longest-processing-time bins: slice indices sorted by cost
    (largest first, ties by index), each given to the rank with the least
    cost so far (ties to the lowest rank).  Returns one sorted index list
    per rank."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * nranks
    bins = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        bins[r].append(i)
        load[r] += costs[i]
    return [sorted(b) for b in bins]


def combine_reports(reports, group=None, device=None) -> dict:
    """The whole problem's report from each rank's solve reports.

    Every report carries ``rel_residual`` = ||r|| / ||b|| of the rank's part,
    ``rhs_norm`` = ||b|| of that part and ``cycles``; the parts are disjoint
    sets of unknowns, so ||r||^2 and ||b||^2 add up over ranks (one SUM
    all-reduce) and the cycle count and the largest per-part residual are
    maxima (one MAX all-reduce)."""
    import torch
    import torch.distributed as dist
    r2 = sum((rp["rel_residual"] * rp["rhs_norm"]) ** 2 for rp in reports)
    b2 = sum(rp["rhs_norm"] ** 2 for rp in reports)
    cyc = max((rp["cycles"] for rp in reports), default=0)
    worst = max((rp["rel_residual"] for rp in reports), default=0.0)
    sums = torch.tensor([r2, b2], dtype=torch.float64, device=device)
    maxs = torch.tensor([float(cyc), worst], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(maxs, op=dist.ReduceOp.MAX, group=group)
    r2, b2 = float(sums[0]), float(sums[1])
    return {"rel_residual": math.sqrt(r2 / b2) if b2 > 0 else math.sqrt(r2),
            "rhs_norm": math.sqrt(b2), "cycles": int(maxs[0]), "rel_residual_max_part": float(maxs[1])}


def screened_poisson_slab(I0, I1, I2, alpha: float, ctl=None, group=None, device=None) -> dict:
    """This rank's contiguous range of slices of a stack ((nz_r, ny, nx) CUDA
    tensors) solved with libgd (Sec. 3.1 screened Poisson, per slice); returns
    the report of the whole stack (all ranks call it together)."""
    from . import gd_destroy, gd_screened_poisson_slices, gd_stack_create
    nz, ny, nx = I0.shape
    reports = []
    if nz > 0:
        s = gd_stack_create(nx, ny, nz)
        try:
            reports.append(gd_screened_poisson_slices(s, I0, I1, I2, alpha, ctl))
        finally:
            gd_destroy(s)
    return combine_reports(reports, group, device)


def batch_screened_poisson_bin(nx, ny, alphas, I0, I1, I2, ctl=None, group=None, device=None) -> dict:
    """This rank's bin of independent slices of different sizes (packed as in
    gd_batch_create) solved with one libgd batch; returns the combined report
    (the largest per-slice residual over all ranks is ``rel_residual_max_part``)."""
    from . import gd_batch_create, gd_batch_destroy, gd_batch_screened_poisson
    reports = []
    if len(nx):
        b = gd_batch_create(list(nx), list(ny), list(alphas))
        try:
            reports.append(gd_batch_screened_poisson(b, I0, I1, I2, ctl))
        finally:
            gd_batch_destroy(b)
    out = combine_reports(reports, group, device)
    out["rel_residual"] = out["rel_residual_max_part"]  # a batch's tolerance holds per slice
    return out
