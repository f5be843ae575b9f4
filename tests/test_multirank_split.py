"""The split of the method across ranks, on CPU ranks (gloo, world size 2).

* Screened Poisson by slices (paper Sec. 3.1: the step has no z term): each
  rank solves its own slices -- a contiguous z-range of a stack, or a
  size-balanced bin of slices of different sizes -- and the pieces, put back
  together, equal the single-domain solution; the residual combined by
  ``shard.combine_reports`` equals the one computed on the whole stack.  The
  per-rank solver here is the FP64 oracle (no GPU in this test); on GPUs it
  is libgd.
* Anisotropic diffusion by z-slabs: an emulation of the protocol on CPU ranks
  -- one-plane halos exchanged after every red-black half-sweep, residual
  norms and the iterate's sum all-reduced, the z-coarsened residual gathered
  on rank 0, solved there and scattered back -- against the single-domain
  oracle: one distributed sweep equals the oracle's sweep, and the
  distributed two-level iteration converges to the exact solution.
"""
import os
import queue
import socket
import time

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1310_0041_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(target, world=2, *args):
    """Runs target(rank, world, port, queue, *args) on `world` spawned ranks
    and returns {rank: the value it put}.  A rank that exits without putting
    its value fails the test at once (the other ranks are terminated)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + args) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    deadline = time.monotonic() + 300
    try:
        while len(out) < world:
            try:
                r, v = q.get(timeout=1.0)
                out[r] = v
                continue
            except queue.Empty:
                pass
            dead = [(i, p.exitcode) for i, p in enumerate(procs) if p.exitcode not in (None, 0)]
            if dead:
                pytest.fail("rank(s) %s exited without a result (exit codes %s)" %
                            ([i for i, _ in dead], [c for _, c in dead]))
            if time.monotonic() > deadline:
                pytest.fail("ranks did not report within 300 s")
    finally:
        if len(out) < world:
            for p in procs:
                if p.is_alive():
                    p.terminate()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


# ---------------------------------------------------------------------------
# host logic
# ---------------------------------------------------------------------------
def test_slabs_and_bins():
    assert shard.slabs(16, 2, align=2) == [(0, 8), (8, 16)]
    assert shard.slabs(10, 3, align=2) == [(0, 4), (4, 8), (8, 10)]
    assert shard.slabs(3, 4) == [(0, 1), (1, 2), (2, 3), (3, 3)]
    for n, k, a in [(128, 8, 2), (37, 5, 1), (9, 2, 4)]:
        sl = shard.slabs(n, k, a)
        assert sl[0][0] == 0 and sl[-1][1] == n
        assert all(s1 == t0 for (_, s1), (t0, _) in zip(sl, sl[1:]))
        assert all(z0 % a == 0 for z0, _ in sl)
    costs = [256 * 256, 4096 * 4096, 300 * 300, 2048 * 2048, 1000 * 1000, 4000 * 4000, 512 * 512]
    bins = shard.balanced_bins(costs, 2)
    assert sorted(i for b in bins for i in b) == list(range(len(costs)))
    loads = [sum(costs[i] for i in b) for b in bins]
    # LPT: no rank carries more than the optimum plus the largest single slice
    assert max(loads) <= sum(costs) / 2 + max(costs)
    assert shard.balanced_bins(costs, 2) == bins  # deterministic


# ---------------------------------------------------------------------------
# screened Poisson by slices
# ---------------------------------------------------------------------------
def _sp_stack_worker(rank, world, port, q):
    dist = _init(rank, world, port)
    from oracle import closed_form as cf
    rng = np.random.default_rng(3)
    nz, ny, nx = 9, 20, 28
    I0 = rng.uniform(0, 255, (nz, ny, nx))
    I1 = rng.uniform(0, 255, (nz, ny, nx))
    z0, z1 = shard.slabs(nz, world)[rank]
    x = cf.sp(I0[z0:z1], I1[z0:z1], 0.01)  # this rank's slices, solved on their own
    # the rank's report: residual of the stored float32 result against its part of b
    from oracle import rhs_sp, apply
    b = rhs_sp(I0[z0:z1], I1[z0:z1], 0.01)
    r = b - apply(x.astype(np.float32).astype(np.float64), 0.01, 1.0, 1.0, 0.0)
    rep = {"rel_residual": float(np.linalg.norm(r) / np.linalg.norm(b)), "rhs_norm": float(np.linalg.norm(b)),
           "cycles": 3 + rank}
    comb = shard.combine_reports([rep])
    parts = [None] * world
    dist.all_gather_object(parts, (z0, z1, x))
    q.put((rank, (comb, parts)))
    dist.destroy_process_group()


def test_sp_stack_split_by_slices_equals_the_single_domain_solution():
    from oracle import closed_form as cf
    from oracle import rhs_sp, apply
    out = _run(_sp_stack_worker)
    rng = np.random.default_rng(3)
    nz, ny, nx = 9, 20, 28
    I0 = rng.uniform(0, 255, (nz, ny, nx))
    I1 = rng.uniform(0, 255, (nz, ny, nx))
    want = cf.sp(I0, I1, 0.01)
    for rank in range(2):
        comb, parts = out[rank]
        got = np.empty_like(want)
        for z0, z1, x in parts:
            got[z0:z1] = x
        assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()
        # the combined residual is the whole stack's
        b = rhs_sp(I0, I1, 0.01)
        r = b - apply(got.astype(np.float32).astype(np.float64), 0.01, 1.0, 1.0, 0.0)
        assert abs(comb["rel_residual"] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-12
        assert comb["cycles"] == 4


def _sp_batch_worker(rank, world, port, q, sides, alphas):
    dist = _init(rank, world, port)
    from oracle import closed_form as cf
    rng = np.random.default_rng(5)
    I0s = [rng.uniform(0, 255, (n, n + 3)) for n in sides]
    I1s = [rng.uniform(0, 255, (n, n + 3)) for n in sides]
    bins = shard.balanced_bins([n * (n + 3) for n in sides], world)
    mine = {i: cf.sp(I0s[i][None], I1s[i][None], alphas[i])[0] for i in bins[rank]}
    parts = [None] * world
    dist.all_gather_object(parts, mine)
    q.put((rank, (bins, parts)))
    dist.destroy_process_group()


def test_sp_batch_split_by_balanced_bins_equals_the_single_domain_solution():
    from oracle import closed_form as cf
    sides = [5, 17, 9, 23, 12, 6, 30]
    alphas = [0.001, 0.05, 0.02, 0.1, 0.003, 0.07, 0.01]
    out = _run(_sp_batch_worker, 2, sides, alphas)
    rng = np.random.default_rng(5)
    I0s = [rng.uniform(0, 255, (n, n + 3)) for n in sides]
    I1s = [rng.uniform(0, 255, (n, n + 3)) for n in sides]
    bins, parts = out[0]
    assert sorted(bins[0] + bins[1]) == list(range(len(sides)))
    got = {}
    for p in parts:
        got.update(p)
    for i, n in enumerate(sides):
        want = cf.sp(I0s[i][None], I1s[i][None], alphas[i])[0]
        assert np.abs(got[i] - want).max() <= 1e-9 * np.abs(want).max()


# ---------------------------------------------------------------------------
# anisotropic diffusion by z-slabs (protocol emulation)
# ---------------------------------------------------------------------------
def _neighbour_terms(x, k, nz, w):
    """Sum of weighted neighbour values and the diagonal of the 6-point
    operator (difference form, Neumann: missing neighbours drop out) on the
    interior planes of a slab with one halo plane on each side; k = global
    plane indices of the interior planes."""
    alpha, bx, by, bz = w
    xi = x[1:-1]
    s = np.zeros_like(xi)
    d = np.full_like(xi, alpha)
    s[:, :, 1:] += bx * xi[:, :, :-1]
    d[:, :, 1:] += bx
    s[:, :, :-1] += bx * xi[:, :, 1:]
    d[:, :, :-1] += bx
    s[:, 1:, :] += by * xi[:, :-1, :]
    d[:, 1:, :] += by
    s[:, :-1, :] += by * xi[:, 1:, :]
    d[:, :-1, :] += by
    lo = (k > 0)[:, None, None].astype(np.float64)
    hi = (k < nz - 1)[:, None, None].astype(np.float64)
    s += bz * (lo * x[:-2] + hi * x[2:])
    d += bz * (lo + hi)
    return s, d


def _exchange(dist, x, rank, world):
    """One-plane halos: send the first and last interior planes to the
    neighbouring ranks, receive theirs into the halo planes."""
    import torch
    reqs = []
    if rank > 0:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(x[1])), rank - 1))
        lo = torch.empty(x.shape[1:], dtype=torch.float64)
        reqs.append(dist.irecv(lo, rank - 1))
    if rank < world - 1:
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(x[-2])), rank + 1))
        hi = torch.empty(x.shape[1:], dtype=torch.float64)
        reqs.append(dist.irecv(hi, rank + 1))
    for r in reqs:
        r.wait()
    if rank > 0:
        x[0] = lo.numpy()
    if rank < world - 1:
        x[-1] = hi.numpy()


def _rb_sweep(dist, x, b, k, nz, w, rank, world):
    """One red-black sweep (red = (i + j + k) even first) with a halo exchange
    after each half-sweep."""
    ny, nx = x.shape[1:]
    par = (k[:, None, None] + np.arange(ny)[None, :, None] + np.arange(nx)[None, None, :]) % 2
    for colour in (0, 1):
        s, d = _neighbour_terms(x, k, nz, w)
        xi = x[1:-1]
        m = par == colour
        xi[m] = ((b + s) / d)[m]
        _exchange(dist, x, rank, world)


def _residual(x, b, k, nz, w):
    s, d = _neighbour_terms(x, k, nz, w)
    return b - (d * x[1:-1] - s)


def _zslab_worker(rank, world, port, q, shape, w, ncycles):
    dist = _init(rank, world, port)
    import torch
    import oracle
    nz, ny, nx = shape
    rng = np.random.default_rng(9)
    I0 = rng.uniform(0, 255, shape)
    z0, z1 = shard.slabs(nz, world, align=2)[rank]
    k = np.arange(z0, z1)
    b_full = oracle.rhs_ad(I0, w[1], w[2])  # the right-hand side has no z term: local
    b = b_full[z0:z1]
    # (1) one distributed sweep from a random start equals the oracle's
    x0 = rng.uniform(0, 255, shape)
    x = np.zeros((z1 - z0 + 2, ny, nx))
    x[1:-1] = x0[z0:z1]
    _exchange(dist, x, rank, world)
    _rb_sweep(dist, x, b, k, nz, w, rank, world)
    sweep_part = x[1:-1].copy()
    # (2) the two-level iteration from zero: z-pair restriction, coarse
    # problem gathered on rank 0, exact there, correction scattered back
    x[:] = 0.0
    bnorm2 = torch.tensor([float((b * b).sum())], dtype=torch.float64)
    dist.all_reduce(bnorm2)
    mean0 = I0.mean()
    hist = []
    wc = (0.0, 2 * w[1], 2 * w[2], w[3])  # P^T A P for z-pairs: 2 Kx, 2 Ky, K_{nz/2}
    for _ in range(ncycles):
        for _ in range(2):
            _rb_sweep(dist, x, b, k, nz, w, rank, world)
        r = _residual(x, b, k, nz, w)
        rc = r[0::2] + r[1::2]  # sum of the two children (R = P^T)
        parts = [None] * world
        dist.all_gather_object(parts, (z0 // 2, rc))
        ec_box = [None]
        if rank == 0:
            rc_full = np.zeros((nz // 2, ny, nx))
            for c0, piece in parts:
                rc_full[c0:c0 + piece.shape[0]] = piece
            # singular (pure Neumann): make the right-hand side exactly consistent
            rc_full -= rc_full.mean()
            # (1e-11: the consistent singular system's rounding floor is
            # near 1e-13, and the bars below need far less)
            ec, info = oracle.cg(rc_full, np.zeros_like(rc_full), *wc, tol=1e-11)
            assert info["status"] == 0, info
            ec_box = [ec]
        dist.broadcast_object_list(ec_box, src=0)
        ec = ec_box[0][z0 // 2:z1 // 2]
        x[1:-1] += np.repeat(ec, 2, axis=0)  # constant prolongation over the z-pair
        _exchange(dist, x, rank, world)
        for _ in range(2):
            _rb_sweep(dist, x, b, k, nz, w, rank, world)
        # mean fix: the iterate's sum all-reduced
        sx = torch.tensor([float(x[1:-1].sum())], dtype=torch.float64)
        dist.all_reduce(sx)
        x[1:-1] += mean0 - float(sx) / (nz * ny * nx)
        _exchange(dist, x, rank, world)
        rr = _residual(x, b, k, nz, w)
        r2 = torch.tensor([float((rr * rr).sum())], dtype=torch.float64)
        dist.all_reduce(r2)
        hist.append(float(np.sqrt(r2 / bnorm2)))
    q.put((rank, (z0, z1, sweep_part, x[1:-1].copy(), hist)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ad_zslab_protocol_matches_the_single_domain_oracle(world):
    import oracle
    from oracle import closed_form as cf
    shape, w = (12, 18, 22), (0.0, 1.0, 1.0, 10.0)
    out = _run(_zslab_worker, world, shape, w, 30)
    rng = np.random.default_rng(9)
    I0 = rng.uniform(0, 255, shape)
    x0 = rng.uniform(0, 255, shape)
    want_sweep = oracle.gs_sweeps(oracle.rhs_ad(I0, 1.0, 1.0), x0, *w, order="redblack", nsweeps=1)
    want = cf.ad(I0, 1.0, 1.0, 10.0)
    got_sweep = np.empty(shape)
    got = np.empty(shape)
    for r in range(world):
        z0, z1, sw, xr, hist = out[r]
        got_sweep[z0:z1] = sw
        got[z0:z1] = xr
    assert np.abs(got_sweep - want_sweep).max() <= 1e-10 * np.abs(want_sweep).max()
    hist = out[0][4]
    assert all(out[r][4] == hist for r in range(world))  # every rank sees the same norms
    assert hist[-1] <= 1e-9, hist
    assert np.abs(got - want).max() <= 1e-6, np.abs(got - want).max()
