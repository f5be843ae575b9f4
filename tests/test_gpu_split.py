"""The slice split of screened Poisson through libgd (shard.py): two ranks
(processes) each solve their own slices on the GPU -- a contiguous slab of
a stack, then a size-balanced bin of slices of different sizes -- and only
their residual norms and cycle counts are all-reduced (gloo on host
tensors).  The two ranks share the one GPU of the box, which is sound here
because their kernels never wait on each other: the only exchange is the
host-side all-reduce after each solve.  The reassembled result equals the
exact per-slice solutions (DCT closed form) within 1e-3."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

NZ, NY, NX, ALPHA = 16, 256, 256, 0.01
SIDES = [300, 64, 520, 128, 257, 96, 410]
ALPHAS = [0.01, 0.05, 0.002, 0.1, 0.02, 0.07, 0.005]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import gdsynth
    import paper_1310_0041_gb300 as gd
    from paper_1310_0041_gb300 import shard
    torch.cuda.set_device(0)
    I0 = gdsynth.em_stack(NX, NY, NZ, seed=31).astype(np.float32)
    I1 = gdsynth.em_stack(NX, NY, NZ, seed=31, photo_seed=77, noise_sigma=0.0).astype(np.float32)
    z0, z1 = shard.slabs(NZ, world)[rank]
    a0 = torch.from_numpy(I0[z0:z1]).cuda()
    a1 = torch.from_numpy(I1[z0:z1]).cuda()
    a2 = torch.empty_like(a0)
    rep = shard.screened_poisson_slab(a0, a1, a2, ALPHA, gd.solve_ctl(30, 1e-8))
    slab = a2.cpu().numpy()
    # a batch of slices of different sizes, split by balanced bins
    B0s, B1s = gdsynth.batch_slices(SIDES, SIDES, seed=5)
    bins = shard.balanced_bins([n * n for n in SIDES], world)
    mine = bins[rank]
    p0 = torch.from_numpy(gdsynth.pack([B0s[i] for i in mine])).cuda()
    p1 = torch.from_numpy(gdsynth.pack([B1s[i] for i in mine])).cuda()
    p2 = torch.empty_like(p0)
    brep = shard.batch_screened_poisson_bin([SIDES[i] for i in mine], [SIDES[i] for i in mine],
                                            [ALPHAS[i] for i in mine], p0, p1, p2, gd.solve_ctl(40, 1e-8))
    pieces = dict(zip(mine, gdsynth.unpack(p2.cpu().numpy(), [SIDES[i] for i in mine],
                                           [SIDES[i] for i in mine])))
    parts = [None] * world
    dist.all_gather_object(parts, ((z0, z1, slab), pieces))
    q.put((rank, (rep, brep, parts)))
    dist.destroy_process_group()


def test_screened_poisson_split_over_two_ranks_on_the_gpu():
    import gdsynth
    from oracle import closed_form as cf
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    rep, brep, parts = out[0]
    assert out[1][0] == rep and out[1][1] == brep  # every rank sees the same combined report
    assert rep["rel_residual"] <= 1e-8 and brep["rel_residual"] <= 1e-8, (rep, brep)
    I0 = gdsynth.em_stack(NX, NY, NZ, seed=31).astype(np.float64)
    I1 = gdsynth.em_stack(NX, NY, NZ, seed=31, photo_seed=77, noise_sigma=0.0).astype(np.float64)
    got = np.empty_like(I0)
    pieces = {}
    for (z0, z1, slab), pc in parts:
        got[z0:z1] = slab
        pieces.update(pc)
    assert np.abs(got - cf.sp(I0, I1, ALPHA)).max() <= 1e-3
    B0s, B1s = gdsynth.batch_slices(SIDES, SIDES, seed=5)
    for i in range(len(SIDES)):
        want = cf.sp(B0s[i][None].astype(np.float64), B1s[i][None].astype(np.float64), ALPHAS[i])[0]
        assert np.abs(pieces[i] - want).max() <= 1e-3, i
