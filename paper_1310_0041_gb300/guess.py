"""Training and use of the learned initial guess, as a sequence of libgd calls.

The network (``include/gd_learn.h``) is trained on pairs that the multigrid
solver itself produces: for a stack I0, the anisotropic-diffusion solution I1
(paper Sec. 3.1, solved by ``gd_diffuse_z`` on the GPU) gives the target
(I1 - I0) / out_scale of every 256 x 256 x 16 tile, the input being
(I0 - in_shift) * in_scale with the slices as channels.  The solver's
V-cycle (Sec. 4.1) accepts any start, so the prediction only sets x0; the
multigrid still runs to the requested residual and judges the result.

Every step runs in libgd's kernels; this module only sequences the calls.
Stacks come from a caller-supplied ``make_stack(seed)`` returning a CUDA
tensor (uint8 or float32) of shape (nz, ny, nx).
"""
from __future__ import annotations

import time

import numpy as np

from . import (gd_destroy, gd_diffuse_z, gd_stack_create, solve_ctl)
from . import learn

IN_SHIFT, IN_SCALE, OUT_SCALE = 128.0, 1.0 / 64.0, 16.0
AD_WEIGHTS = (0.0, 1.0, 1.0, 10.0)


def train_on_solver_pairs(net, make_stack, n_pairs, shape=(1024, 1024, 128), weights=AD_WEIGHTS,
                          tol=1e-6, batch=32, lr=1e-3, lr_final=1e-4, passes=2, seed0=100000,
                          log=None):
    """Trains `net` on about `n_pairs` (tile, target) pairs drawn from fresh
    stacks of `shape`; each stack's tiles are visited `passes` times in
    random batches.  Returns a dict with the losses and timings."""
    import torch
    nx, ny, nz = shape
    th, tw, tc = net.tile_h, net.tile_w, net.c_in
    tiles = (nx // tw) * (ny // th) * (nz // tc)
    n_stacks = max(1, -(-n_pairs // tiles))
    steps_per_stack = max(1, passes * tiles // batch)
    total_steps = n_stacks * steps_per_stack
    xpool = torch.empty((tiles, th, tw, tc), dtype=torch.bfloat16, device="cuda")
    tpool = torch.empty((tiles, th, tw, net.c_out), dtype=torch.float32, device="cuda")
    I1 = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    s = gd_stack_create(nx, ny, nz)
    rng = np.random.default_rng(seed0)
    losses, t_gen, t_solve, t_train = [], 0.0, 0.0, 0.0
    step = 0
    try:
        for k in range(n_stacks):
            t0 = time.time()
            I0 = make_stack(seed0 + k).float()
            torch.cuda.synchronize()
            t1 = time.time()
            gd_diffuse_z(s, I0, I1, weights, solve_ctl(30, tol))
            learn.gd_learn_stack_tiles(I0, None, nx, ny, nz, th, tw, tc, 0, tiles, IN_SHIFT, IN_SCALE,
                                       x=xpool)
            learn.gd_learn_stack_tiles(I1, I0, nx, ny, nz, th, tw, tc, 0, tiles, 0.0, 1.0 / OUT_SCALE,
                                       xf=tpool)
            torch.cuda.synchronize()
            t2 = time.time()
            for _ in range(steps_per_stack):
                frac = step / max(1, total_steps - 1)
                lr_k = lr * (lr_final / lr) ** frac  # geometric decay
                idx = rng.choice(tiles, size=min(batch, tiles), replace=False)
                losses.append(learn.gd_learn_train_step(net, xpool, tpool, idx, lr=lr_k))
                step += 1
            t3 = time.time()
            t_gen += t1 - t0
            t_solve += t2 - t1
            t_train += t3 - t2
            if log and (k % 10 == 0 or k == n_stacks - 1):
                log("stack %d/%d loss %.4g" % (k + 1, n_stacks, float(np.mean(losses[-steps_per_stack:]))))
    finally:
        gd_destroy(s)
    return dict(losses=losses, pairs=n_stacks * tiles, stacks=n_stacks, steps=step,
                seconds_generate=t_gen, seconds_solve=t_solve, seconds_train=t_train)


def learned_start(net, I0, x0):
    """x0 = I0 + OUT_SCALE * net((I0 - IN_SHIFT) * IN_SCALE), tile by tile."""
    nz, ny, nx = I0.shape
    learn.gd_learn_predict_stack(net, I0, nx, ny, nz, IN_SHIFT, IN_SCALE, OUT_SCALE, x0)
    return x0
