"""What the trained network gains: it is trained on the GPU on 20k
(tile, target) pairs that the multigrid solver itself produces, then seeds
the anisotropic diffusion (Sec. 3.1) of held-out 1024 x 1024 x 128 stacks.

Controls: the zero start (the solver's default), the I0 start, and I0 with
the exact low-mode projection (gd_learn_lowmodes) but no network.  Measured
by the relative residual after each V-cycle (Sec. 4.1), which the solver
reports, and the cycles to 1e-6:

* the network's start beats the I0 start after the first two cycles (it has
  learned the local part of the diffusion's correction);
* with the low modes made exact, the learned start beats the zero start
  after each of the first four cycles and needs no more cycles;
* the network adds to the projection alone (first cycle).

The learned start does not save a whole cycle on this workload: that would
take a residual ~13x below the zero start's after four cycles.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_PAIRS = 20000
K = 4


@pytest.fixture(scope="module")
def trained():
    import torch
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    import gdsynth
    import paper_1310_0041_gb300 as gd
    from paper_1310_0041_gb300 import guess, learn
    gd.build()
    gdsynth.build_cuda()
    net = learn.gd_learn_create(16, 16, (16, 32, 64, 128), 256, 256, 32, seed=1)
    rep = guess.train_on_solver_pairs(net, lambda sd: gdsynth.em_stack_cuda(1024, 1024, 128, seed=sd),
                                      N_PAIRS, passes=4, lr=2e-3)
    yield torch, gdsynth, gd, guess, learn, net, rep
    learn.gd_learn_destroy(net)


def histories(trained, seed):
    torch, gdsynth, gd, guess, learn, net, _ = trained
    nx, ny, nz = 1024, 1024, 128
    W = guess.AD_WEIGHTS
    I0 = gdsynth.em_stack_cuda(nx, ny, nz, seed=seed).float()
    out = torch.empty_like(I0)
    s = gd.gd_stack_create(nx, ny, nz)
    try:
        def solve(x0):
            return gd.gd_diffuse_z(s, I0, out, W, gd.solve_ctl(30, 1e-6), x0=x0)
        h = {"zero": solve(None), "I0": solve(I0)}
        x = I0.clone()
        learn.gd_learn_lowmodes(net, I0, x, nx, ny, nz, W, K)
        h["I0+low"] = solve(x)
        x0 = torch.empty_like(I0)
        guess.learned_start(net, I0, x0)
        h["learned"] = solve(x0)
        learn.gd_learn_lowmodes(net, I0, x0, nx, ny, nz, W, K)
        h["learned+low"] = solve(x0)
    finally:
        gd.gd_destroy(s)
    return h


def test_training_lowered_the_loss(trained):
    rep = trained[-1]
    assert rep["pairs"] >= N_PAIRS
    L = rep["losses"]
    assert np.mean(L[-50:]) < 0.6 * np.mean(L[:20])


@pytest.mark.parametrize("seed", [1, 2])
def test_learned_start_against_the_controls(trained, seed):
    h = histories(trained, seed)
    for k in h:
        assert h[k]["status"] == 0 and h[k]["rel_residual"] <= 1e-6, (k, h[k])
    hz, hi, hil = h["zero"]["history"], h["I0"]["history"], h["I0+low"]["history"]
    hl, hll = h["learned"]["history"], h["learned+low"]["history"]
    # the network beats the I0 start after the first two cycles, and in cycles
    for c in (1, 2):
        assert hl[c] <= 0.9 * hi[c], (c, hl, hi)
    assert h["learned"]["cycles"] <= h["I0"]["cycles"]
    # with exact low modes it beats the zero start after each of the first four cycles
    for c in range(1, 5):
        assert hll[c] <= 0.85 * hz[c], (c, hll, hz)
    assert h["learned+low"]["cycles"] <= h["zero"]["cycles"]
    # and it adds to the projection alone
    assert hll[1] <= 0.8 * hil[1], (hll, hil)
