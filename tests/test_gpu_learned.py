"""Parity of the learned initial guess's CUDA kernels with the FP64 reference
``oracle/learned.py``, element by element.

Inputs and weights are first rounded to bfloat16 (the kernels' operand type),
and the reference evaluates each layer in FP64 on those same values, so the
only differences are the kernels' FP32 accumulation order and the bfloat16
rounding of their outputs.  Tolerances:

* one layer, bfloat16 output: |d| <= 2^-7 |ref| + 1e-3 max|ref| (the output
  rounding is at most 2^-9 relative; the rest is accumulation order);
* one layer, float32 output (weight and bias gradients, sums over thousands
  of products): |d| <= 1e-3 max|ref| + 2e-3 |ref|;
* the whole network (eight layers, every activation and activation gradient
  rounded to bfloat16 on the way): relative L2 error of the output and of
  each layer's weight gradient <= 5e-2, cosine >= 0.998.
"""
import numpy as np
import pytest

import oracle.learned as ol

pytestmark = pytest.mark.gpu

ONE_LAYER_REL, ONE_LAYER_ABS = 2.0 ** -7, 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    import paper_1310_0041_gb300 as gd
    from paper_1310_0041_gb300 import learn
    gd.build()
    gd.lib()
    return torch, learn


def bf(torch, a):
    """float64 copy of a rounded to bfloat16, and the bfloat16 CUDA tensor."""
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16)
    return t.to(torch.float64).numpy(), t.cuda()


def nhwc_to_tiles(a):
    """[T][H][W][C] -> list of [C][H][W]."""
    return [np.transpose(t, (2, 0, 1)) for t in a]


def tiles_to_nhwc(ts):
    return np.stack([np.transpose(t, (1, 2, 0)) for t in ts])


def w_to_kernel(w):
    """oracle [co][ci][3][3] -> kernel layout [co][9][ci]."""
    co, ci = w.shape[:2]
    return np.ascontiguousarray(w.reshape(co, ci, 9).transpose(0, 2, 1))


def close_bf16(got, want):
    err = np.abs(got - want)
    bound = ONE_LAYER_REL * np.abs(want) + ONE_LAYER_ABS * max(np.abs(want).max(), 1e-30)
    return bool(np.all(err <= bound)), float(err.max())


def close_f32(got, want):
    err = np.abs(got - want)
    bound = 2e-3 * np.abs(want) + 1e-3 * max(np.abs(want).max(), 1e-30)
    return bool(np.all(err <= bound)), float(err.max())


def concat_input(xa, up, xb):
    """The virtual input [up(xa), xb] of every tile, [C][H][W] each."""
    out = []
    for t in range(len(xa)):
        a = xa[t] if up == 1 else ol.up2(xa[t])
        out.append(a if xb is None else np.concatenate([a, xb[t]]))
    return out


CONV_CASES = [
    # ntiles, h, w, ca, up_a, cb, co, relu, mask
    (2, 16, 16, 16, 1, 0, 16, 1, False),   # e1-like
    (1, 24, 24, 32, 1, 0, 64, 1, False),   # ragged pixel count (576 = 4.5 blocks)
    (3, 8, 8, 128, 2, 64, 64, 1, False),   # d3: [up(e4), e3]
    (2, 16, 16, 32, 2, 16, 16, 1, False),  # d1-like concat
    (2, 8, 8, 64, 1, 0, 192, 0, False),    # input gradient of d3 (192 outputs)
    (2, 16, 16, 16, 1, 0, 48, 0, True),    # masked output
    (2, 32, 32, 16, 1, 0, 128, 0, False),  # N = 128
]


@pytest.mark.parametrize("nt,h,w,ca,up,cb,co,relu,use_mask", CONV_CASES)
def test_conv3x3_forward(env, nt, h, w, ca, up, cb, co, relu, use_mask):
    torch, learn = env
    rng = np.random.default_rng(nt * 1000 + h * 10 + ca + co)
    xa64, xa = bf(torch, rng.normal(size=(nt, h // up, w // up, ca)))
    xb64, xb = (None, None) if cb == 0 else bf(torch, rng.normal(size=(nt, h, w, cb)))
    ci = ca + cb
    wo = rng.normal(0, np.sqrt(2.0 / (9 * ci)), size=(co, ci, 3, 3))
    w64, wk = bf(torch, w_to_kernel(wo))
    wref = w64.reshape(co, 9, ci).transpose(0, 2, 1).reshape(co, ci, 3, 3)
    b = rng.normal(0, 0.1, size=co).astype(np.float32)
    mask64, mask = (None, None)
    if use_mask:
        mask64, mask = bf(torch, rng.normal(size=(nt, h, w, co)))
    y = torch.empty((nt, h, w, co), dtype=torch.bfloat16, device="cuda")
    yf = torch.empty((nt, h, w, co), dtype=torch.float32, device="cuda")
    st = learn.gd_nn_conv3x3(xa, ca, up, xb, cb, nt, h, w, wk, torch.from_numpy(b).cuda(), co, relu,
                             mask, y, yf)
    assert st == 0, learn.last_error()
    xin = concat_input(nhwc_to_tiles(xa64), up, None if xb64 is None else nhwc_to_tiles(xb64))
    ref = []
    for t in range(nt):
        r = ol.conv3x3(xin[t], wref, b.astype(np.float64))
        if relu:
            r = ol.relu(r)
        ref.append(r)
    ref = tiles_to_nhwc(ref)
    if use_mask:
        ref = ref * (mask64 > 0)
    ok, e = close_bf16(y.to(torch.float64).cpu().numpy(), ref)
    assert ok, e
    okf, ef = close_bf16(yf.to(torch.float64).cpu().numpy(), ref)
    assert okf, ef


@pytest.mark.parametrize("nt,h,w,ci,co", [(2, 16, 16, 16, 32), (1, 24, 24, 64, 128), (2, 8, 8, 192, 64)])
def test_input_gradient_by_flipped_weights(env, nt, h, w, ci, co):
    """dx of conv3x3 = a forward convolution of dy with the flipped weights."""
    torch, learn = env
    rng = np.random.default_rng(ci * 7 + co)
    wo = rng.normal(0, 0.1, size=(co, ci, 3, 3))
    w32 = torch.from_numpy(w_to_kernel(wo).astype(np.float32)).cuda()
    w16 = torch.empty((co, 9, ci), dtype=torch.bfloat16, device="cuda")
    wf16 = torch.empty((ci, 9, co), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_nn_flip_weights(w32, co, ci, w16, wf16) == 0
    wref = w16.to(torch.float64).cpu().numpy().reshape(co, 9, ci).transpose(0, 2, 1).reshape(co, ci, 3, 3)
    dy64, dy = bf(torch, rng.normal(size=(nt, h, w, co)))
    dx = torch.empty((nt, h, w, ci), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_nn_conv3x3(dy, co, 1, None, 0, nt, h, w, wf16, None, ci, 0, None, dx, None) == 0
    ref = []
    x_dummy = np.zeros((ci, h, w))
    for t, d in enumerate(nhwc_to_tiles(dy64)):
        ref.append(ol.conv3x3_backward(x_dummy, wref, d)[0])
    ok, e = close_bf16(dx.to(torch.float64).cpu().numpy(), tiles_to_nhwc(ref))
    assert ok, e


@pytest.mark.parametrize("nt,h,w,ca,up,cb,co", [
    (2, 16, 16, 16, 1, 0, 16),
    (1, 24, 24, 32, 1, 0, 64),
    (3, 8, 8, 128, 2, 64, 64),
    (2, 32, 32, 32, 2, 16, 16),
    (2, 16, 16, 64, 1, 0, 128),
])
def test_weight_and_bias_gradients(env, nt, h, w, ca, up, cb, co):
    torch, learn = env
    rng = np.random.default_rng(h * 31 + ca + cb + co)
    xa64, xa = bf(torch, rng.normal(size=(nt, h // up, w // up, ca)))
    xb64, xb = (None, None) if cb == 0 else bf(torch, rng.normal(size=(nt, h, w, cb)))
    ci = ca + cb
    dy64, dy = bf(torch, rng.normal(size=(nt, h, w, co)))
    dw = torch.zeros((co, 9, ci), dtype=torch.float32, device="cuda")
    db = torch.zeros(co, dtype=torch.float32, device="cuda")
    assert learn.gd_nn_conv3x3_wgrad(xa, ca, up, xb, cb, nt, h, w, dy, co, dw) == 0
    assert learn.gd_nn_bias_grad(dy, nt * h * w, co, db) == 0
    xin = concat_input(nhwc_to_tiles(xa64), up, None if xb64 is None else nhwc_to_tiles(xb64))
    w0 = np.zeros((co, ci, 3, 3))
    rdw, rdb = 0.0, 0.0
    for t, d in enumerate(nhwc_to_tiles(dy64)):
        _, gw, gb = ol.conv3x3_backward(xin[t], w0, d)
        rdw, rdb = rdw + gw, rdb + gb
    got = dw.cpu().numpy().astype(np.float64).reshape(co, 9, ci).transpose(0, 2, 1).reshape(co, ci, 3, 3)
    ok, e = close_f32(got, rdw)
    assert ok, e
    ok, e = close_f32(db.cpu().numpy().astype(np.float64), rdb)
    assert ok, e


def test_pool_and_its_gradient_and_upsampling_gradient(env):
    torch, learn = env
    rng = np.random.default_rng(5)
    nt, h, w, c = 2, 16, 24, 32
    x64, x = bf(torch, rng.normal(size=(nt, h, w, c)))
    y = torch.empty((nt, h // 2, w // 2, c), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_nn_pool2(x, nt, h, w, c, y) == 0
    ref = tiles_to_nhwc([ol.pool2(t) for t in nhwc_to_tiles(x64)])
    ok, e = close_bf16(y.to(torch.float64).cpu().numpy(), ref)
    assert ok, e
    # pooling gradient + skip (channels 8.. of a 48-channel tensor), masked
    dp64, dp = bf(torch, rng.normal(size=(nt, h // 2, w // 2, c)))
    sk64, sk = bf(torch, rng.normal(size=(nt, h, w, 48)))
    m64, m = bf(torch, rng.normal(size=(nt, h, w, c)))
    out = torch.empty((nt, h, w, c), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_nn_pool2_backward(dp, sk, 48, 16, m, nt, h, w, c, out) == 0
    ref = []
    for t in range(nt):
        g = ol.pool2_backward(np.transpose(dp64[t], (2, 0, 1))) + np.transpose(sk64[t, :, :, 16:48], (2, 0, 1))
        ref.append(ol.relu_backward(np.transpose(m64[t], (2, 0, 1)), g))
    ok, e = close_bf16(out.to(torch.float64).cpu().numpy(), tiles_to_nhwc(ref))
    assert ok, e
    # upsampling gradient of the first 32 of 48 channels, masked
    dk64, dk = bf(torch, rng.normal(size=(nt, h, w, 48)))
    mc64, mc = bf(torch, rng.normal(size=(nt, h // 2, w // 2, c)))
    o2 = torch.empty((nt, h // 2, w // 2, c), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_nn_up2_backward(dk, 48, c, mc, nt, h // 2, w // 2, o2) == 0
    ref = []
    for t in range(nt):
        g = ol.up2_backward(np.transpose(dk64[t, :, :, :c], (2, 0, 1)))
        ref.append(ol.relu_backward(np.transpose(mc64[t], (2, 0, 1)), g))
    ok, e = close_bf16(o2.to(torch.float64).cpu().numpy(), tiles_to_nhwc(ref))
    assert ok, e


def test_adam_step_matches_oracle(env):
    torch, learn = env
    rng = np.random.default_rng(6)
    n = 1000
    p0 = rng.normal(size=n).astype(np.float32)
    ref = {"a": p0.astype(np.float64)}
    state = {}
    p = torch.from_numpy(p0).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    for t in range(1, 4):
        g0 = rng.normal(size=n).astype(np.float32)
        ol.adam_step(ref, {"a": g0.astype(np.float64)}, state, lr=1e-2)
        assert learn.gd_nn_adam(p, torch.from_numpy(g0).cuda(), m, v, 1e-2, 0.9, 0.999, 1e-8, t) == 0
        assert np.abs(p.cpu().numpy() - ref["a"]).max() <= 1e-5


def test_stack_tiles(env):
    torch, learn = env
    rng = np.random.default_rng(7)
    nz, ny, nx, th, tw, tc = 32, 48, 64, 16, 32, 16
    I = rng.integers(0, 256, size=(nz, ny, nx)).astype(np.float32)
    J = rng.integers(0, 256, size=(nz, ny, nx)).astype(np.float32)
    It, Jt = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    T = (nx // tw) * (ny // th) * (nz // tc)
    x = torch.empty((T - 1, th, tw, tc), dtype=torch.bfloat16, device="cuda")
    assert learn.gd_learn_stack_tiles(It, None, nx, ny, nz, th, tw, tc, 1, T - 1, 128.0, 1 / 64, x=x) == 0
    tf = torch.empty((T, th, tw, tc), dtype=torch.float32, device="cuda")
    assert learn.gd_learn_stack_tiles(Jt, It, nx, ny, nz, th, tw, tc, 0, T, 0.0, 0.5, xf=tf) == 0
    torch.cuda.synchronize()
    xs, ts = x.to(torch.float32).cpu().numpy(), tf.cpu().numpy()
    for t in range(T):
        tx, r = t % (nx // tw), t // (nx // tw)
        ty, tz = r % (ny // th), r // (ny // th)
        win = (slice(tz * tc, (tz + 1) * tc), slice(ty * th, (ty + 1) * th), slice(tx * tw, (tx + 1) * tw))
        want_t = np.transpose((J[win] - I[win]) * 0.5, (1, 2, 0))
        assert np.array_equal(ts[t], want_t)
        if t >= 1:  # (I - 128) / 64 is exact in bfloat16 for integers 0..255
            assert np.array_equal(xs[t - 1], np.transpose((I[win] - 128.0) / 64.0, (1, 2, 0)))


WIDTHS = (16, 32, 64, 128)


def _oracle_params(learn, net, seed):
    """He-normal parameters of the reference, weights rounded to bfloat16 (the
    kernels' copies), small nonzero biases; returns (dict, flat)."""
    import torch
    p = ol.init_params(16, 16, WIDTHS, seed=seed)
    rng = np.random.default_rng(seed + 1)
    for k in p:
        if k.endswith(".b"):
            p[k] = 0.05 * rng.normal(size=p[k].shape)
        else:
            p[k] = torch.from_numpy(p[k].astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    p = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    return p, learn.params_to_flat(net, p)


def rel_l2(got, want):
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-30))


def cosine(a, b):
    return float(np.dot(a.ravel(), b.ravel()) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))


def test_network_forward_and_gradients(env):
    torch, learn = env
    B, H, W = 2, 32, 32
    net = learn.gd_learn_create(16, 16, WIDTHS, H, W, B, seed=0)
    try:
        p, flat = _oracle_params(learn, net, seed=11)
        learn.gd_learn_set_params(net, flat)
        assert np.array_equal(learn.gd_learn_get_params(net), flat)
        rng = np.random.default_rng(12)
        x64, x = bf(torch, rng.integers(0, 256, size=(B, H, W, 16)) / 64.0 - 2.0)
        tgt = rng.normal(size=(B, H, W, 16)).astype(np.float32)
        yf = torch.empty((B, H, W, 16), dtype=torch.float32, device="cuda")
        learn.gd_learn_forward(net, x, B, yf)
        ys, caches = [], []
        for t in range(B):
            y, c = ol.forward(p, np.transpose(x64[t], (2, 0, 1)))
            ys.append(y)
            caches.append(c)
        yref = tiles_to_nhwc(ys)
        got = yf.cpu().numpy().astype(np.float64)
        assert rel_l2(got, yref) <= 5e-2 and cosine(got, yref) >= 0.998, (rel_l2(got, yref), cosine(got, yref))
        # gradients of the batch's mean squared error (the mean over the batch
        # of the per-tile losses, which the reference computes tile by tile)
        loss = learn.gd_learn_train_step(net, x, torch.from_numpy(tgt).cuda(), None, B, lr=0.0)
        gref = None
        lref = 0.0
        for t in range(B):
            tt = np.transpose(tgt[t].astype(np.float64), (2, 0, 1))
            lref += ol.mse(ys[t], tt) / B
            g = ol.backward(p, caches[t], ys[t], tt)
            gref = g if gref is None else {k: gref[k] + g[k] for k in g}
        gref = {k: v / B for k, v in gref.items()}
        assert abs(loss - lref) <= 5e-2 * lref
        g = learn.flat_to_params(net, learn.gd_learn_get_grads(net))
        assert np.array_equal(learn.gd_learn_get_params(net), flat)  # lr = 0: unchanged
        for k in gref:
            r, cs = rel_l2(g[k].astype(np.float64), gref[k]), cosine(g[k].astype(np.float64), gref[k])
            assert r <= 5e-2 and cs >= 0.998, (k, r, cs)
    finally:
        learn.gd_learn_destroy(net)


def test_training_steps_match_oracle_adam_and_lower_the_loss(env):
    """Three Adam steps on the GPU against three of the reference from the same
    start, then a short run that lowers the loss."""
    torch, learn = env
    B, H, W = 1, 16, 16
    net = learn.gd_learn_create(16, 16, WIDTHS, H, W, B, seed=0)
    try:
        p, flat = _oracle_params(learn, net, seed=21)
        learn.gd_learn_set_params(net, flat)
        rng = np.random.default_rng(22)
        x64, x = bf(torch, rng.integers(0, 256, size=(B, H, W, 16)) / 64.0 - 2.0)
        tgt = (0.25 * x64 + 0.1).astype(np.float32)
        t_dev = torch.from_numpy(tgt).cuda()
        state = {}
        xo, to = np.transpose(x64[0], (2, 0, 1)), np.transpose(tgt[0].astype(np.float64), (2, 0, 1))
        p_start = {k: v.copy() for k, v in p.items()}
        for _ in range(3):
            learn.gd_learn_train_step(net, x, t_dev, None, B, lr=1e-3)
            y, c = ol.forward(p, xo)
            ol.adam_step(p, ol.backward(p, c, y, to), state, lr=1e-3)
        got = learn.flat_to_params(net, learn.gd_learn_get_params(net))
        # Adam moves each parameter by about lr * sign(gradient) per step, so a
        # parameter whose gradient is lost in bfloat16 noise may move the other
        # way: the updates are compared as whole vectors per layer
        for k in p:
            du_gpu = got[k].astype(np.float64) - p_start[k]
            du_ref = p[k] - p_start[k]
            if np.linalg.norm(du_ref) == 0:
                continue
            assert rel_l2(du_gpu, du_ref) <= 0.25 and cosine(du_gpu, du_ref) >= 0.97, (k, rel_l2(du_gpu, du_ref))
        losses = [learn.gd_learn_train_step(net, x, t_dev, None, B, lr=3e-3) for _ in range(60)]
        assert losses[-1] < 0.5 * losses[0]
    finally:
        learn.gd_learn_destroy(net)


def test_predict_stack_matches_tiles_and_forward(env):
    torch, learn = env
    nz, ny, nx = 32, 64, 96
    net = learn.gd_learn_create(16, 16, WIDTHS, 32, 32, 4, seed=3)  # 12 tiles in 3 batches
    try:
        rng = np.random.default_rng(8)
        I0 = torch.from_numpy(rng.integers(0, 256, size=(nz, ny, nx)).astype(np.float32)).cuda()
        x0 = torch.empty_like(I0)
        learn.gd_learn_predict_stack(net, I0, nx, ny, nz, 128.0, 1 / 64, 4.0, x0)
        ntiles = (nx // 32) * (ny // 32) * (nz // 16)
        want = I0.clone()
        for t0 in range(0, ntiles, 4):
            xt = torch.empty((4, 32, 32, 16), dtype=torch.bfloat16, device="cuda")
            assert learn.gd_learn_stack_tiles(I0, None, nx, ny, nz, 32, 32, 16, t0, 4, 128.0, 1 / 64, x=xt) == 0
            yf = torch.empty((4, 32, 32, 16), dtype=torch.float32, device="cuda")
            learn.gd_learn_forward(net, xt, 4, yf)
            for k in range(4):
                t = t0 + k
                tx, r = t % (nx // 32), t // (nx // 32)
                ty, tz = r % (ny // 32), r // (ny // 32)
                want[tz * 16:(tz + 1) * 16, ty * 32:(ty + 1) * 32, tx * 32:(tx + 1) * 32] += 4.0 * yf[k].permute(2, 0, 1)
        assert (x0 - want).abs().max().item() <= 1e-4 * max(1.0, want.abs().max().item())
    finally:
        learn.gd_learn_destroy(net)


@pytest.mark.parametrize("shape,K,bz", [((16, 48, 64), 4, 10.0), ((12, 40, 24), 2, 0.1), ((8, 32, 32), 8, 1.0)])
def test_lowmode_projection_matches_closed_form(env, shape, K, bz):
    """After gd_learn_lowmodes, the start's K x K lowest xy cosine modes are
    those of the exact anisotropic-diffusion solution (the oracle's FP64 DCT
    closed form) and every other mode is left as it was."""
    from scipy.fft import dctn
    from oracle import closed_form as cf
    torch, learn = env
    nz, ny, nx = shape
    rng = np.random.default_rng(nz * 100 + K)
    I0 = rng.integers(0, 256, size=shape).astype(np.float32)
    x = (I0 + rng.normal(0, 20, size=shape)).astype(np.float32)
    net = learn.gd_learn_create(16, 16, WIDTHS, 16, 16, 1, seed=0)
    try:
        xd = torch.from_numpy(x).cuda()
        learn.gd_learn_lowmodes(net, torch.from_numpy(I0).cuda(), xd, nx, ny, nz, (0.0, 1.0, 1.0, bz), K)
        got = dctn(xd.cpu().numpy().astype(np.float64), axes=(1, 2), norm="ortho")
    finally:
        learn.gd_learn_destroy(net)
    want_low = dctn(cf.ad(I0.astype(np.float64), 1.0, 1.0, bz), axes=(1, 2), norm="ortho")[:, :K, :K]
    before = dctn(x.astype(np.float64), axes=(1, 2), norm="ortho")
    scale = np.abs(before).max()
    assert np.abs(got[:, :K, :K] - want_low).max() <= 2e-5 * scale
    rest = np.ones(got.shape, bool)
    rest[:, :K, :K] = False
    assert np.abs(got[rest] - before[rest]).max() <= 2e-5 * scale
