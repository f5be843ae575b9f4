/*
 * gd_learn.h -- C ABI of the learned initial guess for the multigrid solves
 * of libgd (gradient-domain processing of EM image stacks, arXiv 1310.0041).
 *
 * The paper has no learned component.  Its multigrid V-cycle (Sec. 4.1)
 * accepts any starting iterate and drives it to the solution of the same
 * discrete system, so a better start only saves cycles; the solver still
 * judges the result by its residual.  This header exposes a small
 * convolutional encoder-decoder that predicts, from a stack I0, the change
 * the anisotropic diffusion makes (I1 - I0, Sec. 3.1 Eq. anisotropic
 * diffusion), to be used as the x0 of gd_diffuse_z.
 *
 * Network (widths c1..c4, 16-32-64-128 by default; 3x3 convolutions, zero
 * padding 1, cross-correlation, bias; pool = 2x2 average; up = 2x nearest;
 * [a, b] = channel concatenation):
 *   e1 = relu(conv(x)) ; e2 = relu(conv(pool e1)) ; e3 = relu(conv(pool e2))
 *   e4 = relu(conv(pool e3)) ; d3 = relu(conv([up e4, e3]))
 *   d2 = relu(conv([up d3, e2])) ; d1 = relu(conv([up d2, e1])) ; y = conv(d1)
 * Loss: mean squared error; optimiser: Adam with bias correction.
 *
 * Data layout: activations are bfloat16, channels last, [tile][h][w][c]
 * (c fastest); every channel count is a multiple of 16, tile heights and
 * widths multiples of 8.  Weights of a layer (co outputs, ci inputs) are
 * [co][9][ci] with tap = 3 dy + dx; the master copy is float32, the kernels
 * read bfloat16 copies.  All arithmetic of the convolutions is bfloat16
 * products accumulated in float32 on the tensor cores (tcgen05, TMEM).
 *
 * Conventions: pointers are device pointers unless a parameter says "host";
 * every call enqueues on the given CUDA stream (NULL = legacy default) and
 * the layer-level calls (gd_nn_*) return after their kernels complete.
 * Status codes are libgd's (gd.h): GD_OK, GD_ERR_INVALID_ARG for sizes the
 * kernels do not take, GD_ERR_OOM, GD_ERR_CUDA, GD_ERR_TIMEOUT when a
 * kernel's bounded wait on its own tensor-core work gave up (the kernel then
 * returns without touching the output further).
 */
#ifndef GD_LEARN_H
#define GD_LEARN_H

#include "gd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- layer-level operations (the network's building blocks) ---- */

/*
 * gd_nn_conv3x3 -- y = act(conv3x3(x, w) + bias) [* (mask > 0)] as an
 * implicit GEMM on the tensor cores.  The input is the channel
 * concatenation [up_a(xa), xb] of two bfloat16 sources: xa
 * [ntiles][h/up_a][w/up_a][ca] (up_a = 1 or 2, nearest upsampling) and,
 * when cb > 0, xb [ntiles][h][w][cb].  w: bfloat16 [co][9][ca + cb];
 * bias: float [co] or NULL; relu: 0 or 1; mask: bfloat16 [ntiles][h][w][co]
 * or NULL.  Outputs (either or both may be NULL): y bfloat16, yf float32,
 * both [ntiles][h][w][co].  ca, cb, co multiples of 16 (cb may be 0),
 * co <= 256.  Used with flipped weights (gd_nn_flip_weights) it is also the
 * input gradient of a convolution.
 */
int gd_nn_conv3x3(const void *xa, int ca, int up_a, const void *xb, int cb, int ntiles, int h, int w,
                  const void *wt, const float *bias, int co, int relu, const void *mask, void *y,
                  float *yf, void *stream);

/*
 * gd_nn_conv3x3_wgrad -- dw[o][tap][i] += sum over pixels p of
 * dy[p][o] * x[p + offset(tap)][i], with x the concatenated input of
 * gd_nn_conv3x3 (same xa, ca, up_a, xb, cb).  dy: bfloat16 [ntiles][h][w][co],
 * co <= 128; dw: float [co][9][ca + cb], accumulated (zero it first).
 */
int gd_nn_conv3x3_wgrad(const void *xa, int ca, int up_a, const void *xb, int cb, int ntiles, int h,
                        int w, const void *dy, int co, float *dw, void *stream);

/* db[o] += sum over pixels of dy[p][o]; dy bfloat16 [npix][co]. */
int gd_nn_bias_grad(const void *dy, long long npix, int co, float *db, void *stream);

/* w16 = bfloat16(w) in the same [co][9][ci] layout, and wf16 [ci][9][co]
 * with wf16[i][8 - tap][o] = w[o][tap][i]: the weights whose convolution is
 * the input gradient (either output may be NULL). */
int gd_nn_flip_weights(const float *w, int co, int ci, void *w16, void *wf16, void *stream);

/* 2x2 average pooling: x [ntiles][h][w][c] -> y [ntiles][h/2][w/2][c]. */
int gd_nn_pool2(const void *x, int ntiles, int h, int w, int c, void *y, void *stream);

/* Input gradient of pooling plus a skip gradient, masked by a ReLU output:
 * out[t][y][x][k] = (dp[t][y/2][x/2][k] / 4 + skip[t][y][x][skip_off + k])
 *                   * (mask[t][y][x][k] > 0)
 * dp [ntiles][h/2][w/2][c]; skip (nullable) has skip_stride channels per
 * pixel; mask and out [ntiles][h][w][c]. */
int gd_nn_pool2_backward(const void *dp, const void *skip, int skip_stride, int skip_off,
                         const void *mask, int ntiles, int h, int w, int c, void *out, void *stream);

/* Input gradient of nearest upsampling, masked by a ReLU output:
 * out[t][y][x][k] = sum over the 2x2 children of dk[t][.][.][k] (k < c, dk
 * has ck channels per pixel) * (mask[t][y][x][k] > 0).  h, w: the coarse
 * size; dk [ntiles][2h][2w][ck]; mask and out [ntiles][h][w][c]. */
int gd_nn_up2_backward(const void *dk, int ck, int c, const void *mask, int ntiles, int h, int w,
                       void *out, void *stream);

/* One Adam step (Kingma & Ba 2015) with bias correction at step t >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  float arrays of n. */
int gd_nn_adam(float *p, const float *g, float *m, float *v, long long n, double lr, double b1,
               double b2, double eps, int t, void *stream);

/* Self-test of the failure path of the tensor-core kernels: a kernel polls
 * an mbarrier that nothing arrives at, `limit` times (1 .. 2^21) with the
 * kernels' try_wait and suspend hint, gives up and raises the same device
 * flag a conv kernel raises when its bounded wait gives up; returns
 * GD_ERR_TIMEOUT (and clears the flag), leaving the context usable. */
int gd_nn_selftest_wait(unsigned limit);

/* ---- tiles of a stack ---- */

/*
 * gd_learn_stack_tiles -- cuts a float32 stack I [nz][ny][nx] (x fastest)
 * into tiles of th x tw pixels and tc slices, the slices becoming channels:
 * x[t][h][w][c] = (I[tz tc + c][ty th + h][tx tw + w] - shift) * scale as
 * bfloat16, tile t = (tz * (ny/th) + ty) * (nx/tw) + tx, for the ntiles
 * tiles starting at tile0.  When I_sub is given the value is
 * (I - I_sub) * scale and the output is float32 (xf) instead: the training
 * target.  nx, ny, nz multiples of tw, th, tc; tc a multiple of 8.  Returns
 * after the transform completes.
 */
int gd_learn_stack_tiles(const float *I, const float *I_sub, int nx, int ny, int nz, int th, int tw,
                         int tc, long long tile0, long long ntiles, double shift, double scale,
                         void *x, float *xf, void *stream);

/* ---- the network ---- */

typedef struct gd_learn gd_learn;

/*
 * gd_learn_create -- a network with c_in input and c_out output channels
 * (multiples of 16), widths[4] (multiples of 16; NULL = 16, 32, 64, 128),
 * for tiles of tile_h x tile_w pixels (multiples of 8) and batches of up to
 * max_batch tiles.  Parameters are drawn He-normal (std sqrt(2 / (9 ci))),
 * biases zero, from `seed`.  Everything is allocated here.
 */
int gd_learn_create(gd_learn **out, int c_in, int c_out, const int *widths, int tile_h, int tile_w,
                    int max_batch, unsigned long long seed, void *stream);
int gd_learn_destroy(gd_learn *L);

/* Number of parameters; flat order: for e1, e2, e3, e4, d3, d2, d1, y: the
 * weights [co][9][ci] then the bias [co]. */
long long gd_learn_param_count(const gd_learn *L);
/* Host float arrays of gd_learn_param_count values. */
int gd_learn_set_params(gd_learn *L, const float *host);
int gd_learn_get_params(gd_learn *L, float *host);
int gd_learn_get_grads(gd_learn *L, float *host);  /* of the last training step */

/* Forward pass on `batch` tiles x (bfloat16 [batch][h][w][c_in]) into yf
 * (float [batch][h][w][c_out]). */
int gd_learn_forward(gd_learn *L, const void *x, int batch, float *yf);

/*
 * gd_learn_train_step -- forward, mean squared error against target
 * (float [.][h][w][c_out]), backward and one Adam step with learning rate
 * lr (lr = 0 leaves the parameters as they are).  x_pool / t_pool hold
 * pool_tiles tiles each; idx_host (host, `batch` indices in
 * [0, pool_tiles)) picks the batch, or NULL for the first `batch` tiles
 * (GD_ERR_INVALID_ARG for an index outside the pool).  *loss (host,
 * nullable) receives the loss before the step.
 */
int gd_learn_train_step(gd_learn *L, const void *x_pool, const float *t_pool, long long pool_tiles,
                        const int *idx_host, int batch, double lr, double *loss);

/*
 * gd_learn_predict_stack -- the learned start of a solve:
 * x0 = I0 + out_scale * net((I0 - in_shift) * in_scale) tile by tile
 * (tiles of tile_h x tile_w pixels and c_in = c_out slices).  I0 and x0
 * float32 [nz][ny][nx], x0 may not alias I0; nx, ny, nz multiples of the
 * tile sizes.
 */
int gd_learn_predict_stack(gd_learn *L, const float *I0, int nx, int ny, int nz, double in_shift,
                           double in_scale, double out_scale, float *x0);

/*
 * gd_learn_lowmodes -- replaces, in every slice z of the start x, the
 * components along the first K x K two-dimensional cosine modes
 * phi_k(x) phi_l(y) (orthonormal DCT-II vectors, the eigenvectors of the
 * Neumann K_nx and K_ny) by those of the exact anisotropic-diffusion
 * solution of I0 with weights w (Sec. 3.1; Sec. 3.2 gives the filter: in
 * the cosine basis the solution of mode (k, l, m) is I0's times
 * (bx lk + by ll) / (bx lk + by ll + bz lm), l_j = 4 sin^2(pi j / 2n), and
 * the mean is kept).  A tile-wise prediction cannot see the whole stack, so
 * its slice means and slow illumination gradients are wrong; those modes are
 * the ones the V-cycle reduces slowly, and here they are made exact.
 * I0, x: float32 [nz][ny][nx] device arrays; K in {1, 2, 4, 8};
 * w.beta_z > 0.  Uses L's stream and a workspace of 3 nz K^2 doubles held
 * by L; returns after the correction is applied.
 */
int gd_learn_lowmodes(gd_learn *L, const float *I0, float *x, int nx, int ny, int nz, gd_weights w, int K);

/* Kernel launches issued by this network since creation. */
long long gd_learn_launch_count(const gd_learn *L);
/* Message of the network's last failure; with L = NULL (or a network with
 * none) the last failure of any call of this header. */
const char *gd_learn_last_error(const gd_learn *L);

#ifdef __cplusplus
}
#endif
#endif
