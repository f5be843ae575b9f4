// gd_kernels.cu -- sm_103a kernels of the gradient-domain multigrid solver.
//
// All kernels are HBM-bandwidth bound stencils on FP32 data (about 1 flop per
// byte moved); none is a dense contraction, so none uses the tensor cores.
//
// Operator at a level (see LevelDev): at voxel (i,j,k)
//   (A x)_p = cx sum_{x-nbrs n}(x_p - x_n) + cy sum_{y-nbrs}(..) + cz sum_{z-nbrs}(..) + m x_p
//   cx = wx My(j) Mz(k), cy = wy Mx(i) Mz(k), cz = wz Mx(i) My(j), m = wm Mx My Mz,
// evaluated in difference form (x_p - x_n), which keeps the rounding error
// relative to the local differences rather than to the voxel values.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "gd.h"
#include "gd_internal.h"

namespace {

constexpr int NT = 256;       // threads per block of the stencil kernels
constexpr int TX = 64;        // z-march tile, x extent
constexpr int TY = 16;        // z-march tile, y extent

__device__ __forceinline__ float mass_of(int i, int n, int s, int l) {
  return (float)((i == n - 1) ? l : s);
}

// Block-wide sum of a double; result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh /* >= 32 */) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    t = (lane < nw) ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  }
  return t;
}

// ---------------------------------------------------------------------------
// Red-black Gauss-Seidel sweep, 2.5D z-march (Sec. 4.1 multi-colour relaxation;
// Sec. 4.1 streaming window: here a window of slices held in shared memory).
//
// One CTA owns a TX x TY column tile and marches along z over a chunk
// [zs, ze) of planes.  At step t it loads plane t+1, relaxes the red voxels
// (i+j+k even) of plane t on the tile plus a 1-voxel ring, then the black
// voxels of plane t-1 on the tile, and writes plane t-1.  Red values on the
// ring are recomputed from the old black values exactly as the neighbouring
// CTA computes them, so the result is the textbook red-black sweep.  Input
// and output are different arrays, so halos always hold old values.
// ---------------------------------------------------------------------------
struct SweepSmem {
  float x[4][TY + 4][TX + 4];   // ring of 4 planes, tile + 2-voxel halo
  float b[2][TY + 2][TX + 2];   // ring of 2 planes, tile + 1-voxel halo
  double red[32];
};

template <bool ZERO_IN, bool SUM_OUT>
__global__ void __launch_bounds__(NT) k_rb_sweep(LevelDev L, const float *__restrict__ xin,
                                                 const float *__restrict__ b,
                                                 float *__restrict__ xout, int zchunk,
                                                 double *__restrict__ partials) {
  constexpr int XW = TX + 4, XH = TY + 4, BW = TX + 2, BH = TY + 2;
  __shared__ SweepSmem sm;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int zs = blockIdx.z * zchunk;
  const int ze = min(zs + zchunk, nz);
  const bool zc = (L.wz != 0.f) && (nz > 1);
  const int tid = threadIdx.x;
  const size_t plane = (size_t)nx * (size_t)ny;
  double acc = 0.0;

  auto load_x = [&](int p) {
    float(*dst)[XW] = sm.x[p & 3];
    const float *src = xin + (size_t)p * plane;
    for (int q = tid; q < XH * XW; q += NT) {
      const int r = q / XW, c = q - r * XW;
      const int gi = i0 - 2 + c, gj = j0 - 2 + r;
      float v = 0.f;
      if (!ZERO_IN && gi >= 0 && gi < nx && gj >= 0 && gj < ny) v = __ldg(src + (size_t)gj * nx + gi);
      dst[r][c] = v;
    }
  };
  auto load_b = [&](int p) {
    float(*dst)[BW] = sm.b[p & 1];
    const float *src = b + (size_t)p * plane;
    for (int q = tid; q < BH * BW; q += NT) {
      const int r = q / BW, c = q - r * BW;
      const int gi = i0 - 1 + c, gj = j0 - 1 + r;
      float v = 0.f;
      if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) v = __ldg(src + (size_t)gj * nx + gi);
      dst[r][c] = v;
    }
  };
  // Gauss-Seidel update of one voxel in shared memory (sy, sx in the halo-2 frame).
  auto relax = [&](int p, int gi, int gj, int sy, int sx, float bv) {
    float(*X)[XW] = sm.x[p & 3];
    const float(*Xm)[XW] = sm.x[(p + 3) & 3];
    const float(*Xp)[XW] = sm.x[(p + 1) & 3];
    const float mx = mass_of(gi, nx, L.sx, L.lx);
    const float my = mass_of(gj, ny, L.sy, L.ly);
    const float mz = mass_of(p, nz, L.sz, L.lz);
    const float cx = L.wx * my * mz, cy = L.wy * mx * mz, cz = L.wz * mx * my;
    const float mm = L.wm * mx * my * mz;
    const float xc = X[sy][sx];
    float ax = mm * xc, dg = mm;
    if (gi > 0) { ax += cx * (xc - X[sy][sx - 1]); dg += cx; }
    if (gi < nx - 1) { ax += cx * (xc - X[sy][sx + 1]); dg += cx; }
    if (gj > 0) { ax += cy * (xc - X[sy - 1][sx]); dg += cy; }
    if (gj < ny - 1) { ax += cy * (xc - X[sy + 1][sx]); dg += cy; }
    if (zc && p > 0) { ax += cz * (xc - Xm[sy][sx]); dg += cz; }
    if (zc && p < nz - 1) { ax += cz * (xc - Xp[sy][sx]); dg += cz; }
    if (dg > 0.f) X[sy][sx] = xc + (bv - ax) / dg;
  };
  auto red = [&](int t) {  // tile + 1 ring, colour (i+j+k) even
    const float(*B)[BW] = sm.b[t & 1];
    for (int q = tid; q < BH * (BW / 2); q += NT) {
      const int r = q / (BW / 2), c2 = q - r * (BW / 2);
      const int gj = j0 - 1 + r;
      const int col = 2 * c2 + ((i0 - 1 + gj + t) & 1);
      const int gi = i0 - 1 + col;
      if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
      relax(t, gi, gj, r + 1, col + 1, B[r][col]);
    }
  };
  auto black = [&](int p) {  // tile only, colour (i+j+k) odd
    const float(*B)[BW] = sm.b[p & 1];
    for (int q = tid; q < TY * (TX / 2); q += NT) {
      const int r = q / (TX / 2), c2 = q - r * (TX / 2);
      const int gj = j0 + r;
      const int col = 2 * c2 + ((i0 + gj + p + 1) & 1);
      const int gi = i0 + col;
      if (gi >= nx || gj >= ny) continue;
      relax(p, gi, gj, r + 2, col + 2, B[r + 1][col + 1]);
    }
  };
  auto store = [&](int p) {
    const float(*X)[XW] = sm.x[p & 3];
    float *dst = xout + (size_t)p * plane;
    for (int q = tid; q < TY * TX; q += NT) {
      const int r = q / TX, c = q - r * TX;
      const int gi = i0 + c, gj = j0 + r;
      if (gi < nx && gj < ny) {
        const float v = X[r + 2][c + 2];
        dst[(size_t)gj * nx + gi] = v;
        if (SUM_OUT) acc += (double)v;
      }
    }
  };

  if (zc) {
    if (zs - 2 >= 0) load_x(zs - 2);
    if (zs - 1 >= 0) load_x(zs - 1);
    for (int t = zs - 1; t <= ze; ++t) {
      if (t + 1 < nz) load_x(t + 1);
      if (t >= 0 && t < nz) load_b(t);
      __syncthreads();
      if (t >= 0 && t < nz) red(t);
      __syncthreads();
      if (t - 1 >= zs) {
        black(t - 1);
        __syncthreads();
        store(t - 1);
      }
      __syncthreads();
    }
  } else {
    for (int t = zs; t < ze; ++t) {
      load_x(t);
      load_b(t);
      __syncthreads();
      red(t);
      __syncthreads();
      black(t);
      __syncthreads();
      store(t);
      __syncthreads();
    }
  }
  if (SUM_OUT) {
    const double s = block_sum(acc, sm.red);
    if (tid == 0) {
      const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      partials[blk * S_NUM + S_E] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Residual r = b - A x, down-sampled by summing the children (Sec. 4.1; the
// Constant discretisation's (1,1) stencil per coarsened axis, Sec. 4.2):
// one thread per coarse cell.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float residual_at(const LevelDev &L, const float *__restrict__ x,
                                             const float *__restrict__ b, int i, int j, int k) {
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const size_t p = ((size_t)k * ny + j) * nx + i;
  const size_t pl = (size_t)nx * ny;
  const float mx = mass_of(i, nx, L.sx, L.lx);
  const float my = mass_of(j, ny, L.sy, L.ly);
  const float mz = mass_of(k, nz, L.sz, L.lz);
  const float cx = L.wx * my * mz, cy = L.wy * mx * mz, cz = L.wz * mx * my;
  const float xc = __ldg(x + p);
  float ax = L.wm * mx * my * mz * xc;
  if (i > 0) ax += cx * (xc - __ldg(x + p - 1));
  if (i < nx - 1) ax += cx * (xc - __ldg(x + p + 1));
  if (j > 0) ax += cy * (xc - __ldg(x + p - nx));
  if (j < ny - 1) ax += cy * (xc - __ldg(x + p + nx));
  if (cz != 0.f) {
    if (k > 0) ax += cz * (xc - __ldg(x + p - pl));
    if (k < nz - 1) ax += cz * (xc - __ldg(x + p + pl));
  }
  return __ldg(b + p) - ax;
}

__global__ void __launch_bounds__(NT) k_residual_restrict(LevelDev F, const float *__restrict__ x,
                                                          const float *__restrict__ b, int fx,
                                                          int fy, int fz, int ncx, int ncy,
                                                          int ncz, float *__restrict__ bc) {
  const size_t total = (size_t)ncx * ncy * ncz;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(idx % ncx);
    const int J = (int)((idx / ncx) % ncy);
    const int K = (int)(idx / ((size_t)ncx * ncy));
    float s = 0.f;
    for (int dk = 0; dk <= fz; ++dk) {
      const int k = (K << fz) + dk;
      if (k >= F.nz) continue;
      for (int dj = 0; dj <= fy; ++dj) {
        const int j = (J << fy) + dj;
        if (j >= F.ny) continue;
        for (int di = 0; di <= fx; ++di) {
          const int i = (I << fx) + di;
          if (i >= F.nx) continue;
          s += residual_at(F, x, b, i, j, k);
        }
      }
    }
    bc[idx] = s;
  }
}

// x += P xc: each coarse value replicated into its children (Sec. 4.2 Constant).
__global__ void __launch_bounds__(NT) k_prolong_add(int nx, int ny, int nz, int fx, int fy, int fz,
                                                    int ncx, int ncy, const float *__restrict__ xc,
                                                    float *__restrict__ x) {
  const size_t total = (size_t)nx * ny * nz;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((size_t)nx * ny));
    const size_t q = ((size_t)(k >> fz) * ncy + (j >> fy)) * ncx + (i >> fx);
    x[p] += __ldg(xc + q);
  }
}

// ---------------------------------------------------------------------------
// Fine-level outer pass: x_new = x + e (+ mean shift) kept as an unevaluated
// float pair (hi, lo); r = b - A x_new with b assembled from the inputs
// (Sec. 3.1: AD b = (bx Kx + by Ky) I0; SP b = alpha I1 + (Kx + Ky) I0);
// FP64 block partial sums of r^2, b^2, x_new and I0.
// ---------------------------------------------------------------------------
// Double-float ("ff") arithmetic on FP32 pairs (hi, lo), value hi + lo:
// Knuth's TwoSum and Dekker's fast renormalisation; products through FMA.
// Intrinsics keep the compiler from contracting or reassociating.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p, e);
}

// Outer pass.  The residual is evaluated in ff arithmetic with ff weights, so
// its rounding error is ~1e-13 of the terms rather than ~1e-7: the refinement
// then converges to the exact (double-weight) system far below 1e-8.
template <int RHS, bool HAS_XL, bool HAS_E>
__global__ void __launch_bounds__(NT) k_outer(OuterArgs a) {
  __shared__ double sh[32];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t pl = (size_t)nx * ny;
  const size_t total = pl * nz;
  float shift = 0.f;
  if (HAS_E && a.mean_fix)
    shift = (float)((a.scalars[S_I0] - a.scalars[S_X] - a.scalars[S_E] * (double)a.e_scale) * a.inv_n);
  // float32 storage only (the plain kernels serve float32 hierarchies)
  const float *ev = static_cast<const float *>(a.e);
  float *rout = static_cast<float *>(a.r_out);
  const ff Wx = {a.bx, a.bx_lo}, Wy = {a.by, a.by_lo}, Wz = {a.bz, a.bz_lo};
  const ff Wa = {a.alpha, a.alpha_lo};
  const ff Rx = {a.rbx, a.rbx_lo}, Ry = {a.rby, a.rby_lo}, Ra = {a.ralpha, a.ralpha_lo};
  double srr = 0.0, sbb = 0.0, sx = 0.0, si = 0.0;
  auto xnew = [&](size_t q) -> ff {
    const float xh = __ldg(a.xh_in + q);
    const float xl = HAS_XL ? __ldg(a.xl_in + q) : 0.f;
    if (HAS_E) return ff_add({xh, xl}, {__fadd_rn(__ldg(ev + q) * a.e_scale, shift), 0.f});
    return {xh, xl};
  };
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / pl);
    const ff xc = xnew(p);
    ff dx = {0.f, 0.f}, dy = {0.f, 0.f}, dz = {0.f, 0.f};
    if (i > 0) dx = ff_add(dx, ff_add(xc, ff_neg(xnew(p - 1))));
    if (i < nx - 1) dx = ff_add(dx, ff_add(xc, ff_neg(xnew(p + 1))));
    if (j > 0) dy = ff_add(dy, ff_add(xc, ff_neg(xnew(p - nx))));
    if (j < ny - 1) dy = ff_add(dy, ff_add(xc, ff_neg(xnew(p + nx))));
    if (a.bz != 0.f) {
      if (k > 0) dz = ff_add(dz, ff_add(xc, ff_neg(xnew(p - pl))));
      if (k < nz - 1) dz = ff_add(dz, ff_add(xc, ff_neg(xnew(p + pl))));
    }
    ff ax = ff_add(ff_mul(dx, Wx), ff_mul(dy, Wy));
    ax = ff_add(ax, ff_mul(dz, Wz));
    ax = ff_add(ax, ff_mul(xc, Wa));
    ff bv;
    if (RHS == RHS_EXPLICIT) {
      bv = {__ldg(a.b + p), 0.f};
    } else {
      // I0 holds integers 0..255 in the workloads; differences and their sums
      // are exact in FP32 for any input below 2^22
      const float ic = __ldg(a.I0 + p);
      float gx = 0.f, gy = 0.f;
      if (i > 0) gx += ic - __ldg(a.I0 + p - 1);
      if (i < nx - 1) gx += ic - __ldg(a.I0 + p + 1);
      if (j > 0) gy += ic - __ldg(a.I0 + p - nx);
      if (j < ny - 1) gy += ic - __ldg(a.I0 + p + nx);
      bv = ff_add(ff_mul({gx, 0.f}, Rx), ff_mul({gy, 0.f}, Ry));
      if (RHS == RHS_SP) bv = ff_add(bv, ff_mul({__ldg(a.I1 + p), 0.f}, Ra));
      si += (double)ic;
    }
    const ff rr = ff_add(bv, ff_neg(ax));
    const float r = __fadd_rn(rr.h, rr.l);
    if (a.xh_out) a.xh_out[p] = xc.h;
    if (a.xl_out) a.xl_out[p] = xc.l;
    if (rout) rout[p] = r * a.r_scale;
    const double rd = (double)rr.h + (double)rr.l;
    const double bd = (double)bv.h + (double)bv.l;
    srr += rd * rd;
    sbb += bd * bd;
    sx += (double)xc.h + (double)xc.l;
  }
  double v;
  v = block_sum(srr, sh);
  if (threadIdx.x == 0) a.partials[(size_t)blockIdx.x * S_NUM + S_RR] = v;
  v = block_sum(sbb, sh);
  if (threadIdx.x == 0) a.partials[(size_t)blockIdx.x * S_NUM + S_BB] = v;
  v = block_sum(sx, sh);
  if (threadIdx.x == 0) a.partials[(size_t)blockIdx.x * S_NUM + S_X] = v;
  v = block_sum(si, sh);
  if (threadIdx.x == 0) a.partials[(size_t)blockIdx.x * S_NUM + S_I0] = v;
}

// Deterministic reduction of the per-block partials (fixed order).
__global__ void __launch_bounds__(1024) k_reduce(const double *__restrict__ partials, int nblocks,
                                                 double *__restrict__ scalars, int lo, int hi,
                                                 int accumulate) {
  __shared__ double sh[32];
  for (int s = lo; s < hi; ++s) {
    double v = 0.0;
    for (int bidx = threadIdx.x; bidx < nblocks; bidx += blockDim.x) v += partials[(size_t)bidx * S_NUM + s];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) scalars[s] = accumulate ? scalars[s] + v : v;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: fast diagonalisation (Lynch, Rice, Thomas 1964).
// out = M_axis applied along one axis; M = V^T (transpose) or V; optional
// multiplication by Dinv (period: Dinv repeats every `period` elements).
// V is row-major n x n, column c = eigenvector c.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) k_axis_apply(int nx, int ny, int nz, int axis,
                                                   const float *__restrict__ V, int transpose,
                                                   const float *__restrict__ in,
                                                   float *__restrict__ out,
                                                   const float *__restrict__ Dinv, int period) {
  const size_t total = (size_t)nx * ny * nz;
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)nx : (size_t)nx * ny);
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
       p += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const int j = (int)((p / nx) % ny);
    const int k = (int)(p / ((size_t)nx * ny));
    const int c = axis == 0 ? i : (axis == 1 ? j : k);
    const size_t base = p - (size_t)c * stride;
    float s = 0.f;
    for (int q = 0; q < n; ++q) {
      const float m = transpose ? V[q * n + c] : V[c * n + q];
      s += m * in[base + (size_t)q * stride];
    }
    if (Dinv) s *= Dinv[p % (size_t)period];
    out[p] = s;
  }
}

__global__ void k_fill(float *p, size_t n, float v) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) p[q] = v;
}

__global__ void k_copy(float *__restrict__ d, const float *__restrict__ s, size_t n) {
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) d[q] = s[q];
}

// 16-byte copy with four loads in flight per thread: many requests
// outstanding at once, which a copy across the CPU-GPU link needs
__global__ void k_copy4(float4 *__restrict__ d, const float4 *__restrict__ s, size_t n4) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; q + 3 * stride < n4; q += 4 * stride) {
    const float4 a = s[q], b = s[q + stride], c = s[q + 2 * stride], e = s[q + 3 * stride];
    d[q] = a;
    d[q + stride] = b;
    d[q + 2 * stride] = c;
    d[q + 3 * stride] = e;
  }
  for (; q < n4; q += stride) d[q] = s[q];
}

int grid_for(size_t n, int per_block, int cap) {
  size_t g = (n + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > (size_t)cap) g = cap;
  return (int)g;
}

}  // namespace

// Number of SMs; filled lazily.
static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      g_num_sms = v;
    else
      g_num_sms = 152;
  }
  return g_num_sms;
}

cudaError_t launch_rb_sweep(const LevelDev &L, const float *xin, const float *b, float *xout,
                            bool zero_in, double *partials_sum, int *nblocks_out, cudaStream_t st) {
  const int gx = (L.nx + TX - 1) / TX, gy = (L.ny + TY - 1) / TY;
  const bool zc = (L.wz != 0.f) && (L.nz > 1);
  // enough CTAs for a few waves (about 7 resident CTAs per SM); coupled
  // chunks pay a 2-plane halo, so keep them at least 8 planes deep
  const long target = (long)num_sms() * 7 * 3;
  long chunks = (target + (long)gx * gy - 1) / ((long)gx * gy);
  const int min_chunk = zc ? 8 : 1;
  long max_chunks = (L.nz + min_chunk - 1) / min_chunk;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  const int zchunk = (int)((L.nz + chunks - 1) / chunks);
  const int gz = (L.nz + zchunk - 1) / zchunk;
  dim3 grid(gx, gy, gz);
  if (nblocks_out) *nblocks_out = gx * gy * gz;
  const bool sum = partials_sum != nullptr;
  if (zero_in) {
    if (sum) k_rb_sweep<true, true><<<grid, NT, 0, st>>>(L, xin, b, xout, zchunk, partials_sum);
    else k_rb_sweep<true, false><<<grid, NT, 0, st>>>(L, xin, b, xout, zchunk, nullptr);
  } else {
    if (sum) k_rb_sweep<false, true><<<grid, NT, 0, st>>>(L, xin, b, xout, zchunk, partials_sum);
    else k_rb_sweep<false, false><<<grid, NT, 0, st>>>(L, xin, b, xout, zchunk, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_residual_restrict(const LevelDev &F, const float *x, const float *b, int fx,
                                     int fy, int fz, float *bc, cudaStream_t st) {
  const int ncx = fx ? (F.nx + 1) / 2 : F.nx;
  const int ncy = fy ? (F.ny + 1) / 2 : F.ny;
  const int ncz = fz ? (F.nz + 1) / 2 : F.nz;
  const size_t n = (size_t)ncx * ncy * ncz;
  k_residual_restrict<<<grid_for(n, NT, num_sms() * 64), NT, 0, st>>>(F, x, b, fx, fy, fz, ncx, ncy, ncz, bc);
  return cudaGetLastError();
}

cudaError_t launch_prolong_add(const LevelDev &F, int fx, int fy, int fz, const float *xc, float *x,
                               cudaStream_t st) {
  const int ncx = fx ? (F.nx + 1) / 2 : F.nx;
  const int ncy = fy ? (F.ny + 1) / 2 : F.ny;
  const size_t n = (size_t)F.nx * F.ny * F.nz;
  k_prolong_add<<<grid_for(n, NT, num_sms() * 64), NT, 0, st>>>(F.nx, F.ny, F.nz, fx, fy, fz, ncx, ncy, xc, x);
  return cudaGetLastError();
}

cudaError_t launch_outer(const OuterArgs &a, int rhs_mode, int *nblocks_out, cudaStream_t st) {
  const size_t n = (size_t)a.nx * a.ny * a.nz;
  const int g = grid_for(n, NT, num_sms() * 8);
  if (nblocks_out) *nblocks_out = g;
  const bool xl = a.xl_in != nullptr, e = a.e != nullptr;
#define GD_OUTER(R)                                                         \
  if (xl && e) k_outer<R, true, true><<<g, NT, 0, st>>>(a);                 \
  else if (xl) k_outer<R, true, false><<<g, NT, 0, st>>>(a);                \
  else if (e) k_outer<R, false, true><<<g, NT, 0, st>>>(a);                 \
  else k_outer<R, false, false><<<g, NT, 0, st>>>(a);
  if (rhs_mode == RHS_EXPLICIT) { GD_OUTER(RHS_EXPLICIT) }
  else if (rhs_mode == RHS_AD) { GD_OUTER(RHS_AD) }
  else { GD_OUTER(RHS_SP) }
#undef GD_OUTER
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partials, int nblocks, double *scalars, int slot_lo,
                          int slot_hi, int accumulate, cudaStream_t st) {
  k_reduce<<<1, 1024, 0, st>>>(partials, nblocks, scalars, slot_lo, slot_hi, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_fdm(int nx, int ny, int nz, const float *Vx, const float *Vy, const float *Vz,
                       const float *Dinv, int batch_z, const float *b, float *x, float *tmp,
                       cudaStream_t st) {
  const size_t n = (size_t)nx * ny * nz;
  const int g = grid_for(n, NT, num_sms() * 8);
  if (batch_z) {
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 0, Vx, 1, b, tmp, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 1, Vy, 1, tmp, x, Dinv, nx * ny);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 1, Vy, 0, x, tmp, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 0, Vx, 0, tmp, x, nullptr, 1);
  } else {
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 0, Vx, 1, b, tmp, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 1, Vy, 1, tmp, x, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 2, Vz, 1, x, tmp, Dinv, (int)n);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 2, Vz, 0, tmp, x, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 1, Vy, 0, x, tmp, nullptr, 1);
    k_axis_apply<<<g, NT, 0, st>>>(nx, ny, nz, 0, Vx, 0, tmp, x, nullptr, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_fill(float *p, size_t n, float v, cudaStream_t st) {
  k_fill<<<grid_for(n, NT, num_sms() * 8), NT, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

cudaError_t launch_copy(float *dst, const float *src, size_t n, cudaStream_t st) {
  k_copy<<<grid_for(n, NT, num_sms() * 8), NT, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_copy_wide(float *dst, const float *src, size_t n, cudaStream_t st) {
  if (((uintptr_t)dst & 15) || ((uintptr_t)src & 15)) return launch_copy(dst, src, n, st);
  const size_t n4 = n / 4;
  if (n4) {
    k_copy4<<<grid_for(n4, NT, num_sms() * 16), NT, 0, st>>>(reinterpret_cast<float4 *>(dst),
                                                            reinterpret_cast<const float4 *>(src), n4);
  }
  if (n % 4) k_copy<<<1, 32, 0, st>>>(dst + 4 * n4, src + 4 * n4, n % 4);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// NPR gradient filter right-hand side (Sec. 7, after Bhat et al. 2010):
//   b = alpha I0 - div(W V),  V = lambda (1 - exp(-|grad I0|^2 / 2 sigma^2)) grad I0
// with forward differences on voxel faces (none leaves the domain); the
// modulation of face p -> p + e_d uses the full forward-difference vector at
// its lower voxel p.  One thread per voxel, neighbours through the caches.
// ---------------------------------------------------------------------------
struct NprArgs {
  int nx, ny, nz;
  float alpha, wx, wy, wz, lam, inv2s2;  // inv2s2 = 1 / (2 sigma^2)
};

__device__ __forceinline__ float npr_at(const float *__restrict__ I0, const NprArgs &a, int i, int j,
                                        int k, int d) {
  // V_d on the face (i,j,k) -> +e_d; 0 when that face leaves the domain
  const size_t pl = (size_t)a.nx * a.ny;
  const size_t o = (size_t)k * pl + (size_t)j * a.nx + i;
  const float c = __ldg(I0 + o);
  const float gx = i + 1 < a.nx ? __ldg(I0 + o + 1) - c : 0.f;
  const float gy = j + 1 < a.ny ? __ldg(I0 + o + a.nx) - c : 0.f;
  const float gz = k + 1 < a.nz ? __ldg(I0 + o + pl) - c : 0.f;
  const float g = d == 0 ? gx : (d == 1 ? gy : gz);
  const float m2 = gx * gx + gy * gy + gz * gz;
  // 1 - exp(-u) = -expm1(-u), accurate for small u
  return a.lam * -expm1f(-m2 * a.inv2s2) * g;
}

__global__ void __launch_bounds__(NT) k_npr_rhs(const float *__restrict__ I0, float *__restrict__ b,
                                                NprArgs a) {
  const size_t pl = (size_t)a.nx * a.ny, n = pl * a.nz;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(q / pl);
    const int j = (int)((q - (size_t)k * pl) / a.nx);
    const int i = (int)(q - (size_t)k * pl - (size_t)j * a.nx);
    float v = a.alpha * __ldg(I0 + q);
    const float w[3] = {a.wx, a.wy, a.wz};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (w[d] == 0.f) continue;
      float in = 0.f;
      if (d == 0 && i > 0) in = npr_at(I0, a, i - 1, j, k, 0);
      if (d == 1 && j > 0) in = npr_at(I0, a, i, j - 1, k, 1);
      if (d == 2 && k > 0) in = npr_at(I0, a, i, j, k - 1, 2);
      v += w[d] * (in - npr_at(I0, a, i, j, k, d));
    }
    b[q] = v;
  }
}

cudaError_t launch_npr_rhs(const float *I0, float *b, int nx, int ny, int nz, double alpha, double wx,
                           double wy, double wz, double lam, double sigma, cudaStream_t st) {
  NprArgs a;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.alpha = (float)alpha;
  a.wx = (float)wx;
  a.wy = (float)wy;
  a.wz = (float)wz;
  a.lam = (float)lam;
  a.inv2s2 = (float)(1.0 / (2.0 * sigma * sigma));
  const size_t n = (size_t)nx * ny * nz;
  k_npr_rhs<<<grid_for(n, NT, num_sms() * 8), NT, 0, st>>>(I0, b, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free relaxation (gd_smooth_noalloc): the out-of-place sweep's
// second array lives in this file-scope device array instead of a per-call
// cudaMalloc.  Host code must not use the symbol as a device address: the
// address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
static __device__ __align__(256) float g_noalloc_scratch[GD_NOALLOC_MAX_VOXELS];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kNoallocMaxDevices] = {};

// A device (or managed) array that the kernels on device `dev` can address:
// device memory of another GPU is refused (without peer access it is an
// illegal address there).
bool noalloc_device_ptr(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// [a, a + n) and [b, b + n) share an element
bool noalloc_overlap(const float *a, const float *b, size_t n) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b, bytes = n * sizeof(float);
  return pa < pb + bytes && pb < pa + bytes;
}

bool noalloc_weight_ok(double v) { return std::isfinite(v) && v >= 0.0; }
}  // namespace

extern "C" int gd_smooth_noalloc(int nx, int ny, int nz, gd_weights w, const float *b, float *x,
                                 int nsweeps, void *cuda_stream) {
  if (nx < 2 || ny < 2 || nz < 1 || !b || !x || nsweeps < 0) return GD_ERR_INVALID_ARG;
  if ((double)nx * (double)ny * (double)nz > (double)GD_NOALLOC_MAX_VOXELS) return GD_ERR_INVALID_ARG;
  // the sweep reads b and x through restrict pointers: they must not overlap
  if (noalloc_overlap(b, x, (size_t)nx * ny * nz)) return GD_ERR_INVALID_ARG;
  if (!noalloc_weight_ok(w.alpha) || !noalloc_weight_ok(w.beta_x) || !noalloc_weight_ok(w.beta_y) ||
      !noalloc_weight_ok(w.beta_z))
    return GD_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GD_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return GD_ERR_UNSUPPORTED;
  if (!noalloc_device_ptr(b, dev) || !noalloc_device_ptr(x, dev)) return GD_ERR_INVALID_ARG;
  float *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return GD_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = static_cast<float *>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)nx * ny * nz;
  const LevelDev L = {nx, ny, nz, 1, 1, 1, 1, 1, 1, (float)w.beta_x, (float)w.beta_y,
                      (float)w.beta_z, (float)w.alpha};
  // sweep k reads x (k even) or the scratch (k odd) and writes the other one
  for (int k = 0; k < nsweeps; ++k) {
    const float *in = (k & 1) ? scratch : x;
    float *out = (k & 1) ? x : scratch;
    if (launch_rb_sweep(L, in, b, out, false, nullptr, nullptr, st) != cudaSuccess) return GD_ERR_CUDA;
  }
  if ((nsweeps & 1) && launch_copy(x, scratch, n, st) != cudaSuccess) return GD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return GD_ERR_CUDA;
  return GD_OK;
}
