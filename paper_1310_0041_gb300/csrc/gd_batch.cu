// gd_batch.cu -- batched screened Poisson on independent slices of different
// sizes (the per-slice system of Sec. 3.1, Eq. screened_poisson:
// (alpha_s + Kx + Ky) I2 = alpha_s I1 + (Kx + Ky) I0 on slice s, with its own
// alpha_s and its own nx_s x ny_s).
//
// The slices decouple (the screened Poisson step has no z term), so one
// multigrid V-cycle runs over all of them at once: every slice has its own
// 2D hierarchy (the planner's coarsening rule applied to nx_s x ny_s), the
// levels of all slices with the same depth are packed into one buffer, and
// each kernel is one persistent launch over a work list of (slice, tile)
// items of that depth.  Slices whose hierarchy ends at depth l are solved
// exactly there (fast diagonalisation, one CTA per slice) between the
// descent and the ascent.  The whole V-cycle is a fixed launch sequence and
// is replayed from a CUDA graph.
//
// Layout of the caller's arrays: slice s occupies elements
// [off_s, off_s + nx_s ny_s) of one packed float32 array, x fastest, with
// off_s = sum over t < s of nx_t ny_t.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "gd.h"
#include "gd_internal.h"

namespace {

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
constexpr int BX = 64, BY = 32;  // tile (cells)
constexpr int BNT = 256;         // threads per CTA
constexpr int XW = BX + 4, XH = BY + 4;  // x box: two-cell halo (the red ring and its neighbours)
constexpr int BW = BX + 2, BH = BY + 2;  // b box: one-cell halo (the red ring)
constexpr int kBMaxLev = 24;
constexpr int kFdmMaxCells = 4096;

// One slice at one level.  The level operator is the Kronecker form of the
// stack solver restricted to a slice:
//   A = wx Kx (x) My + wy Mx (x) Ky + wm Mx (x) My,
// M = diag(children counts, s inside and l for the last cell of an axis).
struct BEntry {
  long long off;   // first element of the slice in this level's packed buffer
  long long coff;  // the same in the next level's buffer (-1: coarsest level)
  int nx, ny;
  int sx, sy, lx, ly;
  int cnx, cny, fx, fy;  // next level's sizes and the axes halved to reach it
  float wx, wy, wm;
  int slice;
};

struct BCoarse {  // coarsest level of one slice
  int lev;        // its depth
  int nx, ny;
  int vx, vy;     // offsets of Vx, Vy in the V table
  int lx, ly;     // offsets of the eigenvalues in the lambda table
  float wx, wy, wm;
  long long off;  // first element in the level's packed buffer
};

struct BLevelPtrs {
  const float *b[kBMaxLev];
  float *x[kBMaxLev];
};

__device__ __forceinline__ bool inside(const BEntry &e, int i, int j) {
  return i >= 0 && i < e.nx && j >= 0 && j < e.ny;
}

// Couplings and diagonal of cell (i, j): cx to each x-neighbour, cy to each
// y-neighbour; neighbours outside the slice are absent (Neumann).
__device__ __forceinline__ void coef(const BEntry &e, int i, int j, float &cx, float &cy, float &dg) {
  const float mx = (i == e.nx - 1) ? (float)e.lx : (float)e.sx;
  const float my = (j == e.ny - 1) ? (float)e.ly : (float)e.sy;
  cx = e.wx * my;
  cy = e.wy * mx;
  const float nbx = (float)((i > 0) + (i < e.nx - 1));
  const float nby = (float)((j > 0) + (j < e.ny - 1));
  dg = cx * nbx + cy * nby + e.wm * mx * my;
}

// Fills two shared-memory boxes (h1 x w1 and h2 x w2, row-major) with
// get1(r, c) and get2(r, c): every global load of the thread is issued
// before the first shared-memory store, so one round trip covers both.
template <int H1, int W1, int H2, int W2, typename G1, typename G2>
__device__ __forceinline__ void load_boxes(float *d1, G1 get1, float *d2, G2 get2) {
  constexpr int N1 = (H1 * W1 + BNT - 1) / BNT, N2 = (H2 * W2 + BNT - 1) / BNT;
  float v1[N1], v2[N2 > 0 ? N2 : 1];
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    const int q = threadIdx.x + k * BNT;
    v1[k] = (q < H1 * W1) ? get1(q / W1, q % W1) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < N2; ++k) {
    const int q = threadIdx.x + k * BNT;
    v2[k] = (q < H2 * W2) ? get2(q / W2, q % W2) : 0.f;
  }
#pragma unroll
  for (int k = 0; k < N1; ++k) {
    const int q = threadIdx.x + k * BNT;
    if (q < H1 * W1) d1[q] = v1[k];
  }
#pragma unroll
  for (int k = 0; k < N2; ++k) {
    const int q = threadIdx.x + k * BNT;
    if (q < H2 * W2) d2[q] = v2[k];
  }
}

// One red-black Gauss-Seidel sweep of every tile of the work list, xin ->
// xout.  Red cells are (i + j) even.  A tile relaxes its red cells and the red
// ring around it (whose values the tile's black cells read), then its black
// cells; a red value depends only on black values of the input, so the ring
// values a CTA computes are the ones the neighbouring tile writes.
template <bool ZERO_IN, bool PROLONG>
__global__ void __launch_bounds__(BNT) k_bsweep(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                int nitems, const float *__restrict__ xin,
                                                const float *__restrict__ b, float *__restrict__ xout,
                                                const float *__restrict__ xc) {
  __shared__ float xs[XH][XW];
  __shared__ float bs[BH][BW];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int i0 = w.y, j0 = w.z;
    load_boxes<XH, XW, BH, BW>(
        &xs[0][0],
        [&](int r, int c) {
          const int gi = i0 - 2 + c, gj = j0 - 2 + r;
          float v = 0.f;
          if (inside(e, gi, gj)) {
            if (!ZERO_IN) v = xin[e.off + (long long)gj * e.nx + gi];
            if (PROLONG) v += xc[e.coff + (long long)(gj >> e.fy) * e.cnx + (gi >> e.fx)];
          }
          return v;
        },
        &bs[0][0],
        [&](int r, int c) {
          const int gi = i0 - 1 + c, gj = j0 - 1 + r;
          return inside(e, gi, gj) ? b[e.off + (long long)gj * e.nx + gi] : 0.f;
        });
    __syncthreads();
    // red cells of the tile and its ring: rows j0-1 .. j0+BY, BW/2 per row
    for (int q = threadIdx.x; q < BH * (BW / 2); q += BNT) {
      const int r = q / (BW / 2), k = q - r * (BW / 2);
      const int gj = j0 - 1 + r;
      const int gi = i0 - 1 + ((i0 - 1 + gj) & 1) + 2 * k;
      if (inside(e, gi, gj)) {
        const int xr = r + 1, xq = gi - i0 + 2;
        float cx, cy, dg;
        coef(e, gi, gj, cx, cy, dg);
        const float s = bs[r][gi - i0 + 1] + cx * (xs[xr][xq - 1] + xs[xr][xq + 1]) +
                        cy * (xs[xr - 1][xq] + xs[xr + 1][xq]);
        xs[xr][xq] = __fdividef(s, dg);
      }
    }
    __syncthreads();
    // black cells of the tile: BX/2 per row
    for (int q = threadIdx.x; q < BY * (BX / 2); q += BNT) {
      const int r = q / (BX / 2), k = q - r * (BX / 2);
      const int gj = j0 + r;
      const int gi = i0 + (((i0 + gj) & 1) ^ 1) + 2 * k;
      if (inside(e, gi, gj)) {
        const int xr = r + 2, xq = gi - i0 + 2;
        float cx, cy, dg;
        coef(e, gi, gj, cx, cy, dg);
        const float s = bs[r + 1][gi - i0 + 1] + cx * (xs[xr][xq - 1] + xs[xr][xq + 1]) +
                        cy * (xs[xr - 1][xq] + xs[xr + 1][xq]);
        xs[xr][xq] = __fdividef(s, dg);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < BY * BX; q += BNT) {
      const int r = q / BX, c = q - r * BX;
      const int gi = i0 + c, gj = j0 + r;
      if (inside(e, gi, gj)) xout[e.off + (long long)gj * e.nx + gi] = xs[r + 2][c + 2];
    }
    __syncthreads();  // the next item reuses the boxes
  }
}

// Residual r = b - A x of a tile into rs (0 outside the slice); xs holds the
// x box with a one-cell halo.
__device__ __forceinline__ void tile_residual(float (*xs)[BW], float (*rs)[BX], const BEntry &e, int i0,
                                              int j0, const float *__restrict__ b) {
  for (int q = threadIdx.x; q < BY * BX; q += BNT) {
    const int r = q / BX, c = q - r * BX;
    const int gi = i0 + c, gj = j0 + r;
    float v = 0.f;
    if (inside(e, gi, gj)) {
      float cx, cy, dg;
      coef(e, gi, gj, cx, cy, dg);
      const float ax = dg * xs[r + 1][c + 1] - cx * (xs[r + 1][c] + xs[r + 1][c + 2]) -
                       cy * (xs[r][c + 1] + xs[r + 2][c + 1]);
      v = b[e.off + (long long)gj * e.nx + gi] - ax;
    }
    rs[r][c] = v;
  }
}

__device__ __forceinline__ void load_xbox1(float (*xs)[BW], const BEntry &e, int i0, int j0,
                                           const float *__restrict__ x) {
  auto get = [&](int r, int c) {
    const int gi = i0 - 1 + c, gj = j0 - 1 + r;
    return inside(e, gi, gj) ? x[e.off + (long long)gj * e.nx + gi] : 0.f;
  };
  load_boxes<BH, BW, 0, 1>(&xs[0][0], get, &xs[0][0], get);
}

// Residual of the tile summed over each coarse cell's children into the next
// level's right-hand side (restriction = transpose of the prolongation).
// Tiles start at even cells, so a coarse cell's children share one tile.
__global__ void __launch_bounds__(BNT) k_brestrict(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                   int nitems, const float *__restrict__ x,
                                                   const float *__restrict__ b, float *__restrict__ bc) {
  __shared__ float xs[BH][BW];
  __shared__ float rs[BY][BX];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int i0 = w.y, j0 = w.z;
    load_xbox1(xs, e, i0, j0, x);
    __syncthreads();
    tile_residual(xs, rs, e, i0, j0, b);
    __syncthreads();
    const int cw = BX >> e.fx, ch = BY >> e.fy;
    for (int q = threadIdx.x; q < cw * ch; q += BNT) {
      const int cr = q / cw, cc = q - cr * cw;
      const int ci = (i0 >> e.fx) + cc, cj = (j0 >> e.fy) + cr;
      if (ci < e.cnx && cj < e.cny) {
        float s = 0.f;
        for (int dy = 0; dy <= e.fy; ++dy)
          for (int dx = 0; dx <= e.fx; ++dx) s += rs[(cr << e.fy) + dy][(cc << e.fx) + dx];
        bc[e.coff + (long long)cj * e.cnx + ci] = s;
      }
    }
    __syncthreads();
  }
}

// Error-free transformations (Knuth's TwoSum): s + e == a + b exactly.
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

// The outer pass of the float-pair refinement at the fine level (unit
// masses and stiffness, A = alpha + Kx + Ky): (h, l) <- (h, l) + e
// (ADD_E; input pair -> output pair, never in place, since neighbouring
// tiles read this tile's cells), then r = bf - A (h + l) with every rounding
// error of the high parts captured, written as the correction's right-hand
// side, and the per-slice sums of r^2 and bf^2 (FP64 slots acc[2 s],
// acc[2 s + 1]; each thread sums its few cells in FP32, the block in FP64).
template <bool ADD_E>
__global__ void __launch_bounds__(BNT) k_bouter(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                int nitems, const float *__restrict__ bf,
                                                const float *__restrict__ hin, const float *__restrict__ lin,
                                                const float *__restrict__ e, float *__restrict__ hout,
                                                float *__restrict__ lout, float *__restrict__ r,
                                                double *__restrict__ acc) {
  __shared__ float hs[BH][BW];
  __shared__ float ls[BH][BW];
  __shared__ double red[2][BNT / 32];
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry en = E[w.x];
    const int i0 = w.y, j0 = w.z, nx = en.nx;
    {
      constexpr int N = (BH * BW + BNT - 1) / BNT;
      float hv[N], lv[N], ev[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int q = threadIdx.x + k * BNT;
        const int rr = q / BW, c = q - rr * BW;
        const int gi = i0 - 1 + c, gj = j0 - 1 + rr;
        hv[k] = lv[k] = ev[k] = 0.f;
        if (q < BH * BW && inside(en, gi, gj)) {
          const long long o = en.off + (long long)gj * nx + gi;
          hv[k] = hin[o];
          lv[k] = lin[o];
          if (ADD_E) ev[k] = e[o];
        }
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const int q = threadIdx.x + k * BNT;
        if (q < BH * BW) {
          float h = hv[k], l = lv[k];
          if (ADD_E) {
            const ff a = two_sum(h, ev[k]);
            const ff v = two_sum(a.h, __fadd_rn(a.l, l));
            h = v.h;
            l = v.l;
          }
          (&hs[0][0])[q] = h;
          (&ls[0][0])[q] = l;
        }
      }
    }
    __syncthreads();
    float s_rr = 0.f, s_bb = 0.f;
    const float alpha = en.wm;
    for (int q = threadIdx.x; q < BY * BX; q += BNT) {
      const int rr = q / BX, c = q - rr * BX;
      const int gi = i0 + c, gj = j0 + rr;
      if (!inside(en, gi, gj)) continue;
      const long long o = en.off + (long long)gj * nx + gi;
      const float hc = hs[rr + 1][c + 1], lc = ls[rr + 1][c + 1];
      if (ADD_E) {
        hout[o] = hc;
        lout[o] = lc;
      } else if (hout != hin) {
        hout[o] = hc;
        lout[o] = lc;
      }
      const float bv = bf[o];
      float hi = bv, lo = 0.f;
      auto sub = [&](float v) {
        const ff t = two_sum(hi, -v);
        hi = t.h;
        lo += t.l;
      };
      auto nb = [&](bool has, float hn, float ln) {
        if (!has) return;
        const ff d = two_sum(hc, -hn);
        sub(d.h);
        lo -= d.l + (lc - ln);
      };
      nb(gi > 0, hs[rr + 1][c], ls[rr + 1][c]);
      nb(gi < nx - 1, hs[rr + 1][c + 2], ls[rr + 1][c + 2]);
      nb(gj > 0, hs[rr][c + 1], ls[rr][c + 1]);
      nb(gj < en.ny - 1, hs[rr + 2][c + 1], ls[rr + 2][c + 1]);
      const float pa = alpha * hc;
      sub(pa);
      lo -= __fmaf_rn(alpha, hc, -pa) + alpha * lc;
      const float rv = hi + lo;
      r[o] = rv;
      s_rr = fmaf(rv, rv, s_rr);
      s_bb = fmaf(bv, bv, s_bb);
    }
    double drr = s_rr, dbb = s_bb;
    for (int o = 16; o > 0; o >>= 1) {
      drr += __shfl_down_sync(0xffffffffu, drr, o);
      dbb += __shfl_down_sync(0xffffffffu, dbb, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      red[0][warp] = drr;
      red[1][warp] = dbb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (int k = 0; k < BNT / 32; ++k) {
        a0 += red[0][k];
        a1 += red[1][k];
      }
      atomicAdd(&acc[2 * en.slice], a0);
      atomicAdd(&acc[2 * en.slice + 1], a1);
    }
    __syncthreads();
  }
}

// I2 = h + l rounded to float32
__global__ void k_bfinal(float *__restrict__ out, const float *__restrict__ h, const float *__restrict__ l,
                         long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    out[q] = __fadd_rn(h[q], l[q]);
}

// Fine right-hand side b = alpha I1 + (Kx + Ky) I0 and the initial float
// pair (x0 or I0, 0).
__global__ void __launch_bounds__(BNT) k_brhs(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                              int nitems, const float *__restrict__ I0,
                                              const float *__restrict__ I1, const float *__restrict__ x0,
                                              float *__restrict__ b, float *__restrict__ x,
                                              float *__restrict__ xl) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int i0 = w.y, j0 = w.z;
    for (int q = threadIdx.x; q < BY * BX; q += BNT) {
      const int r = q / BX, c = q - r * BX;
      const int gi = i0 + c, gj = j0 + r;
      if (!inside(e, gi, gj)) continue;
      const long long o = e.off + (long long)gj * e.nx + gi;
      const float c0 = I0[o];
      float k = 0.f;
      if (gi > 0) k += c0 - I0[o - 1];
      if (gi < e.nx - 1) k += c0 - I0[o + 1];
      if (gj > 0) k += c0 - I0[o - e.nx];
      if (gj < e.ny - 1) k += c0 - I0[o + e.nx];
      b[o] = fmaf(e.wm, I1[o], k);
      x[o] = x0 ? x0[o] : c0;
      xl[o] = 0.f;
    }
  }
}

// Exact solve on each slice's coarsest level by fast diagonalisation:
// x = (Vx (x) Vy) D^-1 (Vx (x) Vy)^T b, D_kl = wm + wx lamx_k + wy lamy_l.
// One CTA per slice; the level is at most kFdmMaxCells cells.
__global__ void __launch_bounds__(BNT) k_bfdm(const BCoarse *__restrict__ C, int ns, const float *__restrict__ V,
                                              const float *__restrict__ lam, BLevelPtrs P) {
  extern __shared__ float fsm[];
  float *B = fsm, *T = fsm + kFdmMaxCells;
  for (int s = blockIdx.x; s < ns; s += gridDim.x) {
    const BCoarse c = C[s];
    const int nx = c.nx, ny = c.ny, n = nx * ny;
    const float *Vx = V + c.vx, *Vy = V + c.vy;
    const float *bl = P.b[c.lev] + c.off;
    float *xl = P.x[c.lev] + c.off;
    for (int q = threadIdx.x; q < n; q += BNT) B[q] = bl[q];
    __syncthreads();
    // T[j][k] = sum_i B[j][i] Vx[i][k]
    for (int q = threadIdx.x; q < n; q += BNT) {
      const int j = q / nx, k = q - j * nx;
      float a = 0.f;
      for (int i = 0; i < nx; ++i) a = fmaf(B[j * nx + i], Vx[i * nx + k], a);
      T[q] = a;
    }
    __syncthreads();
    // B[l][k] = sum_j Vy[j][l] T[j][k] / D_kl
    for (int q = threadIdx.x; q < n; q += BNT) {
      const int l = q / nx, k = q - l * nx;
      float a = 0.f;
      for (int j = 0; j < ny; ++j) a = fmaf(Vy[j * ny + l], T[j * nx + k], a);
      B[q] = a / (c.wm + c.wx * lam[c.lx + k] + c.wy * lam[c.ly + l]);
    }
    __syncthreads();
    // T[j][k] = sum_l Vy[j][l] B[l][k]
    for (int q = threadIdx.x; q < n; q += BNT) {
      const int j = q / nx, k = q - j * nx;
      float a = 0.f;
      for (int l = 0; l < ny; ++l) a = fmaf(Vy[j * ny + l], B[l * nx + k], a);
      T[q] = a;
    }
    __syncthreads();
    // x[j][i] = sum_k Vx[i][k] T[j][k]
    for (int q = threadIdx.x; q < n; q += BNT) {
      const int j = q / nx, i = q - j * nx;
      float a = 0.f;
      for (int k = 0; k < nx; ++k) a = fmaf(Vx[i * nx + k], T[j * nx + k], a);
      xl[q] = a;
    }
    __syncthreads();
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct gd_batch {
  int ns = 0;
  std::vector<int> nx, ny;
  std::vector<double> alpha;
  std::vector<long long> off;  // packed offsets of the slices
  long long nvox = 0;
  int cxy = 16;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int sm_count = 0;
  // levels (packed over the slices that reach them)
  struct Lev {
    long long n = 0;
    float *x = nullptr, *t = nullptr, *b = nullptr;
    BEntry *E = nullptr;            // device
    int ne = 0;
    int4 *items = nullptr;          // tiles of the entries that have a next level
    int nitems = 0;
    int4 *items_all = nullptr;      // tiles of every entry (level 0 only)
    int nitems_all = 0;
  };
  std::vector<Lev> L;
  BCoarse *C = nullptr;  // device, one per slice
  float *V = nullptr, *lam = nullptr;
  int depth_max = 0;
  float *bf = nullptr;                            // fine right-hand side
  float *ph[2] = {nullptr, nullptr}, *pl[2] = {nullptr, nullptr};  // float-pair iterates (ping-pong)
  int cur = 0;                                    // pair holding the iterate
  double *acc = nullptr;    // device [2 ns]
  double *h_acc = nullptr;  // pinned
  float *stage[4] = {nullptr, nullptr, nullptr, nullptr};  // I0, I1, x0, I2 of host callers
  // graph of one V-cycle (+ the residual sums) for (nu1, nu2)
  cudaGraphExec_t gexec = nullptr;
  int g_nu1 = -1, g_nu2 = -1;
  long long launches = 0;
  long long g_launches = 0;
  int occ_sweep = 1, occ_aux = 1;
  std::string err;
};

namespace {

// message of the last gd_batch_create that failed in this thread
thread_local std::string g_create_err;

void bset_err(gd_batch *b, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
}

#define BCK(call)                                                                     \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) {                                                          \
      bset_err(B, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__,   \
               __LINE__);                                                             \
      return GD_ERR_CUDA;                                                             \
    }                                                                                 \
  } while (0)

template <typename T>
int balloc(gd_batch *B, T **p, size_t n) {
  *p = nullptr;
  if (n == 0) return GD_OK;
  if (cudaMalloc((void **)p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    bset_err(B, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    return GD_ERR_OOM;
  }
  return GD_OK;
}

void batch_free(gd_batch *B) {
  if (B->gexec) cudaGraphExecDestroy(B->gexec);
  for (auto &l : B->L) {
    cudaFree(l.x);
    cudaFree(l.t);
    cudaFree(l.b);
    cudaFree(l.E);
    cudaFree(l.items);
    cudaFree(l.items_all);
  }
  cudaFree(B->C);
  cudaFree(B->V);
  cudaFree(B->lam);
  cudaFree(B->acc);
  cudaFree(B->bf);
  for (int k = 0; k < 2; ++k) {
    cudaFree(B->ph[k]);
    cudaFree(B->pl[k]);
  }
  if (B->h_acc) cudaFreeHost(B->h_acc);
  for (auto &p : B->stage) cudaFree(p);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
}

bool dev_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct SliceLevel {
  int nx, ny, sx, sy, lx, ly, fx, fy;
  double wx, wy, wm;
};

// The 2D hierarchy of one slice: the stack planner's rule with no z axis.
// An axis is halved (n_c = ceil(n/2)) when n >= 2 cxy and its interior
// coupling w_d s_e is at least half the largest; stiffness w_d halves per
// coarsening of axis d, masses are the children counts.
std::vector<SliceLevel> slice_levels(int nx, int ny, double alpha, int cxy) {
  std::vector<SliceLevel> v;
  SliceLevel l{nx, ny, 1, 1, 1, 1, 0, 0, 1.0, 1.0, alpha};
  for (int guard = 0; guard < 64; ++guard) {
    const bool can[2] = {l.nx >= 2 * cxy, l.ny >= 2 * cxy};
    const double c[2] = {l.wx * l.sy, l.wy * l.sx};
    const double cm = std::fmax(c[0], c[1]);
    l.fx = can[0] && c[0] >= 0.5 * cm;
    l.fy = can[1] && c[1] >= 0.5 * cm;
    v.push_back(l);
    if (!l.fx && !l.fy) break;
    SliceLevel n = l;
    n.fx = n.fy = 0;
    if (l.fx) {
      n.nx = (l.nx + 1) / 2;
      n.sx = 2 * l.sx;
      n.lx = (l.nx % 2 == 0) ? l.sx + l.lx : l.lx;
      n.wx = 0.5 * l.wx;
    }
    if (l.fy) {
      n.ny = (l.ny + 1) / 2;
      n.sy = 2 * l.sy;
      n.ly = (l.ny % 2 == 0) ? l.sy + l.ly : l.ly;
      n.wy = 0.5 * l.wy;
    }
    l = n;
  }
  return v;
}

void tiles_of(int e, int nx, int ny, std::vector<int4> &out) {
  for (int j0 = 0; j0 < ny; j0 += BY)
    for (int i0 = 0; i0 < nx; i0 += BX) out.push_back(make_int4(e, i0, j0, 0));
}

int grid_for(gd_batch *B, int nitems, int occ) {
  const int g = B->sm_count * std::max(occ, 1);
  return std::max(1, std::min(nitems, g));
}

// One V(nu1, nu2) cycle on the correction equation A e = r: r in L[0].b,
// e (from zero) into L[0].x.  nu1 + nu2 is even, so every level's iterate
// ends in its x buffer.
int bvcycle(gd_batch *B, int nu1, int nu2, cudaStream_t st) {
  const int D = (int)B->L.size();
  std::vector<float *> cur(D, nullptr);
  // descent
  for (int l = 0; l < D; ++l) {
    gd_batch::Lev &v = B->L[l];
    if (v.nitems == 0) continue;  // every slice of this depth is at its coarsest level
    cur[l] = v.x;
    const int g = grid_for(B, v.nitems, B->occ_sweep);
    for (int k = 0; k < nu1; ++k) {
      const bool zero = k == 0;
      float *out = (cur[l] == v.x) ? v.t : v.x;
      if (zero)
        k_bsweep<true, false><<<g, BNT, 0, st>>>(v.E, v.items, v.nitems, nullptr, v.b, out, nullptr);
      else
        k_bsweep<false, false><<<g, BNT, 0, st>>>(v.E, v.items, v.nitems, cur[l], v.b, out, nullptr);
      ++B->launches;
      cur[l] = out;
    }
    k_brestrict<<<grid_for(B, v.nitems, B->occ_aux), BNT, 0, st>>>(v.E, v.items, v.nitems, cur[l], v.b,
                                                                  B->L[l + 1].b);
    ++B->launches;
  }
  // coarsest levels
  BLevelPtrs P;
  std::memset(&P, 0, sizeof P);
  for (int l = 0; l < D && l < kBMaxLev; ++l) {
    P.b[l] = B->L[l].b;
    P.x[l] = B->L[l].x;
  }
  k_bfdm<<<std::min(B->ns, B->sm_count * 4), BNT, 2 * kFdmMaxCells * sizeof(float), st>>>(B->C, B->ns, B->V,
                                                                                         B->lam, P);
  ++B->launches;
  // ascent
  for (int l = D - 1; l >= 0; --l) {
    gd_batch::Lev &v = B->L[l];
    if (v.nitems == 0) continue;
    const int g = grid_for(B, v.nitems, B->occ_sweep);
    for (int k = 0; k < nu2; ++k) {
      float *out = (cur[l] == v.x) ? v.t : v.x;
      if (k == 0)
        k_bsweep<false, true><<<g, BNT, 0, st>>>(v.E, v.items, v.nitems, cur[l], v.b, out, B->L[l + 1].x);
      else
        k_bsweep<false, false><<<g, BNT, 0, st>>>(v.E, v.items, v.nitems, cur[l], v.b, out, nullptr);
      ++B->launches;
      cur[l] = out;
    }
  }
  BCK(cudaGetLastError());
  return GD_OK;
}

// Outer pass: pair cur (+ e) -> pair 1 - cur, r = bf - A x into L[0].b and
// the per-slice sums into acc.
int outer_pass(gd_batch *B, bool add_e) {
  gd_batch::Lev &f = B->L[0];
  const int a = B->cur, o = 1 - B->cur;
  BCK(cudaMemsetAsync(B->acc, 0, 2 * B->ns * sizeof(double), B->stream));
  const int g = grid_for(B, f.nitems_all, B->occ_aux);
  if (add_e)
    k_bouter<true><<<g, BNT, 0, B->stream>>>(f.E, f.items_all, f.nitems_all, B->bf, B->ph[a], B->pl[a], f.x,
                                             B->ph[o], B->pl[o], f.b, B->acc);
  else
    k_bouter<false><<<g, BNT, 0, B->stream>>>(f.E, f.items_all, f.nitems_all, B->bf, B->ph[a], B->pl[a],
                                              nullptr, B->ph[o], B->pl[o], f.b, B->acc);
  ++B->launches;
  BCK(cudaGetLastError());
  B->cur = o;
  return GD_OK;
}

// Reads the per-slice sums: max over slices of ||r_s|| / ||b_s|| and the
// total ||b||.
int read_rel(gd_batch *B, double *rel_max, double *bnorm, double *slice_rel) {
  BCK(cudaMemcpyAsync(B->h_acc, B->acc, 2 * B->ns * sizeof(double), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  double m = 0.0, bb = 0.0;
  for (int s = 0; s < B->ns; ++s) {
    const double r2 = B->h_acc[2 * s], b2 = B->h_acc[2 * s + 1];
    const double rel = b2 > 0.0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
    if (slice_rel) slice_rel[s] = rel;
    m = std::isnan(rel) ? rel : (std::isnan(m) ? m : std::fmax(m, rel));
    bb += b2;
  }
  *rel_max = m;
  *bnorm = std::sqrt(bb);
  return GD_OK;
}

int ensure_graph(gd_batch *B, int nu1, int nu2) {
  if (B->gexec && B->g_nu1 == nu1 && B->g_nu2 == nu2) return GD_OK;
  if (B->gexec) {
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
  }
  if (!B->cap_stream) BCK(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  const long long l0 = B->launches;
  BCK(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int st = bvcycle(B, nu1, nu2, B->cap_stream);
  cudaError_t e = cudaStreamEndCapture(B->cap_stream, &graph);
  B->g_launches = B->launches - l0;
  B->launches = l0;
  if (st != GD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) {
    bset_err(B, "graph capture failed: %s", cudaGetErrorString(e));
    return GD_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&B->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B->gexec = nullptr;
    bset_err(B, "graph instantiation failed: %s", cudaGetErrorString(e));
    return GD_ERR_CUDA;
  }
  B->g_nu1 = nu1;
  B->g_nu2 = nu2;
  return GD_OK;
}

int batch_build(gd_batch *B) {
  const int ns = B->ns;
  std::vector<std::vector<SliceLevel>> H(ns);
  int D = 0;
  for (int s = 0; s < ns; ++s) {
    H[s] = slice_levels(B->nx[s], B->ny[s], B->alpha[s], B->cxy);
    D = std::max(D, (int)H[s].size());
    const SliceLevel &c = H[s].back();
    if ((long long)c.nx * c.ny > kFdmMaxCells) {
      bset_err(B, "slice %d (%d x %d): its coarsest level has %d x %d cells, above the %d the "
                  "batched direct solve takes (aspect ratio too large)",
               s, B->nx[s], B->ny[s], c.nx, c.ny, kFdmMaxCells);
      return GD_ERR_UNSUPPORTED;
    }
  }
  if (D > kBMaxLev) {
    bset_err(B, "too many levels (%d)", D);
    return GD_ERR_UNSUPPORTED;
  }
  B->depth_max = D;
  B->L.assign(D, gd_batch::Lev());
  // per level: entries (slices that reach it) and packed offsets
  std::vector<std::vector<BEntry>> E(D);
  std::vector<std::vector<int>> eidx(ns, std::vector<int>());
  for (int l = 0; l < D; ++l) {
    long long o = 0;
    for (int s = 0; s < ns; ++s) {
      if (l >= (int)H[s].size()) continue;
      const SliceLevel &v = H[s][l];
      BEntry e;
      std::memset(&e, 0, sizeof e);
      e.off = o;
      e.coff = -1;
      e.nx = v.nx;
      e.ny = v.ny;
      e.sx = v.sx;
      e.sy = v.sy;
      e.lx = v.lx;
      e.ly = v.ly;
      e.fx = v.fx;
      e.fy = v.fy;
      e.wx = (float)v.wx;
      e.wy = (float)v.wy;
      e.wm = (float)v.wm;
      e.slice = s;
      eidx[s].push_back((int)E[l].size());
      E[l].push_back(e);
      o += (long long)v.nx * v.ny;
    }
    B->L[l].n = o;
  }
  for (int s = 0; s < ns; ++s)
    for (size_t l = 0; l + 1 < H[s].size(); ++l) {
      BEntry &e = E[l][eidx[s][l]];
      const BEntry &c = E[l + 1][eidx[s][l + 1]];
      e.coff = c.off;
      e.cnx = c.nx;
      e.cny = c.ny;
    }
  // work lists and buffers
  int st;
  for (int l = 0; l < D; ++l) {
    gd_batch::Lev &v = B->L[l];
    std::vector<int4> it, all;
    for (int k = 0; k < (int)E[l].size(); ++k) {
      const BEntry &e = E[l][k];
      if (e.coff >= 0) tiles_of(k, e.nx, e.ny, it);
      if (l == 0) tiles_of(k, e.nx, e.ny, all);
    }
    v.ne = (int)E[l].size();
    v.nitems = (int)it.size();
    v.nitems_all = (int)all.size();
    if ((st = balloc(B, &v.x, (size_t)v.n)) != GD_OK) return st;
    if ((st = balloc(B, &v.b, (size_t)v.n)) != GD_OK) return st;
    if (v.nitems > 0 && (st = balloc(B, &v.t, (size_t)v.n)) != GD_OK) return st;
    if ((st = balloc(B, &v.E, E[l].size())) != GD_OK) return st;
    if ((st = balloc(B, &v.items, it.size())) != GD_OK) return st;
    if ((st = balloc(B, &v.items_all, all.size())) != GD_OK) return st;
    BCK(cudaMemcpy(v.E, E[l].data(), E[l].size() * sizeof(BEntry), cudaMemcpyHostToDevice));
    if (!it.empty()) BCK(cudaMemcpy(v.items, it.data(), it.size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (!all.empty())
      BCK(cudaMemcpy(v.items_all, all.data(), all.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  const size_t n0 = (size_t)B->L[0].n;
  if ((st = balloc(B, &B->bf, n0)) != GD_OK) return st;
  for (int k = 0; k < 2; ++k) {
    if ((st = balloc(B, &B->ph[k], n0)) != GD_OK) return st;
    if ((st = balloc(B, &B->pl[k], n0)) != GD_OK) return st;
  }
  // coarsest levels: eigen-decompositions shared by equal (n, s, l) axes
  std::map<std::tuple<int, int, int>, std::pair<int, int>> cache;  // -> (V offset, lambda offset)
  std::vector<float> Vt, Lt;
  auto axis = [&](int n, int sfac, int last) {
    auto key = std::make_tuple(n, sfac, last);
    auto f = cache.find(key);
    if (f != cache.end()) return f->second;
    std::vector<float> V;
    std::vector<double> lam;
    axis_eig(n, sfac, last, V, lam);
    std::pair<int, int> r((int)Vt.size(), (int)Lt.size());
    Vt.insert(Vt.end(), V.begin(), V.end());
    for (double x : lam) Lt.push_back((float)x);
    cache[key] = r;
    return r;
  };
  std::vector<BCoarse> C(ns);
  for (int s = 0; s < ns; ++s) {
    const int l = (int)H[s].size() - 1;
    const SliceLevel &v = H[s][l];
    const BEntry &e = E[l][eidx[s][l]];
    const auto ax = axis(v.nx, v.sx, v.lx);
    const auto ay = axis(v.ny, v.sy, v.ly);
    C[s] = BCoarse{l, v.nx, v.ny, ax.first, ay.first, ax.second, ay.second,
                   (float)v.wx, (float)v.wy, (float)v.wm, e.off};
  }
  if ((st = balloc(B, &B->C, C.size())) != GD_OK) return st;
  if ((st = balloc(B, &B->V, Vt.size())) != GD_OK) return st;
  if ((st = balloc(B, &B->lam, Lt.size())) != GD_OK) return st;
  BCK(cudaMemcpy(B->C, C.data(), C.size() * sizeof(BCoarse), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(B->V, Vt.data(), Vt.size() * sizeof(float), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(B->lam, Lt.data(), Lt.size() * sizeof(float), cudaMemcpyHostToDevice));
  if ((st = balloc(B, &B->acc, 2 * (size_t)ns)) != GD_OK) return st;
  if (cudaMallocHost((void **)&B->h_acc, 2 * (size_t)ns * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    B->h_acc = nullptr;
    bset_err(B, "pinned allocation failed");
    return GD_ERR_OOM;
  }
  BCK(cudaFuncSetAttribute(k_bfdm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(2 * kFdmMaxCells * sizeof(float))));
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, dev));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_sweep, k_bsweep<false, true>, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_aux, k_bouter<true>, BNT, 0));
  return GD_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gd_batch_create(gd_batch **out, int nslices, const int *nx, const int *ny, const double *alpha,
                    int coarsest_xy, void *stream) {
  g_create_err.clear();
  if (!out) return GD_ERR_INVALID_ARG;
  *out = nullptr;
  if (nslices < 1 || !nx || !ny || !alpha) {
    g_create_err = "nslices >= 1 and the nx, ny and alpha arrays are required";
    return GD_ERR_INVALID_ARG;
  }
  if (coarsest_xy == 0) coarsest_xy = 16;
  if (coarsest_xy < 2 || coarsest_xy > 4096) {
    g_create_err = "coarsest_xy must be 0 or in [2, 4096]";
    return GD_ERR_INVALID_ARG;
  }
  long long tot = 0;
  for (int s = 0; s < nslices; ++s) {
    if (nx[s] < 1 || ny[s] < 1 || nx[s] > (1 << 20) || ny[s] > (1 << 20)) {
      g_create_err = "slice " + std::to_string(s) + ": sizes must be in [1, 2^20]";
      return GD_ERR_INVALID_ARG;
    }
    if (!(std::isfinite(alpha[s]) && alpha[s] > 0.0)) {
      g_create_err = "slice " + std::to_string(s) + ": alpha must be finite and > 0";
      return GD_ERR_INVALID_ARG;
    }
    tot += (long long)nx[s] * ny[s];
  }
  std::unique_ptr<gd_batch> B(new gd_batch);
  B->ns = nslices;
  B->nx.assign(nx, nx + nslices);
  B->ny.assign(ny, ny + nslices);
  B->alpha.assign(alpha, alpha + nslices);
  B->off.resize(nslices);
  long long o = 0;
  for (int s = 0; s < nslices; ++s) {
    B->off[s] = o;
    o += (long long)nx[s] * ny[s];
  }
  B->nvox = tot;
  B->cxy = coarsest_xy;
  B->stream = static_cast<cudaStream_t>(stream);
  const int st = batch_build(B.get());
  if (st != GD_OK) {
    g_create_err = B->err;
    batch_free(B.get());
    return st;
  }
  *out = B.release();
  return GD_OK;
}

long long gd_batch_voxels(const gd_batch *b) { return b ? b->nvox : -1; }

long long gd_batch_offset(const gd_batch *b, int slice) {
  if (!b || slice < 0 || slice >= b->ns) return -1;
  return b->off[slice];
}

int gd_batch_levels(const gd_batch *b) { return b ? b->depth_max : -1; }

long long gd_batch_launch_count(const gd_batch *b) { return b ? b->launches : -1; }

const char *gd_batch_last_error(const gd_batch *b) { return b ? b->err.c_str() : g_create_err.c_str(); }

int gd_batch_screened_poisson(gd_batch *B, const float *I0, const float *I1, float *I2,
                              const gd_solve_ctl *ctl, const float *x0, gd_report *rep,
                              double *slice_rel) {
  if (rep) {
    std::memset(rep, 0, sizeof *rep);
    rep->rel_residual_out = NAN;
  }
  if (!B) return GD_ERR_INVALID_ARG;
  if (!I0 || !I1 || !I2) {
    bset_err(B, "I0, I1 and I2 are required");
    if (rep) rep->status = GD_ERR_INVALID_ARG;
    return GD_ERR_INVALID_ARG;
  }
  gd_solve_ctl c = {20, 1e-6, 2, 2, 0, 0};
  if (ctl) c = *ctl;
  if (c.max_cycles < 0 || c.nu1 < 1 || c.nu1 > 8 || c.nu2 < 1 || c.nu2 > 8 || ((c.nu1 + c.nu2) & 1) ||
      !(c.rel_tol >= 0.0) || (c.rel_tol <= 0.0 && c.max_cycles <= 0) ||
      (c.coarsest_xy != 0 && c.coarsest_xy != B->cxy)) {
    bset_err(B, "invalid solve control (max_cycles %d, rel_tol %g, nu1 %d, nu2 %d: nu1 + nu2 must be "
                "even; coarsest_xy %d: 0 or the batch's %d)",
             c.max_cycles, c.rel_tol, c.nu1, c.nu2, c.coarsest_xy, B->cxy);
    if (rep) rep->status = GD_ERR_INVALID_ARG;
    return GD_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)B->nvox;
  // device views of the caller's arrays (host arrays are staged)
  const float *in[3] = {I0, I1, x0};
  const float *dv[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k) {
    if (!in[k]) continue;
    if (dev_ptr(in[k])) {
      dv[k] = in[k];
      continue;
    }
    if (!B->stage[k]) {
      const int st = balloc(B, &B->stage[k], n);
      if (st != GD_OK) return st;
    }
    BCK(cudaMemcpyAsync(B->stage[k], in[k], n * sizeof(float), cudaMemcpyHostToDevice, B->stream));
    dv[k] = B->stage[k];
  }
  gd_batch::Lev &f = B->L[0];
  B->cur = 0;
  k_brhs<<<grid_for(B, f.nitems_all, B->occ_aux), BNT, 0, B->stream>>>(f.E, f.items_all, f.nitems_all, dv[0],
                                                                       dv[1], dv[2], B->bf, B->ph[0], B->pl[0]);
  ++B->launches;
  BCK(cudaGetLastError());
  int st = outer_pass(B, false);
  if (st != GD_OK) return st;
  double rel = 0.0, bn = 0.0;
  if ((st = read_rel(B, &rel, &bn, slice_rel)) != GD_OK) return st;
  if (rep) {
    rep->levels = B->depth_max;
    rep->rhs_norm = bn;
    rep->history[0] = rel;
  }
  const double rel0 = rel;
  int cycles = 0;
  int status = GD_OK;
  if ((st = ensure_graph(B, c.nu1, c.nu2)) != GD_OK) return st;
  while (!(rel <= c.rel_tol) && cycles < c.max_cycles) {
    BCK(cudaGraphLaunch(B->gexec, B->stream));
    B->launches += B->g_launches;
    if ((st = outer_pass(B, true)) != GD_OK) return st;
    ++cycles;
    if ((st = read_rel(B, &rel, &bn, slice_rel)) != GD_OK) return st;
    if (rep && cycles < GD_HISTORY) rep->history[cycles] = rel;
    if (!std::isfinite(rel)) {
      status = GD_ERR_DIVERGED;
      bset_err(B, "the residual is not finite after cycle %d", cycles);
      break;
    }
  }
  if (status == GD_OK && !(rel <= c.rel_tol)) {
    status = GD_ERR_NOT_CONVERGED;
    bset_err(B, "relative residual %.3g after %d cycles (tolerance %.3g)", rel, cycles, c.rel_tol);
  }
  // result: the pair rounded to float32
  float *out = dev_ptr(I2) ? I2 : nullptr;
  if (!out) {
    if (!B->stage[3]) {
      if ((st = balloc(B, &B->stage[3], n)) != GD_OK) return st;
    }
    out = B->stage[3];
  }
  k_bfinal<<<B->sm_count * 8, 256, 0, B->stream>>>(out, B->ph[B->cur], B->pl[B->cur], (long long)n);
  ++B->launches;
  BCK(cudaGetLastError());
  if (out != I2) BCK(cudaMemcpyAsync(I2, out, n * sizeof(float), cudaMemcpyDeviceToHost, B->stream));
  BCK(cudaStreamSynchronize(B->stream));
  if (rep) {
    rep->status = status;
    rep->cycles = cycles;
    rep->rel_residual = rel;
    rep->rho_per_cycle = (cycles > 0 && rel0 > 0.0) ? std::pow(rel / rel0, 1.0 / cycles) : NAN;
  }
  return status;
}

int gd_batch_destroy(gd_batch *b) {
  if (!b) return GD_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return GD_OK;
}

}  // extern "C"
