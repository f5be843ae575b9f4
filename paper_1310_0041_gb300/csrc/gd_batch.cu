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
// Internal layout: every slice level is stored with a row pitch rounded up
// to 4 floats (rows and slices 16-byte aligned); the padding cells hold 0.
//
// The level kernels are row marches by one warp over a strip of 128 columns:
// lane l holds the float4 of columns x0 - 4 + 4 l, lanes 1..30 own the 120
// columns x0 .. x0 + 119 and lanes 0 and 31 carry the halo (their cells are
// computed, never stored).  The warp walks down a chunk of rows keeping the
// previous rows in registers: no shared memory, no CTA barrier.
constexpr int BNT = 256;  // threads per CTA
constexpr int WPB = BNT / 32;
constexpr int SW = 120;   // owned columns of a strip
constexpr int CH = 64;    // default rows of a chunk (even; gd_batch_tune picks another)
constexpr int TX = 64, TY = 32;  // tiles of the element-wise kernels
constexpr int kBMaxLev = 24;
constexpr int kFdmMaxCells = 4096;
constexpr unsigned FULL = 0xffffffffu;

// One slice at one level.  The level operator is the Kronecker form of the
// stack solver restricted to a slice:
//   A = wx Kx (x) My + wy Mx (x) Ky + wm Mx (x) My,
// M = diag(children counts, s inside and l for the last cell of an axis).
struct BEntry {
  long long off;   // first element of the slice in this level's buffer
  long long coff;  // the same in the next level's buffer (-1: coarsest level)
  long long uoff;  // level 0: first element of the slice in the caller's packed arrays
  int nx, ny, pitch;
  int sx, sy, lx, ly;
  int cnx, cny, cpitch, fx, fy;  // next level and the axes halved to reach it
  float wx, wy, wm;
  int slice;
};

struct BCoarse {  // coarsest level of one slice
  int lev;        // its depth
  int nx, ny, pitch;
  int vx, vy;     // offsets of Vx, Vy in the V table
  int lx, ly;     // offsets of the eigenvalues in the lambda table
  float wx, wy, wm;
  long long off;  // first element in the level's buffer
};

struct BLevelPtrs {
  const float *b[kBMaxLev];
  float *x[kBMaxLev];
};

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ float4 f4(float a) { return make_float4(a, a, a, a); }
__device__ __forceinline__ float cmp(const float4 &v, int c) {
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
__device__ __forceinline__ void set(float4 &v, int c, float a) {
  if (c == 0) v.x = a;
  else if (c == 1) v.y = a;
  else if (c == 2) v.z = a;
  else v.w = a;
}

// The lane's four columns: inside flags, masses along x and x-neighbour counts.
struct Cols {
  int gi;     // first column
  bool mem;   // the float4 lies inside the row pitch
  bool own;   // and the lane owns it (lanes 1..30)
  bool in[4];
  float mx[4], nbx[4];
  __device__ __forceinline__ Cols(const BEntry &e, int x0, int lane) {
    gi = x0 - 4 + 4 * lane;
    mem = gi >= 0 && gi < e.pitch;
    own = mem && lane >= 1 && lane <= 30;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = gi + c;
      in[c] = i >= 0 && i < e.nx;
      mx[c] = (i == e.nx - 1) ? (float)e.lx : (float)e.sx;
      nbx[c] = (float)((i > 0) + (i < e.nx - 1));
    }
  }
  __device__ __forceinline__ float4 mask(float4 v) const {
    return make_float4(in[0] ? v.x : 0.f, in[1] ? v.y : 0.f, in[2] ? v.z : 0.f, in[3] ? v.w : 0.f);
  }
};

// Couplings of row t: cx to each x-neighbour; per cell cy = wy mx and the
// diagonal cx nbx + cy nby + wm mx my.
struct RowK {
  float cx, my, nby;
  __device__ __forceinline__ RowK(const BEntry &e, int t) {
    my = (t == e.ny - 1) ? (float)e.ly : (float)e.sy;
    cx = e.wx * my;
    nby = (float)((t > 0) + (t < e.ny - 1));
  }
};

// Gauss-Seidel value of cell c of a row: (b + cx (l + r) + cy (u + d)) / diag.
__device__ __forceinline__ float relax(const BEntry &e, const Cols &C, const RowK &k, int c, float bv,
                                       float lr, float ud) {
  const float cy = e.wy * C.mx[c];
  const float dg = k.cx * C.nbx[c] + cy * k.nby + e.wm * C.mx[c] * k.my;
  return __fdividef(bv + k.cx * lr + cy * ud, dg);
}

// Residual b - A x at cell c of a row.
__device__ __forceinline__ float resid(const BEntry &e, const Cols &C, const RowK &k, int c, float bv,
                                       float xv, float lr, float ud) {
  const float cy = e.wy * C.mx[c];
  const float dg = k.cx * C.nbx[c] + cy * k.nby + e.wm * C.mx[c] * k.my;
  return bv - (dg * xv - k.cx * lr - cy * ud);
}

// One red-black Gauss-Seidel sweep, xin -> xout, over the strip items
// (entry, x0, ys, ye).  Red cells are (i + j) even.  At step t the warp
// relaxes the red cells of row t (from the old black values of rows t-1,
// t, t+1) and then the black cells of row t-1 (from the new red values of
// rows t-2, t-1, t), which completes row t-1.  Rows ys-1 and ye get their
// red pass only (the chunk's halo rows); a red value depends only on old
// black values, so neighbouring chunks and strips compute the same ones.
// ZERO_IN: the input is 0.  PROLONG: the input is xin plus the next level's
// value of each cell's parent (piecewise-constant prolongation).
template <bool ZERO_IN, bool PROLONG>
__global__ void __launch_bounds__(BNT) k_bsweep(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                const int *__restrict__ nitems_p, const float *__restrict__ xin,
                                                const float *__restrict__ b, float *__restrict__ xout,
                                                const float *__restrict__ xc) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * WPB;
  const int nitems = *nitems_p;  // read at run time: the list shrinks as slices converge
  for (int it = blockIdx.x * WPB + (threadIdx.x >> 5); it < nitems; it += nw) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int ys = w.z, ye = w.w, ny = e.ny;
    const Cols C(e, w.y, lane);
    const long long rb = e.off + C.gi;
    // raw rows of x and their parents' values (PROLONG); the sum is formed
    // when a row enters the window, so the loads of a row stay in flight
    // for a step
    auto ldx = [&](int t) -> float4 {
      return (!ZERO_IN && t >= 0 && t < ny && C.mem) ? ld4(xin + rb + (long long)t * e.pitch) : f4(0.f);
    };
    auto ldc = [&](int t) -> float4 {
      if (!PROLONG || t < 0 || t >= ny || !C.mem) return f4(0.f);
      const float *cp = xc + e.coff + (long long)(t >> e.fy) * e.cpitch;
      if (e.fx) {
        const float2 c = ld2(cp + (C.gi >> 1));
        return make_float4(c.x, c.x, c.y, c.y);
      }
      return ld4(cp + C.gi);
    };
    auto corr = [&](float4 v, float4 c) -> float4 {
      if (!PROLONG) return v;
      return C.mask(make_float4(v.x + c.x, v.y + c.y, v.z + c.z, v.w + c.w));
    };
    auto ldb = [&](int t) -> float4 {
      return (t >= 0 && t < ny && C.mem) ? ld4(b + rb + (long long)t * e.pitch) : f4(0.f);
    };
    float4 xm2 = f4(0.f), xm1 = corr(ldx(ys - 2), ldc(ys - 2)), xcur = corr(ldx(ys - 1), ldc(ys - 1));
    float4 xp1 = corr(ldx(ys), ldc(ys)), xp2 = ldx(ys + 1), cp2 = ldc(ys + 1);
    float4 bm1 = f4(0.f), b0 = ldb(ys - 1), bp1 = ldb(ys);
    for (int t = ys - 1; t <= ye; ++t) {
      // row t + 3 reuses its parents' row when the pair's first row had it
      const float4 xn = ldx(t + 3), bn = ldb(t + 2);
      const float4 cn = (PROLONG && e.fy && ((t + 3) & 1) && t + 3 < ny) ? cp2 : ldc(t + 3);
      // red cells of row t
      float4 xr = xcur;
      if (t >= 0 && t < ny) {
        const RowK k(e, t);
        const float lw = __shfl_up_sync(FULL, xcur.w, 1), rx = __shfl_down_sync(FULL, xcur.x, 1);
        if ((t & 1) == 0) {
          xr.x = relax(e, C, k, 0, b0.x, lw + xcur.y, xm1.x + xp1.x);
          xr.z = relax(e, C, k, 2, b0.z, xcur.y + xcur.w, xm1.z + xp1.z);
        } else {
          xr.y = relax(e, C, k, 1, b0.y, xcur.x + xcur.z, xm1.y + xp1.y);
          xr.w = relax(e, C, k, 3, b0.w, xcur.z + rx, xm1.w + xp1.w);
        }
        xr = C.mask(xr);
      }
      // black cells of row t - 1, which is then complete
      const int j = t - 1;
      float4 xb = xm1;
      if (j >= ys && j < ye) {
        const RowK k(e, j);
        const float lw = __shfl_up_sync(FULL, xm1.w, 1), rx = __shfl_down_sync(FULL, xm1.x, 1);
        if ((j & 1) != 0) {
          xb.x = relax(e, C, k, 0, bm1.x, lw + xm1.y, xm2.x + xr.x);
          xb.z = relax(e, C, k, 2, bm1.z, xm1.y + xm1.w, xm2.z + xr.z);
        } else {
          xb.y = relax(e, C, k, 1, bm1.y, xm1.x + xm1.z, xm2.y + xr.y);
          xb.w = relax(e, C, k, 3, bm1.w, xm1.z + rx, xm2.w + xr.w);
        }
        xb = C.mask(xb);
        if (C.own) st4(xout + rb + (long long)j * e.pitch, xb);
      }
      xm2 = xb;
      xm1 = xr;
      xcur = xp1;
      xp1 = corr(xp2, cp2);
      xp2 = xn;
      cp2 = cn;
      bm1 = b0;
      b0 = bp1;
      bp1 = bn;
    }
  }
}

// Residual of x summed over each coarse cell's children into the next
// level's right-hand side (restriction = transpose of the prolongation).
// Chunks start at even rows and strips at even columns, so a coarse cell's
// children lie in one lane's float4 and one chunk.
__global__ void __launch_bounds__(BNT) k_brestrict(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                   const int *__restrict__ nitems_p, const float *__restrict__ x,
                                                   const float *__restrict__ b, float *__restrict__ bc) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * WPB;
  const int nitems = *nitems_p;
  for (int it = blockIdx.x * WPB + (threadIdx.x >> 5); it < nitems; it += nw) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int ys = w.z, ye = w.w, ny = e.ny;
    const Cols C(e, w.y, lane);
    const long long rb = e.off + C.gi;
    auto ldx = [&](int t) -> float4 {
      return (t >= 0 && t < ny && C.mem) ? ld4(x + rb + (long long)t * e.pitch) : f4(0.f);
    };
    auto ldb = [&](int t) -> float4 {
      return (t >= 0 && t < ny && C.mem) ? ld4(b + rb + (long long)t * e.pitch) : f4(0.f);
    };
    float4 xm = ldx(ys - 1), xcur = ldx(ys), xp = ldx(ys + 1), xpp = ldx(ys + 2);
    float4 b0 = ldb(ys), bp = ldb(ys + 1);
    float4 acc = f4(0.f);
    for (int t = ys; t < ye; ++t) {
      const float4 xn = ldx(t + 3), bn = ldb(t + 2);
      const RowK k(e, t);
      const float lw = __shfl_up_sync(FULL, xcur.w, 1), rx = __shfl_down_sync(FULL, xcur.x, 1);
      float4 r;
      r.x = resid(e, C, k, 0, b0.x, xcur.x, lw + xcur.y, xm.x + xp.x);
      r.y = resid(e, C, k, 1, b0.y, xcur.y, xcur.x + xcur.z, xm.y + xp.y);
      r.z = resid(e, C, k, 2, b0.z, xcur.z, xcur.y + xcur.w, xm.z + xp.z);
      r.w = resid(e, C, k, 3, b0.w, xcur.w, xcur.z + rx, xm.w + xp.w);
      r = C.mask(r);
      const bool first = e.fy && (t & 1) == 0;
      acc.x += r.x;
      acc.y += r.y;
      acc.z += r.z;
      acc.w += r.w;
      if (!first || t == ny - 1) {
        if (C.own) {
          float *cp = bc + e.coff + (long long)(t >> e.fy) * e.cpitch;
          if (e.fx)
            st2(cp + (C.gi >> 1), make_float2(acc.x + acc.y, acc.z + acc.w));
          else
            st4(cp + C.gi, acc);
        }
        acc = f4(0.f);
      }
      xm = xcur;
      xcur = xp;
      xp = xpp;
      xpp = xn;
      b0 = bp;
      bp = bn;
    }
  }
}

// Error-free transformation (Knuth's TwoSum): s + e == a + b exactly.
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
// masses and stiffness, A = alpha + Kx + Ky): (h, l) <- (h, l) + e (ADD_E;
// from the input pair to the output pair, never in place, since
// neighbouring strips read this strip's cells), then r = bf - A (h + l) with
// every rounding error of the high parts captured, written as the
// correction's right-hand side, and the per-slice sums of r^2 and bf^2 (FP64
// slots acc[2 s], acc[2 s + 1]; lanes sum in FP32, the warp in FP64).
// PAIR = false while the residual is large: the low words are neither read
// nor written (both buffers' low words are still zero then), h += e is a
// plain FP32 add and its rounding stays far below the residual.
template <bool ADD_E, bool PAIR = true>
__global__ void __launch_bounds__(BNT) k_bouter(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                int nitems, const float *__restrict__ bf,
                                                const float *__restrict__ hin, const float *__restrict__ lin,
                                                const float *__restrict__ ein, float *__restrict__ hout,
                                                float *__restrict__ lout, float *__restrict__ r,
                                                double *__restrict__ acc) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * WPB;
  for (int it = blockIdx.x * WPB + (threadIdx.x >> 5); it < nitems; it += nw) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int ys = w.z, ye = w.w, ny = e.ny;
    const Cols C(e, w.y, lane);
    const long long rb = e.off + C.gi;
    const float alpha = e.wm;
    // the updated pair of row t (0 outside)
    auto ldp = [&](int t, float4 &h, float4 &l) {
      h = l = f4(0.f);
      if (t < 0 || t >= ny || !C.mem) return;
      const long long o = rb + (long long)t * e.pitch;
      h = ld4(hin + o);
      if (PAIR) l = ld4(lin + o);
      if (ADD_E && !PAIR) {
        const float4 d = ld4(ein + o);
        h = make_float4(h.x + d.x, h.y + d.y, h.z + d.z, h.w + d.w);
      } else if (ADD_E) {
        const float4 d = ld4(ein + o);
        float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
        const float dv[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const ff a = two_sum(hv[c], dv[c]);
          const ff s = two_sum(a.h, __fadd_rn(a.l, lv[c]));
          hv[c] = s.h;
          lv[c] = s.l;
        }
        h = make_float4(hv[0], hv[1], hv[2], hv[3]);
        l = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
    };
    auto ldb = [&](int t) -> float4 {
      return (t >= 0 && t < ny && C.mem) ? ld4(bf + rb + (long long)t * e.pitch) : f4(0.f);
    };
    float4 hm, lm, hc, lc, hp, lp;
    ldp(ys - 1, hm, lm);
    ldp(ys, hc, lc);
    ldp(ys + 1, hp, lp);
    float4 b0 = ldb(ys);
    float s_rr = 0.f, s_bb = 0.f;
    for (int t = ys; t < ye; ++t) {
      float4 hn, ln;
      ldp(t + 2, hn, ln);
      const float4 bn = ldb(t + 1);
      const float hlw = __shfl_up_sync(FULL, hc.w, 1), llw = __shfl_up_sync(FULL, lc.w, 1);
      const float hrx = __shfl_down_sync(FULL, hc.x, 1), lrx = __shfl_down_sync(FULL, lc.x, 1);
      const float hcv[4] = {hc.x, hc.y, hc.z, hc.w}, lcv[4] = {lc.x, lc.y, lc.z, lc.w};
      const float hmv[4] = {hm.x, hm.y, hm.z, hm.w}, lmv[4] = {lm.x, lm.y, lm.z, lm.w};
      const float hpv[4] = {hp.x, hp.y, hp.z, hp.w}, lpv[4] = {lp.x, lp.y, lp.z, lp.w};
      const float bv4[4] = {b0.x, b0.y, b0.z, b0.w};
      float rv4[4];
      const bool up = t > 0, dn = t < ny - 1;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = C.gi + c;
        const float hcc = hcv[c], lcc = lcv[c];
        float hi = bv4[c], lo = 0.f;
        auto sub = [&](float v) {
          const ff s = two_sum(hi, -v);
          hi = s.h;
          lo += s.l;
        };
        auto nb = [&](bool has, float hn_, float ln_) {
          if (!has) return;
          const ff d = two_sum(hcc, -hn_);
          sub(d.h);
          lo -= d.l + (lcc - ln_);
        };
        nb(i > 0, c == 0 ? hlw : hcv[c - 1], c == 0 ? llw : lcv[c - 1]);
        nb(i < e.nx - 1, c == 3 ? hrx : hcv[c + 1], c == 3 ? lrx : lcv[c + 1]);
        nb(up, hmv[c], lmv[c]);
        nb(dn, hpv[c], lpv[c]);
        const float pa = alpha * hcc;
        sub(pa);
        lo -= __fmaf_rn(alpha, hcc, -pa) + alpha * lcc;
        const float rr = (C.in[c] && C.own) ? hi + lo : 0.f;
        rv4[c] = rr;
        s_rr = fmaf(rr, rr, s_rr);
        if (C.in[c] && C.own) s_bb = fmaf(bv4[c], bv4[c], s_bb);
      }
      if (C.own) {
        const long long o = rb + (long long)t * e.pitch;
        st4(r + o, make_float4(rv4[0], rv4[1], rv4[2], rv4[3]));
        st4(hout + o, C.mask(hc));
        if (PAIR) st4(lout + o, C.mask(lc));
      }
      hm = hc;
      lm = lc;
      hc = hp;
      lc = lp;
      hp = hn;
      lp = ln;
      b0 = bn;
    }
    double drr = s_rr, dbb = s_bb;
    for (int o = 16; o > 0; o >>= 1) {
      drr += __shfl_down_sync(FULL, drr, o);
      dbb += __shfl_down_sync(FULL, dbb, o);
    }
    if (lane == 0) {
      atomicAdd(&acc[2 * e.slice], drr);
      atomicAdd(&acc[2 * e.slice + 1], dbb);
    }
  }
}

// Fine right-hand side b = alpha I1 + (Kx + Ky) I0 and the initial float
// pair (x0 or I0, 0), from the caller's packed arrays to the internal
// layout; one 64 x 32 tile per item (entry, i0, j0).
__global__ void __launch_bounds__(BNT) k_brhs(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                              int nitems, const float *__restrict__ I0,
                                              const float *__restrict__ I1, const float *__restrict__ x0,
                                              float *__restrict__ b, float *__restrict__ xh,
                                              float *__restrict__ xl) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int i0 = w.y, j0 = w.z, nx = e.nx;
    for (int q = threadIdx.x; q < TX * TY; q += BNT) {
      const int gi = i0 + (q % TX), gj = j0 + q / TX;
      if (gi >= nx || gj >= e.ny) continue;
      const long long u = e.uoff + (long long)gj * nx + gi;
      const long long o = e.off + (long long)gj * e.pitch + gi;
      const float c0 = I0[u];
      float k = 0.f;
      if (gi > 0) k += c0 - I0[u - 1];
      if (gi < nx - 1) k += c0 - I0[u + 1];
      if (gj > 0) k += c0 - I0[u - nx];
      if (gj < e.ny - 1) k += c0 - I0[u + nx];
      b[o] = fmaf(e.wm, I1[u], k);
      xh[o] = x0 ? x0[u] : c0;
      xl[o] = 0.f;
    }
  }
}

// I2 = h + l rounded to float32, from the internal layout to the caller's
// packed array.
__global__ void __launch_bounds__(BNT) k_bfinal(const BEntry *__restrict__ E, const int4 *__restrict__ items,
                                                int nitems, const float *__restrict__ h0,
                                                const float *__restrict__ l0, const float *__restrict__ h1,
                                                const float *__restrict__ l1, const int *__restrict__ fin,
                                                float *__restrict__ out) {
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int4 w = items[it];
    const BEntry e = E[w.x];
    const int i0 = w.y, j0 = w.z;
    // the pair buffer holding this slice's final iterate
    const float *h = fin[e.slice] ? h1 : h0, *l = fin[e.slice] ? l1 : l0;
    for (int q = threadIdx.x; q < TX * TY; q += BNT) {
      const int gi = i0 + (q % TX), gj = j0 + q / TX;
      if (gi >= e.nx || gj >= e.ny) continue;
      const long long o = e.off + (long long)gj * e.pitch + gi;
      out[e.uoff + (long long)gj * e.nx + gi] = __fadd_rn(h[o], l[o]);
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
    for (int q = threadIdx.x; q < n; q += BNT) B[q] = bl[(q / nx) * c.pitch + q % nx];
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
      xl[j * c.pitch + i] = a;
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
  int device = 0;  // current at creation; caller device arrays must live there
  int sm_count = 0;
  // levels (packed over the slices that reach them)
  struct Lev {
    long long n = 0;
    float *x = nullptr, *t = nullptr, *b = nullptr;
    BEntry *E = nullptr;            // device
    int ne = 0;
    int4 *items = nullptr;          // strips of the entries that have a next level (active ones first)
    int nitems = 0;                 // all entries' strips (the buffer's size; the graph's grids)
    int *cnt = nullptr;             // device: strips of the active entries (read by the kernels)
    int4 *strips_all = nullptr;     // level 0: strips of every entry (outer pass), active ones first
    int nstrips_all = 0;            // of the active entries
    int nstrips_all_cap = 0;        // of every entry (the buffer's size)
    int4 *tiles_all = nullptr;      // level 0: 64 x 32 tiles of every entry (input / output)
    int ntiles_all = 0;
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
  int occ_sweep = 1, occ_aux = 1, occ_tile = 1;
  int occ_zero = 1, occ_prolong = 1, occ_restrict = 1;  // each variant's own occupancy
  std::vector<std::vector<BEntry>> Eh;  // host copies of the entries, per level
  int chunk = CH;                       // rows per work item of the row marches
  // slices still iterating (the work lists hold only theirs once some have
  // converged), their last relative residuals and squared rhs norms, and the
  // pair buffer that holds each slice's final iterate
  std::vector<char> active;
  std::vector<double> srel, sbb;
  std::vector<int> fin;
  int *d_fin = nullptr;
  int *d_cnt = nullptr;  // device: one active-strip count per level
  bool filtered = false;
  double last_bytes = 0.0;  // algorithmic bytes of the last solve (the work actually done)
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
    cudaFree(l.strips_all);
    cudaFree(l.tiles_all);
  }
  cudaFree(B->C);
  cudaFree(B->V);
  cudaFree(B->lam);
  cudaFree(B->acc);
  cudaFree(B->d_fin);
  cudaFree(B->d_cnt);
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

// A device array of a GPU other than `dev` (the batch's): refused, since the
// batch's kernels would read it from the wrong device.
bool other_dev_ptr(const void *p, int dev) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return dev >= 0 && at.type == cudaMemoryTypeDevice && at.device != dev;
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
  for (int j0 = 0; j0 < ny; j0 += TY)
    for (int i0 = 0; i0 < nx; i0 += TX) out.push_back(make_int4(e, i0, j0, 0));
}

// strips of 120 columns by chunks of `ch` rows (even), row-chunk major so
// that neighbouring warps take neighbouring strips (shared halos in L2)
void strips_of(int e, int nx, int ny, int ch, std::vector<int4> &out) {
  for (int ys = 0; ys < ny; ys += ch)
    for (int x0 = 0; x0 < nx; x0 += SW) out.push_back(make_int4(e, x0, ys, std::min(ys + ch, ny)));
}

int pitch_of(int nx) { return (nx + 3) & ~3; }

// CTAs for a launch over n items: one item per CTA (tile kernels) or per warp
int grid_for(gd_batch *B, int nitems, int occ, bool warp_items = true) {
  const int need = warp_items ? (nitems + WPB - 1) / WPB : nitems;
  const int g = B->sm_count * std::max(occ, 1);
  return std::max(1, std::min(need, g));
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
    const int g = grid_for(B, v.nitems, B->occ_sweep), gz = grid_for(B, v.nitems, B->occ_zero);
    for (int k = 0; k < nu1; ++k) {
      const bool zero = k == 0;
      float *out = (cur[l] == v.x) ? v.t : v.x;
      if (zero)
        k_bsweep<true, false><<<gz, BNT, 0, st>>>(v.E, v.items, v.cnt, nullptr, v.b, out, nullptr);
      else
        k_bsweep<false, false><<<g, BNT, 0, st>>>(v.E, v.items, v.cnt, cur[l], v.b, out, nullptr);
      ++B->launches;
      cur[l] = out;
    }
    k_brestrict<<<grid_for(B, v.nitems, B->occ_restrict), BNT, 0, st>>>(v.E, v.items, v.cnt, cur[l], v.b,
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
    const int g = grid_for(B, v.nitems, B->occ_sweep), gp = grid_for(B, v.nitems, B->occ_prolong);
    for (int k = 0; k < nu2; ++k) {
      float *out = (cur[l] == v.x) ? v.t : v.x;
      if (k == 0)
        k_bsweep<false, true><<<gp, BNT, 0, st>>>(v.E, v.items, v.cnt, cur[l], v.b, out, B->L[l + 1].x);
      else
        k_bsweep<false, false><<<g, BNT, 0, st>>>(v.E, v.items, v.cnt, cur[l], v.b, out, nullptr);
      ++B->launches;
      cur[l] = out;
    }
  }
  BCK(cudaGetLastError());
  return GD_OK;
}

// Outer pass: pair cur (+ e) -> pair 1 - cur, r = bf - A x into L[0].b and
// the per-slice sums into acc.
int outer_pass(gd_batch *B, bool add_e, bool pair = true) {
  gd_batch::Lev &f = B->L[0];
  const int a = B->cur, o = 1 - B->cur;
  BCK(cudaMemsetAsync(B->acc, 0, 2 * B->ns * sizeof(double), B->stream));
  const int g = grid_for(B, f.nstrips_all, B->occ_aux);
  if (add_e && !pair)
    k_bouter<true, false><<<g, BNT, 0, B->stream>>>(f.E, f.strips_all, f.nstrips_all, B->bf, B->ph[a],
                                                    B->pl[a], f.x, B->ph[o], B->pl[o], f.b, B->acc);
  else if (add_e)
    k_bouter<true><<<g, BNT, 0, B->stream>>>(f.E, f.strips_all, f.nstrips_all, B->bf, B->ph[a], B->pl[a],
                                             f.x, B->ph[o], B->pl[o], f.b, B->acc);
  else
    k_bouter<false><<<g, BNT, 0, B->stream>>>(f.E, f.strips_all, f.nstrips_all, B->bf, B->ph[a], B->pl[a],
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
  B->srel.resize(B->ns, 0.0);
  B->sbb.resize(B->ns, 0.0);
  for (int s = 0; s < B->ns; ++s) {
    if (B->active.empty() || B->active[s]) {  // converged slices keep their last values
      const double r2 = B->h_acc[2 * s], b2 = B->h_acc[2 * s + 1];
      B->srel[s] = b2 > 0.0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
      B->sbb[s] = b2;
    }
    const double rel = B->srel[s];
    if (slice_rel) slice_rel[s] = rel;
    m = std::isnan(rel) ? rel : (std::isnan(m) ? m : std::fmax(m, rel));
    bb += B->sbb[s];
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

// Cells (padded rows) of the fine level over the slices still iterating.
double n_active_fine(const gd_batch *B) {
  double n0 = 0.0;
  for (const BEntry &e : B->Eh[0])
    if (B->active.empty() || B->active[e.slice]) n0 += (double)e.pitch * e.ny;
  return n0;
}

// Algorithmic bytes of one V(nu1, nu2) cycle with its outer pass over the
// slices still iterating (all of them when `active` is empty).
double cycle_bytes(const gd_batch *B, int nu1, int nu2) {
  double cyc = 0.0;
  for (size_t l = 0; l < B->Eh.size(); ++l) {
    double nf = 0.0, nc = 0.0, n0 = 0.0;
    for (const BEntry &e : B->Eh[l]) {
      if (!B->active.empty() && !B->active[e.slice]) continue;
      if (l == 0) n0 += (double)e.pitch * e.ny;
      if (e.coff < 0) continue;
      nf += (double)e.pitch * e.ny;
      nc += (double)e.cpitch * e.cny;
    }
    // sweeps (the first from zero: 8 B, the others 12 B; the prolongation
    // adds 4 B per coarse cell), restriction (8 B + 4 B per coarse cell),
    // and at level 0 the outer pass (28 B)
    cyc += nf * (8.0 + 12.0 * (nu1 - 1)) + nf * 12.0 * nu2 + 4.0 * nc + nf * 8.0 + 4.0 * nc + 28.0 * n0;
  }
  return cyc;
}

// Host work lists of the active slices (all slices when `all`) for chunks of
// `ch` rows: per level the strips of the entries that have a next level, and
// at level 0 the strips of every entry (the outer pass).
void host_lists(const gd_batch *B, int ch, bool all, std::vector<std::vector<int4>> &it,
                std::vector<int4> &sa) {
  it.assign(B->L.size(), std::vector<int4>());
  sa.clear();
  for (size_t l = 0; l < B->L.size(); ++l)
    for (int k = 0; k < (int)B->Eh[l].size(); ++k) {
      const BEntry &e = B->Eh[l][k];
      if (!all && !B->active.empty() && !B->active[e.slice]) continue;
      if (e.coff >= 0) strips_of(k, e.nx, e.ny, ch, it[l]);
      if (l == 0) strips_of(k, e.nx, e.ny, ch, sa);
    }
}

// (Re)builds the row-march work lists for chunks of `ch` rows, every slice
// included; the buffers keep this size, so a captured V-cycle stays valid
// when filter_lists later shrinks their contents.
int build_lists(gd_batch *B, int ch) {
  int st;
  std::vector<std::vector<int4>> it;
  std::vector<int4> sa;
  host_lists(B, ch, true, it, sa);
  if (!B->d_cnt && (st = balloc(B, &B->d_cnt, (size_t)B->L.size())) != GD_OK) return st;
  std::vector<int> cnt(B->L.size());
  for (size_t l = 0; l < B->L.size(); ++l) {
    gd_batch::Lev &v = B->L[l];
    cudaFree(v.items);
    cudaFree(v.strips_all);
    v.items = v.strips_all = nullptr;
    v.nitems = (int)it[l].size();
    v.cnt = B->d_cnt + l;
    cnt[l] = v.nitems;
    if ((st = balloc(B, &v.items, it[l].size())) != GD_OK) return st;
    if (!it[l].empty())
      BCK(cudaMemcpy(v.items, it[l].data(), it[l].size() * sizeof(int4), cudaMemcpyHostToDevice));
    if (l == 0) {
      v.nstrips_all = v.nstrips_all_cap = (int)sa.size();
      if ((st = balloc(B, &v.strips_all, sa.size())) != GD_OK) return st;
      if (!sa.empty())
        BCK(cudaMemcpy(v.strips_all, sa.data(), sa.size() * sizeof(int4), cudaMemcpyHostToDevice));
    }
  }
  BCK(cudaMemcpy(B->d_cnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice));
  B->chunk = ch;
  if (B->gexec) {  // the graph holds the old buffers
    cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
    B->g_nu1 = B->g_nu2 = -1;
  }
  return GD_OK;
}

// Writes the active slices' strips into the front of the existing list
// buffers and their counts into d_cnt (stream-ordered, then synchronised):
// the kernels read the counts at run time, so the captured V-cycle stays
// valid as slices leave.
int filter_lists(gd_batch *B) {
  std::vector<std::vector<int4>> it;
  std::vector<int4> sa;
  host_lists(B, B->chunk, false, it, sa);
  std::vector<int> cnt(B->L.size());
  for (size_t l = 0; l < B->L.size(); ++l) {
    gd_batch::Lev &v = B->L[l];
    cnt[l] = (int)it[l].size();
    if (cnt[l] > v.nitems) return GD_ERR_CUDA;  // cannot happen: a subset of the full list
    if (cnt[l])
      BCK(cudaMemcpyAsync(v.items, it[l].data(), it[l].size() * sizeof(int4), cudaMemcpyHostToDevice,
                          B->stream));
  }
  gd_batch::Lev &f = B->L[0];
  if ((int)sa.size() > f.nstrips_all_cap) return GD_ERR_CUDA;
  if (!sa.empty())
    BCK(cudaMemcpyAsync(f.strips_all, sa.data(), sa.size() * sizeof(int4), cudaMemcpyHostToDevice, B->stream));
  f.nstrips_all = (int)sa.size();
  BCK(cudaMemcpyAsync(B->d_cnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  BCK(cudaStreamSynchronize(B->stream));  // the host vectors go out of scope
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
      e.uoff = B->off[s];
      e.nx = v.nx;
      e.ny = v.ny;
      e.pitch = pitch_of(v.nx);
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
      o += (long long)e.pitch * v.ny;
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
      e.cpitch = c.pitch;
    }
  // work lists and buffers
  int st;
  for (int l = 0; l < D; ++l) {
    gd_batch::Lev &v = B->L[l];
    std::vector<int4> ta;
    for (int k = 0; k < (int)E[l].size() && l == 0; ++k) tiles_of(k, E[l][k].nx, E[l][k].ny, ta);
    long long fc = 0;  // cells of the entries that have a next level (they need a sweep buffer)
    for (const BEntry &e : E[l])
      if (e.coff >= 0) fc += (long long)e.pitch * e.ny;
    v.ne = (int)E[l].size();
    v.ntiles_all = (int)ta.size();
    if ((st = balloc(B, &v.x, (size_t)v.n)) != GD_OK) return st;
    if ((st = balloc(B, &v.b, (size_t)v.n)) != GD_OK) return st;
    if (fc > 0 && (st = balloc(B, &v.t, (size_t)v.n)) != GD_OK) return st;
    // padding cells hold 0 from here on: every kernel writes 0 there
    BCK(cudaMemset(v.x, 0, (size_t)v.n * sizeof(float)));
    BCK(cudaMemset(v.b, 0, (size_t)v.n * sizeof(float)));
    if (v.t) BCK(cudaMemset(v.t, 0, (size_t)v.n * sizeof(float)));
    if ((st = balloc(B, &v.E, E[l].size())) != GD_OK) return st;
    if ((st = balloc(B, &v.tiles_all, ta.size())) != GD_OK) return st;
    BCK(cudaMemcpy(v.E, E[l].data(), E[l].size() * sizeof(BEntry), cudaMemcpyHostToDevice));
    if (!ta.empty())
      BCK(cudaMemcpy(v.tiles_all, ta.data(), ta.size() * sizeof(int4), cudaMemcpyHostToDevice));
  }
  B->Eh = E;
  if ((st = build_lists(B, CH)) != GD_OK) return st;
  const size_t n0 = (size_t)B->L[0].n;
  if ((st = balloc(B, &B->bf, n0)) != GD_OK) return st;
  BCK(cudaMemset(B->bf, 0, n0 * sizeof(float)));
  for (int k = 0; k < 2; ++k) {
    if ((st = balloc(B, &B->ph[k], n0)) != GD_OK) return st;
    if ((st = balloc(B, &B->pl[k], n0)) != GD_OK) return st;
    BCK(cudaMemset(B->ph[k], 0, n0 * sizeof(float)));
    BCK(cudaMemset(B->pl[k], 0, n0 * sizeof(float)));
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
    C[s] = BCoarse{l, v.nx, v.ny, e.pitch, ax.first, ay.first, ax.second, ay.second,
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
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_sweep, k_bsweep<false, false>, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_zero, k_bsweep<true, false>, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_prolong, k_bsweep<false, true>, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_restrict, k_brestrict, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_aux, k_bouter<true>, BNT, 0));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B->occ_tile, k_brhs, BNT, 0));
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
  if (cudaGetDevice(&B->device) != cudaSuccess) {
    cudaGetLastError();
    B->device = -1;
  }
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

int gd_batch_traffic(const gd_batch *b, int nu1, int nu2, double *per_cycle, double *per_solve) {
  if (!b || nu1 < 1 || nu2 < 1) return GD_ERR_INVALID_ARG;
  gd_batch tmp_view;  // every slice active
  tmp_view.Eh = b->Eh;
  const double n0 = (double)b->L[0].n;
  if (per_cycle) *per_cycle = cycle_bytes(&tmp_view, nu1, nu2);
  // right-hand side (reads I0, I1; writes bf, h, l), first outer pass
  // (reads bf, h, l; writes h, l, r), output (reads h, l; writes I2)
  if (per_solve) *per_solve = 20.0 * (double)b->nvox + 24.0 * n0 + 12.0 * n0;
  return GD_OK;
}

double gd_batch_last_traffic(const gd_batch *b) { return b ? b->last_bytes : -1.0; }

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
  for (int k = 0; k < 4; ++k) {
    const void *p = k < 3 ? (const void *)in[k] : (const void *)I2;
    if (other_dev_ptr(p, B->device)) {
      bset_err(B, "array %p lives on another device than the batch's (device %d)", p, B->device);
      if (rep) rep->status = GD_ERR_INVALID_ARG;
      return GD_ERR_INVALID_ARG;
    }
  }
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
  // every slice iterates again
  B->active.assign(B->ns, 1);
  B->fin.assign(B->ns, 0);
  B->srel.assign(B->ns, 0.0);
  B->sbb.assign(B->ns, 0.0);
  if (B->filtered) {  // every slice iterates again: the full lists, same buffers
    const int st0 = filter_lists(B);
    if (st0 != GD_OK) return st0;
    B->filtered = false;
  }
  k_brhs<<<grid_for(B, f.ntiles_all, B->occ_tile, false), BNT, 0, B->stream>>>(
      f.E, f.tiles_all, f.ntiles_all, dv[0], dv[1], dv[2], B->bf, B->ph[0], B->pl[0]);
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
  // slices at tolerance leave the work lists (their iterate stays in the
  // pair buffer that holds it); the lists shrink at most once per cycle
  auto retire = [&]() -> int {
    int left = 0, newly = 0;
    for (int q = 0; q < B->ns; ++q) {
      if (!B->active[q]) continue;
      if (B->srel[q] <= c.rel_tol) {
        B->active[q] = 0;
        B->fin[q] = B->cur;
        ++newly;
      } else {
        ++left;
      }
    }
    if (newly > 0 && left > 0 && cycles < c.max_cycles) {
      const int r = filter_lists(B);
      if (r != GD_OK) return r;
      B->filtered = true;
    }
    return GD_OK;
  };
  if ((st = retire()) != GD_OK) return st;
  double bytes = 20.0 * (double)B->nvox + 36.0 * (double)f.n;  // input, first outer pass, output
  bool exact = false;
  while (!(rel <= c.rel_tol) && cycles < c.max_cycles) {
    bytes += cycle_bytes(B, c.nu1, c.nu2);
    if (B->gexec) {
      BCK(cudaGraphLaunch(B->gexec, B->stream));
      B->launches += B->g_launches;
    } else if ((st = bvcycle(B, c.nu1, c.nu2, B->stream)) != GD_OK) {
      return st;
    }
    // plain FP32 updates while the residual is large; from 1e-4 on (and from
    // then on always) the pair carries the low words
    if (rel < 1e-4) exact = true;
    if ((st = outer_pass(B, true, exact)) != GD_OK) return st;
    bytes -= exact ? 0.0 : 8.0 * (double)n_active_fine(B);
    ++cycles;
    if ((st = read_rel(B, &rel, &bn, slice_rel)) != GD_OK) return st;
    if ((st = retire()) != GD_OK) return st;
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
  B->last_bytes = bytes;
  for (int q = 0; q < B->ns; ++q)
    if (B->active[q]) B->fin[q] = B->cur;
  if (!B->d_fin && (st = balloc(B, &B->d_fin, (size_t)B->ns)) != GD_OK) return st;
  BCK(cudaMemcpyAsync(B->d_fin, B->fin.data(), B->ns * sizeof(int), cudaMemcpyHostToDevice, B->stream));
  k_bfinal<<<grid_for(B, f.ntiles_all, B->occ_tile, false), BNT, 0, B->stream>>>(
      f.E, f.tiles_all, f.ntiles_all, B->ph[0], B->pl[0], B->ph[1], B->pl[1], B->d_fin, out);
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

int gd_batch_tune(gd_batch *B, int *chunk_out) {
  if (!B) return GD_ERR_INVALID_ARG;
  // every candidate runs the same V(2, 2) cycle on whatever the buffers
  // hold (the timing does not depend on the values); the next solve starts
  // from its own right-hand side
  static const int cand[] = {32, 64, 128, 256};
  B->active.assign(B->ns, 1);
  B->filtered = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  int best = B->chunk;
  float best_ms = 0.f;
  int st = GD_OK;
  for (int c : cand) {
    if ((st = build_lists(B, c)) != GD_OK) break;
    if ((st = bvcycle(B, 2, 2, B->stream)) != GD_OK) break;  // warm-up
    cudaEventRecord(e0, B->stream);
    for (int r = 0; r < 2 && st == GD_OK; ++r) st = bvcycle(B, 2, 2, B->stream);
    cudaEventRecord(e1, B->stream);
    if (st != GD_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      bset_err(B, "tuning run failed: %s", cudaGetErrorString(cudaGetLastError()));
      st = GD_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best_ms == 0.f || ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == GD_OK) st = build_lists(B, best);
  if (chunk_out) *chunk_out = B->chunk;
  return st;
}

int gd_batch_destroy(gd_batch *b) {
  if (!b) return GD_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  delete b;
  return GD_OK;
}

}  // extern "C"
