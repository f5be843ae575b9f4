// gd_zmarch.cu -- TMA-pipelined 2.5D z-march kernels for sm_103a.
//
// A CTA owns a 64 x 16 column tile of one level and marches along z over a
// chunk of planes.  Planes of each input array arrive in a shared-memory ring
// by TMA (cp.async.bulk.tensor.3d, one elected thread, mbarrier completion),
// PF planes ahead of their first use, so HBM latency is hidden without extra
// threads.  Boxes start at x = i0 - 4 (16-byte aligned coordinates) and are
// 72 floats wide; the tensor map zero-fills outside the array.
//
// k_zsweep: one red-black Gauss-Seidel sweep (Sec. 4.1 multi-colour
//   relaxation) with optional fusions:
//     ZERO_IN   the input iterate is zero (first pre-sweep of a correction);
//     PROLONG   x <- x + P x_c before relaxing (first post-sweep: the
//               up-sampled coarse correction of Sec. 4.1, replication
//               stencil of Sec. 4.2);
//     RESTRICT  after relaxing, r = b - A x is summed over the children into
//               the coarse right-hand side (last pre-sweep: residual and
//               down-sampling of Sec. 4.1);
//     SUM       the block sums of the written iterate (mean fix of AD).
//   Pipeline per step t: red of plane t on the tile + (H-1) ring, black of
//   plane t-1 on the tile + (H-2) ring, store plane t-1, residual of plane
//   t-2 (RESTRICT).  Ring margins recompute neighbours' values exactly as the
//   neighbouring CTA does, so the result is the textbook red-black sweep.
//
// k_zouter: fine-level outer pass of the iterative refinement: x_new = x + e
//   (+ mean shift) as a float pair, r = b - A x_new in double-float arithmetic
//   with b assembled from I0 (and I1), and FP64 block partial sums.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>

#include "gd_internal.h"

namespace {

constexpr int ZX = 64;            // tile x extent
constexpr int ZY = 16;            // tile y extent
constexpr int ZNT = 256;          // threads per CTA
constexpr int BOXW = ZX + 8;      // box width: tile + 4 on each side (16-byte aligned start)
constexpr int PF = 2;             // planes in flight ahead of use
constexpr uint32_t WAIT_LIMIT = 1u << 22;  // bounded mbarrier polling

__host__ __device__ constexpr int pad32(int n) { return (n + 31) & ~31; }  // 128-byte slots

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = su32(bar);
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_plane(float *dst, const CUtensorMap *map, int x, int y, int z,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ float mass_of(int i, int n, int s, int l) {
  return (float)((i == n - 1) ? l : s);
}

// Checks a CTA makes before any TMA: the dynamic shared-memory base is
// 128-byte aligned (slot offsets are multiples of 128 bytes), it holds `bytes`
// within the CTA's shared window, and the tensor-map parameter is 64-byte
// aligned.  Returns 0 or an error code (2: smem base, 3: tensor map, 4: size).
__device__ __forceinline__ int tma_preflight(const void *smem_base, size_t bytes, const void *map) {
  uint32_t dyn = 0;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  if ((su32(smem_base) & 127u) != 0) return 2;
  if (((uintptr_t)map & 63u) != 0) return 3;
  if (bytes > dyn) return 4;
  return 0;
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
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

// Ring bookkeeping for one input array: planes [lo, hi] are loaded, plane p
// lives in slot (p - lo) % DEPTH and completes phase ((p - lo) / DEPTH) & 1.
template <int DEPTH>
struct Ring {
  int lo, hi;
  __device__ __forceinline__ bool has(int p) const { return p >= lo && p <= hi; }
  __device__ __forceinline__ int slot(int p) const { return (p - lo) % DEPTH; }
  __device__ __forceinline__ uint32_t parity(int p) const { return ((p - lo) / DEPTH) & 1; }
};

// ===========================================================================
// red-black sweep
// ===========================================================================
template <bool RESTRICT>
struct SweepGeo {
  static constexpr int H = RESTRICT ? 3 : 2;     // x box halo in y
  static constexpr int XH = ZY + 2 * H;          // x box rows
  static constexpr int BH = ZY + 2 * (H - 1);    // b box rows
  static constexpr int XR = (RESTRICT ? 5 : 4) + PF;
  static constexpr int BR = (RESTRICT ? 3 : 2) + PF;
  static constexpr int XS = pad32(XH * BOXW);    // floats per x slot
  static constexpr int BS = pad32(BH * BOXW);
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(float) * ((size_t)XR * XS + (size_t)BR * BS + ZX * ZY) +
           sizeof(uint64_t) * (XR + BR) + sizeof(double) * 32 + 16;
  }
};

template <bool ZERO_IN, bool PROLONG, bool RESTRICT, bool SUM>
__global__ void __launch_bounds__(ZNT) k_zsweep(const __grid_constant__ CUtensorMap tmx,
                                                const __grid_constant__ CUtensorMap tmb,
                                                const ZSweepArgs a) {
  using G = SweepGeo<RESTRICT>;
  constexpr int H = G::H;
  extern __shared__ __align__(128) unsigned char smem[];
  float *xs = reinterpret_cast<float *>(smem);
  float *bs = xs + G::XR * G::XS;
  float *acc = bs + G::BR * G::BS;
  uint64_t *xbar = reinterpret_cast<uint64_t *>(acc + ZX * ZY);
  uint64_t *bbar = xbar + G::XR;
  double *dsh = reinterpret_cast<double *>(bbar + G::BR);
  __shared__ int abort_flag;

  const LevelDev &L = a.L;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * ZY;
  const int zs = blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, nz);
  const bool zc = (L.wz != 0.f) && (nz > 1);
  const int R = RESTRICT ? 1 : 0;
  const int t0 = zc ? zs - 1 - R : zs;
  const int t1 = zc ? ze + R : ze - 1;
  const int lagb = zc ? 1 : 0, lagr = zc ? 2 : 0;
  const int red_lo = zc ? max(zs - 1 - R, 0) : zs, red_hi = zc ? min(ze + R, nz - 1) : ze - 1;
  const int blk_lo = zc ? max(zs - R, 0) : zs, blk_hi = zc ? min(ze - 1 + R, nz - 1) : ze - 1;
  Ring<G::XR> rx;
  rx.lo = zc ? max(t0 - 1, 0) : zs;
  rx.hi = zc ? min(t1 + 1, nz - 1) : ze - 1;
  Ring<G::BR> rb;
  rb.lo = zc ? max(t0, 0) : zs;
  rb.hi = zc ? min(t1, nz - 1) : ze - 1;
  const size_t plane = (size_t)nx * ny;

  if (tid == 0) {
    abort_flag = 0;
    int e = tma_preflight(smem, G::smem_bytes(), &tmx);
    if (!e) e = tma_preflight(smem, G::smem_bytes(), &tmb);
    if (e) {
      abort_flag = e;
      a.err[0] = (double)e;
    } else {
      for (int s = 0; s < G::XR; ++s) mbar_init(&xbar[s], 1);
      for (int s = 0; s < G::BR; ++s) mbar_init(&bbar[s], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (abort_flag) return;  // nothing issued yet

  int xissued = rx.lo - 1, bissued = rb.lo - 1;  // meaningful in thread 0
  auto issue_x = [&](int p) {
    if (ZERO_IN || !rx.has(p)) return;
    const int s = rx.slot(p);
    mbar_expect_tx(&xbar[s], (uint32_t)(G::XH * BOXW * sizeof(float)));
    tma_plane(xs + s * G::XS, &tmx, i0 - 4, j0 - H, p, &xbar[s]);
    xissued = p;
  };
  auto issue_b = [&](int p) {
    if (!rb.has(p)) return;
    const int s = rb.slot(p);
    mbar_expect_tx(&bbar[s], (uint32_t)(G::BH * BOXW * sizeof(float)));
    tma_plane(bs + s * G::BS, &tmb, i0 - 4, j0 - (H - 1), p, &bbar[s]);
    bissued = p;
  };
  const int xnext0 = zc ? t0 + 1 + PF : t0 + PF;  // first plane issued inside the loop
  if (tid == 0) {
    for (int p = rx.lo; p < xnext0 && p <= rx.hi; ++p) issue_x(p);
    for (int p = rb.lo; p < t0 + PF && p <= rb.hi; ++p) issue_b(p);
  }
  int xready = rx.lo - 1, bready = rb.lo - 1;
  auto xslot = [&](int p) -> float * { return xs + rx.slot(p) * G::XS; };
  auto bslot = [&](int p) -> float * { return bs + rb.slot(p) * G::BS; };

  // Make x planes up to `upto` usable: wait for TMA (or zero-fill), add P x_c.
  auto ready_x = [&](int upto) {
    upto = min(upto, rx.hi);
    for (int p = xready + 1; p <= upto; ++p) {
      float *X = xslot(p);
      if (ZERO_IN) {
        for (int q = tid; q < G::XH * BOXW; q += ZNT) X[q] = 0.f;
      } else {
        if (!mbar_wait(&xbar[rx.slot(p)], rx.parity(p))) {
          abort_flag = 1;
          return;
        }
        if (PROLONG) {
          const size_t cpl = (size_t)(p >> a.fz) * a.ncy;
          for (int q = tid; q < G::XH * BOXW; q += ZNT) {
            const int r = q / BOXW, c = q - r * BOXW;
            const int gi = i0 - 4 + c, gj = j0 - H + r;
            if (gi >= 0 && gi < nx && gj >= 0 && gj < ny)
              X[q] += __ldg(a.xc + (cpl + (gj >> a.fy)) * a.ncx + (gi >> a.fx));
          }
        }
      }
      xready = p;
    }
  };
  auto ready_b = [&](int upto) {
    upto = min(upto, rb.hi);
    for (int p = bready + 1; p <= upto; ++p) {
      if (!mbar_wait(&bbar[rb.slot(p)], rb.parity(p))) {
        abort_flag = 1;
        return;
      }
      bready = p;
    }
  };

  // (A x)_p terms at one voxel, difference form; returns A x, diag in *dg.
  auto apply_at = [&](const float *X, const float *Xm, const float *Xp, int sy, int sx, int gi,
                      int gj, int p, float &dg) -> float {
    const float mx = mass_of(gi, nx, L.sx, L.lx);
    const float my = mass_of(gj, ny, L.sy, L.ly);
    const float mz = mass_of(p, nz, L.sz, L.lz);
    const float cx = L.wx * my * mz, cy = L.wy * mx * mz, cz = L.wz * mx * my;
    const float mm = L.wm * mx * my * mz;
    const int o = sy * BOXW + sx;
    const float xc = X[o];
    float ax = mm * xc;
    dg = mm;
    if (gi > 0) { ax += cx * (xc - X[o - 1]); dg += cx; }
    if (gi < nx - 1) { ax += cx * (xc - X[o + 1]); dg += cx; }
    if (gj > 0) { ax += cy * (xc - X[o - BOXW]); dg += cy; }
    if (gj < ny - 1) { ax += cy * (xc - X[o + BOXW]); dg += cy; }
    if (zc && p > 0) { ax += cz * (xc - Xm[o]); dg += cz; }
    if (zc && p < nz - 1) { ax += cz * (xc - Xp[o]); dg += cz; }
    return ax;
  };
  auto relax_plane = [&](int p, int ring, int colour) {
    float *X = xslot(p);
    const float *Xm = (zc && p > 0) ? xslot(p - 1) : X;
    const float *Xp = (zc && p < nz - 1) ? xslot(p + 1) : X;
    const float *B = bslot(p);
    const int W = ZX + 2 * ring, Hh = ZY + 2 * ring;
    const int half = W / 2;
    for (int q = tid; q < Hh * half; q += ZNT) {
      const int r = q / half, c2 = q - r * half;
      const int gj = j0 - ring + r;
      // colour 0 (red): gi + gj + p even; gi = i0 - ring + col, i0 even
      const int col = 2 * c2 + ((ring + gj + p + colour) & 1);
      const int gi = i0 - ring + col;
      if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
      const int sy = gj - (j0 - H), sx = gi - (i0 - 4);
      float dg;
      const float ax = apply_at(X, Xm, Xp, sy, sx, gi, gj, p, dg);
      const float bv = B[(gj - (j0 - (H - 1))) * BOXW + sx];
      if (dg > 0.f) X[sy * BOXW + sx] = X[sy * BOXW + sx] + (bv - ax) / dg;
    }
  };
  double sum = 0.0;
  auto store = [&](int p) {
    const float *X = xslot(p);
    const int r = tid >> 4, c = (tid & 15) * 4;
    const int gi = i0 + c, gj = j0 + r;
    if (gi < nx && gj < ny) {
      const float4 v = *reinterpret_cast<const float4 *>(X + (r + H) * BOXW + 4 + c);
      *reinterpret_cast<float4 *>(a.xout + (size_t)p * plane + (size_t)gj * nx + gi) = v;
      if (SUM) sum += (double)v.x + (double)v.y + (double)v.z + (double)v.w;
    }
  };
  auto restrict_plane = [&](int p) {
    const float *X = xslot(p);
    const float *Xm = (zc && p > 0) ? xslot(p - 1) : X;
    const float *Xp = (zc && p < nz - 1) ? xslot(p + 1) : X;
    const float *B = bslot(p);
    const int fx = a.fx, fy = a.fy, fz = a.fz;
    const int CW = ZX >> fx, CH = ZY >> fy;
    const size_t cpl = (size_t)(p >> fz) * a.ncy;
    for (int q = tid; q < CW * CH; q += ZNT) {
      const int cr = q / CW, cc = q - cr * CW;
      float s = 0.f;
      for (int dr = 0; dr <= fy; ++dr)
        for (int dc = 0; dc <= fx; ++dc) {
          const int gi = i0 + (cc << fx) + dc, gj = j0 + (cr << fy) + dr;
          if (gi >= nx || gj >= ny) continue;
          const int sy = gj - (j0 - H), sx = gi - (i0 - 4);
          float dg;
          const float ax = apply_at(X, Xm, Xp, sy, sx, gi, gj, p, dg);
          s += B[(gj - (j0 - (H - 1))) * BOXW + sx] - ax;
        }
      const int I = (i0 >> fx) + cc, J = (j0 >> fy) + cr;
      if (fz && (p & 1) == 0 && p != nz - 1) {
        acc[q] = s;  // first child plane: keep for the second
      } else {
        if (fz && (p & 1) == 1) s += acc[q];
        if (I < a.ncx && J < a.ncy) a.bc[(cpl + J) * a.ncx + I] = s;
      }
    }
  };

  for (int t = t0; t <= t1; ++t) {
    if (tid == 0) {
      fence_proxy_async();
      issue_x(zc ? t + 1 + PF : t + PF);
      issue_b(t + PF);
    }
    ready_x(zc ? t + 1 : t);
    ready_b(t);
    __syncthreads();
    if (abort_flag) break;
    if (t >= red_lo && t <= red_hi) relax_plane(t, H - 1, 0);
    __syncthreads();
    const int pb = t - lagb;
    if (pb >= blk_lo && pb <= blk_hi) relax_plane(pb, H - 2, 1);
    __syncthreads();
    if (pb >= zs && pb < ze) store(pb);
    if (RESTRICT) {
      const int pr = t - lagr;
      if (pr >= zs && pr < ze) restrict_plane(pr);
    }
    __syncthreads();
  }
  if (abort_flag) {
    // a TMA completion did not arrive in time: flag it, give the copies this
    // CTA still has in flight a bounded wait to land, and leave
    if (tid == 0) {
      a.err[0] = 1.0;
      for (int p = xready + 1; p <= xissued; ++p) mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
      for (int p = bready + 1; p <= bissued; ++p) mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
    }
    return;
  }
  if (SUM) {
    const double s = block_sum(sum, dsh);
    if (tid == 0) {
      const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[blk * S_NUM + S_E] = s;
    }
  }
}

// ===========================================================================
// outer pass (double-float residual of the float-pair iterate)
// ===========================================================================
struct ff {
  float h, l;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, {-b.h, -b.l}); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p, e);
}

struct OuterGeo {
  static constexpr int BH = ZY + 2;              // rows: tile + 1 halo
  static constexpr int S = pad32(BH * BOXW);
  static constexpr int XR = 3 + PF;              // x_new planes t-1..t+1 + in flight
  static constexpr int ER = 3 + PF;              // corrections: same planes and lag as x
  static constexpr int IR = 1 + PF;
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(float) * (size_t)S * (2 * XR + ER + 2 * IR) +
           sizeof(uint64_t) * (2 * XR + ER + 2 * IR) + sizeof(double) * 32 + 16;
  }
};

template <int RHS, bool HAS_XL, bool HAS_E>
__global__ void __launch_bounds__(ZNT) k_zouter(const __grid_constant__ CUtensorMap tmh,
                                                const __grid_constant__ CUtensorMap tml,
                                                const __grid_constant__ CUtensorMap tme,
                                                const __grid_constant__ CUtensorMap tmi0,
                                                const __grid_constant__ CUtensorMap tmi1,
                                                const OuterArgs a, int zchunk, double *err) {
  using G = OuterGeo;
  constexpr int S = G::S;
  extern __shared__ __align__(128) unsigned char smem[];
  float *hs = reinterpret_cast<float *>(smem);    // XR slots: x_new high parts
  float *ls = hs + G::XR * S;                     // XR slots: x_new low parts
  float *es = ls + G::XR * S;                     // ER slots: corrections
  float *i0s = es + G::ER * S;                    // IR slots: I0 (or explicit b)
  float *i1s = i0s + G::IR * S;                   // IR slots: I1
  uint64_t *hb = reinterpret_cast<uint64_t *>(i1s + G::IR * S);
  uint64_t *lb = hb + G::XR;
  uint64_t *eb = lb + G::XR;
  uint64_t *ib0 = eb + G::ER;
  uint64_t *ib1 = ib0 + G::IR;
  double *dsh = reinterpret_cast<double *>(ib1 + G::IR);
  __shared__ int abort_flag;

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * ZY;
  const int zs = blockIdx.z * zchunk, ze = min(zs + zchunk, nz);
  const bool zc = (a.bz != 0.f) && (nz > 1);
  const size_t plane = (size_t)nx * ny;
  const int t0 = zc ? zs - 1 : zs, t1 = ze - 1;
  Ring<G::XR> rx;
  rx.lo = zc ? max(zs - 1, 0) : zs;
  rx.hi = zc ? min(ze, nz - 1) : ze - 1;
  Ring<G::ER> re;  // same planes as x
  re.lo = rx.lo;
  re.hi = rx.hi;
  Ring<G::IR> ri;
  ri.lo = zs;
  ri.hi = ze - 1;
  constexpr bool SP = RHS == RHS_SP;
  constexpr uint32_t BOXB = (uint32_t)(G::BH * BOXW * sizeof(float));

  if (tid == 0) {
    abort_flag = 0;
    int e = tma_preflight(smem, G::smem_bytes(), &tmh);
    if (!e && HAS_XL) e = tma_preflight(smem, G::smem_bytes(), &tml);
    if (!e && HAS_E) e = tma_preflight(smem, G::smem_bytes(), &tme);
    if (!e) e = tma_preflight(smem, G::smem_bytes(), &tmi0);
    if (!e && SP) e = tma_preflight(smem, G::smem_bytes(), &tmi1);
    if (e) {
      abort_flag = e;
      err[0] = (double)e;
    } else {
      for (int s = 0; s < G::XR; ++s) { mbar_init(&hb[s], 1); mbar_init(&lb[s], 1); }
      for (int s = 0; s < G::ER; ++s) mbar_init(&eb[s], 1);
      for (int s = 0; s < G::IR; ++s) { mbar_init(&ib0[s], 1); mbar_init(&ib1[s], 1); }
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (abort_flag) return;  // nothing issued yet

  int xissued = rx.lo - 1, iissued = ri.lo - 1;  // meaningful in thread 0
  auto issue_x = [&](int p) {
    if (!rx.has(p)) return;
    xissued = p;
    const int s = rx.slot(p);
    mbar_expect_tx(&hb[s], BOXB);
    tma_plane(hs + s * S, &tmh, i0 - 4, j0 - 1, p, &hb[s]);
    if (HAS_XL) {
      mbar_expect_tx(&lb[s], BOXB);
      tma_plane(ls + s * S, &tml, i0 - 4, j0 - 1, p, &lb[s]);
    }
    if (HAS_E) {
      const int se = re.slot(p);
      mbar_expect_tx(&eb[se], BOXB);
      tma_plane(es + se * S, &tme, i0 - 4, j0 - 1, p, &eb[se]);
    }
  };
  auto issue_i = [&](int p) {
    if (!ri.has(p)) return;
    iissued = p;
    const int s = ri.slot(p);
    mbar_expect_tx(&ib0[s], BOXB);
    tma_plane(i0s + s * S, &tmi0, i0 - 4, j0 - 1, p, &ib0[s]);
    if (SP) {
      mbar_expect_tx(&ib1[s], BOXB);
      tma_plane(i1s + s * S, &tmi1, i0 - 4, j0 - 1, p, &ib1[s]);
    }
  };
  const int xnext0 = zc ? t0 + 1 + PF : t0 + PF;
  if (tid == 0) {
    for (int p = rx.lo; p < xnext0 && p <= rx.hi; ++p) issue_x(p);
    for (int p = ri.lo; p < t0 + PF && p <= ri.hi; ++p) issue_i(p);
  }
  float shift = 0.f;
  if (HAS_E && a.mean_fix)
    shift = (float)((a.scalars[S_I0] - a.scalars[S_X] - a.scalars[S_E]) * a.inv_n);
  int xready = rx.lo - 1, iready = ri.lo - 1;
  auto ready_x = [&](int upto) {
    upto = min(upto, rx.hi);
    for (int p = xready + 1; p <= upto; ++p) {
      const int s = rx.slot(p);
      const uint32_t ph = rx.parity(p);
      bool ok = mbar_wait(&hb[s], ph);
      if (HAS_XL) ok = mbar_wait(&lb[s], ph) && ok;
      if (HAS_E) ok = mbar_wait(&eb[re.slot(p)], re.parity(p)) && ok;
      if (!ok) {
        abort_flag = 1;
        return;
      }
      float *Hs = hs + s * S, *Ls = ls + s * S;
      const float *Es = es + re.slot(p) * S;
      for (int q = tid; q < G::BH * BOXW; q += ZNT) {
        const float h = Hs[q];
        const float l = HAS_XL ? Ls[q] : 0.f;
        if (HAS_E) {
          const ff v = ff_add({h, l}, {__fadd_rn(Es[q], shift), 0.f});
          Hs[q] = v.h;
          Ls[q] = v.l;
        } else if (!HAS_XL) {
          Ls[q] = 0.f;
        }
      }
      xready = p;
    }
  };
  auto ready_i = [&](int upto) {
    upto = min(upto, ri.hi);
    for (int p = iready + 1; p <= upto; ++p) {
      bool ok = mbar_wait(&ib0[ri.slot(p)], ri.parity(p));
      if (SP) ok = mbar_wait(&ib1[ri.slot(p)], ri.parity(p)) && ok;
      if (!ok) {
        abort_flag = 1;
        return;
      }
      iready = p;
    }
  };
  const ff Wx = {a.bx, a.bx_lo}, Wy = {a.by, a.by_lo}, Wz = {a.bz, a.bz_lo};
  const ff Wa = {a.alpha, a.alpha_lo};
  const ff Rx = {a.rbx, a.rbx_lo}, Ry = {a.rby, a.rby_lo}, Ra = {a.ralpha, a.ralpha_lo};
  double srr = 0.0, sbb = 0.0, sx = 0.0, si = 0.0;

  auto residual_plane = [&](int p) {
    const int s = rx.slot(p);
    const float *Hc = hs + s * S, *Lc = ls + s * S;
    const bool hm = zc && p > 0, hp = zc && p < nz - 1;
    const float *Hm = hm ? hs + rx.slot(p - 1) * S : Hc, *Lm = hm ? ls + rx.slot(p - 1) * S : Lc;
    const float *Hp = hp ? hs + rx.slot(p + 1) * S : Hc, *Lp = hp ? ls + rx.slot(p + 1) * S : Lc;
    const float *I0 = i0s + ri.slot(p) * S, *I1 = i1s + ri.slot(p) * S;
    for (int q = tid; q < ZX * ZY; q += ZNT) {
      const int r = q >> 6, c = q & 63;
      const int gi = i0 + c, gj = j0 + r;
      if (gi >= nx || gj >= ny) continue;
      const int o = (r + 1) * BOXW + 4 + c;
      const ff xc = {Hc[o], Lc[o]};
      ff dx = {0.f, 0.f}, dy = {0.f, 0.f}, dz = {0.f, 0.f};
      if (gi > 0) dx = ff_add(dx, ff_sub(xc, {Hc[o - 1], Lc[o - 1]}));
      if (gi < nx - 1) dx = ff_add(dx, ff_sub(xc, {Hc[o + 1], Lc[o + 1]}));
      if (gj > 0) dy = ff_add(dy, ff_sub(xc, {Hc[o - BOXW], Lc[o - BOXW]}));
      if (gj < ny - 1) dy = ff_add(dy, ff_sub(xc, {Hc[o + BOXW], Lc[o + BOXW]}));
      if (hm) dz = ff_add(dz, ff_sub(xc, {Hm[o], Lm[o]}));
      if (hp) dz = ff_add(dz, ff_sub(xc, {Hp[o], Lp[o]}));
      ff ax = ff_add(ff_mul(dx, Wx), ff_mul(dy, Wy));
      ax = ff_add(ax, ff_mul(dz, Wz));
      ax = ff_add(ax, ff_mul(xc, Wa));
      ff bv;
      if (RHS == RHS_EXPLICIT) {
        bv = {I0[o], 0.f};
      } else {
        const float ic = I0[o];
        float gx = 0.f, gy = 0.f;
        if (gi > 0) gx += ic - I0[o - 1];
        if (gi < nx - 1) gx += ic - I0[o + 1];
        if (gj > 0) gy += ic - I0[o - BOXW];
        if (gj < ny - 1) gy += ic - I0[o + BOXW];
        bv = ff_add(ff_mul({gx, 0.f}, Rx), ff_mul({gy, 0.f}, Ry));
        if (SP) bv = ff_add(bv, ff_mul({I1[o], 0.f}, Ra));
        si += (double)ic;
      }
      const ff rr = ff_sub(bv, ax);
      const size_t g = (size_t)p * plane + (size_t)gj * nx + gi;
      if (a.xh_out) {
        a.xh_out[g] = xc.h;
        a.xl_out[g] = xc.l;
      }
      if (a.r_out) a.r_out[g] = __fadd_rn(rr.h, rr.l);
      const double rd = (double)rr.h + (double)rr.l;
      const double bd = (double)bv.h + (double)bv.l;
      srr += rd * rd;
      sbb += bd * bd;
      sx += (double)xc.h + (double)xc.l;
    }
  };

  for (int t = t0; t <= t1; ++t) {
    if (tid == 0) {
      fence_proxy_async();
      issue_x(zc ? t + 1 + PF : t + PF);
      issue_i(t + PF);
    }
    ready_x(zc ? t + 1 : t);
    ready_i(t);
    __syncthreads();
    if (abort_flag) break;
    if (t >= zs) residual_plane(t);
    __syncthreads();
  }
  if (abort_flag) {
    if (tid == 0) {
      err[0] = 1.0;
      for (int p = xready + 1; p <= xissued; ++p) {
        mbar_wait(&hb[rx.slot(p)], rx.parity(p));
        if (HAS_XL) mbar_wait(&lb[rx.slot(p)], rx.parity(p));
        if (HAS_E) mbar_wait(&eb[re.slot(p)], re.parity(p));
      }
      for (int p = iready + 1; p <= iissued; ++p) {
        mbar_wait(&ib0[ri.slot(p)], ri.parity(p));
        if (SP) mbar_wait(&ib1[ri.slot(p)], ri.parity(p));
      }
    }
    return;
  }
  const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  double v;
  v = block_sum(srr, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_RR] = v;
  v = block_sum(sbb, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_BB] = v;
  v = block_sum(sx, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_X] = v;
  v = block_sum(si, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_I0] = v;
}

// ===========================================================================
// host side: tensor maps and launchers
// ===========================================================================
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_encode_state = 0;  // 0 unknown, 1 ok, -1 unavailable

bool encoder() {
  if (g_encode_state == 0) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess && fn) {
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
      g_encode_state = 1;
    } else {
      cudaGetLastError();
      g_encode_state = -1;
    }
  }
  return g_encode_state == 1;
}

// 3D map over a float32 [nz][ny][nx] array with a (BOXW x rows x 1) box.
bool make_map(CUtensorMap *m, const float *base, int nx, int ny, int nz, int rows) {
  if (!encoder() || !base) return false;
  if (((uintptr_t)base & 15) != 0 || (nx & 3) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)BOXW, (cuuint32_t)rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides,
                  box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      n = 152;
  }
  return n;
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// z chunking: a few waves of resident CTAs; coupled chunks are even and >= 16
// planes deep (each chunk re-reads a few halo planes)
int pick_zchunk(int tiles, int nz, bool coupled, int ctas_per_sm) {
  const long target = (long)sm_count() * ctas_per_sm * 4;
  long chunks = (target + tiles - 1) / tiles;
  const int min_chunk = coupled ? 16 : 1;
  const long max_chunks = (nz + min_chunk - 1) / min_chunk;
  if (chunks > max_chunks) chunks = max_chunks;
  if (chunks < 1) chunks = 1;
  int zc = (int)((nz + chunks - 1) / chunks);
  if (coupled && (zc & 1)) ++zc;
  return zc;
}

template <bool Z, bool P, bool R, bool S>
cudaError_t run_zsweep(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a, dim3 grid,
                       cudaStream_t st) {
  const size_t bytes = SweepGeo<R>::smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem(k_zsweep<Z, P, R, S>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_zsweep<Z, P, R, S><<<grid, ZNT, bytes, st>>>(mx, mb, a);
  return cudaGetLastError();
}

template <int RHS, bool XL, bool E>
cudaError_t run_zouter(const CUtensorMap *m, const OuterArgs &a, int zchunk, double *err, dim3 grid,
                       cudaStream_t st) {
  const size_t bytes = OuterGeo::smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem(k_zouter<RHS, XL, E>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_zouter<RHS, XL, E><<<grid, ZNT, bytes, st>>>(m[0], m[1], m[2], m[3], m[4], a, zchunk, err);
  return cudaGetLastError();
}

}  // namespace

bool zmarch_usable(const LevelDev &L) { return encoder() && (L.nx & 3) == 0; }

cudaError_t launch_zsweep(ZSweepArgs a, const float *xin, const float *b, bool zero_in, bool prolong,
                          bool restrict_, bool sum, int *nblocks_out, cudaStream_t st) {
  const LevelDev &L = a.L;
  const bool R = restrict_;
  const int rows_x = ZY + 2 * (R ? 3 : 2), rows_b = ZY + 2 * (R ? 2 : 1);
  CUtensorMap mx, mb;
  std::memset(&mx, 0, sizeof mx);
  if (!zero_in && !make_map(&mx, xin, L.nx, L.ny, L.nz, rows_x)) return cudaErrorNotSupported;
  if (zero_in && !make_map(&mx, b, L.nx, L.ny, L.nz, rows_x)) return cudaErrorNotSupported;
  if (!make_map(&mb, b, L.nx, L.ny, L.nz, rows_b)) return cudaErrorNotSupported;
  if (((uintptr_t)a.xout & 15) != 0) return cudaErrorNotSupported;
  const int gx = (L.nx + ZX - 1) / ZX, gy = (L.ny + ZY - 1) / ZY;
  const bool coupled = (L.wz != 0.f) && (L.nz > 1);
  a.zchunk = pick_zchunk(gx * gy, L.nz, coupled, R ? 2 : 3);
  const int gz = (L.nz + a.zchunk - 1) / a.zchunk;
  if (nblocks_out) *nblocks_out = gx * gy * gz;
  dim3 grid(gx, gy, gz);
  if (zero_in && !prolong && !R && !sum) return run_zsweep<true, false, false, false>(mx, mb, a, grid, st);
  if (zero_in && !prolong && R && !sum) return run_zsweep<true, false, true, false>(mx, mb, a, grid, st);
  if (!zero_in && !prolong && R && !sum) return run_zsweep<false, false, true, false>(mx, mb, a, grid, st);
  if (!zero_in && prolong && !R && !sum) return run_zsweep<false, true, false, false>(mx, mb, a, grid, st);
  if (!zero_in && prolong && !R && sum) return run_zsweep<false, true, false, true>(mx, mb, a, grid, st);
  if (!zero_in && !prolong && !R && !sum) return run_zsweep<false, false, false, false>(mx, mb, a, grid, st);
  if (!zero_in && !prolong && !R && sum) return run_zsweep<false, false, false, true>(mx, mb, a, grid, st);
  if (!zero_in && prolong && R && !sum) return run_zsweep<false, true, true, false>(mx, mb, a, grid, st);
  return cudaErrorNotSupported;
}

cudaError_t launch_zouter(const OuterArgs &a, int rhs_mode, double *err, int *nblocks_out,
                          cudaStream_t st) {
  if ((a.nx & 3) != 0) return cudaErrorNotSupported;
  const int rows = ZY + 2;
  CUtensorMap m[5];
  std::memset(m, 0, sizeof m);
  const float *rhs0 = rhs_mode == RHS_EXPLICIT ? a.b : a.I0;
  if (!make_map(&m[0], a.xh_in, a.nx, a.ny, a.nz, rows)) return cudaErrorNotSupported;
  if (a.xl_in && !make_map(&m[1], a.xl_in, a.nx, a.ny, a.nz, rows)) return cudaErrorNotSupported;
  if (a.e && !make_map(&m[2], a.e, a.nx, a.ny, a.nz, rows)) return cudaErrorNotSupported;
  if (!make_map(&m[3], rhs0, a.nx, a.ny, a.nz, rows)) return cudaErrorNotSupported;
  if (rhs_mode == RHS_SP && !make_map(&m[4], a.I1, a.nx, a.ny, a.nz, rows)) return cudaErrorNotSupported;
  const int gx = (a.nx + ZX - 1) / ZX, gy = (a.ny + ZY - 1) / ZY;
  const bool coupled = (a.bz != 0.f) && (a.nz > 1);
  const int zchunk = pick_zchunk(gx * gy, a.nz, coupled, 2);
  const int gz = (a.nz + zchunk - 1) / zchunk;
  if (nblocks_out) *nblocks_out = gx * gy * gz;
  dim3 grid(gx, gy, gz);
  const bool xl = a.xl_in != nullptr, e = a.e != nullptr;
#define GD_ZO(R)                                                     \
  if (xl && e) return run_zouter<R, true, true>(m, a, zchunk, err, grid, st);   \
  if (xl) return run_zouter<R, true, false>(m, a, zchunk, err, grid, st);       \
  if (e) return run_zouter<R, false, true>(m, a, zchunk, err, grid, st);        \
  return run_zouter<R, false, false>(m, a, zchunk, err, grid, st);
  if (rhs_mode == RHS_EXPLICIT) { GD_ZO(RHS_EXPLICIT) }
  if (rhs_mode == RHS_AD) { GD_ZO(RHS_AD) }
  GD_ZO(RHS_SP)
#undef GD_ZO
}

int zouter_max_blocks(int nx, int ny, int nz) {
  const int gx = (nx + ZX - 1) / ZX, gy = (ny + ZY - 1) / ZY;
  return gx * gy * nz;
}
