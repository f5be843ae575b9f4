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
//     SUM       the block sums of the written iterate (mean fix of AD).
//   Pipeline per step t: red of plane t on the tile + 1 ring, black of plane
//   t-1 on the tile, store plane t-1.  The ring recomputes the neighbouring
//   CTA's red values exactly as it does, so the result is the textbook
//   red-black sweep.
//
// k_zrestrict: residual r = b - A x and its down-sampling (sum over the
//   children of each coarse cell, Sec. 4.1 / 4.2) into the next level's
//   right-hand side.
//
// k_zouter: fine-level outer pass of the iterative refinement: x_new = x + e
//   (+ mean shift) as a float pair, r = b - A x_new in double-float arithmetic
//   with b assembled from I0 (and I1), and FP64 block partial sums.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <cstring>
#include <type_traits>

#include "gd_internal.h"

namespace {

constexpr int ZX = 64;            // tile x extent
constexpr int ZY = 16;            // tile y extent
constexpr int ZNT = 256;          // threads per CTA
constexpr int NTY = ZNT / ZX;      // thread rows of the tile-cell map
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
// (p - lo) is never negative; power-of-two depths make these masks and shifts.
template <int DEPTH>
struct Ring {
  int lo, hi;
  __device__ __forceinline__ bool has(int p) const { return p >= lo && p <= hi; }
  __device__ __forceinline__ int slot(int p) const { return (int)((uint32_t)(p - lo) % DEPTH); }
  __device__ __forceinline__ uint32_t parity(int p) const {
    return ((uint32_t)(p - lo) / DEPTH) & 1;
  }
};

// ===========================================================================
// red-black sweep
// ===========================================================================
// Dynamic shared memory of the z-march kernels, addressed with 32-bit float
// offsets (slots are multiples of 32 floats, i.e. 128 bytes).
extern __shared__ __align__(128) float zsm[];

struct SweepGeo {
  static constexpr int H = 2;                    // x box halo in y
  static constexpr int XH = ZY + 2 * H;          // x box rows
  static constexpr int BH = ZY + 2 * (H - 1);    // b box rows
  // ring depths: planes in use plus PF in flight, rounded up to a power of two
  static constexpr int XR = 8;                   // needs 4 + PF
  static constexpr int BR = 4;                   // needs 2 + PF
  static_assert(XR >= 4 + PF && BR >= 2 + PF, "ring depth");
  static constexpr int XS = pad32(XH * BOXW);    // floats per x slot
  static constexpr int BS = pad32(BH * BOXW);
  static constexpr int BOFF = XR * XS;           // b slots
  static constexpr int MOFF = BOFF + BR * BS;    // mbarriers
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(float) * (size_t)MOFF + sizeof(uint64_t) * (XR + BR) + sizeof(double) * 32 + 16;
  }
};

template <bool ZERO_IN, bool PROLONG, bool SUM, bool UNIFORM>
__global__ void __launch_bounds__(ZNT, 2) k_zsweep(const __grid_constant__ CUtensorMap tmx,
                                                   const __grid_constant__ CUtensorMap tmb,
                                                   const ZSweepArgs a) {
  using G = SweepGeo;
  constexpr int H = G::H;
  uint64_t *xbar = reinterpret_cast<uint64_t *>(zsm + G::MOFF);
  uint64_t *bbar = xbar + G::XR;
  double *dsh = reinterpret_cast<double *>(bbar + G::BR);
  __shared__ int abort_flag;

  const LevelDev &L = a.L;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * ZY;
  const int zs = blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, nz);
  const bool zc = (L.wz != 0.f) && (nz > 1);
  const int t0 = zc ? zs - 1 : zs;
  const int t1 = zc ? ze : ze - 1;
  const int lagb = zc ? 1 : 0;
  const int red_lo = zc ? max(zs - 1, 0) : zs, red_hi = zc ? min(ze, nz - 1) : ze - 1;
  const int blk_lo = zs, blk_hi = ze - 1;
  Ring<G::XR> rx;
  rx.lo = zc ? max(t0 - 1, 0) : zs;
  rx.hi = zc ? min(t1 + 1, nz - 1) : ze - 1;
  Ring<G::BR> rb;
  rb.lo = zc ? max(t0, 0) : zs;
  rb.hi = zc ? min(t1, nz - 1) : ze - 1;
  const size_t plane = (size_t)nx * ny;

  if (tid == 0) {
    abort_flag = 0;
    int e = tma_preflight(zsm, G::smem_bytes(), &tmx);
    if (!e) e = tma_preflight(zsm, G::smem_bytes(), &tmb);
    if (e) {
      abort_flag = e;
      a.err[0] = (double)e;
    } else {
      for (int q = 0; q < G::XR; ++q) mbar_init(&xbar[q], 1);
      for (int q = 0; q < G::BR; ++q) mbar_init(&bbar[q], 1);
      fence_mbar_init();
    }
  }
  if (ZERO_IN) {
    // x is never loaded: cells outside the domain must read 0 for good, and
    // every cell inside is written before it is read
    for (int q = tid; q < G::XR * G::XS; q += ZNT) zsm[q] = 0.f;
  }
  __syncthreads();
  if (abort_flag) return;  // nothing issued yet

  int xissued = rx.lo - 1, bissued = rb.lo - 1;  // thread 0
  auto issue_x = [&](int p) {
    if (ZERO_IN || !rx.has(p)) return;
    const int q = rx.slot(p);
    mbar_expect_tx(&xbar[q], (uint32_t)(G::XH * BOXW * sizeof(float)));
    tma_plane(zsm + q * G::XS, &tmx, i0 - 4, j0 - H, p, &xbar[q]);
    xissued = p;
  };
  auto issue_b = [&](int p) {
    if (!rb.has(p)) return;
    const int q = rb.slot(p);
    mbar_expect_tx(&bbar[q], (uint32_t)(G::BH * BOXW * sizeof(float)));
    tma_plane(zsm + G::BOFF + q * G::BS, &tmb, i0 - 4, j0 - (H - 1), p, &bbar[q]);
    bissued = p;
  };
  const int xnext0 = zc ? t0 + 1 + PF : t0 + PF;
  if (tid == 0) {
    for (int p = rx.lo; p < xnext0 && p <= rx.hi; ++p) issue_x(p);
    for (int p = rb.lo; p < t0 + PF && p <= rb.hi; ++p) issue_b(p);
  }
  int xready = rx.lo - 1, bready = rb.lo - 1;  // planes made usable (all threads)
  int xwait = rx.lo - 1, bwait = rb.lo - 1;    // planes whose wait succeeded (warp 0)
  auto xo = [&](int p) { return rx.slot(p) * G::XS; };
  auto bo = [&](int p) { return G::BOFF + rb.slot(p) * G::BS; };

  // ---- per-thread constants ----
  // Tile cells: thread (tx, ty) owns column tx and rows of the row pairs
  // ty, ty + NTY, ...; in a colour phase it takes the row of each pair with the
  // right parity, so the 32 lanes of a warp alternate between two rows
  // (row stride 72 floats = 8 banks) and never share a bank.
  const int tx = tid % ZX, ty = tid / ZX;
  const int gi = i0 + tx;
  const bool col_in = gi < nx;
  const float nbx = (float)((gi > 0) + (gi < nx - 1));
  const float cxu = L.wx * (float)L.sy * (float)L.sz;
  const float cyu = L.wy * (float)L.sx * (float)L.sz;
  const float czu = zc ? L.wz * (float)L.sx * (float)L.sy : 0.f;
  const float mmu = L.wm * (float)L.sx * (float)L.sy * (float)L.sz;

  // Gauss-Seidel update of one cell: x = (b + sum_n c_n x_n) / diag.  Cells
  // outside the domain read 0 and are never written; missing neighbours are
  // left out of the diagonal by the neighbour counts.  RED0: the first red
  // pass of a zero iterate (all neighbours are 0).
  auto cell = [&](auto red0_c, int xop, int xmo, int xpo, int bop, int so, int gci, int gcj,
                  float mz, float zmf, float zpf, float nbxc) {
    constexpr bool RED0 = decltype(red0_c)::value;
    float cx = cxu, cy = cyu, cz = czu, mm = mmu;
    if (!UNIFORM) {
      const float mx = mass_of(gci, nx, L.sx, L.lx), my = mass_of(gcj, ny, L.sy, L.ly);
      cx = L.wx * my * mz;
      cy = L.wy * mx * mz;
      cz = zc ? L.wz * mx * my : 0.f;
      mm = L.wm * mx * my * mz;
    }
    const float nby = (float)((gcj > 0) + (gcj < ny - 1));
    const float dg = cx * nbxc + cy * nby + cz * (zmf + zpf) + mm;
    const float bv = zsm[bop + so - BOXW];
    float v;
    if (RED0) {
      v = __fdividef(bv, dg);
    } else {
      float sacc = cx * (zsm[xop + so - 1] + zsm[xop + so + 1]) +
                   cy * (zsm[xop + so - BOXW] + zsm[xop + so + BOXW]);
      if (zc) sacc += cz * (zmf * zsm[xmo + so] + zpf * zsm[xpo + so]);
      v = __fdividef(bv + sacc, dg);
    }
    zsm[xop + so] = v;
  };
  // Fast path: a uniform level and a tile whose cells and their neighbours
  // all lie inside the domain in x and y (z faces are handled by zmf / zpf).
  const bool fast = UNIFORM && (i0 >= 3) && (i0 + ZX + 3 <= nx) && (j0 >= 3) && (j0 + ZY + 3 <= ny);
  // Ring cells of this thread (red ring H-1, black ring H-2), decoded once.
  constexpr int RMAX = 1;  // ring cells per thread: ceil(164 / 256)
  int rso[RMAX], rpar[RMAX], rgi[RMAX], rgj[RMAX], rring[RMAX];
#pragma unroll
  for (int m = 0; m < RMAX; ++m) {
    rso[m] = -1;
    rpar[m] = rgi[m] = rgj[m] = rring[m] = 0;
    const int RG = H - 1;  // widest ring (the red one)
    const int WR = ZX + 2 * RG, NTB = RG * WR, NLR = ZY * RG;
    const int q = tid + m * ZNT;
    if (q < 2 * NTB + 2 * NLR) {
      int row, col;
      if (q < NTB) {
        row = -RG + q / WR; col = -RG + q % WR;
      } else if (q < 2 * NTB) {
        row = ZY + (q - NTB) / WR; col = -RG + (q - NTB) % WR;
      } else if (q < 2 * NTB + NLR) {
        row = (q - 2 * NTB) / RG; col = -RG + (q - 2 * NTB) % RG;
      } else {
        row = (q - 2 * NTB - NLR) / RG; col = ZX + (q - 2 * NTB - NLR) % RG;
      }
      const int gci = i0 + col, gcj = j0 + row;
      if (gci >= 0 && gci < nx && gcj >= 0 && gcj < ny) {
        rso[m] = (row + H) * BOXW + 4 + col;
        rpar[m] = (gci + gcj) & 1;
        rgi[m] = gci;
        rgj[m] = gcj;
        // distance of the cell outside the tile (1 or 2)
        const int dx = col < 0 ? -col : (col >= ZX ? col - ZX + 1 : 0);
        const int dy = row < 0 ? -row : (row >= ZY ? row - ZY + 1 : 0);
        rring[m] = dx > dy ? dx : dy;
      }
    }
  }
  auto relax = [&](auto ring_c, auto colour_c, int p) {
    constexpr int RING = decltype(ring_c)::value;
    constexpr int COLOUR = decltype(colour_c)::value;
    constexpr bool RED0 = ZERO_IN && COLOUR == 0;
    const std::integral_constant<bool, RED0> red0;
    const int xop = xo(p);
    const bool hm = zc && p > 0, hp = zc && p < nz - 1;
    const int xmo = hm ? xo(p - 1) : xop, xpo = hp ? xo(p + 1) : xop;
    const int bop = bo(p);
    const float zmf = hm ? 1.f : 0.f, zpf = hp ? 1.f : 0.f;
    const float mz = mass_of(p, nz, L.sz, L.lz);
    const int d = (tx + p + COLOUR) & 1;  // i0, j0 even
    if (fast) {
      const float idg = 1.f / (2.f * (cxu + cyu) + czu * (zmf + zpf) + mmu);
      const float czm = czu * zmf, czp = czu * zpf;
#pragma unroll
      for (int k = 0; k < ZY / (2 * NTY); ++k) {
        const int so = (2 * (ty + NTY * k) + d + H) * BOXW + 4 + tx;
        const float bv = zsm[bop + so - BOXW];
        float v;
        if (RED0) {
          v = bv * idg;
        } else {
          const float *xc = zsm + xop + so;
          float sacc = cxu * (xc[-1] + xc[1]) + cyu * (xc[-BOXW] + xc[BOXW]);
          if (zc) sacc += czm * zsm[xmo + so] + czp * zsm[xpo + so];
          v = (bv + sacc) * idg;
        }
        zsm[xop + so] = v;
      }
    } else {
#pragma unroll
      for (int k = 0; k < ZY / (2 * NTY); ++k) {
        const int row = 2 * (ty + NTY * k) + d;
        const int gj = j0 + row;
        if (col_in && gj < ny)
          cell(red0, xop, xmo, xpo, bop, (row + H) * BOXW + 4 + tx, gi, gj, mz, zmf, zpf, nbx);
      }
    }
    if constexpr (RING > 0) {
#pragma unroll
      for (int m = 0; m < RMAX; ++m) {
        if (rso[m] >= 0 && rring[m] <= RING && ((rpar[m] + p) & 1) == COLOUR) {
          const float nbxc = (float)((rgi[m] > 0) + (rgi[m] < nx - 1));
          cell(red0, xop, xmo, xpo, bop, rso[m], rgi[m], rgj[m], mz, zmf, zpf, nbxc);
        }
      }
    }
  };
  // double-float block sums in FP32 (the FP64 pipe is narrow)
  float sum_h = 0.f, sum_l = 0.f;
  auto store = [&](int p) {
    const int xop = xo(p);
#pragma unroll
    for (int q = tid; q < ZX * ZY / 4; q += ZNT) {
      const int r = q >> 4, c = (q & 15) * 4;
      const int gci = i0 + c, gcj = j0 + r;
      if (gci < nx && gcj < ny) {
        const float4 v = *reinterpret_cast<const float4 *>(zsm + xop + (r + H) * BOXW + 4 + c);
        *reinterpret_cast<float4 *>(a.xout + (size_t)p * plane + (size_t)gcj * nx + gci) = v;
        if (SUM) {
          const float s4 = (v.x + v.y) + (v.z + v.w);
          const float sn = sum_h + s4;
          const float bb = sn - sum_h;
          sum_l += (sum_h - (sn - bb)) + (s4 - bb);
          sum_h = sn;
        }
      }
    }
  };
  // Prolongation: this thread's slot cells (columns 4-H .. 68+H-1 are the
  // only ones any stage reads) and their offsets within a coarse plane.
  constexpr int PW = ZX + 2 * H;
  constexpr int PMAX = PROLONG ? (G::XH * PW + ZNT - 1) / ZNT : 1;
  int pso[PMAX], pco[PMAX];
  float pv[PMAX];
  int pf_plane = -1;  // plane whose coarse values are in pv
#pragma unroll
  for (int m = 0; m < PMAX; ++m) {
    pso[m] = -1;
    pco[m] = 0;
    pv[m] = 0.f;
    const int q = tid + m * ZNT;
    if (PROLONG && q < G::XH * PW) {
      const int r = q / PW, c = q - r * PW + (4 - H);
      const int gci = i0 - 4 + c, gcj = j0 - H + r;
      if (gci >= 0 && gci < nx && gcj >= 0 && gcj < ny) {
        pso[m] = r * BOXW + c;
        pco[m] = (gcj >> a.fy) * a.ncx + (gci >> a.fx);
      }
    }
  }

  for (int t = t0; t <= t1; ++t) {
    if (tid == 0) {
      fence_proxy_async();
      issue_x(zc ? t + 1 + PF : t + PF);
      issue_b(t + PF);
    }
    // one warp waits for the planes of this step, then the barrier releases all
    const int ux = min(zc ? t + 1 : t, rx.hi), ub = min(t, rb.hi);
    // Without the prolongation every warp waits for this step's planes itself
    // (no barrier needed); with it, warp 0 waits, the barrier releases the CTA
    // and the coarse correction is added before anyone relaxes.
    if (!PROLONG || warp == 0) {
      bool ok = true;
      if (!ZERO_IN)
        for (int p = xwait + 1; p <= ux && ok; ++p) {
          ok = mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
          if (ok) xwait = p;
        }
      for (int p = bwait + 1; p <= ub && ok; ++p) {
        ok = mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
        if (ok) bwait = p;
      }
      if (!ok) abort_flag = 1;
    }
    const int xprev = xready;
    if (ux > xready) xready = ux;
    if (ub > bready) bready = ub;
    if (PROLONG) {
      __syncthreads();
      if (abort_flag) break;
      // the up-sampled coarse correction, added once to every plane loaded;
      // the values of the next plane were requested one step ahead
      for (int p = xprev + 1; p <= xready; ++p) {
        const int xop = xo(p);
        if (p == pf_plane) {
#pragma unroll
          for (int m = 0; m < PMAX; ++m)
            if (pso[m] >= 0) zsm[xop + pso[m]] += pv[m];
        } else {
          const float *xcp = a.xc + (size_t)(p >> a.fz) * a.ncy * a.ncx;
#pragma unroll
          for (int m = 0; m < PMAX; ++m)
            if (pso[m] >= 0) zsm[xop + pso[m]] += __ldg(xcp + pco[m]);
        }
      }
      pf_plane = xready + 1;
      if (pf_plane <= rx.hi) {
        const float *xcp = a.xc + (size_t)(pf_plane >> a.fz) * a.ncy * a.ncx;
#pragma unroll
        for (int m = 0; m < PMAX; ++m) pv[m] = pso[m] >= 0 ? __ldg(xcp + pco[m]) : 0.f;
      }
      __syncthreads();
    }
    if (t >= red_lo && t <= red_hi)
      relax(std::integral_constant<int, H - 1>(), std::integral_constant<int, 0>(), t);
    __syncthreads();
    if (abort_flag) break;
    const int pb = t - lagb;
    if (pb >= blk_lo && pb <= blk_hi)
      relax(std::integral_constant<int, H - 2>(), std::integral_constant<int, 1>(), pb);
    __syncthreads();
    if (pb >= zs && pb < ze) store(pb);
    // the next issue targets x(t-2) / b(t-1), whose last reads (black of
    // plane t-1) precede the barrier above
  }
  if (abort_flag) {
    // a TMA completion did not arrive in time: flag it, give the copies this
    // CTA still has in flight a bounded wait to land, and leave
    if (tid == 0) {
      a.err[0] = 1.0;
      for (int p = xwait + 1; p <= xissued; ++p) mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
      for (int p = bwait + 1; p <= bissued; ++p) mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
    }
    return;
  }
  if (SUM) {
    const double sv = block_sum((double)sum_h + (double)sum_l, dsh);
    if (tid == 0) {
      const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[blk * S_NUM + S_E] = sv;
    }
  }
}

// ===========================================================================
// residual + down-sampling
// ===========================================================================
struct RestrictGeo {
  static constexpr int XH = ZY + 2;              // x box rows: tile + 1 halo
  static constexpr int XR = 8;                   // x planes t-1..t+1 + PF in flight
  static constexpr int BR = 4;                   // b plane t + PF in flight
  static_assert(XR >= 3 + PF && BR >= 1 + PF, "ring depth");
  static constexpr int XS = pad32(XH * BOXW);
  static constexpr int BS = pad32(ZY * ZX);      // b box: the tile only
  static constexpr int BOFF = XR * XS;
  static constexpr int ROFF = BOFF + BR * BS;    // residual of a plane, two buffers
  static constexpr int AOFF = ROFF + 2 * ZX * ZY;  // first child plane's sums
  static constexpr int MOFF = AOFF + ZX * ZY;
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(float) * (size_t)MOFF + sizeof(uint64_t) * (XR + BR) + 16;
  }
};

template <bool UNIFORM>
__global__ void __launch_bounds__(ZNT, 2) k_zrestrict(const __grid_constant__ CUtensorMap tmx,
                                                      const __grid_constant__ CUtensorMap tmb,
                                                      const ZSweepArgs a) {
  using G = RestrictGeo;
  uint64_t *xbar = reinterpret_cast<uint64_t *>(zsm + G::MOFF);
  uint64_t *bbar = xbar + G::XR;
  __shared__ int abort_flag;
  const LevelDev &L = a.L;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int tid = threadIdx.x;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * ZY;
  const int zs = blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, nz);
  const bool zc = (L.wz != 0.f) && (nz > 1);
  Ring<G::XR> rx;
  rx.lo = zc ? max(zs - 1, 0) : zs;
  rx.hi = zc ? min(ze, nz - 1) : ze - 1;
  Ring<G::BR> rb;
  rb.lo = zs;
  rb.hi = ze - 1;
  if (tid == 0) {
    abort_flag = 0;
    int e = tma_preflight(zsm, G::smem_bytes(), &tmx);
    if (!e) e = tma_preflight(zsm, G::smem_bytes(), &tmb);
    if (e) {
      abort_flag = e;
      a.err[0] = (double)e;
    } else {
      for (int q = 0; q < G::XR; ++q) mbar_init(&xbar[q], 1);
      for (int q = 0; q < G::BR; ++q) mbar_init(&bbar[q], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (abort_flag) return;
  int xissued = rx.lo - 1, bissued = rb.lo - 1;  // thread 0
  auto issue_x = [&](int p) {
    if (!rx.has(p)) return;
    const int q = rx.slot(p);
    mbar_expect_tx(&xbar[q], (uint32_t)(G::XH * BOXW * sizeof(float)));
    tma_plane(zsm + q * G::XS, &tmx, i0 - 4, j0 - 1, p, &xbar[q]);
    xissued = p;
  };
  auto issue_b = [&](int p) {
    if (!rb.has(p)) return;
    const int q = rb.slot(p);
    mbar_expect_tx(&bbar[q], (uint32_t)(ZY * ZX * sizeof(float)));
    tma_plane(zsm + G::BOFF + q * G::BS, &tmb, i0, j0, p, &bbar[q]);
    bissued = p;
  };
  // step t: residual of plane t (needs x of t-1, t, t+1)
  const int t0 = zs, t1 = ze - 1;
  const int xnext0 = zc ? t0 + 1 + PF : t0 + PF;
  if (tid == 0) {
    for (int p = rx.lo; p < xnext0 && p <= rx.hi; ++p) issue_x(p);
    for (int p = rb.lo; p < t0 + PF && p <= rb.hi; ++p) issue_b(p);
  }
  int xwait = rx.lo - 1, bwait = rb.lo - 1;  // warp 0
  const int tx = tid % ZX, ty = tid / ZX;
  const int gi = i0 + tx;
  const bool col_in = gi < nx;
  const float nbx = (float)((gi > 0) + (gi < nx - 1));
  const float cxu = L.wx * (float)L.sy * (float)L.sz;
  const float cyu = L.wy * (float)L.sx * (float)L.sz;
  const float czu = zc ? L.wz * (float)L.sx * (float)L.sy : 0.f;
  const float mmu = L.wm * (float)L.sx * (float)L.sy * (float)L.sz;
  const int fx = a.fx, fy = a.fy, fz = a.fz;
  const int CW = ZX >> fx, CH = ZY >> fy;
  for (int t = t0; t <= t1; ++t) {
    if (tid == 0) {
      fence_proxy_async();
      issue_x(zc ? t + 1 + PF : t + PF);
      issue_b(t + PF);
    }
    const int ux = min(zc ? t + 1 : t, rx.hi), ub = min(t, rb.hi);
    {
      // every warp waits for its planes itself
      bool ok = true;
      for (int p = xwait + 1; p <= ux && ok; ++p) {
        ok = mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
        if (ok) xwait = p;
      }
      for (int p = bwait + 1; p <= ub && ok; ++p) {
        ok = mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
        if (ok) bwait = p;
      }
      if (!ok) abort_flag = 1;
    }
    const int p = t;
    const int roff = G::ROFF + (t & 1) * ZX * ZY;  // residual buffer of this step
    const int xop = rx.slot(p) * G::XS;
    const bool hm = zc && p > 0, hp = zc && p < nz - 1;
    const int xmo = hm ? rx.slot(p - 1) * G::XS : xop, xpo = hp ? rx.slot(p + 1) * G::XS : xop;
    const int bop = G::BOFF + rb.slot(p) * G::BS;
    const float zmf = hm ? 1.f : 0.f, zpf = hp ? 1.f : 0.f;
    const float mz = mass_of(p, nz, L.sz, L.lz);
    const float czm = czu * zmf, czp = czu * zpf;
#pragma unroll
    for (int k = 0; k < ZY / NTY; ++k) {
      const int row = ty + NTY * k, gj = j0 + row;
      float rv = 0.f;
      if (col_in && gj < ny) {
        const int so = (row + 1) * BOXW + 4 + tx;
        float cx = cxu, cy = cyu, cz = czu, mm = mmu;
        if (!UNIFORM) {
          const float mx = mass_of(gi, nx, L.sx, L.lx), my = mass_of(gj, ny, L.sy, L.ly);
          cx = L.wx * my * mz;
          cy = L.wy * mx * mz;
          cz = zc ? L.wz * mx * my : 0.f;
          mm = L.wm * mx * my * mz;
        }
        const float nby = (float)((gj > 0) + (gj < ny - 1));
        const float dg = cx * nbx + cy * nby + cz * (zmf + zpf) + mm;
        const float *xc = zsm + xop + so;
        float sacc = cx * (xc[-1] + xc[1]) + cy * (xc[-BOXW] + xc[BOXW]);
        if (zc) sacc += (UNIFORM ? czm : cz * zmf) * zsm[xmo + so] + (UNIFORM ? czp : cz * zpf) * zsm[xpo + so];
        rv = zsm[bop + row * ZX + tx] + sacc - dg * xc[0];  // b - A x
      }
      zsm[roff + row * ZX + tx] = rv;
    }
    __syncthreads();
    if (abort_flag) break;
    const size_t cpl = (size_t)(p >> fz) * a.ncy;
    for (int q = tid; q < CW * CH; q += ZNT) {
      const int cr = q / CW, cc = q - cr * CW;
      const float *r0 = zsm + roff + (cr << fy) * ZX + (cc << fx);
      float sv = r0[0];
      if (fx) sv += r0[1];
      if (fy) {
        sv += r0[ZX];
        if (fx) sv += r0[ZX + 1];
      }
      const int I = (i0 >> fx) + cc, J = (j0 >> fy) + cr;
      if (fz && (p & 1) == 0 && p != nz - 1) {
        zsm[G::AOFF + q] = sv;  // first child plane: keep for the second
      } else {
        if (fz && (p & 1) == 1) sv += zsm[G::AOFF + q];
        if (I < a.ncx && J < a.ncy) a.bc[(cpl + J) * a.ncx + I] = sv;
      }
    }
    // The next issue targets x(t-5) / b(t-2): dead.  The next step writes the
    // other residual buffer; this one is rewritten two steps on, after the
    // next step's barrier.
  }
  if (abort_flag) {
    if (tid == 0) {
      a.err[0] = 1.0;
      for (int p = xwait + 1; p <= xissued; ++p) mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
      for (int p = bwait + 1; p <= bissued; ++p) mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
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
struct OuterGeo {
  static constexpr int BH = ZY + 2;              // rows: tile + 1 halo
  static constexpr int S = pad32(BH * BOXW);
  static constexpr int XR = 3 + PF;              // x_new planes t-1..t+1 + in flight
  static constexpr int ER = 3 + PF;              // corrections: same planes and lag as x
  static constexpr int IR = 1 + PF;              // inputs: plane t + in flight
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(float) * (size_t)S * (2 * XR + ER + 2 * IR) +
           sizeof(uint64_t) * (2 * XR + ER + 2 * IR) + sizeof(double) * 32 + 16;
  }
};

template <int RHS, bool HAS_XL, bool HAS_E, bool ACCURATE>
__global__ void __launch_bounds__(ZNT, 2) k_zouter(const __grid_constant__ CUtensorMap tmh,
                                                const __grid_constant__ CUtensorMap tml,
                                                const __grid_constant__ CUtensorMap tme,
                                                const __grid_constant__ CUtensorMap tmi0,
                                                const __grid_constant__ CUtensorMap tmi1,
                                                const OuterArgs a, int zchunk, double *err) {
  using G = OuterGeo;
  constexpr int S = G::S;
  float *hs = zsm;                                // XR slots: x_new high parts
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
  // the low word of the float pair is carried only in exact passes (and read
  // whenever the caller passes one)
  constexpr bool USE_L = HAS_XL || (HAS_E && ACCURATE);
  constexpr uint32_t BOXB = (uint32_t)(G::BH * BOXW * sizeof(float));

  if (tid == 0) {
    abort_flag = 0;
    int e = tma_preflight(zsm, G::smem_bytes(), &tmh);
    if (!e && HAS_XL) e = tma_preflight(zsm, G::smem_bytes(), &tml);
    if (!e && HAS_E) e = tma_preflight(zsm, G::smem_bytes(), &tme);
    if (!e) e = tma_preflight(zsm, G::smem_bytes(), &tmi0);
    if (!e && SP) e = tma_preflight(zsm, G::smem_bytes(), &tmi1);
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
      if (HAS_E || (USE_L && !HAS_XL)) {
        for (int q = tid; q < G::BH * BOXW; q += ZNT) {
          const float h = Hs[q];
          const float l = HAS_XL ? Ls[q] : 0.f;
          if (HAS_E && ACCURATE) {
            const ff v = ff_add({h, l}, {__fadd_rn(Es[q], shift), 0.f});
            Hs[q] = v.h;
            Ls[q] = v.l;
          } else if (HAS_E) {
            Hs[q] = __fadd_rn(h, __fadd_rn(Es[q], shift));
            if (USE_L) Ls[q] = l;
          } else {
            Ls[q] = 0.f;
          }
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
  // per-thread sums in FP32 (r^2, b^2, I0) and double-float (x); FP64 only
  // once per block
  float srr = 0.f, sbb = 0.f, si = 0.f, sxh = 0.f, sxl = 0.f;
  auto add_x = [&](float v) {
    const ff t = two_sum(sxh, v);
    sxh = t.h;
    sxl += t.l;
  };

  auto residual_plane = [&](int p) {
    const int s = rx.slot(p);
    const float *Hc = hs + s * S, *Lc = ls + s * S;
    const bool hm = zc && p > 0, hp = zc && p < nz - 1;
    const float *Hm = hm ? hs + rx.slot(p - 1) * S : Hc, *Lm = hm ? ls + rx.slot(p - 1) * S : Lc;
    const float *Hp = hp ? hs + rx.slot(p + 1) * S : Hc, *Lp = hp ? ls + rx.slot(p + 1) * S : Lc;
    const float *I0 = i0s + ri.slot(p) * S, *I1 = i1s + ri.slot(p) * S;
#pragma unroll 1
    for (int q = tid; q < ZX * ZY; q += ZNT) {
      const int r = q >> 6, c = q & 63;
      const int gi = i0 + c, gj = j0 + r;
      if (gi >= nx || gj >= ny) continue;
      const int o = (r + 1) * BOXW + 4 + c;
      const bool w = gi > 0, e = gi < nx - 1, so = gj > 0, no = gj < ny - 1;
      const float hc = Hc[o], lc = USE_L ? Lc[o] : 0.f;
      // right-hand side: I0 differences are exact (integer-valued inputs)
      float gx = 0.f, gy = 0.f, bh, bl = 0.f;
      if (RHS == RHS_EXPLICIT) {
        bh = I0[o];
      } else {
        const float ic = I0[o];
        if (w) gx += ic - I0[o - 1];
        if (e) gx += ic - I0[o + 1];
        if (so) gy += ic - I0[o - BOXW];
        if (no) gy += ic - I0[o + BOXW];
        si += ic;
      }
      float rv, rr_h, rr_l;
      if (!ACCURATE) {
        // FP32 differences of the float pair: error ~1e-7 of the local terms
        float dx = 0.f, dy = 0.f, dz = 0.f;
        if (USE_L) {
          if (w) dx += (hc - Hc[o - 1]) + (lc - Lc[o - 1]);
          if (e) dx += (hc - Hc[o + 1]) + (lc - Lc[o + 1]);
          if (so) dy += (hc - Hc[o - BOXW]) + (lc - Lc[o - BOXW]);
          if (no) dy += (hc - Hc[o + BOXW]) + (lc - Lc[o + BOXW]);
          if (hm) dz += (hc - Hm[o]) + (lc - Lm[o]);
          if (hp) dz += (hc - Hp[o]) + (lc - Lp[o]);
        } else {
          if (w) dx += hc - Hc[o - 1];
          if (e) dx += hc - Hc[o + 1];
          if (so) dy += hc - Hc[o - BOXW];
          if (no) dy += hc - Hc[o + BOXW];
          if (hm) dz += hc - Hm[o];
          if (hp) dz += hc - Hp[o];
        }
        const float ax = a.bx * dx + a.by * dy + a.bz * dz + a.alpha * (hc + lc);
        if (RHS != RHS_EXPLICIT) {
          bh = a.rbx * gx + a.rby * gy;
          if (SP) bh += a.ralpha * I1[o];
        }
        rv = bh - ax;
        rr_h = rv;
        rr_l = 0.f;
      } else {
        // compensated evaluation: every rounding error of the hi parts is
        // captured by an error-free transformation and summed into `lo`
        float lo = 0.f;
        auto axis = [&](bool has1, float h1, float l1, bool has2, float h2, float l2, float wh,
                        float wl, float &ph) {
          float t1 = 0.f, t2 = 0.f, la = 0.f;
          if (has1) { const ff d = two_sum(hc, -h1); t1 = d.h; la += d.l + (lc - l1); }
          if (has2) { const ff d = two_sum(hc, -h2); t2 = d.h; la += d.l + (lc - l2); }
          const ff S2 = two_sum(t1, t2);
          la += S2.l;
          const float pp = S2.h * wh;
          lo += __fmaf_rn(S2.h, wh, -pp) + S2.h * wl + la * wh;
          ph = pp;
        };
        float px, py, pz = 0.f;
        auto lo_at = [&](const float *Ls, int oo) { return USE_L ? Ls[oo] : 0.f; };
        axis(w, w ? Hc[o - 1] : 0.f, w ? lo_at(Lc, o - 1) : 0.f, e, e ? Hc[o + 1] : 0.f,
             e ? lo_at(Lc, o + 1) : 0.f, a.bx, a.bx_lo, px);
        axis(so, so ? Hc[o - BOXW] : 0.f, so ? lo_at(Lc, o - BOXW) : 0.f, no,
             no ? Hc[o + BOXW] : 0.f, no ? lo_at(Lc, o + BOXW) : 0.f, a.by, a.by_lo, py);
        if (zc) axis(hm, Hm[o], lo_at(Lm, o), hp, Hp[o], lo_at(Lp, o), a.bz, a.bz_lo, pz);
        const float pa = hc * a.alpha;
        lo += __fmaf_rn(hc, a.alpha, -pa) + hc * a.alpha_lo + lc * a.alpha;
        ff A = two_sum(px, py);
        lo += A.l;
        A = two_sum(A.h, pz);
        lo += A.l;
        A = two_sum(A.h, pa);
        lo += A.l;
        // b as a pair
        if (RHS != RHS_EXPLICIT) {
          const float qx = gx * a.rbx, qy = gy * a.rby;
          bl = __fmaf_rn(gx, a.rbx, -qx) + gx * a.rbx_lo + __fmaf_rn(gy, a.rby, -qy) + gy * a.rby_lo;
          ff Bv = two_sum(qx, qy);
          bl += Bv.l;
          if (SP) {
            const float i1 = I1[o];
            const float qa = i1 * a.ralpha;
            bl += __fmaf_rn(i1, a.ralpha, -qa) + i1 * a.ralpha_lo;
            Bv = two_sum(Bv.h, qa);
            bl += Bv.l;
          }
          bh = Bv.h;
        }
        const ff Rv = two_sum(bh, -A.h);
        rr_h = Rv.h;
        rr_l = Rv.l + (bl - lo);
        rv = rr_h + rr_l;
      }
      const size_t g = (size_t)p * plane + (size_t)gj * nx + gi;
      if (a.xh_out) a.xh_out[g] = hc;
      if (USE_L && a.xl_out) a.xl_out[g] = lc;
      if (a.r_out) a.r_out[g] = rv;
      srr += rv * rv;
      sbb += bh * bh;
      add_x(hc);
      sxl += lc;
      (void)rr_h;
      (void)rr_l;
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
  v = block_sum((double)srr, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_RR] = v;
  v = block_sum((double)sbb, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_BB] = v;
  v = block_sum((double)sxh + (double)sxl, dsh);
  if (tid == 0) a.partials[blk * S_NUM + S_X] = v;
  v = block_sum((double)si, dsh);
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

// 3D map over a float32 [nz][ny][nx] array with a (width x rows x 1) box.
bool make_map(CUtensorMap *m, const float *base, int nx, int ny, int nz, int width, int rows) {
  if (!encoder() || !base) return false;
  if (((uintptr_t)base & 15) != 0 || (nx & 3) != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
  const cuuint32_t box[3] = {(cuuint32_t)width, (cuuint32_t)rows, 1};
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

template <bool Z, bool P, bool S, bool U>
cudaError_t run_zsweep_u(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a,
                         dim3 grid, cudaStream_t st) {
  const size_t bytes = SweepGeo::smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem(k_zsweep<Z, P, S, U>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_zsweep<Z, P, S, U><<<grid, ZNT, bytes, st>>>(mx, mb, a);
  return cudaGetLastError();
}
bool level_uniform(const LevelDev &L) { return L.sx == L.lx && L.sy == L.ly && L.sz == L.lz; }
template <bool Z, bool P, bool S>
cudaError_t run_zsweep(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a, dim3 grid,
                       cudaStream_t st) {
  if (level_uniform(a.L)) return run_zsweep_u<Z, P, S, true>(mx, mb, a, grid, st);
  return run_zsweep_u<Z, P, S, false>(mx, mb, a, grid, st);
}
template <bool U>
cudaError_t run_zrestrict(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a,
                          dim3 grid, cudaStream_t st) {
  const size_t bytes = RestrictGeo::smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem(k_zrestrict<U>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_zrestrict<U><<<grid, ZNT, bytes, st>>>(mx, mb, a);
  return cudaGetLastError();
}

template <int RHS, bool XL, bool E, bool ACC>
cudaError_t run_zouter(const CUtensorMap *m, const OuterArgs &a, int zchunk, double *err, dim3 grid,
                       cudaStream_t st) {
  const size_t bytes = OuterGeo::smem_bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = set_smem(k_zouter<RHS, XL, E, ACC>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_zouter<RHS, XL, E, ACC><<<grid, ZNT, bytes, st>>>(m[0], m[1], m[2], m[3], m[4], a, zchunk, err);
  return cudaGetLastError();
}

}  // namespace

bool zmarch_usable(const LevelDev &L) { return encoder() && (L.nx & 3) == 0; }

cudaError_t launch_zsweep(ZSweepArgs a, const float *xin, const float *b, bool zero_in, bool prolong,
                          bool sum, int *nblocks_out, cudaStream_t st) {
  const LevelDev &L = a.L;
  const int rows_x = ZY + 2 * SweepGeo::H, rows_b = ZY + 2 * (SweepGeo::H - 1);
  CUtensorMap mx, mb;
  std::memset(&mx, 0, sizeof mx);
  if (!make_map(&mx, zero_in ? b : xin, L.nx, L.ny, L.nz, BOXW, rows_x)) return cudaErrorNotSupported;
  if (!make_map(&mb, b, L.nx, L.ny, L.nz, BOXW, rows_b)) return cudaErrorNotSupported;
  if (((uintptr_t)a.xout & 15) != 0) return cudaErrorNotSupported;
  const int gx = (L.nx + ZX - 1) / ZX, gy = (L.ny + ZY - 1) / ZY;
  const bool coupled = (L.wz != 0.f) && (L.nz > 1);
  a.zchunk = pick_zchunk(gx * gy, L.nz, coupled, 3);
  const int gz = (L.nz + a.zchunk - 1) / a.zchunk;
  if (nblocks_out) *nblocks_out = gx * gy * gz;
  dim3 grid(gx, gy, gz);
  if (zero_in && !prolong && !sum) return run_zsweep<true, false, false>(mx, mb, a, grid, st);
  if (!zero_in && prolong && !sum) return run_zsweep<false, true, false>(mx, mb, a, grid, st);
  if (!zero_in && prolong && sum) return run_zsweep<false, true, true>(mx, mb, a, grid, st);
  if (!zero_in && !prolong && !sum) return run_zsweep<false, false, false>(mx, mb, a, grid, st);
  if (!zero_in && !prolong && sum) return run_zsweep<false, false, true>(mx, mb, a, grid, st);
  return cudaErrorNotSupported;
}

cudaError_t launch_zrestrict(ZSweepArgs a, const float *x, const float *b, cudaStream_t st) {
  const LevelDev &L = a.L;
  CUtensorMap mx, mb;
  if (!make_map(&mx, x, L.nx, L.ny, L.nz, BOXW, ZY + 2)) return cudaErrorNotSupported;
  if (!make_map(&mb, b, L.nx, L.ny, L.nz, ZX, ZY)) return cudaErrorNotSupported;
  const int gx = (L.nx + ZX - 1) / ZX, gy = (L.ny + ZY - 1) / ZY;
  const bool coupled = (L.wz != 0.f) && (L.nz > 1);
  a.zchunk = pick_zchunk(gx * gy, L.nz, coupled || a.fz, 3);
  if (a.fz && (a.zchunk & 1)) ++a.zchunk;  // both children of a coarse plane in one chunk
  const int gz = (L.nz + a.zchunk - 1) / a.zchunk;
  dim3 grid(gx, gy, gz);
  if (level_uniform(L)) return run_zrestrict<true>(mx, mb, a, grid, st);
  return run_zrestrict<false>(mx, mb, a, grid, st);
}

cudaError_t launch_zouter(const OuterArgs &a, int rhs_mode, double *err, int *nblocks_out,
                          cudaStream_t st) {
  if ((a.nx & 3) != 0) return cudaErrorNotSupported;
  const int rows = ZY + 2;
  CUtensorMap m[5];
  std::memset(m, 0, sizeof m);
  const float *rhs0 = rhs_mode == RHS_EXPLICIT ? a.b : a.I0;
  if (!make_map(&m[0], a.xh_in, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (a.xl_in && !make_map(&m[1], a.xl_in, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (a.e && !make_map(&m[2], a.e, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (!make_map(&m[3], rhs0, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (rhs_mode == RHS_SP && !make_map(&m[4], a.I1, a.nx, a.ny, a.nz, BOXW, rows))
    return cudaErrorNotSupported;
  const int gx = (a.nx + ZX - 1) / ZX, gy = (a.ny + ZY - 1) / ZY;
  const bool coupled = (a.bz != 0.f) && (a.nz > 1);
  const int zchunk = pick_zchunk(gx * gy, a.nz, coupled, 2);
  const int gz = (a.nz + zchunk - 1) / zchunk;
  if (nblocks_out) *nblocks_out = gx * gy * gz;
  dim3 grid(gx, gy, gz);
  const bool xl = a.xl_in != nullptr, e = a.e != nullptr;
#define GD_ZO2(R, ACC)                                                          \
  if (xl && e) return run_zouter<R, true, true, ACC>(m, a, zchunk, err, grid, st);  \
  if (xl) return run_zouter<R, true, false, ACC>(m, a, zchunk, err, grid, st);      \
  if (e) return run_zouter<R, false, true, ACC>(m, a, zchunk, err, grid, st);       \
  return run_zouter<R, false, false, ACC>(m, a, zchunk, err, grid, st);
#define GD_ZO(R)                \
  if (a.accurate) {             \
    GD_ZO2(R, true)             \
  } else {                      \
    GD_ZO2(R, false)            \
  }
  if (rhs_mode == RHS_EXPLICIT) { GD_ZO(RHS_EXPLICIT) }
  if (rhs_mode == RHS_AD) { GD_ZO(RHS_AD) }
  GD_ZO(RHS_SP)
#undef GD_ZO
}

int zouter_max_blocks(int nx, int ny, int nz) {
  const int gx = (nx + ZX - 1) / ZX, gy = (ny + ZY - 1) / ZY;
  return gx * gy * nz;
}
