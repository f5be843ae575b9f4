// gd_zmarch.cu -- TMA-pipelined 2.5D z-march kernels for sm_103a.
//
// A CTA owns a column tile of one level (64 x 32 cells for the sweep and the
// restriction, 64 x 16 for the outer pass) and marches along z over a chunk
// of planes.  Planes of each input array arrive in a shared-memory ring by
// TMA (cp.async.bulk.tensor.3d issued by one lane of a service warp, mbarrier
// completion) a few planes ahead of their first use.  Boxes start at
// x = i0 - 4 (16-byte aligned coordinates) and are 72 floats wide; the tensor
// map zero-fills outside the array.  Tile threads own float4 groups of cells:
// x-neighbours come from the neighbouring lanes (shuffles), y-neighbours from
// shared memory, z-neighbours from the thread's own registers.
//
// k_zsweep: one red-black Gauss-Seidel sweep (Sec. 4.1 multi-colour
//   relaxation) with optional fusions:
//     ZERO_IN   the input iterate is zero (first pre-sweep of a correction);
//     PROLONG   x <- x + P x_c before relaxing (first post-sweep: the
//               up-sampled coarse correction of Sec. 4.1, replication
//               stencil of Sec. 4.2);
//     SUM       the block sums of the written iterate (mean fix of AD).
//   Pipeline per step t: red of plane t on the tile + 1 ring, black of plane
//   t-1 on the tile, stored from registers; one CTA barrier per plane.  The
//   ring recomputes the neighbouring CTA's red values exactly as it does, so
//   the result is the textbook red-black sweep.
//
// k_zrestrict: residual r = b - A x and its down-sampling (sum over the
//   children of each coarse cell, Sec. 4.1 / 4.2) into the next level's
//   right-hand side.  Producer/consumer ring, no CTA barrier per plane.
//
// k_zouter: fine-level outer pass of the iterative refinement: x_new = x + e
//   (+ mean shift) as a float pair, r = b - A x_new in double-float arithmetic
//   with b assembled from I0 (and I1), and FP64 block partial sums.
//   Producer/consumer ring, no CTA barrier per plane.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "gd_internal.h"

// The file compiles as one translation unit, or in parts that the build
// compiles in parallel (-DGD_ZMARCH_PART=0 .. 4): part 0 holds the launchers'
// front ends and the restriction, parts 1 and 2 the sweep instantiations
// over float32 and bfloat16 levels, parts 3 and 4 the outer pass's over a
// float32 and a bfloat16 correction.  Each kernel instantiation belongs to
// exactly one part.
#ifndef GD_ZMARCH_PART
#define GD_ZMARCH_PART -1
#endif
#define GD_ZM_PART(n) (GD_ZMARCH_PART < 0 || GD_ZMARCH_PART == (n))
#if GD_ZMARCH_PART >= 0
#pragma nv_diag_suppress 177  // helpers that another part uses
#endif

// sweep launchers by element type of the level (esz_c: the coarse level's)
cudaError_t zsweep_f32(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc, const ZSweepArgs &a,
                       bool zero_in, bool prolong, bool sum, int esz_c, dim3 grid, int *nblocks_out,
                       cudaStream_t st);
cudaError_t zsweep_bf16(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc, const ZSweepArgs &a,
                        bool zero_in, bool prolong, bool sum, int esz_c, dim3 grid, int *nblocks_out,
                        cudaStream_t st);
// outer-pass launchers by element type of the correction e
cudaError_t zouter_f32(const CUtensorMap *m, const OuterArgs &a, int rhs_mode, double *err, dim3 grid,
                       int *nblocks_out, cudaStream_t st);
cudaError_t zouter_bf16(const CUtensorMap *m, const OuterArgs &a, int rhs_mode, double *err, dim3 grid,
                        int *nblocks_out, cudaStream_t st);

namespace {

constexpr int ZX = 64;            // tile x extent
constexpr int BOXW = ZX + 8;      // box width: tile + 4 on each side (16-byte aligned start)
constexpr uint32_t WAIT_LIMIT = 1u << 21;  // bounded mbarrier polling (at most ~1 s)

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
  // each try_wait may suspend the thread up to the hint (ns) while the phase
  // is incomplete, so a waiting warp issues few instructions
  const uint32_t a = su32(bar);
  const uint32_t hint_ns = 500;
  for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(hint_ns)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_plane(void *dst, const CUtensorMap *map, int x, int y, int z,
                                          uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}
// L2 prefetch of one box of a tensor (no shared memory, no completion)
__device__ __forceinline__ void prefetch_plane(const CUtensorMap *map, int x, int y, int z) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"((uint64_t)map),
               "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

#if GD_ZM_PART(0)
// Self-test of the bounded wait: one thread initialises an mbarrier that
// expects one arrival, never arrives, and polls it `limit` times with the
// same try_wait and suspend hint the kernels use; a wait that gives up sets
// *flag to 1 and the kernel returns normally.
__global__ void k_wait_selftest(uint32_t limit, int *flag) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  const uint32_t a = su32(&bar);
  const uint32_t hint_ns = 500;
  bool done = false;
  for (uint32_t it = 0; it < limit && !done; ++it) {
    uint32_t d;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(d)
        : "r"(a), "r"(0u), "r"(hint_ns)
        : "memory");
    done = d != 0;
  }
  *flag = done ? 0 : 1;
}
#endif


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
// Dynamic shared memory of the z-march kernels, addressed with 32-bit element
// offsets (slots are multiples of 128 bytes).
extern __shared__ __align__(128) float zsm[];

// ---- storage types ----
// The hierarchy's arrays are float32, or bfloat16 in the mixed-precision mode
// (arithmetic is float32 either way).  A TMA box must start on a 16-byte
// boundary: boxes start 4 floats / 8 halves left of the tile and are 72 / 80
// elements wide.  Four consecutive cells are one float4 / one 8-byte pair of
// half2.
template <typename T>
struct St;
template <>
struct St<float> {
  static constexpr int W = 72, OFF = 4;
  __device__ static __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
  __device__ static __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
  __device__ static __forceinline__ float ld1(const float *p) { return *p; }
  __device__ static __forceinline__ void st1(float *p, float v) { *p = v; }
  __device__ static __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
  __device__ static __forceinline__ float2 ldg2(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
  __device__ static __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
  __device__ static __forceinline__ void stg2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <>
struct St<__nv_bfloat16> {
  static constexpr int W = 80, OFF = 8;
  __device__ static __forceinline__ float4 cvt(uint2 u) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static __forceinline__ uint2 pack(float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
  }
  __device__ static __forceinline__ float4 ld4(const __nv_bfloat16 *p) { return cvt(*reinterpret_cast<const uint2 *>(p)); }
  __device__ static __forceinline__ void st4(__nv_bfloat16 *p, float4 v) { *reinterpret_cast<uint2 *>(p) = pack(v); }
  __device__ static __forceinline__ float ld1(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
  __device__ static __forceinline__ void st1(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
  __device__ static __forceinline__ float4 ldg4(const __nv_bfloat16 *p) {
    return cvt(__ldg(reinterpret_cast<const uint2 *>(p)));
  }
  __device__ static __forceinline__ float2 ldg2(const __nv_bfloat16 *p) {
    const unsigned u = __ldg(reinterpret_cast<const unsigned *>(p));
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
  }
  __device__ static __forceinline__ float2 ld2(const __nv_bfloat16 *p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p));
  }
  __device__ static __forceinline__ void stg2(__nv_bfloat16 *p, float2 v) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
  }
};
// the 16-bit storage type of the mixed mode
using half_t = __nv_bfloat16;
// slot sizes are multiples of 128 bytes
template <typename T>
__host__ __device__ constexpr int pad128(int n) {
  return (n + (int)(128 / sizeof(T)) - 1) / (int)(128 / sizeof(T)) * (int)(128 / sizeof(T));
}



// Sweep tiles are 64 x 32: eight tile warps (two float4 cells per thread),
// a service warp (TMA issue, mbarrier polling) and a ring warp (the red ring).
constexpr int SY = 32;  // sweep tile rows

template <typename T, typename TC = T, bool PRO = false>
struct SweepGeo {
  static constexpr int W = St<T>::W, OFF = St<T>::OFF;
  static constexpr int H = 2;                    // x box halo rows
  static constexpr int XH = SY + 2 * H;          // x box rows j0-2 .. j0+SY+1
  static constexpr int BH = SY + 2 * (H - 1);    // b box rows j0-1 .. j0+SY
  static constexpr int PFS = 2;                  // x planes in flight ahead of use
  // b planes in flight: the prolongation sweep gives up one (its b copies
  // land within one step) so that its two coarse staging slots fit beside
  // the rings at two CTAs per SM
  static constexpr int PFSB = PRO ? 1 : 2;
  // ring depths: an x plane is last read two steps after its red pass (its
  // red cells are the z-neighbours of the next black pass but one), a b
  // plane one step after it (by the black pass)
  static constexpr int XR = 6;                   // needs PFS + 4
  static constexpr int BR = PFSB + 2;
  static_assert(XR >= PFS + 4, "ring depth");
  static constexpr int XS = pad128<T>(XH * W);   // elements per x slot
  static constexpr int BS = pad128<T>(BH * W);
  static constexpr int BOFF = XR * XS;           // b slots
  // coarse staging (prolongation): two slots, each the largest coarse box:
  // the x box's extent in coarse elements, or 80 wide for a bfloat16 level
  // under a float32 one (its box starts 8 elements left of the tile, which is
  // where 16-byte alignment puts it)
  static constexpr int CW_MAX = (sizeof(T) == 4 && sizeof(TC) == 2) ? 80 : W;
  static constexpr size_t CSB = PRO ? (XH * CW_MAX * sizeof(TC) + 127) / 128 * 128 : 0;
  static constexpr size_t COFF_B = sizeof(T) * (size_t)(BOFF + BR * BS);  // bytes
  static constexpr size_t MOFF_B = COFF_B + 2 * CSB;                      // mbarriers (bytes)
  static constexpr int TILE_WARPS = 8;
  static constexpr int NT = 32 * (TILE_WARPS + 2);  // + the service and ring warps
  static constexpr int SVC = 32 * TILE_WARPS;       // first thread of the service warp
  // red ring cells of one colour: the in-plane neighbours of tile cells that
  // lie outside the tile (corners are nobody's neighbour), relaxed by the
  // ring warp while the service warp issues copies and polls
  static constexpr int NRING = ZX + SY;          // (2 ZX + 2 SY) / 2
  static constexpr int RING_IT = NRING / 32;
  static_assert(NRING % 32 == 0, "ring cells per lane");
  __host__ __device__ static constexpr size_t smem_bytes() {
    return MOFF_B + sizeof(uint64_t) * (XR + BR + 2) + sizeof(double) * 32 + 16;
  }
};

// Thread layout of the tile: a tile thread owns two float4 cells, rows r and
// r + 16 of one column of four, where warp w's half-warps take rows
// r = 4 (w / 2) + (w % 2) and r + 2.  All rows of a warp have the same
// parity, so colour branches are warp-uniform.  The z-neighbours of a cell
// are the same thread's (its previous plane in registers, older planes and b
// from the shared-memory rings), so one CTA barrier per plane orders all the
// in-plane exchanges.
template <typename T, typename TC, bool ZERO_IN, bool PROLONG, bool SUM, bool UNIFORM, bool COUPLED>
__global__ void __launch_bounds__(SweepGeo<T, TC, PROLONG>::NT, 2) k_zsweep(const __grid_constant__ CUtensorMap tmx,
                                                               const __grid_constant__ CUtensorMap tmb,
                                                               const __grid_constant__ CUtensorMap tmc,
                                                               const ZSweepArgs a) {
  using G = SweepGeo<T, TC, PROLONG>;
  using S = St<T>;
  constexpr int H = G::H;
  constexpr int PFS = G::PFS;
  constexpr int XS = G::XS;
  constexpr int W = G::W, OFF = G::OFF;
  constexpr bool zc = COUPLED;  // the launcher passes wz != 0 && nz > 1
  T *sm = reinterpret_cast<T *>(zsm);
  auto lds4 = [&](int off) { return S::ld4(sm + off); };
  auto sts4 = [&](int off, float4 v) { S::st4(sm + off, v); };
  uint64_t *xbar = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(zsm) + G::MOFF_B);
  uint64_t *bbar = xbar + G::XR;
  uint64_t *cbar = bbar + G::BR;  // coarse staging slots (prolongation)
  double *dsh = reinterpret_cast<double *>(cbar + 2);
  TC *cstage = reinterpret_cast<TC *>(reinterpret_cast<char *>(zsm) + G::COFF_B);
  __shared__ int abort_flag;

  const LevelDev &L = a.L;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool tile = warp < G::TILE_WARPS;
  const bool svc = warp == G::TILE_WARPS;
  const bool rwarp = warp == G::TILE_WARPS + 1;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * SY;
  const int zs = blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, nz);
  const int t0 = zc ? zs - 1 : zs;
  const int t1 = zc ? ze : ze - 1;
  constexpr int lagb = zc ? 1 : 0;
  const int red_lo = zc ? max(zs - 1, 0) : zs, red_hi = zc ? min(ze, nz - 1) : ze - 1;
  const int blk_lo = zs, blk_hi = ze - 1;
  Ring<G::XR> rx;
  rx.lo = zc ? max(t0 - 1, 0) : zs;
  rx.hi = zc ? min(t1 + 1, nz - 1) : ze - 1;
  Ring<G::BR> rb;
  rb.lo = zc ? max(t0, 0) : zs;
  rb.hi = zc ? min(t1, nz - 1) : ze - 1;
  const size_t plane = (size_t)nx * ny;

  if (tid == G::SVC) {
    abort_flag = 0;
    int e = tma_preflight(zsm, G::smem_bytes(), &tmx);
    if (!e) e = tma_preflight(zsm, G::smem_bytes(), &tmb);
    if (!e && PROLONG && a.cpf) e = tma_preflight(zsm, G::smem_bytes(), &tmc);
    if (e) {
      abort_flag = e;
      a.err[0] = (double)e;
    } else {
      for (int q = 0; q < G::XR; ++q) mbar_init(&xbar[q], 1);
      for (int q = 0; q < G::BR; ++q) mbar_init(&bbar[q], 1);
      for (int q = 0; q < 2; ++q) mbar_init(&cbar[q], 1);
      fence_mbar_init();
    }
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ZERO_IN) {
    // x is never loaded: cells outside the domain and the black ring must
    // read 0 for good; every other cell is written before it is read
    for (int q = tid; q < G::XR * XS / 4; q += G::NT) sts4(4 * q, zero4);
  }
  __syncthreads();
  if (abort_flag) return;  // nothing issued yet

  int xissued = rx.lo - 1, bissued = rb.lo - 1;  // issuing thread
  auto issue_x = [&](int p) {
    if (ZERO_IN || !rx.has(p)) return;
    const int q = rx.slot(p);
    mbar_expect_tx(&xbar[q], (uint32_t)(G::XH * W * sizeof(T)));
    tma_plane(sm + q * XS, &tmx, i0 - OFF, j0 - H, p, &xbar[q]);
    xissued = p;
  };
  auto issue_b = [&](int p) {
    if (!rb.has(p)) return;
    const int q = rb.slot(p);
    mbar_expect_tx(&bbar[q], (uint32_t)(G::BH * W * sizeof(T)));
    tma_plane(sm + G::BOFF + q * G::BS, &tmb, i0 - OFF, j0 - (H - 1), p, &bbar[q]);
    bissued = p;
  };
  // x plane issued at step t, and the last x plane a step reads or corrects
  auto x_issue_at = [&](int t) { return t + (zc ? 1 : 0) + PFS; };
  auto x_need_at = [&](int t) { return t + (zc ? 1 : 0) + (PROLONG ? 1 : 0); };
  // ---- coarse staging of the prolongation: step t corrects x plane
  // corr_plane(t) from coarse plane corr_plane(t) >> fz, which the service
  // lane brings by TMA into one of two slots a step ahead (a slot is reused
  // once the steps that read its previous plane are past a CTA barrier)
  const bool stage = PROLONG && a.cpf;
  constexpr int AC = 16 / (int)sizeof(TC);  // TMA x alignment in coarse elements
  // the coarse box: its x start (16-byte aligned) and extent
  const int cxs = a.fx ? (i0 >> 1) - AC : (G::CW_MAX != W ? i0 - 8 : i0 - OFF);
  const int cw = a.fx ? 32 + 2 * AC : G::CW_MAX, ch = a.fy ? G::XH / 2 : G::XH;
  auto corr_plane = [&](int t) { return zc ? t + 2 : t + 1; };
  const int c_lo = corr_plane(t0) >> a.fz;
  int cissued = c_lo - 1, cwait = c_lo - 1;
  auto cslot = [&](int c) { return (c - c_lo) & 1; };
  auto cpar = [&](int c) { return (uint32_t)((c - c_lo) >> 1) & 1u; };
  auto issue_c_for = [&](int t) {
    if (!stage || corr_plane(t) > rx.hi) return;
    const int c = corr_plane(t) >> a.fz;
    for (int q = cissued + 1; q <= c; ++q) {
      const int sl = cslot(q);
      mbar_expect_tx(&cbar[sl], (uint32_t)(cw * ch * (int)sizeof(TC)));
      tma_plane(cstage + sl * (int)(G::CSB / sizeof(TC)), &tmc, cxs, (j0 - H) >> a.fy, q, &cbar[sl]);
      cissued = q;
    }
  };
  auto wait_c_for = [&](int t) -> bool {
    if (!stage || corr_plane(t) > rx.hi) return true;
    const int c = min(corr_plane(t) >> a.fz, cissued);
    bool ok = true;
    for (int q = cwait + 1; q <= c && ok; ++q) {
      ok = mbar_wait(&cbar[cslot(q)], cpar(q));
      if (ok) cwait = q;
    }
    return ok;
  };
  if (tid == G::SVC) {
    for (int p = rx.lo; p < x_issue_at(t0) && p <= rx.hi; ++p) issue_x(p);
    for (int p = rb.lo; p < t0 + G::PFSB && p <= rb.hi; ++p) issue_b(p);
    issue_c_for(t0);
    issue_c_for(t0 + 1);
  }
  int xwait = rx.lo - 1, bwait = rb.lo - 1;  // planes whose wait succeeded (service warp)
  auto wait_planes = [&](int ux, int ub) -> bool {
    bool ok = true;
    if (!ZERO_IN)
      for (int p = xwait + 1; p <= min(ux, rx.hi) && ok; ++p) {
        ok = mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
        if (ok) xwait = p;
      }
    for (int p = bwait + 1; p <= min(ub, rb.hi) && ok; ++p) {
      ok = mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
      if (ok) bwait = p;
    }
    return ok;
  };
  auto xo = [&](int p) { return rx.slot(p) * XS; };
  auto bo = [&](int p) { return G::BOFF + rb.slot(p) * G::BS; };

  // ---- coefficients ----
  const float cxu = L.wx * (float)L.sy * (float)L.sz;
  const float cyu = L.wy * (float)L.sx * (float)L.sz;
  const float czu = zc ? L.wz * (float)L.sx * (float)L.sy : 0.f;
  const float mmu = L.wm * (float)L.sx * (float)L.sy * (float)L.sz;
  // Fast path: a uniform level and a tile whose cells, ring and the ring's
  // neighbours all lie inside the domain in x and y (z faces: zmf / zpf).
  const bool fast = UNIFORM && (i0 >= 3) && (i0 + ZX + 3 <= nx) && (j0 >= 3) && (j0 + SY + 3 <= ny);
  // inverse diagonals of the fast path with two / one z-neighbours
  const float idg2 = 1.f / (2.f * (cxu + cyu) + 2.f * czu + mmu);
  const float idg1 = 1.f / (2.f * (cxu + cyu) + czu + mmu);
  struct PlaneK {
    float mz, zmf, zpf, idg, czm, czp;
  };
  auto plane_k = [&](int p) {
    PlaneK k;
    const bool hm = zc && p > 0, hp = zc && p < nz - 1;
    k.zmf = hm ? 1.f : 0.f;
    k.zpf = hp ? 1.f : 0.f;
    k.mz = mass_of(p, nz, L.sz, L.lz);
    k.czm = hm ? czu : 0.f;
    k.czp = hp ? czu : 0.f;
    k.idg = (hm && hp) ? idg2 : idg1;
    return k;
  };
  // Gauss-Seidel value of cell (ci, cj):
  //   (b + cx (x-neighbours) + cy (y-neighbours) + cz (z-neighbours)) / diag
  // sxn / syn are the sums of the x / y neighbours.  Cells outside the domain
  // read 0; the neighbour counts leave them out of the diagonal.
  auto gs = [&](auto fast_c, auto red0_c, const PlaneK &k, float bv, float sxn, float syn, float zm,
                float zp, int ci, int cj) -> float {
    constexpr bool RED0 = decltype(red0_c)::value;
    if constexpr (decltype(fast_c)::value) {
      if (RED0) return bv * k.idg;
      return (bv + cxu * sxn + cyu * syn + k.czm * zm + k.czp * zp) * k.idg;
    }
    float cx = cxu, cy = cyu, cz = czu, mm = mmu;
    if (!UNIFORM) {
      const float mx = mass_of(ci, nx, L.sx, L.lx), my = mass_of(cj, ny, L.sy, L.ly);
      cx = L.wx * my * k.mz;
      cy = L.wy * mx * k.mz;
      cz = zc ? L.wz * mx * my : 0.f;
      mm = L.wm * mx * my * k.mz;
    }
    const float nbx = (float)((ci > 0) + (ci < nx - 1));
    const float nby = (float)((cj > 0) + (cj < ny - 1));
    const float dg = cx * nbx + cy * nby + cz * (k.zmf + k.zpf) + mm;
    if (RED0) return __fdividef(bv, dg);
    return __fdividef(bv + cx * sxn + cy * syn + cz * (k.zmf * zm + k.zpf * zp), dg);
  };

  // ---- tile threads: two float4 cells ----
  const int c4 = lane & 15;
  const int r0 = 4 * ((warp & 7) >> 1) + (warp & 1) + 2 * (lane >> 4);
  const int gi = i0 + 4 * c4, gj0 = j0 + r0, gj1 = gj0 + 16;
  const bool act0 = tile && gi < nx && gj0 < ny;  // nx % 4 == 0: all four cells or none
  const bool act1 = tile && gi < nx && gj1 < ny;
  const int so0 = (r0 + H) * W + OFF + 4 * c4, so1 = so0 + 16 * W;
  const int go0 = gj0 * nx + gi, go1 = go0 + 16 * nx;  // in-plane offsets

  // ---- ring warp: red ring cell m of this lane for colour class P ----
  // Class P holds the cells with (col + row) & 1 = P (i0 + j0 even), so the
  // red ring of plane t is class t & 1.  Decoded on the fly (no registers
  // held across the loop); off < 0 marks a cell outside the domain.
  auto ring_cell = [&](int m, int P, int &off, int &ci, int &cj) {
    const int q = lane + 32 * m;
    int row, col;
    if (q < ZX / 2) {
      row = -1;
      col = (P ^ 1) + 2 * q;
    } else if (q < ZX) {
      row = SY;
      col = P + 2 * (q - ZX / 2);
    } else if (q < ZX + SY / 2) {
      col = -1;
      row = (P ^ 1) + 2 * (q - ZX);
    } else {
      col = ZX;
      row = P + 2 * (q - ZX - SY / 2);
    }
    ci = i0 + col;
    cj = j0 + row;
    off = (ci >= 0 && ci < nx && cj >= 0 && cj < ny) ? (row + H) * W + OFF + col : -1;
  };

  // ---- prolongation by replication: every float4 of the x box inside the
  // domain gets the coarse value of each of its cells (with x coarsened the
  // four cells take two coarse values; nx % 4 == 0 keeps both loads aligned).
  // Thread tid takes float4 column tid % QW of box rows tid / QW + k RP, so
  // its columns (fine, staged and coarse) and its validity in x are fixed.
  constexpr int QW = W / 4;                       // float4 columns of the box
  constexpr int RP = G::NT / QW;                  // box rows per pass
  constexpr int KP = PROLONG ? (G::XH + RP - 1) / RP : 1;
  const int ccq = tid % QW, crr = tid / QW;
  const int cgi = i0 - OFF + 4 * ccq;
  const bool cxok = PROLONG && crr < RP && cgi >= 0 && cgi < nx;
  const bool cunmasked = !a.fx && !a.fy;
  const int cxoff = crr * W + 4 * ccq;  // this thread's first float4 in an x slot
  // its first coarse value in a staging slot (unmasked form: row crr
  // included)
  const int ccoff = ((cgi >> a.fx) - cxs) + (cunmasked ? crr * cw : 0);
  auto add4 = [&](int so, float4 c) {
    float4 v = lds4(so);
    v.x += c.x;
    v.y += c.y;
    v.z += c.z;
    v.w += c.w;
    sts4(so, v);
  };
  // the staged form: x plane p += its coarse values from the staging slot
  auto correct_staged = [&](int p) {
    const TC *cs = cstage + cslot(p >> a.fz) * (int)(G::CSB / sizeof(TC)) + ccoff;
    const int xop = xo(p) + cxoff;
    if (cunmasked) {
      // the staged box has the x box's cells, and the copy's zero fill gives
      // every cell outside the domain a correction of 0: no masks
      if (crr < RP) {
#pragma unroll
        for (int k = 0; k < KP; ++k)
          if (k + 1 < KP || crr + k * RP < G::XH) add4(xop + k * RP * W, St<TC>::ld4(cs + k * RP * cw));
      }
      return;
    }
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const int rr = crr + k * RP, gcj = j0 - H + rr;
      if (cxok && rr < G::XH && gcj >= 0 && gcj < ny) {
        const TC *q = cs + (a.fy ? rr >> 1 : rr) * cw;
        float4 c;
        if (a.fx) {
          const float2 c2 = St<TC>::ld2(q);
          c = make_float4(c2.x, c2.x, c2.y, c2.y);
        } else {
          c = St<TC>::ld4(q);
        }
        add4(xop + k * RP * W, c);
      }
    }
  };
  // the direct form (no coarse tensor map, and the planes before the first
  // step): the coarse values come from global memory
  const int ccol = max(cgi, 0) >> a.fx;
  int corrected = rx.lo - 1;  // planes that hold the coarse correction
  auto correct_upto = [&](int u) {
    for (int p = corrected + 1; p <= min(u, rx.hi); ++p) {
      const TC *xcp = reinterpret_cast<const TC *>(a.xc) + (size_t)(p >> a.fz) * a.ncy * a.ncx + ccol;
      const int xop = xo(p) + cxoff;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        const int rr = crr + k * RP, gcj = j0 - H + rr;
        if (cxok && rr < G::XH && gcj >= 0 && gcj < ny) {
          const TC *q = xcp + (size_t)(gcj >> a.fy) * a.ncx;
          float4 c;
          if (a.fx) {
            const float2 c2 = St<TC>::ldg2(q);
            c = make_float4(c2.x, c2.x, c2.y, c2.y);
          } else {
            c = St<TC>::ldg4(q);
          }
          add4(xop + k * RP * W, c);
        }
      }
      corrected = p;
    }
  };

  // The service warp polls the mbarriers for the planes of the next step
  // just before the CTA barrier that releases that step.
  bool failed = false;
  if (svc) failed = !wait_planes(x_need_at(t0), t0) || !wait_c_for(t0);
  if (__syncthreads_or(failed)) abort_flag = 1;
  if (PROLONG && !abort_flag) {
    // the planes the first step reads get their correction before it
    correct_upto(zc ? t0 + 1 : t0);
    __syncthreads();
  }

  float4 cp0 = zero4, cp1 = zero4;    // plane t-1 after its red pass
  bool have_prev = false;             // cp holds plane t-1
  // double-float block sums in FP32 (the FP64 pipe is narrow)
  float sum_h = 0.f, sum_l = 0.f;
  auto acc = [&](float4 f) {
    const float s4 = (f.x + f.y) + (f.z + f.w);
    const float sn = sum_h + s4;
    const float bb = sn - sum_h;
    sum_l += (sum_h - (sn - bb)) + (s4 - bb);
    sum_h = sn;
  };
  const unsigned FULL = 0xffffffffu;

  // The step loop, specialised for fast tiles (constant coefficients) and
  // the rest, so that neither path pays for the other.
  auto march = [&](auto fast_c) {
    const std::integral_constant<bool, ZERO_IN> red0;
    const std::false_type nored0;
    // red value of the two cells of a float4 with colour pattern E (cells 0
    // and 2 when E, else 1 and 3); e is the neighbour across the float4 edge
    auto red2 = [&](auto e_c, const PlaneK &k, float4 xc, float4 xu, float4 xd, float4 xm, float4 xp,
                    float4 bv, float e, int cj, float4 &out) {
      if constexpr (decltype(e_c)::value) {
        out.x = gs(fast_c, red0, k, bv.x, e + xc.y, xu.x + xd.x, xm.x, xp.x, gi, cj);
        out.z = gs(fast_c, red0, k, bv.z, xc.y + xc.w, xu.z + xd.z, xm.z, xp.z, gi + 2, cj);
        out.y = xc.y;
        out.w = xc.w;
      } else {
        out.y = gs(fast_c, red0, k, bv.y, xc.x + xc.z, xu.y + xd.y, xm.y, xp.y, gi + 1, cj);
        out.w = gs(fast_c, red0, k, bv.w, xc.z + e, xu.w + xd.w, xm.w, xp.w, gi + 3, cj);
        out.x = xc.x;
        out.z = xc.z;
      }
    };
    auto black2 = [&](auto e_c, const PlaneK &k, float4 yc, float4 yu, float4 yd, float4 ym, float4 yp,
                      float4 yb, float e, int cj, float4 &out) {
      out = yc;
      if constexpr (decltype(e_c)::value) {
        out.x = gs(fast_c, nored0, k, yb.x, e + yc.y, yu.x + yd.x, ym.x, yp.x, gi, cj);
        out.z = gs(fast_c, nored0, k, yb.z, yc.y + yc.w, yu.z + yd.z, ym.z, yp.z, gi + 2, cj);
      } else {
        out.y = gs(fast_c, nored0, k, yb.y, yc.x + yc.z, yu.y + yd.y, ym.y, yp.y, gi + 1, cj);
        out.w = gs(fast_c, nored0, k, yb.w, yc.z + e, yu.w + yd.w, ym.w, yp.w, gi + 3, cj);
      }
    };
    int xs_t = ((t0 - rx.lo + G::XR) % G::XR) * XS;  // slot offset of plane t (rolled each step)
    for (int t = t0; t <= t1; ++t) {
      if (tid == G::SVC) {
        fence_proxy_async();
        issue_x(x_issue_at(t));
        issue_b(t + G::PFSB);
        issue_c_for(t + 1);
        // prolongation: warm L2 with the coarse box of the plane corrected
        // two steps on (its staging copy, issued a step later, then hits L2)
        if (PROLONG) {
          const int pn = corr_plane(t) + 2;
          if (a.cpf && pn <= rx.hi) prefetch_plane(&tmc, cxs, (j0 - H) >> a.fy, pn >> a.fz);
        }
      }
      const int xs_p = (xs_t == (G::XR - 1) * XS) ? 0 : xs_t + XS;   // plane t + 1
      const int xs_m = (xs_t == 0) ? (G::XR - 1) * XS : xs_t - XS;   // plane t - 1
      const int xs_mm = (xs_m == 0) ? (G::XR - 1) * XS : xs_m - XS;  // plane t - 2
      if (PROLONG) {
        if (stage) {
          if (corr_plane(t) <= rx.hi) correct_staged(corr_plane(t));
        } else {
          correct_upto(corr_plane(t));
        }
      }

      // ---- red pass of plane t ----
      const bool do_red = t >= red_lo && t <= red_hi;
      float4 cc0 = cp0, cc1 = cp1, bv0 = zero4, bv1 = zero4;
      if (do_red) {
        const PlaneK k = plane_k(t);
        const int bs = bo(t) - W;  // b rows start one row below x rows
        if (tile) {
          bv0 = lds4(bs + so0);
          bv1 = lds4(bs + so1);
          float4 xc0 = zero4, xu0 = zero4, xd0 = zero4, xp0 = zero4, xm0 = zero4;
          float4 xc1 = zero4, xu1 = zero4, xd1 = zero4, xp1 = zero4, xm1 = zero4;
          if (!ZERO_IN) {
            xc0 = lds4(xs_t + so0);
            xu0 = lds4(xs_t + so0 - W);
            xd0 = lds4(xs_t + so0 + W);
            xc1 = lds4(xs_t + so1);
            xu1 = lds4(xs_t + so1 - W);
            xd1 = lds4(xs_t + so1 + W);
            if (zc) {
              if (k.zpf != 0.f) {
                xp0 = lds4(xs_p + so0);
                xp1 = lds4(xs_p + so1);
              }
              if (k.zmf != 0.f) {
                if (have_prev) {
                  xm0 = cp0;
                  xm1 = cp1;
                } else {
                  xm0 = lds4(xs_m + so0);
                  xm1 = lds4(xs_m + so1);
                }
              }
            }
          }
          if (((gj0 + t) & 1) == 0) {  // red cells 0 and 2
            float e0 = 0.f, e1 = 0.f;
            if (!ZERO_IN) {
              e0 = __shfl_up_sync(FULL, xc0.w, 1, 16);
              e1 = __shfl_up_sync(FULL, xc1.w, 1, 16);
              if (c4 == 0) {
                e0 = S::ld1(sm + xs_t + so0 - 1);
                e1 = S::ld1(sm + xs_t + so1 - 1);
              }
            }
            red2(std::true_type(), k, xc0, xu0, xd0, xm0, xp0, bv0, e0, gj0, cc0);
            red2(std::true_type(), k, xc1, xu1, xd1, xm1, xp1, bv1, e1, gj1, cc1);
          } else {  // red cells 1 and 3
            float e0 = 0.f, e1 = 0.f;
            if (!ZERO_IN) {
              e0 = __shfl_down_sync(FULL, xc0.x, 1, 16);
              e1 = __shfl_down_sync(FULL, xc1.x, 1, 16);
              if (c4 == 15) {
                e0 = S::ld1(sm + xs_t + so0 + 4);
                e1 = S::ld1(sm + xs_t + so1 + 4);
              }
            }
            red2(std::false_type(), k, xc0, xu0, xd0, xm0, xp0, bv0, e0, gj0, cc0);
            red2(std::false_type(), k, xc1, xu1, xd1, xm1, xp1, bv1, e1, gj1, cc1);
          }
          if (act0) sts4(xs_t + so0, cc0);
          else cc0 = zero4;
          if (act1) sts4(xs_t + so1, cc1);
          else cc1 = zero4;
        } else if (rwarp) {
          // red ring cells of plane t
#pragma unroll
          for (int m = 0; m < G::RING_IT; ++m) {
            int off, ci, cj;
            ring_cell(m, t & 1, off, ci, cj);
            if (off >= 0) {
              const float bq = S::ld1(sm + bs + off);
              float v;
              if (ZERO_IN) {
                v = gs(fast_c, red0, k, bq, 0.f, 0.f, 0.f, 0.f, ci, cj);
              } else {
                const T *xq = sm + xs_t + off;
                const float zm = (zc && k.zmf != 0.f) ? S::ld1(sm + xs_m + off) : 0.f;
                const float zp = (zc && k.zpf != 0.f) ? S::ld1(sm + xs_p + off) : 0.f;
                v = gs(fast_c, red0, k, bq, S::ld1(xq - 1) + S::ld1(xq + 1),
                       S::ld1(xq - W) + S::ld1(xq + W), zm, zp, ci, cj);
              }
              S::st1(sm + xs_t + off, v);
            }
          }
        }
      }
      if (!zc) {
        // uncoupled planes: the black pass of plane t reads this red pass
        if (svc && !failed && t < t1) failed = !wait_planes(x_need_at(t + 1), t + 1) || !wait_c_for(t + 1);
        if (__syncthreads_or(failed)) {
          abort_flag = 1;
          break;
        }
      }

      // ---- black pass of plane pb = t - lagb ----
      const int pb = t - lagb;
      if (tile) {
        if (pb >= blk_lo && pb <= blk_hi) {
          const PlaneK k = plane_k(pb);
          const int xob = zc ? xs_m : xs_t;
          const float4 yc0 = zc ? cp0 : cc0, yc1 = zc ? cp1 : cc1;  // plane pb after red
          const int bsb = bo(pb) - W;
          const float4 yb0 = lds4(bsb + so0), yb1 = lds4(bsb + so1);  // b(pb)
          const float4 yu0 = lds4(xob + so0 - W), yd0 = lds4(xob + so0 + W);
          const float4 yu1 = lds4(xob + so1 - W), yd1 = lds4(xob + so1 + W);
          // red cells of plane pb - 1 (z-neighbours below; coupled case)
          float4 ym0 = zero4, ym1 = zero4;
          if (zc && k.zmf != 0.f) {
            ym0 = lds4(xs_mm + so0);
            ym1 = lds4(xs_mm + so1);
          }
          float4 f0, f1;
          if (((gj0 + pb) & 1) != 0) {  // black cells 0 and 2
            float e0 = __shfl_up_sync(FULL, yc0.w, 1, 16);
            float e1 = __shfl_up_sync(FULL, yc1.w, 1, 16);
            if (c4 == 0) {
              e0 = S::ld1(sm + xob + so0 - 1);
              e1 = S::ld1(sm + xob + so1 - 1);
            }
            black2(std::true_type(), k, yc0, yu0, yd0, ym0, cc0, yb0, e0, gj0, f0);
            black2(std::true_type(), k, yc1, yu1, yd1, ym1, cc1, yb1, e1, gj1, f1);
          } else {  // black cells 1 and 3
            float e0 = __shfl_down_sync(FULL, yc0.x, 1, 16);
            float e1 = __shfl_down_sync(FULL, yc1.x, 1, 16);
            if (c4 == 15) {
              e0 = S::ld1(sm + xob + so0 + 4);
              e1 = S::ld1(sm + xob + so1 + 4);
            }
            black2(std::false_type(), k, yc0, yu0, yd0, ym0, cc0, yb0, e0, gj0, f0);
            black2(std::false_type(), k, yc1, yu1, yd1, ym1, cc1, yb1, e1, gj1, f1);
          }
          T *xo_pb = reinterpret_cast<T *>(a.xout) + (size_t)pb * plane;
          if (act0) {
            S::st4(xo_pb + go0, f0);
            if (SUM) acc(f0);
          }
          if (act1) {
            S::st4(xo_pb + go1, f1);
            if (SUM) acc(f1);
          }
        }
        if (zc) {
          cp0 = cc0;
          cp1 = cc1;
        }
      }
      have_prev = do_red;
      if (zc) {
        // the next black pass reads this red pass; slots of old planes are free
        if (svc && !failed && t < t1) failed = !wait_planes(x_need_at(t + 1), t + 1) || !wait_c_for(t + 1);
        if (__syncthreads_or(failed)) {
          abort_flag = 1;
          break;
        }
      }
      xs_t = xs_p;
    }
  };
  if (!abort_flag) {
    if constexpr (UNIFORM) {
      if (fast)
        march(std::true_type());
      else
        march(std::false_type());
    } else {
      march(std::false_type());
    }
  }
  if (abort_flag) {
    // a TMA completion did not arrive in time: flag it, give the copies this
    // CTA still has in flight a bounded wait to land, and leave
    if (tid == G::SVC) {
      a.err[0] = 1.0;
      for (int p = xwait + 1; p <= xissued; ++p) mbar_wait(&xbar[rx.slot(p)], rx.parity(p));
      for (int p = bwait + 1; p <= bissued; ++p) mbar_wait(&bbar[rb.slot(p)], rb.parity(p));
      for (int q = cwait + 1; q <= cissued; ++q) mbar_wait(&cbar[cslot(q)], cpar(q));
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
// Producer/consumer rings for the streaming kernels: the service warp's
// first lane issues each plane once its slot has been released by all tile
// warps (an "empty" mbarrier per slot, one arrival per tile warp); tile warps
// wait on the slot's "full" mbarrier (TMA completion) and release it after
// their last read.  No CTA barrier is needed inside the plane loop.
template <int DEPTH>
struct PcRing {
  int lo, hi;
  __device__ __forceinline__ bool has(int p) const { return p >= lo && p <= hi; }
  __device__ __forceinline__ int slot(int p) const { return (p - lo) % DEPTH; }
  __device__ __forceinline__ uint32_t parity(int p) const { return ((p - lo) / DEPTH) & 1; }
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

template <typename T>
struct RestrictGeo {
  static constexpr int W = St<T>::W, OFF = St<T>::OFF;
  static constexpr int XH = SY + 2;              // x box rows j0-1 .. j0+SY
  static constexpr int XR = 6;                   // x planes t, t+1 + 4 in flight
  static constexpr int BR = 4;                   // b plane t + 3 in flight
  static constexpr int XS = pad128<T>(XH * W);
  static constexpr int BS = ZX * SY;             // b box: the tile only
  static constexpr int BOFF = XR * XS;
  static constexpr int MOFF = BOFF + BR * BS;
  static constexpr int TILE_WARPS = 8;
  static constexpr int NT = 32 * (TILE_WARPS + 1);
  static constexpr int SVC = 32 * TILE_WARPS;
  __host__ __device__ static constexpr size_t smem_bytes() {
    return sizeof(T) * (size_t)MOFF + sizeof(uint64_t) * 2 * (XR + BR) + 16;
  }
};

// Residual r = b - A x of a level and its down-sampling into the next
// level's right-hand side.  A tile thread owns rows 2k and 2k + 1 of one
// column of four cells, so the children of a coarse cell in x and y are its
// own; children in z are two consecutive planes of the march.
template <typename T, typename TC, bool UNIFORM, bool COUPLED>
__global__ void __launch_bounds__(RestrictGeo<T>::NT, 2) k_zrestrict(const __grid_constant__ CUtensorMap tmx,
                                                                    const __grid_constant__ CUtensorMap tmb,
                                                                    const ZSweepArgs a) {
  using G = RestrictGeo<T>;
  using S = St<T>;
  constexpr int W = G::W, OFF = G::OFF;
  constexpr bool zc = COUPLED;
  T *sm = reinterpret_cast<T *>(zsm);
  auto lds4 = [&](int off) { return S::ld4(sm + off); };
  uint64_t *xfull = reinterpret_cast<uint64_t *>(sm + G::MOFF);
  uint64_t *bfull = xfull + G::XR;
  uint64_t *xempty = bfull + G::BR;
  uint64_t *bempty = xempty + G::XR;
  __shared__ int abort_flag;
  const LevelDev &L = a.L;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * SY;
  const int zs = blockIdx.z * a.zchunk, ze = min(zs + a.zchunk, nz);
  PcRing<G::XR> rx;
  rx.lo = zc ? max(zs - 1, 0) : zs;
  rx.hi = zc ? min(ze, nz - 1) : ze - 1;
  PcRing<G::BR> rb;
  rb.lo = zs;
  rb.hi = ze - 1;
  if (tid == G::SVC) {
    abort_flag = 0;
    int e = tma_preflight(zsm, G::smem_bytes(), &tmx);
    if (!e) e = tma_preflight(zsm, G::smem_bytes(), &tmb);
    if (e) {
      abort_flag = e;
      a.err[0] = (double)e;
    } else {
      for (int q = 0; q < G::XR; ++q) {
        mbar_init(&xfull[q], 1);
        mbar_init(&xempty[q], G::TILE_WARPS);
      }
      for (int q = 0; q < G::BR; ++q) {
        mbar_init(&bfull[q], 1);
        mbar_init(&bempty[q], G::TILE_WARPS);
      }
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (abort_flag) return;

  if (warp == G::TILE_WARPS) {
    // ---- producer: planes in the order the tile warps need them ----
    if (lane == 0) {
      bool ok = true;
      int px = rx.lo, pb = rb.lo;
      int xdone = rx.lo - 1, bdone = rb.lo - 1;  // issued planes
      while (ok && (px <= rx.hi || pb <= rb.hi)) {
        // x(p) is first needed one step before b(p) (coupled levels)
        const bool take_x = px <= rx.hi && (pb > rb.hi || px <= pb + (zc ? 1 : 0));
        if (take_x) {
          const int q = rx.slot(px);
          if (px - G::XR >= rx.lo) ok = mbar_wait(&xempty[q], rx.parity(px - G::XR));
          if (ok) {
            fence_proxy_async();
            mbar_expect_tx(&xfull[q], (uint32_t)(G::XH * W * sizeof(T)));
            tma_plane(sm + q * G::XS, &tmx, i0 - OFF, j0 - 1, px, &xfull[q]);
            xdone = px++;
          }
        } else {
          const int q = rb.slot(pb);
          if (pb - G::BR >= rb.lo) ok = mbar_wait(&bempty[q], rb.parity(pb - G::BR));
          if (ok) {
            fence_proxy_async();
            mbar_expect_tx(&bfull[q], (uint32_t)(ZX * SY * sizeof(T)));
            tma_plane(sm + G::BOFF + q * G::BS, &tmb, i0, j0, pb, &bfull[q]);
            bdone = pb++;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        a.err[0] = 1.0;
      }
      // every issued copy lands before the CTA may exit (bounded waits)
      for (int p = max(xdone - G::XR + 1, rx.lo); p <= xdone; ++p) mbar_wait(&xfull[rx.slot(p)], rx.parity(p));
      for (int p = max(bdone - G::BR + 1, rb.lo); p <= bdone; ++p) mbar_wait(&bfull[rb.slot(p)], rb.parity(p));
    }
    __syncthreads();
    return;
  }

  // ---- tile warps ----
  const int c4 = lane & 15, kr = 2 * warp + (lane >> 4);  // rows 2 kr, 2 kr + 1
  const int gi = i0 + 4 * c4, gj0 = j0 + 2 * kr, gj1 = gj0 + 1;
  const bool colin = gi < nx;
  const bool act0 = colin && gj0 < ny, act1 = colin && gj1 < ny;
  const int so0 = (2 * kr + 1) * W + OFF + 4 * c4, so1 = so0 + W;
  const int sb0 = (2 * kr) * ZX + 4 * c4, sb1 = sb0 + ZX;
  const float cxu = L.wx * (float)L.sy * (float)L.sz;
  const float cyu = L.wy * (float)L.sx * (float)L.sz;
  const float czu = zc ? L.wz * (float)L.sx * (float)L.sy : 0.f;
  const float mmu = L.wm * (float)L.sx * (float)L.sy * (float)L.sz;
  const bool fast = UNIFORM && i0 >= 1 && i0 + ZX + 1 <= nx && j0 >= 1 && j0 + SY + 1 <= ny;
  const int fx = a.fx, fy = a.fy, fz = a.fz;
  const unsigned FULL = 0xffffffffu;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  bool failed = false;
  int xw = rx.lo - 1, bw = rb.lo - 1;  // planes this warp has waited for
  // (a failed wait is made warp-uniform, so the shuffles stay convergent)
  auto need_x = [&](int p) {
    for (int q = xw + 1; q <= min(p, rx.hi) && !failed; ++q) {
      failed = !mbar_wait(&xfull[rx.slot(q)], rx.parity(q));
      if (!failed) xw = q;
    }
    failed = __any_sync(FULL, failed);
  };
  auto need_b = [&](int p) {
    for (int q = bw + 1; q <= min(p, rb.hi) && !failed; ++q) {
      failed = !mbar_wait(&bfull[rb.slot(q)], rb.parity(q));
      if (!failed) bw = q;
    }
    failed = __any_sync(FULL, failed);
  };
  auto release_x = [&](int p) {
    __syncwarp();
    if (lane == 0 && rx.has(p)) mbar_arrive(&xempty[rx.slot(p)]);
  };
  auto release_b = [&](int p) {
    __syncwarp();
    if (lane == 0 && rb.has(p)) mbar_arrive(&bempty[rb.slot(p)]);
  };
  // residual of one cell; sxn / syn: sums of its x / y neighbours
  auto res = [&](auto fast_c, float bv, float xv, float sxn, float syn, float zm, float zp, float zmf,
                 float zpf, float mz, int ci, int cj) -> float {
    if constexpr (decltype(fast_c)::value) {
      const float dg = 2.f * (cxu + cyu) + czu * (zmf + zpf) + mmu;
      return bv + cxu * sxn + cyu * syn + czu * (zm + zp) - dg * xv;
    }
    float cx = cxu, cy = cyu, cz = czu, mm = mmu;
    if (!UNIFORM) {
      const float mx = mass_of(ci, nx, L.sx, L.lx), my = mass_of(cj, ny, L.sy, L.ly);
      cx = L.wx * my * mz;
      cy = L.wy * mx * mz;
      cz = zc ? L.wz * mx * my : 0.f;
      mm = L.wm * mx * my * mz;
    }
    const float nbx = (float)((ci > 0) + (ci < nx - 1));
    const float nby = (float)((cj > 0) + (cj < ny - 1));
    const float dg = cx * nbx + cy * nby + cz * (zmf + zpf) + mm;
    return bv + cx * sxn + cy * syn + cz * (zmf * zm + zpf * zp) - dg * xv;
  };
  float4 acc0 = zero4, acc1 = zero4;  // first child plane's sums (z coarsened)
  auto march = [&](auto fast_c) {
    float4 xm0 = zero4, xm1 = zero4, xc0 = zero4, xc1 = zero4;
    const int t0 = zs, t1 = ze - 1;
    if (zc && t0 > 0) {
      need_x(t0 - 1);
      const int o = rx.slot(t0 - 1) * G::XS;
      xm0 = lds4(o + so0);
      xm1 = lds4(o + so1);
      release_x(t0 - 1);
    }
    need_x(t0);
    {
      const int o = rx.slot(t0) * G::XS;
      xc0 = lds4(o + so0);
      xc1 = lds4(o + so1);
    }
    for (int t = t0; t <= t1 && !failed; ++t) {
      const bool hm = zc && t > 0, hp = zc && t < nz - 1;
      need_x(zc ? t + 1 : t);
      need_b(t);
      if (failed) break;
      const int o = rx.slot(t) * G::XS, ob = G::BOFF + rb.slot(t) * G::BS;
      float4 xn0 = zero4, xn1 = zero4;
      if (hp) {
        const int on = rx.slot(t + 1) * G::XS;
        xn0 = lds4(on + so0);
        xn1 = lds4(on + so1);
      }
      const float4 xu = lds4(o + so0 - W), xd = lds4(o + so1 + W);
      const float4 b0 = lds4(ob + sb0), b1 = lds4(ob + sb1);
      // x-neighbours across the float4 edges
      float l0 = __shfl_up_sync(FULL, xc0.w, 1, 16), l1 = __shfl_up_sync(FULL, xc1.w, 1, 16);
      float r0 = __shfl_down_sync(FULL, xc0.x, 1, 16), r1 = __shfl_down_sync(FULL, xc1.x, 1, 16);
      if (c4 == 0) {
        l0 = S::ld1(sm + o + so0 - 1);
        l1 = S::ld1(sm + o + so1 - 1);
      }
      if (c4 == 15) {
        r0 = S::ld1(sm + o + so0 + 4);
        r1 = S::ld1(sm + o + so1 + 4);
      }
      release_x(t);
      release_b(t);
      const float zmf = hm ? 1.f : 0.f, zpf = hp ? 1.f : 0.f;
      const float mz = mass_of(t, nz, L.sz, L.lz);
      float4 q0, q1;
      q0.x = res(fast_c, b0.x, xc0.x, l0 + xc0.y, xu.x + xc1.x, xm0.x, xn0.x, zmf, zpf, mz, gi, gj0);
      q0.y = res(fast_c, b0.y, xc0.y, xc0.x + xc0.z, xu.y + xc1.y, xm0.y, xn0.y, zmf, zpf, mz, gi + 1, gj0);
      q0.z = res(fast_c, b0.z, xc0.z, xc0.y + xc0.w, xu.z + xc1.z, xm0.z, xn0.z, zmf, zpf, mz, gi + 2, gj0);
      q0.w = res(fast_c, b0.w, xc0.w, xc0.z + r0, xu.w + xc1.w, xm0.w, xn0.w, zmf, zpf, mz, gi + 3, gj0);
      q1.x = res(fast_c, b1.x, xc1.x, l1 + xc1.y, xc0.x + xd.x, xm1.x, xn1.x, zmf, zpf, mz, gi, gj1);
      q1.y = res(fast_c, b1.y, xc1.y, xc1.x + xc1.z, xc0.y + xd.y, xm1.y, xn1.y, zmf, zpf, mz, gi + 1, gj1);
      q1.z = res(fast_c, b1.z, xc1.z, xc1.y + xc1.w, xc0.z + xd.z, xm1.z, xn1.z, zmf, zpf, mz, gi + 2, gj1);
      q1.w = res(fast_c, b1.w, xc1.w, xc1.z + r1, xc0.w + xd.w, xm1.w, xn1.w, zmf, zpf, mz, gi + 3, gj1);
      if (!act0) q0 = zero4;
      if (!act1) q1 = zero4;
      // children of the coarse cells: x pairs in the float4, y pairs in the
      // two rows, z pairs over two steps
      float4 s0, s1;
      if (fx) {
        s0 = make_float4(q0.x + q0.y, q0.z + q0.w, 0.f, 0.f);
        s1 = make_float4(q1.x + q1.y, q1.z + q1.w, 0.f, 0.f);
      } else {
        s0 = q0;
        s1 = q1;
      }
      if (fy) {
        s0.x += s1.x;
        s0.y += s1.y;
        s0.z += s1.z;
        s0.w += s1.w;
      }
      if (fz && (t & 1) == 0 && t != nz - 1) {
        acc0 = s0;
        acc1 = s1;
      } else {
        if (fz && (t & 1) == 1) {
          s0.x += acc0.x;
          s0.y += acc0.y;
          s0.z += acc0.z;
          s0.w += acc0.w;
          s1.x += acc1.x;
          s1.y += acc1.y;
          s1.z += acc1.z;
          s1.w += acc1.w;
        }
        TC *cpl = reinterpret_cast<TC *>(a.bc) + (size_t)(t >> fz) * a.ncy * a.ncx;
        const int I = (i0 + 4 * c4) >> fx;
        const int J0 = gj0 >> fy;
        if (colin) {
          if (fx) {
            if (gj0 < ny) St<TC>::stg2(cpl + (size_t)J0 * a.ncx + I, make_float2(s0.x, s0.y));
            if (!fy && gj1 < ny) St<TC>::stg2(cpl + (size_t)(J0 + 1) * a.ncx + I, make_float2(s1.x, s1.y));
          } else {
            if (gj0 < ny) St<TC>::st4(cpl + (size_t)J0 * a.ncx + I, s0);
            if (!fy && gj1 < ny) St<TC>::st4(cpl + (size_t)(J0 + 1) * a.ncx + I, s1);
          }
        }
      }
      xm0 = xc0;
      xm1 = xc1;
      xc0 = xn0;
      xc1 = xn1;
      if (!zc && t < t1) {
        // uncoupled: the next plane's own rows are read in its own step
        need_x(t + 1);
        if (!failed) {
          const int on = rx.slot(t + 1) * G::XS;
          xc0 = lds4(on + so0);
          xc1 = lds4(on + so1);
        }
      }
    }
  };
  if (fast)
    march(std::true_type());
  else
    march(std::false_type());
  if (failed) {
    abort_flag = 1;
    a.err[0] = 1.0;
  }
  __syncthreads();
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
  static constexpr int OY = 16;                  // tile rows
  static constexpr int BH = OY + 2;              // box rows j0-1 .. j0+OY
  static constexpr int S = pad32(BH * BOXW);     // floats per box
  static constexpr int SI1 = ZX * OY;            // I1 box: the tile only
  static constexpr int XR = 4;                   // x planes t, t+1 + 2 in flight
  static constexpr int IR = 3;                   // input plane t + 2 in flight
  static constexpr int TILE_WARPS = 8;
  static constexpr int NT = 32 * (TILE_WARPS + 1);
  static constexpr int SVC = 32 * TILE_WARPS;
  // An x slot holds the high part, the low part (if read) and the correction
  // (if added, float32 or float16: esz bytes per element, its own box width)
  // of one plane; an input slot holds I0 (or b) and I1 (SP).  Sizes in bytes.
  __host__ __device__ static constexpr int ebytes(int esz) {
    return esz == 2 ? 2 * pad128<half_t>(BH * St<half_t>::W) : 4 * S;
  }
  __host__ __device__ static constexpr int xstride(bool xl, bool e, int esz) {
    return 4 * S * (1 + xl) + (e ? ebytes(esz) : 0);
  }
  __host__ __device__ static constexpr int istride(bool sp) { return 4 * (S + (sp ? SI1 : 0)); }
  __host__ __device__ static constexpr size_t smem_bytes(bool xl, bool e, bool sp, int esz) {
    return (size_t)(XR * xstride(xl, e, esz) + IR * istride(sp)) +
           sizeof(uint64_t) * 2 * (XR + IR) + sizeof(double) * 32 + 16;
  }
};

// Outer pass of the iterative refinement on the fine level: x_new = x + e
// (+ mean shift) as a float pair, the residual r = b - A x_new with b
// assembled from I0 (and I1), and block sums (r^2, b^2, x, I0).  A tile
// thread owns one float4 of the 64 x 16 tile; the updated values of its
// neighbours' cells are recomputed from the shared-memory planes (rows above
// and below, the row ends) or taken from the neighbouring lanes (shuffles)
// and from its own registers (z), so no thread writes shared memory and the
// planes stream through a producer/consumer ring without CTA barriers.
template <typename TE, int RHS, bool HAS_XL, bool HAS_E, bool ACCURATE>
__global__ void __launch_bounds__(OuterGeo::NT, ACCURATE ? 2 : 3) k_zouter(const __grid_constant__ CUtensorMap tmh,
                                                            const __grid_constant__ CUtensorMap tml,
                                                            const __grid_constant__ CUtensorMap tme,
                                                            const __grid_constant__ CUtensorMap tmi0,
                                                            const __grid_constant__ CUtensorMap tmi1,
                                                            const OuterArgs a, int zchunk, double *err) {
  using G = OuterGeo;
  constexpr int S = G::S;
  constexpr bool SP = RHS == RHS_SP;
  constexpr int ESZ = (int)sizeof(TE);
  constexpr int XSTB = G::xstride(HAS_XL, HAS_E, ESZ), ISTB = G::istride(SP);  // bytes
  constexpr int LOFF = S;                                 // floats, within an x slot
  constexpr int EOFFB = 4 * S * (1 + (HAS_XL ? 1 : 0));  // bytes, within an x slot
  constexpr int WE = St<TE>::W, OFFE = St<TE>::OFF;
  char *const smb = reinterpret_cast<char *>(zsm);
  auto xslot = [&](int q) { return reinterpret_cast<float *>(smb + q * XSTB); };
  auto islot = [&](int q) { return reinterpret_cast<float *>(smb + G::XR * XSTB + q * ISTB); };
  // the low word of the float pair is carried only in exact passes (and read
  // whenever the caller passes one)
  constexpr bool USE_L = HAS_XL || (HAS_E && ACCURATE);
  uint64_t *xfull = reinterpret_cast<uint64_t *>(smb + G::XR * XSTB + G::IR * ISTB);
  uint64_t *ifull = xfull + G::XR;
  uint64_t *xempty = ifull + G::IR;
  uint64_t *iempty = xempty + G::XR;
  double *dsh = reinterpret_cast<double *>(iempty + G::IR);
  __shared__ int abort_flag;

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = blockIdx.x * ZX, j0 = blockIdx.y * G::OY;
  const int zs = blockIdx.z * zchunk, ze = min(zs + zchunk, nz);
  const bool zc = (a.bz != 0.f) && (nz > 1);
  const size_t plane = (size_t)nx * ny;
  PcRing<G::XR> rx;
  rx.lo = zc ? max(zs - 1, 0) : zs;
  rx.hi = zc ? min(ze, nz - 1) : ze - 1;
  PcRing<G::IR> ri;
  ri.lo = zs;
  ri.hi = ze - 1;
  constexpr uint32_t BOXB = (uint32_t)(G::BH * BOXW * sizeof(float));

  if (tid == G::SVC) {
    abort_flag = 0;
    const size_t bytes = G::smem_bytes(HAS_XL, HAS_E, SP, ESZ);
    int e = tma_preflight(zsm, bytes, &tmh);
    if (!e && HAS_XL) e = tma_preflight(zsm, bytes, &tml);
    if (!e && HAS_E) e = tma_preflight(zsm, bytes, &tme);
    if (!e) e = tma_preflight(zsm, bytes, &tmi0);
    if (!e && SP) e = tma_preflight(zsm, bytes, &tmi1);
    if (e) {
      abort_flag = e;
      err[0] = (double)e;
    } else {
      for (int q = 0; q < G::XR; ++q) {
        mbar_init(&xfull[q], 1);
        mbar_init(&xempty[q], G::TILE_WARPS);
      }
      for (int q = 0; q < G::IR; ++q) {
        mbar_init(&ifull[q], 1);
        mbar_init(&iempty[q], G::TILE_WARPS);
      }
      fence_mbar_init();
    }
  }
  __syncthreads();
  if (abort_flag) return;  // nothing issued yet

  // per-thread sums in FP32 (r^2, b^2, I0) and double-float (x); FP64 only
  // once per block
  float srr = 0.f, sbb = 0.f, si = 0.f, sxh = 0.f, sxl = 0.f;
  float rmx = 0.f;  // max |r| (for the scale of a float16 residual)

  if (warp == G::TILE_WARPS) {
    // ---- producer: planes in the order the tile warps need them ----
    if (lane == 0) {
      bool ok = true;
      int px = rx.lo, pi = ri.lo;
      int xdone = rx.lo - 1, idone = ri.lo - 1;
      while (ok && (px <= rx.hi || pi <= ri.hi)) {
        const bool take_x = px <= rx.hi && (pi > ri.hi || px <= pi + (zc ? 1 : 0));
        if (take_x) {
          const int q = rx.slot(px);
          if (px - G::XR >= rx.lo) ok = mbar_wait(&xempty[q], rx.parity(px - G::XR));
          if (ok) {
            fence_proxy_async();
            float *xb = xslot(q);
            mbar_expect_tx(&xfull[q], BOXB * (1 + (HAS_XL ? 1 : 0)) +
                                          (HAS_E ? (uint32_t)(G::BH * WE * ESZ) : 0u));
            tma_plane(xb, &tmh, i0 - 4, j0 - 1, px, &xfull[q]);
            if (HAS_XL) tma_plane(xb + LOFF, &tml, i0 - 4, j0 - 1, px, &xfull[q]);
            if (HAS_E) tma_plane(smb + q * XSTB + EOFFB, &tme, i0 - OFFE, j0 - 1, px, &xfull[q]);
            xdone = px++;
          }
        } else {
          const int q = ri.slot(pi);
          if (pi - G::IR >= ri.lo) ok = mbar_wait(&iempty[q], ri.parity(pi - G::IR));
          if (ok) {
            fence_proxy_async();
            float *ib = islot(q);
            mbar_expect_tx(&ifull[q], BOXB + (SP ? (uint32_t)(G::SI1 * sizeof(float)) : 0u));
            tma_plane(ib, &tmi0, i0 - 4, j0 - 1, pi, &ifull[q]);
            if (SP) tma_plane(ib + S, &tmi1, i0, j0, pi, &ifull[q]);
            idone = pi++;
          }
        }
      }
      if (!ok) {
        abort_flag = 1;
        err[0] = 1.0;
      }
      // every issued copy lands before the CTA may exit (bounded waits)
      for (int p = max(xdone - G::XR + 1, rx.lo); p <= xdone; ++p) mbar_wait(&xfull[rx.slot(p)], rx.parity(p));
      for (int p = max(idone - G::IR + 1, ri.lo); p <= idone; ++p) mbar_wait(&ifull[ri.slot(p)], ri.parity(p));
    }
  } else {
    // ---- tile warps ----
    const unsigned FULL = 0xffffffffu;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const int c4 = lane & 15, r = 2 * warp + (lane >> 4);
    const int gi = i0 + 4 * c4, gj = j0 + r;
    const bool act = gi < nx && gj < ny;
    const int so = (r + 1) * BOXW + 4 + 4 * c4;  // box row 0 is j0 - 1
    const int si1 = r * ZX + 4 * c4;
    float shift = 0.f;
    if (HAS_E && a.mean_fix)
      shift = (float)((a.scalars[S_I0] - a.scalars[S_X] - a.scalars[S_E] * (double)a.e_scale) * a.inv_n);
    const float esc = a.e_scale;
    bool failed = false;
    int xw = rx.lo - 1, iw = ri.lo - 1;
    auto need_x = [&](int p) {
      for (int q = xw + 1; q <= min(p, rx.hi) && !failed; ++q) {
        failed = !mbar_wait(&xfull[rx.slot(q)], rx.parity(q));
        if (!failed) xw = q;
      }
      failed = __any_sync(FULL, failed);
    };
    auto need_i = [&](int p) {
      for (int q = iw + 1; q <= min(p, ri.hi) && !failed; ++q) {
        failed = !mbar_wait(&ifull[ri.slot(q)], ri.parity(q));
        if (!failed) iw = q;
      }
      failed = __any_sync(FULL, failed);
    };
    auto release_x = [&](int p) {
      __syncwarp();
      if (lane == 0 && rx.has(p)) mbar_arrive(&xempty[rx.slot(p)]);
    };
    auto release_i = [&](int p) {
      __syncwarp();
      if (lane == 0 && ri.has(p)) mbar_arrive(&iempty[ri.slot(p)]);
    };
    // the updated iterate (a float pair) at one cell / four cells of x slot
    // q; rr is the box row, col the column relative to the tile
    auto upd1 = [&](int q, int rr, int col, float &h, float &l) {
      const float *xb = xslot(q);
      const int off = rr * BOXW + 4 + col;
      h = xb[off];
      l = HAS_XL ? xb[LOFF + off] : 0.f;
      if (HAS_E) {
        const TE *eb = reinterpret_cast<const TE *>(smb + q * XSTB + EOFFB);
        const float e = __fadd_rn(St<TE>::ld1(eb + rr * WE + OFFE + col) * esc, shift);
        if (ACCURATE) {
          const ff v = ff_add({h, l}, {e, 0.f});
          h = v.h;
          l = v.l;
        } else {
          h = __fadd_rn(h, e);
        }
      }
      if (!USE_L) l = 0.f;
    };
    auto upd4 = [&](int q, int rr, int col, float4 &h, float4 &l) {
      const float *xb = xslot(q);
      const int off = rr * BOXW + 4 + col;
      h = *reinterpret_cast<const float4 *>(xb + off);
      l = HAS_XL ? *reinterpret_cast<const float4 *>(xb + LOFF + off) : zero4;
      if (HAS_E) {
        const TE *eb = reinterpret_cast<const TE *>(smb + q * XSTB + EOFFB);
        const float4 e = St<TE>::ld4(eb + rr * WE + OFFE + col);
        float hv[4] = {h.x, h.y, h.z, h.w}, lv[4] = {l.x, l.y, l.z, l.w};
        const float ev[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float ee = __fadd_rn(ev[c] * esc, shift);
          if (ACCURATE) {
            const ff v = ff_add({hv[c], lv[c]}, {ee, 0.f});
            hv[c] = v.h;
            lv[c] = v.l;
          } else {
            hv[c] = __fadd_rn(hv[c], ee);
          }
        }
        h = make_float4(hv[0], hv[1], hv[2], hv[3]);
        l = make_float4(lv[0], lv[1], lv[2], lv[3]);
      }
      if (!USE_L) l = zero4;
    };
    auto add_x = [&](float v) {
      const ff t = two_sum(sxh, v);
      sxh = t.h;
      sxl += t.l;
    };
    // residual at one cell from its value (hc, lc), its neighbours' values
    // and presence flags (missing neighbours contribute no difference), the
    // I0 values around it (gradient right-hand side) and I1
    auto cell = [&](float hc, float lc, bool w, float hw, float lw, bool e, float he, float le, bool s,
                    float hs, float ls, bool n, float hn, float ln, bool m, float hm, float lm, bool p,
                    float hp, float lp, float ic, float iw_, float ie, float is, float in_, float i1,
                    float &bh_out) -> float {
      float gx = 0.f, gy = 0.f, bh, bl = 0.f;
      if (RHS == RHS_EXPLICIT) {
        bh = ic;
      } else {
        gx = (w ? ic - iw_ : 0.f) + (e ? ic - ie : 0.f);
        gy = (s ? ic - is : 0.f) + (n ? ic - in_ : 0.f);
      }
      float rv;
      if (!ACCURATE) {
        // FP32 differences of the float pair: error ~1e-7 of the local terms
        // (the low words enter only when the pair is carried)
        auto d = [&](bool has, float h, float l) -> float {
          if (!has) return 0.f;
          return USE_L ? (hc - h) + (lc - l) : hc - h;
        };
        const float dx = d(w, hw, lw) + d(e, he, le);
        const float dy = d(s, hs, ls) + d(n, hn, ln);
        const float dz = d(m, hm, lm) + d(p, hp, lp);
        const float ax = a.bx * dx + a.by * dy + a.bz * dz + a.alpha * (USE_L ? hc + lc : hc);
        if (RHS != RHS_EXPLICIT) {
          bh = a.rbx * gx + a.rby * gy;
          if (SP) bh += a.ralpha * i1;
        }
        rv = bh - ax;
      } else {
        // compensated evaluation: every rounding error of the hi parts is
        // captured by an error-free transformation and summed into `lo`
        float lo = 0.f;
        auto axis = [&](bool has1, float h1, float l1, bool has2, float h2, float l2, float wh, float wl) {
          float t1 = 0.f, t2 = 0.f, la = 0.f;
          if (has1) {
            const ff d = two_sum(hc, -h1);
            t1 = d.h;
            la += d.l + (lc - l1);
          }
          if (has2) {
            const ff d = two_sum(hc, -h2);
            t2 = d.h;
            la += d.l + (lc - l2);
          }
          const ff S2 = two_sum(t1, t2);
          la += S2.l;
          const float pp = S2.h * wh;
          lo += __fmaf_rn(S2.h, wh, -pp) + S2.h * wl + la * wh;
          return pp;
        };
        const float px = axis(w, hw, lw, e, he, le, a.bx, a.bx_lo);
        const float py = axis(s, hs, ls, n, hn, ln, a.by, a.by_lo);
        const float pz = zc ? axis(m, hm, lm, p, hp, lp, a.bz, a.bz_lo) : 0.f;
        const float pa = hc * a.alpha;
        lo += __fmaf_rn(hc, a.alpha, -pa) + hc * a.alpha_lo + lc * a.alpha;
        ff A = two_sum(px, py);
        lo += A.l;
        A = two_sum(A.h, pz);
        lo += A.l;
        A = two_sum(A.h, pa);
        lo += A.l;
        if (RHS != RHS_EXPLICIT) {
          const float qx = gx * a.rbx, qy = gy * a.rby;
          bl = __fmaf_rn(gx, a.rbx, -qx) + gx * a.rbx_lo + __fmaf_rn(gy, a.rby, -qy) + gy * a.rby_lo;
          ff Bv = two_sum(qx, qy);
          bl += Bv.l;
          if (SP) {
            const float qa = i1 * a.ralpha;
            bl += __fmaf_rn(i1, a.ralpha, -qa) + i1 * a.ralpha_lo;
            Bv = two_sum(Bv.h, qa);
            bl += Bv.l;
          }
          bh = Bv.h;
        }
        const ff Rv = two_sum(bh, -A.h);
        rv = Rv.h + (Rv.l + (bl - lo));
      }
      bh_out = bh;
      return rv;
    };

    // The plane loop, specialised for tiles whose cells all have their four
    // in-plane neighbours inside the domain (presence flags constant).
    const bool fast = i0 >= 1 && i0 + ZX + 1 <= nx && j0 >= 1 && j0 + G::OY + 1 <= ny;
    auto march = [&](auto fast_c) {
      constexpr bool F = decltype(fast_c)::value;
      const bool w0 = F || gi > 0, e3 = F || gi + 3 < nx - 1, sn = F || gj > 0, nn = F || gj < ny - 1;
      float4 hm4 = zero4, lm4 = zero4, hc4 = zero4, lc4 = zero4;  // planes t-1, t (own cells)
      const int t0 = zs, t1 = ze - 1;
      if (zc && t0 > 0) {
        need_x(t0 - 1);
        upd4(rx.slot(t0 - 1), r + 1, 4 * c4, hm4, lm4);
        release_x(t0 - 1);
      }
      need_x(t0);
      if (!failed) upd4(rx.slot(t0), r + 1, 4 * c4, hc4, lc4);
      for (int t = t0; t <= t1 && !failed; ++t) {
        const bool hm = zc && t > 0, hp = zc && t < nz - 1;
        float4 hp4 = zero4, lp4 = zero4;
        if (hp) {
          need_x(t + 1);
          if (failed) break;
          upd4(rx.slot(t + 1), r + 1, 4 * c4, hp4, lp4);
        }
        need_i(t);
        if (failed) break;
        const int qx = rx.slot(t);
        const float *ib = islot(ri.slot(t));
        float4 hu, lu, hd, ld;
        upd4(qx, r, 4 * c4, hu, lu);
        upd4(qx, r + 2, 4 * c4, hd, ld);
        // x-neighbours across the float4 edges: the neighbouring lane's cells,
        // or the shared-memory planes at the tile's ends
        float hw = __shfl_up_sync(FULL, hc4.w, 1, 16), lw = __shfl_up_sync(FULL, lc4.w, 1, 16);
        float he = __shfl_down_sync(FULL, hc4.x, 1, 16), le = __shfl_down_sync(FULL, lc4.x, 1, 16);
        if (c4 == 0) upd1(qx, r + 1, -1, hw, lw);
        if (c4 == 15) upd1(qx, r + 1, 4 * c4 + 4, he, le);
        const float4 ic = *reinterpret_cast<const float4 *>(ib + so);
        float4 iu = zero4, id = zero4;
        float iw_ = 0.f, ie_ = 0.f;
        if (RHS != RHS_EXPLICIT) {
          iu = *reinterpret_cast<const float4 *>(ib + so - BOXW);
          id = *reinterpret_cast<const float4 *>(ib + so + BOXW);
          iw_ = __shfl_up_sync(FULL, ic.w, 1, 16);
          ie_ = __shfl_down_sync(FULL, ic.x, 1, 16);
          if (c4 == 0) iw_ = ib[so - 1];
          if (c4 == 15) ie_ = ib[so + 4];
        }
        const float4 i1 = SP ? *reinterpret_cast<const float4 *>(ib + S + si1) : zero4;
        release_x(t);
        release_i(t);
        if (act) {
          float rv[4], bh[4];
          rv[0] = cell(hc4.x, lc4.x, w0, hw, lw, true, hc4.y, lc4.y, sn, hu.x, lu.x, nn, hd.x, ld.x, hm,
                       hm4.x, lm4.x, hp, hp4.x, lp4.x, ic.x, iw_, ic.y, iu.x, id.x, i1.x, bh[0]);
          rv[1] = cell(hc4.y, lc4.y, true, hc4.x, lc4.x, true, hc4.z, lc4.z, sn, hu.y, lu.y, nn, hd.y, ld.y,
                       hm, hm4.y, lm4.y, hp, hp4.y, lp4.y, ic.y, ic.x, ic.z, iu.y, id.y, i1.y, bh[1]);
          rv[2] = cell(hc4.z, lc4.z, true, hc4.y, lc4.y, true, hc4.w, lc4.w, sn, hu.z, lu.z, nn, hd.z, ld.z,
                       hm, hm4.z, lm4.z, hp, hp4.z, lp4.z, ic.z, ic.y, ic.w, iu.z, id.z, i1.z, bh[2]);
          rv[3] = cell(hc4.w, lc4.w, true, hc4.z, lc4.z, e3, he, le, sn, hu.w, lu.w, nn, hd.w, ld.w, hm,
                       hm4.w, lm4.w, hp, hp4.w, lp4.w, ic.w, ic.z, ie_, iu.w, id.w, i1.w, bh[3]);
          const size_t g = (size_t)t * plane + (size_t)gj * nx + gi;
          if (a.xh_out) *reinterpret_cast<float4 *>(a.xh_out + g) = hc4;
          if (USE_L && a.xl_out) *reinterpret_cast<float4 *>(a.xl_out + g) = lc4;
          if (a.r_out)
            St<TE>::st4(reinterpret_cast<TE *>(a.r_out) + g,
                        make_float4(rv[0] * a.r_scale, rv[1] * a.r_scale, rv[2] * a.r_scale, rv[3] * a.r_scale));
          rmx = fmaxf(rmx, fmaxf(fmaxf(fabsf(rv[0]), fabsf(rv[1])), fmaxf(fabsf(rv[2]), fabsf(rv[3]))));
  #pragma unroll
          for (int c = 0; c < 4; ++c) {
            srr += rv[c] * rv[c];
            sbb += bh[c] * bh[c];
          }
          add_x((hc4.x + hc4.y) + (hc4.z + hc4.w));
          sxl += (lc4.x + lc4.y) + (lc4.z + lc4.w);
          if (RHS != RHS_EXPLICIT) si += (ic.x + ic.y) + (ic.z + ic.w);
        }
        hm4 = hc4;
        lm4 = lc4;
        hc4 = hp4;
        lc4 = lp4;
        if (!zc && t < t1) {
          // uncoupled: the next plane's own cells are read in its own step
          need_x(t + 1);
          if (!failed) upd4(rx.slot(t + 1), r + 1, 4 * c4, hc4, lc4);
        }
      }
    };
    if (fast)
      march(std::true_type());
    else
      march(std::false_type());
    if (failed) {
      abort_flag = 1;
      err[0] = 1.0;
    }
  }
  __syncthreads();
  if (abort_flag) return;
  if (a.rmax) {
    for (int o = 16; o > 0; o >>= 1) rmx = fmaxf(rmx, __shfl_xor_sync(0xffffffffu, rmx, o));
    // non-negative floats order as their bit patterns
    if (lane == 0 && rmx > 0.f) atomicMax(a.rmax, __float_as_uint(rmx));
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

// 3D map over a float32 / float16 (esz = 4 / 2 bytes) [nz][ny][nx] array with a
// (width x rows x 1) box; rows must be 16-byte multiples (TMA strides).
bool make_map(CUtensorMap *m, const void *base, int nx, int ny, int nz, int width, int rows, int esz) {
  if (!encoder() || !base) return false;
  if (((uintptr_t)base & 15) != 0 || ((size_t)nx * esz) % 16 != 0) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * esz, (cuuint64_t)nx * ny * esz};
  const cuuint32_t box[3] = {(cuuint32_t)width, (cuuint32_t)rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return g_encode(m, esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                  const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
bool make_map(CUtensorMap *m, const float *base, int nx, int ny, int nz, int width, int rows) {
  return make_map(m, static_cast<const void *>(base), nx, ny, nz, width, rows, 4);
}
int box_w(int esz) { return esz == 2 ? St<half_t>::W : St<float>::W; }

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

// z chunking.  A CTA marches one chunk of planes of one column tile; all
// CTAs of a launch do (nearly) the same work, so a launch takes about
// ceil(CTAs / resident slots) CTA durations, and a CTA's duration grows with
// its chunk plus the planes it touches beyond it (coupled levels: the red
// pass below the chunk and the x planes around it, about three planes; one
// for the pipeline fill otherwise).  The chunk count minimises that product:
// a nearly empty last wave costs as much as a full one.  Chunks are even on
// coupled levels and where z is coarsened (both children of a coarse plane
// in one chunk).
struct ZPlan {
  int tiles, nz;
  bool coupled, even;
  int *nblocks_out;
};
int pick_zchunk(const ZPlan &p, int slots) {
  const int h = p.coupled ? 3 : 1;
  const int min_chunk = p.coupled ? 4 : 1;
  const int max_chunks = std::max(1, p.nz / min_chunk);
  long best_cost = -1;
  int best = p.nz + (p.even && (p.nz & 1) ? 1 : 0);
  for (int c = 1; c <= max_chunks; ++c) {
    int zc = (p.nz + c - 1) / c;
    if (p.even && (zc & 1)) ++zc;
    const long gz = (p.nz + zc - 1) / zc;
    const long waves = ((long)p.tiles * gz + slots - 1) / slots;
    const long cost = waves * (zc + h);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = zc;
    }
  }
  return best;
}
// resident CTAs of one instantiation on the whole GPU (queried once)
template <typename K>
int resident_slots(K kernel, int threads, size_t smem, int &cache) {
  if (!cache) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    cache = n * sm_count();
  }
  return cache;
}
// fills in the z extent of the grid and the chunk for one instantiation
template <typename K>
int plan_z(K kernel, int threads, size_t smem, int &cache, const ZPlan &p, dim3 &grid) {
  const int zc = pick_zchunk(p, resident_slots(kernel, threads, smem, cache));
  grid.z = (p.nz + zc - 1) / zc;
  if (p.nblocks_out) *p.nblocks_out = (int)(grid.x * grid.y * grid.z);
  return zc;
}

template <typename T, typename TC, bool Z, bool P, bool S, bool U, bool C>
cudaError_t run_zsweep_uc(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc,
                          const ZSweepArgs &a0, dim3 grid, const ZPlan &zp, cudaStream_t st) {
  const size_t bytes = SweepGeo<T, TC, P>::smem_bytes();
  static bool attr = false;
  static int slots = 0;
  if (!attr) {
    cudaError_t e = set_smem(k_zsweep<T, TC, Z, P, S, U, C>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  ZSweepArgs a = a0;
  a.zchunk = plan_z(k_zsweep<T, TC, Z, P, S, U, C>, SweepGeo<T, TC, P>::NT, bytes, slots, zp, grid);
  k_zsweep<T, TC, Z, P, S, U, C><<<grid, SweepGeo<T, TC, P>::NT, bytes, st>>>(mx, mb, mc, a);
  return cudaGetLastError();
}
bool level_uniform(const LevelDev &L) { return L.sx == L.lx && L.sy == L.ly && L.sz == L.lz; }
bool level_coupled(const LevelDev &L) { return L.wz != 0.f && L.nz > 1; }
template <typename T, typename TC, bool Z, bool P, bool S>
cudaError_t run_zsweep(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc,
                       const ZSweepArgs &a, dim3 grid, const ZPlan &zp, cudaStream_t st) {
  const bool u = level_uniform(a.L), c = level_coupled(a.L);
  if (u && c) return run_zsweep_uc<T, TC, Z, P, S, true, true>(mx, mb, mc, a, grid, zp, st);
  if (u) return run_zsweep_uc<T, TC, Z, P, S, true, false>(mx, mb, mc, a, grid, zp, st);
  if (c) return run_zsweep_uc<T, TC, Z, P, S, false, true>(mx, mb, mc, a, grid, zp, st);
  return run_zsweep_uc<T, TC, Z, P, S, false, false>(mx, mb, mc, a, grid, zp, st);
}
// the five sweep variants of a V-cycle; the coarse type matters only with
// the prolongation
template <typename T, typename TC>
cudaError_t run_zsweep_variant(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc,
                               const ZSweepArgs &a, bool zero_in, bool prolong, bool sum, dim3 grid,
                               const ZPlan &zp, cudaStream_t st) {
  if (zero_in && !prolong && !sum) return run_zsweep<T, T, true, false, false>(mx, mb, mc, a, grid, zp, st);
  if (!zero_in && prolong && !sum) return run_zsweep<T, TC, false, true, false>(mx, mb, mc, a, grid, zp, st);
  if (!zero_in && prolong && sum) return run_zsweep<T, TC, false, true, true>(mx, mb, mc, a, grid, zp, st);
  if (!zero_in && !prolong && !sum) return run_zsweep<T, T, false, false, false>(mx, mb, mc, a, grid, zp, st);
  if (!zero_in && !prolong && sum) return run_zsweep<T, T, false, false, true>(mx, mb, mc, a, grid, zp, st);
  return cudaErrorNotSupported;
}
template <typename T, typename TC, bool U, bool C>
cudaError_t run_zrestrict(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a0,
                          dim3 grid, const ZPlan &zp, cudaStream_t st) {
  const size_t bytes = RestrictGeo<T>::smem_bytes();
  static bool attr = false;
  static int slots = 0;
  if (!attr) {
    cudaError_t e = set_smem(k_zrestrict<T, TC, U, C>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  ZSweepArgs a = a0;
  a.zchunk = plan_z(k_zrestrict<T, TC, U, C>, RestrictGeo<T>::NT, bytes, slots, zp, grid);
  k_zrestrict<T, TC, U, C><<<grid, RestrictGeo<T>::NT, bytes, st>>>(mx, mb, a);
  return cudaGetLastError();
}
template <typename T, typename TC>
cudaError_t run_zrestrict_t(const CUtensorMap &mx, const CUtensorMap &mb, const ZSweepArgs &a,
                            dim3 grid, const ZPlan &zp, cudaStream_t st) {
  const bool u = level_uniform(a.L), c = level_coupled(a.L);
  if (u && c) return run_zrestrict<T, TC, true, true>(mx, mb, a, grid, zp, st);
  if (u) return run_zrestrict<T, TC, true, false>(mx, mb, a, grid, zp, st);
  if (c) return run_zrestrict<T, TC, false, true>(mx, mb, a, grid, zp, st);
  return run_zrestrict<T, TC, false, false>(mx, mb, a, grid, zp, st);
}

template <typename TE, int RHS, bool XL, bool E, bool ACC>
cudaError_t run_zouter(const CUtensorMap *m, const OuterArgs &a, const ZPlan &zp, double *err, dim3 grid,
                       cudaStream_t st) {
  const size_t bytes = OuterGeo::smem_bytes(XL, E, RHS == RHS_SP, (int)sizeof(TE));
  static bool attr = false;
  static int slots = 0;
  if (!attr) {
    cudaError_t e = set_smem(k_zouter<TE, RHS, XL, E, ACC>, bytes);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int zchunk = plan_z(k_zouter<TE, RHS, XL, E, ACC>, OuterGeo::NT, bytes, slots, zp, grid);
  k_zouter<TE, RHS, XL, E, ACC><<<grid, OuterGeo::NT, bytes, st>>>(m[0], m[1], m[2], m[3], m[4], a, zchunk,
                                                                    err);
  return cudaGetLastError();
}
template <typename TE>
cudaError_t run_zouter_t(const CUtensorMap *m, const OuterArgs &a, int rhs_mode, const ZPlan &zp, double *err,
                         dim3 grid, cudaStream_t st) {
  const bool xl = a.xl_in != nullptr, e = a.e != nullptr;
#define GD_ZO2(R, ACC)                                                              \
  if (xl && e) return run_zouter<TE, R, true, true, ACC>(m, a, zp, err, grid, st);  \
  if (xl) return run_zouter<TE, R, true, false, ACC>(m, a, zp, err, grid, st);      \
  if (e) return run_zouter<TE, R, false, true, ACC>(m, a, zp, err, grid, st);       \
  return run_zouter<TE, R, false, false, ACC>(m, a, zp, err, grid, st);
#define GD_ZO(R)    \
  if (a.accurate) { \
    GD_ZO2(R, true) \
  } else {          \
    GD_ZO2(R, false) \
  }
  if (rhs_mode == RHS_EXPLICIT) { GD_ZO(RHS_EXPLICIT) }
  if (rhs_mode == RHS_AD) { GD_ZO(RHS_AD) }
  GD_ZO(RHS_SP)
#undef GD_ZO
#undef GD_ZO2
}

}  // namespace

#if GD_ZM_PART(1)
cudaError_t zsweep_f32(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc, const ZSweepArgs &a,
                       bool zero_in, bool prolong, bool sum, int esz_c, dim3 grid, int *nblocks_out,
                       cudaStream_t st) {
  const ZPlan zp{(int)(grid.x * grid.y), a.L.nz, level_coupled(a.L), level_coupled(a.L), nblocks_out};
  if (esz_c == 2 && prolong)
    return run_zsweep_variant<float, half_t>(mx, mb, mc, a, zero_in, prolong, sum, grid, zp, st);
  return run_zsweep_variant<float, float>(mx, mb, mc, a, zero_in, prolong, sum, grid, zp, st);
}
#endif

#if GD_ZM_PART(2)
cudaError_t zsweep_bf16(const CUtensorMap &mx, const CUtensorMap &mb, const CUtensorMap &mc, const ZSweepArgs &a,
                        bool zero_in, bool prolong, bool sum, int esz_c, dim3 grid, int *nblocks_out,
                        cudaStream_t st) {
  const ZPlan zp{(int)(grid.x * grid.y), a.L.nz, level_coupled(a.L), level_coupled(a.L), nblocks_out};
  if (esz_c == 2 || !prolong)
    return run_zsweep_variant<half_t, half_t>(mx, mb, mc, a, zero_in, prolong, sum, grid, zp, st);
  return run_zsweep_variant<half_t, float>(mx, mb, mc, a, zero_in, prolong, sum, grid, zp, st);
}
#endif

#if GD_ZM_PART(3) || GD_ZM_PART(4)
namespace {
ZPlan outer_plan(const OuterArgs &a, dim3 grid, int *nblocks_out) {
  const bool coupled = (a.bz != 0.f) && (a.nz > 1);
  return ZPlan{(int)(grid.x * grid.y), a.nz, coupled, coupled, nblocks_out};
}
}  // namespace
#endif
#if GD_ZM_PART(3)
cudaError_t zouter_f32(const CUtensorMap *m, const OuterArgs &a, int rhs_mode, double *err, dim3 grid,
                       int *nblocks_out, cudaStream_t st) {
  return run_zouter_t<float>(m, a, rhs_mode, outer_plan(a, grid, nblocks_out), err, grid, st);
}
#endif
#if GD_ZM_PART(4)
cudaError_t zouter_bf16(const CUtensorMap *m, const OuterArgs &a, int rhs_mode, double *err, dim3 grid,
                        int *nblocks_out, cudaStream_t st) {
  return run_zouter_t<half_t>(m, a, rhs_mode, outer_plan(a, grid, nblocks_out), err, grid, st);
}
#endif

#if GD_ZM_PART(0)
bool zmarch_usable(const LevelDev &L, int esz) { return encoder() && ((size_t)L.nx * esz) % 16 == 0; }

cudaError_t launch_zsweep(ZSweepArgs a, const void *xin, const void *b, bool zero_in, bool prolong,
                          bool sum, int esz, int esz_c, int *nblocks_out, cudaStream_t st) {
  const LevelDev &L = a.L;
  const int rows_x = SweepGeo<float>::XH, rows_b = SweepGeo<float>::BH;
  CUtensorMap mx, mb;
  std::memset(&mx, 0, sizeof mx);
  if (!make_map(&mx, zero_in ? b : xin, L.nx, L.ny, L.nz, box_w(esz), rows_x, esz)) return cudaErrorNotSupported;
  if (!make_map(&mb, b, L.nx, L.ny, L.nz, box_w(esz), rows_b, esz)) return cudaErrorNotSupported;
  if (((uintptr_t)a.xout & 15) != 0) return cudaErrorNotSupported;
  const int gx = (L.nx + ZX - 1) / ZX, gy = (L.ny + SY - 1) / SY;
  dim3 grid(gx, gy, 1);
  // prolongation: a map over the coarse level for the staging copies (and
  // L2 prefetches) of the boxes the correction reads (x: 32 coarse cells +
  // alignment margins when x is coarsened, else the fine box -- 80 wide from
  // 8 cells left of the tile for a bfloat16 level under a float32 one, where
  // 16-byte alignment puts its start; y: the 36 fine box rows, or 18 when y
  // is coarsened).  Without the map the correction loads from global memory.
  CUtensorMap mc = mx;
  a.cpf = 0;
  if (prolong) {
    const int ac = 16 / esz_c, ncz = a.fz ? (L.nz + 1) / 2 : L.nz;
    const int cw = a.fx ? 32 + 2 * ac : (esz == 4 && esz_c == 2 ? 80 : box_w(esz)), ch = a.fy ? rows_x / 2 : rows_x;
    // (a coarse level whose rows break TMA's alignment is simply not prefetched)
    a.cpf = make_map(&mc, a.xc, a.ncx, a.ncy, ncz, cw, ch, esz_c) ? 1 : 0;
    if (!a.cpf) mc = mx;
  }
  if (esz == 4) return zsweep_f32(mx, mb, mc, a, zero_in, prolong, sum, esz_c, grid, nblocks_out, st);
  return zsweep_bf16(mx, mb, mc, a, zero_in, prolong, sum, esz_c, grid, nblocks_out, st);
}

cudaError_t launch_zrestrict(ZSweepArgs a, const void *x, const void *b, int esz, int esz_c, cudaStream_t st) {
  const LevelDev &L = a.L;
  CUtensorMap mx, mb;
  if (!make_map(&mx, x, L.nx, L.ny, L.nz, box_w(esz), RestrictGeo<float>::XH, esz)) return cudaErrorNotSupported;
  if (!make_map(&mb, b, L.nx, L.ny, L.nz, ZX, SY, esz)) return cudaErrorNotSupported;
  if (((uintptr_t)a.bc & 15) != 0) return cudaErrorNotSupported;
  const int gx = (L.nx + ZX - 1) / ZX, gy = (L.ny + SY - 1) / SY;
  const bool coupled = level_coupled(L);
  const ZPlan zp{gx * gy, L.nz, coupled, coupled || a.fz != 0, nullptr};
  dim3 grid(gx, gy, 1);
  if (esz == 4 && esz_c == 2) return run_zrestrict_t<float, half_t>(mx, mb, a, grid, zp, st);
  if (esz == 4) return run_zrestrict_t<float, float>(mx, mb, a, grid, zp, st);
  if (esz_c == 2) return run_zrestrict_t<half_t, half_t>(mx, mb, a, grid, zp, st);
  return run_zrestrict_t<half_t, float>(mx, mb, a, grid, zp, st);
}

cudaError_t launch_zouter(const OuterArgs &a, int rhs_mode, int esz_e, double *err, int *nblocks_out,
                          cudaStream_t st) {
  if ((a.nx & 3) != 0 || ((size_t)a.nx * esz_e) % 16 != 0) return cudaErrorNotSupported;
  const int rows = OuterGeo::BH;
  CUtensorMap m[5];
  std::memset(m, 0, sizeof m);
  const float *rhs0 = rhs_mode == RHS_EXPLICIT ? a.b : a.I0;
  if (!make_map(&m[0], a.xh_in, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (a.xl_in && !make_map(&m[1], a.xl_in, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (a.e && !make_map(&m[2], a.e, a.nx, a.ny, a.nz, box_w(esz_e), rows, esz_e)) return cudaErrorNotSupported;
  if (!make_map(&m[3], rhs0, a.nx, a.ny, a.nz, BOXW, rows)) return cudaErrorNotSupported;
  if (rhs_mode == RHS_SP && !make_map(&m[4], a.I1, a.nx, a.ny, a.nz, ZX, OuterGeo::OY))
    return cudaErrorNotSupported;
  if (((uintptr_t)a.xh_out & 15) || ((uintptr_t)a.xl_out & 15) || ((uintptr_t)a.r_out & 15))
    return cudaErrorNotSupported;
  const int gx = (a.nx + ZX - 1) / ZX, gy = (a.ny + OuterGeo::OY - 1) / OuterGeo::OY;
  dim3 grid(gx, gy, 1);
  if (esz_e == 2) return zouter_bf16(m, a, rhs_mode, err, grid, nblocks_out, st);
  return zouter_f32(m, a, rhs_mode, err, grid, nblocks_out, st);
}

int zouter_max_blocks(int nx, int ny, int nz) {
  const int gx = (nx + ZX - 1) / ZX, gy = (ny + OuterGeo::OY - 1) / OuterGeo::OY;
  return gx * gy * nz;
}

// Runs k_wait_selftest (one CTA) and returns 1 if its wait gave up, 0 if it
// completed, or -1 on a CUDA error.
int zmarch_wait_selftest(unsigned limit, cudaStream_t st) {
  int *d = nullptr;
  if (cudaMalloc((void **)&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  int h = -1;
  cudaMemsetAsync(d, 0xff, sizeof(int), st);
  k_wait_selftest<<<1, 32, 0, st>>>(limit, d);
  cudaError_t e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return -1;
  return h;
}
#endif  // GD_ZM_PART(0)
