// gd_hybrid.cu -- the "Hybrid" discretisation of Sec. 4.2: the 6-point
// operator at the finest level, first-order B-spline transfers ((1/2, 1, 1/2)
// along each halved axis) and Galerkin coarse operators P^T A P, which are
// 27-point stencils (Sec. 4.2, "Hybrid").
//
// Every level's operator keeps the Kronecker form of the fine one,
//   A = wx Kx (x) My (x) Mz + wy Mx (x) Ky (x) Mz + wz Mx (x) My (x) Kz + wm Mx (x) My (x) Mz,
// with per-axis tridiagonal factors (K_d, M_d): at the fine level K_d is the
// 1D Neumann Laplacian and M_d = I; one level down along a halved axis they
// become P^T K_d P and P^T M_d P (the Galerkin product of a Kronecker
// operator is the Kronecker product of the per-axis Galerkin products).  The
// kernels rebuild the 27 coefficients of a cell from the three rows of its
// factors, so no stencil is stored.
//
// Relaxation on the 27-point levels is Gauss-Seidel with eight colours (the
// parities of i, j and k; same-colour cells are never neighbours), the four
// in-plane colours of a plane fused in one z-march launch (k_h_gsf).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "gd_internal.h"

namespace {

constexpr int HNT = 256;

// 4-byte asynchronous copy; ok = false writes 0 (no global access)
__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Tiles and boxes of the 27-point residual's z-march: a CTA owns a
// GZ_TX x GZ_TY column tile; a plane's box is the tile, one row above and
// below and four columns left and right (a 16-byte aligned start).
constexpr int GZ_TX = 64, GZ_TY = 16, GZ_NT = 256;
constexpr int GZ_BW = GZ_TX + 8, GZ_BH = GZ_TY + 2;  // box: columns i0-4 .., rows j0-1 ..
constexpr int GZ_BC = GZ_BW * GZ_BH;
constexpr int GZ_MAX_CHUNKS = 64;

__device__ __forceinline__ void cp_async16z(float *dst, const float *src, bool ok) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(ok ? 16 : 0)
               : "memory");
}

// One Gauss-Seidel sweep of a 27-point level with the in-plane colours
// fused, out of place.  The eight colours (parities of i, j, k) run in the
// order (i, j) = (0,0), (1,0), (0,1), (1,1) on the even planes, then the same
// on the odd planes: on a coupled level, launch pz = 0 reads every plane
// from xin and writes the even planes to xout, then launch pz = 1 reads the
// odd planes from xin and their even neighbours from xout and writes the odd
// planes to xout; an uncoupled level takes the four colours on every plane
// in one launch.  A CTA owns an FS_TX x FS_TY tile of a plane and relaxes colour c
// (c = px + 2 py) on the tile and a ring of 3 - c cells around it in shared
// memory, in place: colour c + 1 on a ring one narrower reads exactly the
// colour-c values it needs.  Ring cells are computed from the same values,
// with the same arithmetic, as by the CTA that owns them, so the result does
// not depend on the tiling; only tile cells are written.  The CTA marches z
// with the planes in a shared-memory ring (cp.async, a step ahead).
constexpr int FS_TX = 64, FS_TY = 32, FS_NT = 256;
constexpr int FS_R = 4;                                    // box margin (ring 3 + its neighbours)
constexpr int FS_BW = FS_TX + 2 * FS_R, FS_BH = FS_TY + 2 * FS_R;
constexpr int FS_BC = FS_BW * FS_BH;
constexpr int FS_CPT = 3;  // colour cells per thread and colour (<= (64 + 6)(32 + 6) / 4 / 256)
static_assert(((FS_TX + 6) / 2) * ((FS_TY + 6) / 2) <= FS_CPT * FS_NT, "colour cells per thread");
__host__ __device__ constexpr size_t gsf_smem(bool zc) { return (zc ? 5 : 2) * (size_t)FS_BC * sizeof(float); }

template <bool ZC>
__global__ void __launch_bounds__(FS_NT, 3) k_h_gsf(HLevelDev L, int pz, int zchunk, int vec,
                                                   const float *__restrict__ xc, const float *xn,
                                                   const float *__restrict__ b, float *xout) {
  extern __shared__ __align__(16) float fsm[];
  float *cur = fsm;                // two slots: the updated planes k, k + 2 (or k, k + 1)
  float *nbs = fsm + 2 * FS_BC;    // three slots: neighbour planes (coupled levels)
  // factor rows of the box's columns and rows ([K|M][tap][column / row]),
  // taps that leave the domain set to 0 (boundary cells' coefficients)
  __shared__ float fx[2][3][FS_BW], fy[2][3][FS_BH];
  const int tid = threadIdx.x;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i0 = blockIdx.x * FS_TX, j0 = blockIdx.y * FS_TY;
  for (int q = tid; q < 3 * FS_BW; q += FS_NT) {
    const int c = q % FS_BW, t = q / FS_BW, gi = i0 - FS_R + c, nb = gi + t - 1;
    const bool ok = gi >= 0 && gi < nx && nb >= 0 && nb < nx;
    fx[0][t][c] = ok ? L.kx[3 * gi + t] : 0.f;
    fx[1][t][c] = ok ? L.mx[3 * gi + t] : 0.f;
  }
  for (int q = tid; q < 3 * FS_BH; q += FS_NT) {
    const int c = q % FS_BH, t = q / FS_BH, gj = j0 - FS_R + c, nb = gj + t - 1;
    const bool ok = gj >= 0 && gj < ny && nb >= 0 && nb < ny;
    fy[0][t][c] = ok ? L.ky[3 * gj + t] : 0.f;
    fy[1][t][c] = ok ? L.my[3 * gj + t] : 0.f;
  }
  // (the first step's barrier orders these writes before their use)
  const int zs = blockIdx.z * zchunk, ze = min(zs + zchunk, nz);
  const size_t plane = (size_t)nx * ny;
  const int kstep = ZC ? 2 : 1;
  const int k0 = ZC ? zs + ((zs & 1) != pz ? 1 : 0) : zs;

  auto load_box = [&](float *dst, const float *src, int p) {
    const bool pin = p >= 0 && p < nz;
    if (vec) {
      for (int q = tid; q < FS_BC / 4; q += FS_NT) {
        const int c4 = q % (FS_BW / 4), rr = q / (FS_BW / 4);
        const int gi = i0 - FS_R + 4 * c4, gj = j0 - FS_R + rr;
        const bool ok = pin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        cp_async16z(dst + 4 * q, ok ? src + (size_t)p * plane + (size_t)gj * nx + gi : src, ok);
      }
    } else {
      for (int q = tid; q < FS_BC; q += FS_NT) {
        const int c = q % FS_BW, rr = q / FS_BW;
        const int gi = i0 - FS_R + c, gj = j0 - FS_R + rr;
        const bool ok = pin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        cp_async4(dst + q, ok ? src + (size_t)p * plane + (size_t)gj * nx + gi : src, ok);
      }
    }
  };
  auto cur_slot = [&](int k) { return cur + (((k - k0) / kstep) & 1) * FS_BC; };
  auto nb_slot = [&](int p) { return nbs + (((p - k0 + 1) >> 1) % 3) * FS_BC; };  // p = k0 - 1, k0 + 1, ...

  // colour c's cells on the tile and a ring of 3 - c: the m-th of this thread
  auto colour_cell = [&](int c, int m, int &ci, int &cj) -> bool {
    const int px = c & 1, py = c >> 1, d = 3 - c;
    int ia = max(i0 - d, 0), ja = max(j0 - d, 0);
    const int ib = min(i0 + FS_TX - 1 + d, nx - 1), jb = min(j0 + FS_TY - 1 + d, ny - 1);
    ia += (ia & 1) != px;
    ja += (ja & 1) != py;
    if (ia > ib || ja > jb) return false;
    const int ncx = (ib - ia) / 2 + 1, ncy = (jb - ja) / 2 + 1;
    const int q = tid + m * FS_NT;
    if (q >= ncx * ncy) return false;
    ci = ia + 2 * (q % ncx);
    cj = ja + 2 * (q / ncx);
    return true;
  };

  // this thread's colour cells are the same on every plane: their box
  // coordinates packed as bx | by << 8, bit 16 set when the cell's x and y
  // factor rows are the uniform interior rows, bit 17 when it lies in the
  // tile (-1: none), computed once
  int cell[4][FS_CPT];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int m = 0; m < FS_CPT; ++m) {
      int ci, cj;
      if (colour_cell(c, m, ci, cj)) {
        const bool xyint = ci >= L.ilo[0] && ci <= L.ihi[0] && cj >= L.ilo[1] && cj <= L.ihi[1];
        const bool tile = ci >= i0 && ci < i0 + FS_TX && cj >= j0 && cj < j0 + FS_TY;
        cell[c][m] = (ci - i0 + FS_R) | ((cj - j0 + FS_R) << 8) | (xyint ? 1 << 16 : 0) | (tile ? 1 << 17 : 0);
      } else {
        cell[c][m] = -1;
      }
    }
  if (ZC) {
    load_box(cur_slot(k0), xc, k0);
    load_box(nb_slot(k0 - 1), xn, k0 - 1);
    load_box(nb_slot(k0 + 1), xn, k0 + 1);
  } else {
    load_box(cur_slot(k0), xc, k0);
  }
  cp_async_commit();
  for (int k = k0; k < ze; k += kstep) {
    // the right-hand side of this step's cells (all four colours)
    float bq[4][FS_CPT];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int m = 0; m < FS_CPT; ++m) {
        const int pk = cell[c][m];
        bq[c][m] = pk >= 0 ? b[(size_t)k * plane + (size_t)(j0 - FS_R + ((pk >> 8) & 255)) * nx + (i0 - FS_R + (pk & 255))]
                           : 0.f;
      }
    cp_async_wait0();
    __syncthreads();  // this step's planes have landed; every thread is past the previous step
    if (k + kstep < ze) {
      load_box(cur_slot(k + kstep), xc, k + kstep);
      if (ZC) load_box(nb_slot(k + 3), xn, k + 3);
    }
    cp_async_commit();
    float *pc = cur_slot(k);
    const float *pm = ZC ? nb_slot(k - 1) : pc, *pp = ZC ? nb_slot(k + 1) : pc;
    // per-plane z factors (general path)
    float Z1[3] = {0.f, 0.f, 0.f}, MZ[3] = {0.f, 0.f, 0.f};
    {
      const float *kz = L.kz + 3 * k, *mz = L.mz + 3 * k;
      if (ZC) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (k + c - 1 >= 0 && k + c - 1 < nz) {
            MZ[c] = mz[c];
            Z1[c] = L.wz * kz[c] + L.wm * mz[c];
          }
      } else {
        MZ[1] = mz[1];
        Z1[1] = L.wm * mz[1];
      }
    }
    const bool zint = !ZC || (k >= L.ilo[2] && k <= L.ihi[2]);
    const float idg_int = 1.f / L.cst[13];  // interior cells' diagonal, inverted once
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int m = 0; m < FS_CPT; ++m) {
        const int pk = cell[c][m];
        if (pk < 0) continue;
        const int bx = pk & 255, by = (pk >> 8) & 255;
        const int ci = i0 - FS_R + bx, cj = j0 - FS_R + by;
        const int o = by * FS_BW + bx;
        // columns bx - 1 .. bx + 1 of a row as two aligned float2 loads; bx
        // has the colour's x parity (i0 and FS_R are even), known here
        const int o2 = (by - 1) * FS_BW + ((bx - 1) & ~1);
        const bool odd = (c & 1) != 0;
        auto row3 = [&](const float *pl, int bb, float &v0, float &v1, float &v2) {
          const float2 lo = *reinterpret_cast<const float2 *>(pl + o2 + bb * FS_BW);
          const float2 hi = *reinterpret_cast<const float2 *>(pl + o2 + bb * FS_BW + 2);
          v0 = odd ? lo.x : lo.y;
          v1 = odd ? lo.y : hi.x;
          v2 = odd ? hi.x : hi.y;
        };
        float ax = 0.f, dg;
        if (zint && (pk & (1 << 16))) {
          float az[3] = {0.f, 0.f, 0.f};  // one chain per plane
#pragma unroll
          for (int zc = 0; zc < 3; ++zc) {
            if (!ZC && zc != 1) continue;
            const float *pl = zc == 0 ? pm : (zc == 1 ? pc : pp);
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              float v0, v1, v2;
              row3(pl, bb, v0, v1, v2);
              const float *cs = L.cst + zc * 9 + bb * 3;
              az[zc] = fmaf(cs[0], v0, fmaf(cs[1], v1, fmaf(cs[2], v2, az[zc])));
            }
          }
          ax = (az[0] + az[2]) + az[1];
          dg = 0.f;  // interior: the reciprocal of the constant diagonal below
        } else {
          // cf(a, b, c) = mx(a) P(b, c) + kx(a) Q(b, c), P = my(b) Z1(c) +
          // wy ky(b) MZ(c), Q = wx my(b) MZ(c) (the per-axis factoring; taps
          // leaving the domain are 0 in the tables)
          const float kx0 = fx[0][0][bx], kx1 = fx[0][1][bx], kx2 = fx[0][2][bx];
          const float mx0 = fx[1][0][bx], mx1 = fx[1][1][bx], mx2 = fx[1][2][bx];
          float dgp = 0.f, dgq = 0.f;
#pragma unroll
          for (int zc = 0; zc < 3; ++zc) {
            if (!ZC && zc != 1) continue;
            const float *pl = zc == 0 ? pm : (zc == 1 ? pc : pp);
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              const float myb = fy[1][bb][by], kyb = fy[0][bb][by];
              const float P = myb * Z1[zc] + L.wy * kyb * MZ[zc], Q = L.wx * myb * MZ[zc];
              if (zc == 1 && bb == 1) {
                dgp = P;
                dgq = Q;
              }
              float v0, v1, v2;
              row3(pl, bb, v0, v1, v2);
              ax = fmaf(fmaf(mx0, P, kx0 * Q), v0, ax);
              ax = fmaf(fmaf(mx1, P, kx1 * Q), v1, ax);
              ax = fmaf(fmaf(mx2, P, kx2 * Q), v2, ax);
            }
          }
          dg = fmaf(mx1, dgp, kx1 * dgq);
        }
        const float v = dg == 0.f ? pc[o] + (bq[c][m] - ax) * idg_int : pc[o] + (bq[c][m] - ax) / dg;
        pc[o] = v;
        if (pk & (1 << 17)) xout[(size_t)k * plane + (size_t)cj * nx + ci] = v;
      }
      if (c < 3) __syncthreads();
    }
  }
  cp_async_wait0();
}

// r = b - A x as a z-march (SIX: the fine 6-point operator of the Hybrid
// discretisation with Neumann neighbour counts; else the level's 27-point
// Kronecker operator).  Same tiles and boxes as the colour sweep, an
// eight-plane ring with copies two planes ahead; a thread owns four
// consecutive cells of one row.  Tiles whose cells all have the uniform
// interior factor rows use the level's 27 interior coefficients; the others
// form each cell's coefficients from its factor rows (the same per-axis
// factoring as the sweep, taps leaving the domain set to 0).
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

// RZ (coupled levels halved along z only): instead of r, the coarse
// right-hand side bc = P^T r of the B-spline transfer, accumulated per column
// in registers (coarse plane K takes 1/2 r(2K - 1) + r(2K) + 1/2 r(2K + 1),
// the last odd fine plane all of its residual when K + 1 does not exist);
// chunks are even, each also evaluates the plane before it for that plane's
// half, and the chunk holding fine plane 2K stores coarse plane K.
template <bool ZC, bool SIX, bool RZ = false>
__global__ void __launch_bounds__(GZ_NT, 3) k_h_residz(HLevelDev L, int zchunk, int vec, int vec_br,
                                                      const float *__restrict__ x, const float *__restrict__ b,
                                                      float *__restrict__ r, float *__restrict__ bc = nullptr,
                                                      int ncz = 0) {
  constexpr int NS = 8;
  __shared__ __align__(16) float ring[NS][GZ_BC];
  // factor rows of the box's columns and rows ([K|M][tap][column / row]),
  // taps that leave the domain set to 0 (boundary cells' coefficients)
  __shared__ float fx[2][3][GZ_BW], fy[2][3][GZ_BH];
  const int tid = threadIdx.x;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i0 = blockIdx.x * GZ_TX, j0 = blockIdx.y * GZ_TY;
  const int zs = blockIdx.z * zchunk, ze = min(zs + zchunk, nz);
  const size_t plane = (size_t)nx * ny;
  if (!SIX) {
    for (int q = tid; q < 3 * GZ_BW; q += GZ_NT) {
      const int c = q % GZ_BW, t = q / GZ_BW, gi = i0 - 4 + c, nb = gi + t - 1;
      const bool ok = gi >= 0 && gi < nx && nb >= 0 && nb < nx;
      fx[0][t][c] = ok ? L.kx[3 * gi + t] : 0.f;
      fx[1][t][c] = ok ? L.mx[3 * gi + t] : 0.f;
    }
    for (int q = tid; q < 3 * GZ_BH; q += GZ_NT) {
      const int c = q % GZ_BH, t = q / GZ_BH, gj = j0 - 1 + c, nb = gj + t - 1;
      const bool ok = gj >= 0 && gj < ny && nb >= 0 && nb < ny;
      fy[0][t][c] = ok ? L.ky[3 * gj + t] : 0.f;
      fy[1][t][c] = ok ? L.my[3 * gj + t] : 0.f;
    }
    // (the first step's barrier orders these writes before their use)
  }
  auto load_plane = [&](int p) {
    float *dst = ring[(p + NS) & (NS - 1)];
    const bool pin = p >= 0 && p < nz;
    if (vec) {
      for (int q = tid; q < GZ_BC / 4; q += GZ_NT) {
        const int c4 = q % (GZ_BW / 4), rr = q / (GZ_BW / 4);
        const int gi = i0 - 4 + 4 * c4, gj = j0 - 1 + rr;
        const bool ok = pin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        cp_async16z(dst + 4 * q, ok ? x + (size_t)p * plane + (size_t)gj * nx + gi : x, ok);
      }
    } else {
      for (int q = tid; q < GZ_BC; q += GZ_NT) {
        const int c = q % GZ_BW, rr = q / GZ_BW;
        const int gi = i0 - 4 + c, gj = j0 - 1 + rr;
        const bool ok = pin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
        cp_async4(dst + q, ok ? x + (size_t)p * plane + (size_t)gj * nx + gi : x, ok);
      }
    }
    cp_async_commit();
  };
  const int l = tid & 15, ty = tid >> 4;
  const int gi0 = i0 + 4 * l, gj = j0 + ty;
  const bool row_in = gj < ny && gi0 < nx;
  // all four cells interior in x and y (z is checked per plane)
  const bool xy_int = gi0 >= L.ilo[0] && gi0 + 3 <= L.ihi[0] && gj >= L.ilo[1] && gj <= L.ihi[1];
  const int cb = 4 * l;  // box column of the float4 left of the cells

  // the first plane evaluated (RZ: the one before the chunk, for its half)
  const int ks = (RZ && zs > 0) ? zs - 1 : zs;
  // one copy group per plane, two planes ahead of the step that reads them
  if (ZC) {
    load_plane(ks - 1);
    load_plane(ks);
    load_plane(ks + 1);
    load_plane(ks + 2);
  } else {
    load_plane(ks);
    load_plane(ks + 1);
  }
  float carry[4] = {0.f, 0.f, 0.f, 0.f};  // RZ: the half of r(2K - 1) owed to coarse plane K
  // b of this thread's cells, loaded a step ahead of its use
  const size_t orow = (size_t)gj * nx + gi0;
  auto load_b = [&](int k, float *bv) {
    if (!row_in || k >= ze) return;
    const float *bp = b + (size_t)k * plane + orow;
    if (vec_br) {
      const float4 t = *reinterpret_cast<const float4 *>(bp);
      bv[0] = t.x;
      bv[1] = t.y;
      bv[2] = t.z;
      bv[3] = t.w;
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) bv[m] = gi0 + m < nx ? bp[m] : 0.f;
    }
  };
  float bn[4] = {0.f, 0.f, 0.f, 0.f};
  load_b(ks, bn);
  for (int k = ks; k < ze; ++k) {
    float bk[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) bk[m] = bn[m];
    load_b(k + 1, bn);
    load_plane(ZC ? k + 3 : k + 2);
    cp_async_wait2();  // all but the last two issued planes have landed: k + 1 (ZC) / k
    __syncthreads();
    if (row_in) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const bool fast = !SIX && xy_int && (!ZC || (k >= L.ilo[2] && k <= L.ihi[2]));
      float Z1[3] = {0.f, 0.f, 0.f}, MZ[3] = {0.f, 0.f, 0.f};
      if (!SIX && !fast) {
        const float *kz = L.kz + 3 * k, *mz = L.mz + 3 * k;
        if (ZC) {
#pragma unroll
          for (int c = 0; c < 3; ++c)
            if (k + c - 1 >= 0 && k + c - 1 < nz) {
              MZ[c] = mz[c];
              Z1[c] = L.wz * kz[c] + L.wm * mz[c];
            }
        } else {
          MZ[1] = mz[1];
          Z1[1] = L.wm * mz[1];
        }
      }
      float xo[4] = {0.f, 0.f, 0.f, 0.f};  // the cells' own values
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (!ZC && c != 1) continue;
        const float *pl = ring[(k + c - 1 + NS) & (NS - 1)];
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          if (SIX && c != 1 && bb != 1) continue;
          const int ro = (ty + bb) * GZ_BW + cb;  // box row of gj + bb - 1
          const float4 lf = *reinterpret_cast<const float4 *>(pl + ro);
          const float4 md = *reinterpret_cast<const float4 *>(pl + ro + 4);
          const float4 rt = *reinterpret_cast<const float4 *>(pl + ro + 8);
          const float v[6] = {lf.w, md.x, md.y, md.z, md.w, rt.x};
          if (c == 1 && bb == 1) {
            xo[0] = md.x;
            xo[1] = md.y;
            xo[2] = md.z;
            xo[3] = md.w;
          }
          if (SIX) {
            // neighbour sums only; the diagonal is applied below
            if (c == 1 && bb == 1) {
#pragma unroll
              for (int m = 0; m < 4; ++m) acc[m] += L.wx * (v[m] + v[m + 2]);
            } else if (c == 1) {
#pragma unroll
              for (int m = 0; m < 4; ++m) acc[m] += L.wy * v[m + 1];
            } else {
#pragma unroll
              for (int m = 0; m < 4; ++m) acc[m] += L.wz * v[m + 1];
            }
          } else if (fast) {
            const float *cs = L.cst + c * 9 + bb * 3;
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[m] = fmaf(cs[0], v[m], fmaf(cs[1], v[m + 1], fmaf(cs[2], v[m + 2], acc[m])));
          } else {
            // cf(a, bb, c) = mx(a) P + kx(a) Q with the row's P, Q below (the
            // per-axis factoring; taps leaving the domain are 0 in the tables)
            const float myb = fy[1][bb][ty + 1], kyb = fy[0][bb][ty + 1];
            const float P = myb * Z1[c] + L.wy * kyb * MZ[c], Q = L.wx * myb * MZ[c];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int col = cb + 4 + m;  // box column of cell m
#pragma unroll
              for (int aa = 0; aa < 3; ++aa)
                acc[m] = fmaf(fmaf(fx[1][aa][col], P, fx[0][aa][col] * Q), v[m + aa], acc[m]);
            }
          }
        }
      }
      const size_t o = (size_t)k * plane + (size_t)gj * nx + gi0;
      if (SIX) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int gi = gi0 + m;
          float cnt = L.wm;
          cnt += L.wx * (float)((gi > 0) + (gi < nx - 1));
          cnt += L.wy * (float)((gj > 0) + (gj < ny - 1));
          if (ZC) cnt += L.wz * (float)((k > 0) + (k < nz - 1));
          acc[m] = cnt * xo[m] - acc[m];
        }
      }
      if (RZ) {
        float rv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rv[m] = bk[m] - acc[m];
        bool store = false;
        int K = 0;
        float cv[4];
        if ((k & 1) == 0) {
          // even fine plane 2K: its whole residual, plus the half carried
          K = k >> 1;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            cv[m] = carry[m] + rv[m];
            carry[m] = cv[m];  // (completed by the next, odd, plane)
          }
          store = k == nz - 1;  // no plane 2K + 1: coarse plane K is complete
        } else {
          // odd fine plane 2K + 1: half to K (all of it when K + 1 does not
          // exist), half carried to K + 1
          K = (k - 1) >> 1;
          const bool last = ((k + 1) >> 1) >= ncz;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            const float h = last ? rv[m] : 0.5f * rv[m];
            cv[m] = carry[m] + h;
            carry[m] = last ? 0.f : 0.5f * rv[m];
          }
          store = 2 * K >= zs;  // plane 2K in this chunk (not the one before it)
        }
        if (store) {
          const size_t oc = (size_t)K * plane + orow;
          if (vec_br) {  // (vec_br covers bc here)
            *reinterpret_cast<float4 *>(bc + oc) = make_float4(cv[0], cv[1], cv[2], cv[3]);
          } else {
#pragma unroll
            for (int m = 0; m < 4; ++m)
              if (gi0 + m < nx) bc[oc + m] = cv[m];
          }
        }
      } else if (vec_br) {  // nx % 4 == 0 and 16-byte aligned b, r: the four cells are one float4
        *reinterpret_cast<float4 *>(r + o) = make_float4(bk[0] - acc[0], bk[1] - acc[1], bk[2] - acc[2], bk[3] - acc[3]);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m)
          if (gi0 + m < nx) r[o + m] = bk[m] - acc[m];
      }
    }
  }
  cp_async_wait0();
}

// Fine cells of coarse cell I along one axis, with the weights of
// P (first-order B-spline, vertex-centred): fine 2I has weight 1, fine 2I-1
// and 2I+1 weight 1/2, except a fine cell with a single parent (the last
// cell of an even extent), which has weight 1.  An axis that is not halved
// maps I to I with weight 1.
__device__ __forceinline__ int children(int I, int nf, int nc, int f, int *idx, float *w) {
  if (!f) {
    idx[0] = I;
    w[0] = 1.f;
    return 1;
  }
  int m = 0;
  const int c = 2 * I;
  idx[m] = c;
  w[m++] = 1.f;
  if (c - 1 >= 0) {
    idx[m] = c - 1;
    w[m++] = 0.5f;  // fine c-1 lies between coarse I-1 and I
  }
  if (c + 1 < nf) {
    idx[m] = c + 1;
    w[m++] = (I + 1 < nc) ? 0.5f : 1.f;
  }
  return m;
}

// Coarse right-hand side bc = P^T r (P = Px (x) Py (x) Pz).
__global__ void __launch_bounds__(HNT) k_h_restrict(int nx, int ny, int nz, int fx, int fy, int fz, int cnx,
                                                    int cny, int cnz, const float *__restrict__ r,
                                                    float *__restrict__ bc) {
  const long long n = (long long)cnx * cny * cnz;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int I = (int)(q % cnx);
    const long long t = q / cnx;
    const int J = (int)(t % cny), K = (int)(t / cny);
    int ix[3], iy[3], iz[3];
    float wx[3], wy[3], wz[3];
    const int mx = children(I, nx, cnx, fx, ix, wx);
    const int my = children(J, ny, cny, fy, iy, wy);
    const int mz = children(K, nz, cnz, fz, iz, wz);
    float s = 0.f;
    for (int c = 0; c < mz; ++c)
      for (int b = 0; b < my; ++b) {
        const float *rr = r + ((long long)iz[c] * ny + iy[b]) * nx;
        const float wyz = wy[b] * wz[c];
        for (int a = 0; a < mx; ++a) s = fmaf(wx[a] * wyz, rr[ix[a]], s);
      }
    bc[q] = s;
  }
}

// Parents of fine cell i along one axis with their weights (rows of P).
__device__ __forceinline__ int parents(int i, int nc, int f, int *idx, float *w) {
  if (!f) {
    idx[0] = i;
    w[0] = 1.f;
    return 1;
  }
  if ((i & 1) == 0) {
    idx[0] = i >> 1;
    w[0] = 1.f;
    return 1;
  }
  const int I = i >> 1;
  if (I + 1 < nc) {
    idx[0] = I;
    idx[1] = I + 1;
    w[0] = w[1] = 0.5f;
    return 2;
  }
  idx[0] = I;
  w[0] = 1.f;
  return 1;
}

// x += P e (the coarse correction, first-order B-spline prolongation).
__global__ void __launch_bounds__(HNT) k_h_prolong(int nx, int ny, int nz, int fx, int fy, int fz, int cnx,
                                                   int cny, int cnz, const float *__restrict__ e,
                                                   float *__restrict__ x) {
  const long long n = (long long)nx * ny * nz;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int i = (int)(q % nx);
    const long long t = q / nx;
    const int j = (int)(t % ny), k = (int)(t / ny);
    int ix[2], iy[2], iz[2];
    float wx[2], wy[2], wz[2];
    const int mx = parents(i, cnx, fx, ix, wx);
    const int my = parents(j, cny, fy, iy, wy);
    const int mz = parents(k, cnz, fz, iz, wz);
    float s = 0.f;
    for (int c = 0; c < mz; ++c)
      for (int b = 0; b < my; ++b) {
        const float *er = e + ((long long)iz[c] * cny + iy[b]) * cnx;
        const float wyz = wy[b] * wz[c];
        for (int a = 0; a < mx; ++a) s = fmaf(wx[a] * wyz, er[ix[a]], s);
      }
    x[q] += s;
  }
}

int grid_of(long long n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const long long g = (n + HNT - 1) / HNT;
  return (int)(g < (long long)sms * 8 ? (g > 0 ? g : 1) : (long long)sms * 8);
}

}  // namespace

namespace {
// z chunks of a residual launch: as for the other z-march kernels, the
// chunk count minimises ceil(CTAs / resident slots) x (chunk + the planes
// loaded beyond it)
template <typename K>
int resid_chunk(K kernel, int slot_idx, long tiles, int nz, int h) {
  static int slots_cache[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int &slots = slots_cache[slot_idx];
  if (!slots) {
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, GZ_NT, 0) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    slots = occ * (sms > 0 ? sms : 1);
  }
  long best = -1;
  int zc = nz;
  for (int c = 1; c <= std::min(nz, GZ_MAX_CHUNKS); ++c) {
    const int q = (nz + c - 1) / c;
    const long gz = (nz + q - 1) / q;
    const long cost = ((tiles * gz + slots - 1) / slots) * (q + h);
    if (best < 0 || cost < best) {
      best = cost;
      zc = q;
    }
  }
  return zc;
}
}  // namespace


namespace {
// resident CTAs of a kernel with dynamic shared memory, then the z chunks
// as for the other z-march kernels
template <typename K>
int plan_chunk_dyn(K kernel, int threads, size_t smem, int &slots, long tiles, int nz, int h) {
  if (!slots) {
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    slots = occ * (sms > 0 ? sms : 1);
  }
  long best = -1;
  int zc = nz;
  for (int c = 1; c <= std::min(nz, GZ_MAX_CHUNKS); ++c) {
    const int q = (nz + c - 1) / c;
    const long gz = (nz + q - 1) / q;
    const long cost = ((tiles * gz + slots - 1) / slots) * (q + h);
    if (best < 0 || cost < best) {
      best = cost;
      zc = q;
    }
  }
  return zc;
}
template <bool ZC>
cudaError_t run_gsf(const HLevelDev &L, const float *x, float *xout, const float *b, cudaStream_t st) {
  static bool attr = false;
  static int slots = 0;
  const size_t smem = gsf_smem(ZC);
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_h_gsf<ZC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int gx = (L.nx + FS_TX - 1) / FS_TX, gy = (L.ny + FS_TY - 1) / FS_TY;
  const int vec = ((L.nx & 3) == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)xout & 15) == 0) ? 1 : 0;
  const int chunk = plan_chunk_dyn(k_h_gsf<ZC>, FS_NT, smem, slots, (long)gx * gy, L.nz, ZC ? 3 : 1);
  const dim3 grid(gx, gy, (L.nz + chunk - 1) / chunk);
  if (ZC) {
    // even planes' colours from x into xout, then the odd planes' with their
    // (updated) even neighbours from xout
    k_h_gsf<true><<<grid, FS_NT, smem, st>>>(L, 0, chunk, vec, x, x, b, xout);
    k_h_gsf<true><<<grid, FS_NT, smem, st>>>(L, 1, chunk, vec, x, xout, b, xout);
  } else {
    k_h_gsf<false><<<grid, FS_NT, smem, st>>>(L, 0, chunk, vec, x, x, b, xout);
  }
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_h_gsf(const HLevelDev &L, const float *x, float *xout, const float *b, cudaStream_t st) {
  if (L.wz != 0.f && L.nz > 1) return run_gsf<true>(L, x, xout, b, st);
  return run_gsf<false>(L, x, xout, b, st);
}

int h_gsf_launches(const HLevelDev &L) { return (L.wz != 0.f && L.nz > 1) ? 2 : 1; }

cudaError_t launch_h_resid(const HLevelDev &L, bool six, const float *x, const float *b, float *r,
                           cudaStream_t st) {
  const bool zc = L.wz != 0.f && L.nz > 1;
  const int gx = (L.nx + GZ_TX - 1) / GZ_TX, gy = (L.ny + GZ_TY - 1) / GZ_TY;
  const long tiles = (long)gx * gy;
  const bool nx4 = (L.nx & 3) == 0;
  const int vec = (nx4 && ((uintptr_t)x & 15) == 0) ? 1 : 0;
  const int vec_br = (nx4 && ((uintptr_t)b & 15) == 0 && ((uintptr_t)r & 15) == 0) ? 1 : 0;
  int chunk;
#define GD_RZ(Z, S, I)                                                                    \
  chunk = resid_chunk(k_h_residz<Z, S>, I, tiles, L.nz, Z ? 3 : 1);                          \
  k_h_residz<Z, S><<<dim3(gx, gy, (L.nz + chunk - 1) / chunk), GZ_NT, 0, st>>>(L, chunk, vec, vec_br, x, b, r);
  if (six) {
    if (zc) {
      GD_RZ(true, true, 2)
    } else {
      GD_RZ(false, true, 3)
    }
  } else {
    if (zc) {
      GD_RZ(true, false, 4)
    } else {
      GD_RZ(false, false, 5)
    }
  }
#undef GD_RZ
  return cudaGetLastError();
}

cudaError_t launch_h_resid_rz(const HLevelDev &L, bool six, const float *x, const float *b, float *bc, int ncz,
                              cudaStream_t st) {
  const int gx = (L.nx + GZ_TX - 1) / GZ_TX, gy = (L.ny + GZ_TY - 1) / GZ_TY;
  const long tiles = (long)gx * gy;
  const bool nx4 = (L.nx & 3) == 0;
  const int vec = (nx4 && ((uintptr_t)x & 15) == 0) ? 1 : 0;
  const int vec_bc = (nx4 && ((uintptr_t)b & 15) == 0 && ((uintptr_t)bc & 15) == 0) ? 1 : 0;
  int chunk;
#define GD_RZZ(S, I)                                                                                   \
  chunk = resid_chunk(k_h_residz<true, S, true>, I, tiles, L.nz, 3);                                    \
  chunk += chunk & 1; /* even: both fine planes 2K, 2K + 1 of a coarse plane in one chunk */          \
  k_h_residz<true, S, true><<<dim3(gx, gy, (L.nz + chunk - 1) / chunk), GZ_NT, 0, st>>>(                \
      L, chunk, vec, vec_bc, x, b, nullptr, bc, ncz);
  if (six) {
    GD_RZZ(true, 6)
  } else {
    GD_RZZ(false, 7)
  }
#undef GD_RZZ
  return cudaGetLastError();
}

cudaError_t launch_h_restrict(int nx, int ny, int nz, int fx, int fy, int fz, int cnx, int cny, int cnz,
                              const float *r, float *bc, cudaStream_t st) {
  k_h_restrict<<<grid_of((long long)cnx * cny * cnz), HNT, 0, st>>>(nx, ny, nz, fx, fy, fz, cnx, cny, cnz, r,
                                                                    bc);
  return cudaGetLastError();
}

cudaError_t launch_h_prolong(int nx, int ny, int nz, int fx, int fy, int fz, int cnx, int cny, int cnz,
                             const float *e, float *x, cudaStream_t st) {
  k_h_prolong<<<grid_of((long long)nx * ny * nz), HNT, 0, st>>>(nx, ny, nz, fx, fy, fz, cnx, cny, cnz, e, x);
  return cudaGetLastError();
}

// ===========================================================================
// The "Linear" discretisation (Sec. 4.2): the same Kronecker form with the
// fine factors K_n and the P1 mass (1/6) tridiag(1, [2, 4, ..., 4, 2], 1), so
// the fine operator is 27-point too.  Its outer pass evaluates the
// right-hand side once and the residual of the float-pair iterate with
// compensated sums (the 27 coefficients nearly cancel on smooth data; plain
// FP32 sums would lose ~1e-5 of the right-hand side, and FP64 is slow here).
// ===========================================================================
namespace {

__device__ __forceinline__ void block_sums(double a, double b, double *partials, int sa, int sb) {
  __shared__ double red[2][HNT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < HNT / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    if (sa >= 0) partials[(size_t)blockIdx.x * S_NUM + sa] = s0;
    if (sb >= 0) partials[(size_t)blockIdx.x * S_NUM + sb] = s1;
  }
}

// Integer-weighted Kronecker sums, compensated, as a z-march.  With the fine
// factors scaled to integers (K_n as is, the P1 mass times 6), the four sums
//   S_kx = (Kx My Mz) x, S_ky = (Mx Ky Mz) x, S_kz = (Mx My Kz) x,
//   S_m = (Mx My Mz) x
// are separable: three-tap filters along z (Mz x, Kz x), then y (My, Ky),
// then x (Kx, Mx), with shared intermediates -- 27 taps per cell for all
// four instead of 4 x 27.  Every tap is a float pair times a small integer
// (TwoProd) added by TwoSum, so the sums come out exact to ~1e-12 of their
// terms (the 27 coefficients nearly cancel on smooth data; plain FP32 would
// lose ~1e-5 of the right-hand side), and the weighted combination is done
// in float-pair arithmetic too (GB300's FP64 rate is 1/64 of its FP32 rate).
//
// A CTA owns an LZ_TX x LZ_TY column tile and marches z over a chunk of
// planes.  cp.async brings each plane's box (the tile and a one-cell ring,
// zero outside the domain) into a ring of four planes (k - 1, k, k + 1 in
// use, k + 2 in flight); per plane the z, y and x stages each write shared
// memory, with a CTA barrier between them.
constexpr int LZ_TX = 32, LZ_TY = 16, LZ_NT = 256;
constexpr int LZ_BW = LZ_TX + 2, LZ_BH = LZ_TY + 2;  // box
constexpr int LZ_BC = LZ_BW * LZ_BH;                 // box cells
constexpr int LZ_YC = LZ_BW * LZ_TY;                 // y-stage cells
constexpr int LZ_NS = 4;                             // planes in the ring
constexpr int LZ_MAX_CHUNKS = 64;
enum { LZ_RESID = 0, LZ_RHS = 1 };

struct DF {
  float h, l;
};
// v += w S, the double w split as (wh, wl)
__device__ __forceinline__ void df_wadd(DF &v, float wh, float wl, DF S) {
  const float p = wh * S.h;
  const float e = fmaf(wh, S.h, -p) + fmaf(wh, S.l, wl * S.h);
  const float t = v.h + p;
  const float bb = t - v.h;
  const float err = (v.h - (t - bb)) + (p - bb);
  v.h = t;
  v.l += err + e;
}
// P0 x0 + P1 x1 + P2 x2 for float pairs x_t and weights whose products with
// any float are exact (the integer-scaled fine factors: 0, +-1, 2, 4): the
// high products added by two TwoSums, the low parts by one rounded sum
__device__ __forceinline__ DF df_tap3(float P0, float2 x0, float P1, float2 x1, float P2, float2 x2) {
  const float p0 = P0 * x0.x, p1 = P1 * x1.x, p2 = P2 * x2.x;
  float s1 = p0 + p1;
  float bb = s1 - p0;
  const float e1 = (p0 - (s1 - bb)) + (p1 - bb);
  const float s2 = s1 + p2;
  bb = s2 - s1;
  const float e2 = (s1 - (s2 - bb)) + (p2 - bb);
  return DF{s2, (e1 + e2) + fmaf(P0, x0.y, fmaf(P1, x1.y, P2 * x2.y))};
}

struct LzArgs {
  // RESID: a0 = h, a1 = l of the iterate; RHS: a0 = I0, a1 = I1 (no low words)
  const float *a0, *a1;
  const float *bh, *bl;  // RESID: the right-hand side pair
  float *r;              // RESID: r = b - A x (nullable)
  float *oh, *ol;        // RHS: the right-hand side pair
  double *partials;      // RESID: sums of r^2 and b^2 per block
  // weights split as float pairs (RESID: ax, ay, az, am; RHS: gx, gy, gm)
  float wh[4], wl[4];
  int zchunk;
  int want_kz, want_m;
};

template <bool ZC, int MODE>
__global__ void __launch_bounds__(LZ_NT, 2) k_lz(HLevelDev L, LzArgs a) {
  __shared__ __align__(16) float ring[LZ_NS][2][LZ_BC];  // per plane: a0, a1
  __shared__ __align__(16) float2 zst[2][LZ_BC];         // z stage: two float pairs
  __shared__ __align__(16) float2 yst[3][LZ_YC];         // y stage: three float pairs
  __shared__ float wx[2][3][LZ_BW], wy[2][3][LZ_BH];     // [K|M][tap][box column / row]
  __shared__ double red[2][LZ_NT / 32];
  const int tid = threadIdx.x;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const int i0 = blockIdx.x * LZ_TX, j0 = blockIdx.y * LZ_TY;
  const int zs0 = blockIdx.z * a.zchunk, ze = min(zs0 + a.zchunk, nz);
  const size_t plane = (size_t)nx * ny;
  const bool y3 = MODE == LZ_RESID ? a.want_kz != 0 : a.want_m != 0;  // third y / z sum in use

  // factor rows of the box's columns and rows, taps that leave the domain set to 0
  for (int q = tid; q < 3 * LZ_BW; q += LZ_NT) {
    const int c = q % LZ_BW, t = q / LZ_BW, gi = i0 - 1 + c, nb = gi + t - 1;
    const bool ok = gi >= 0 && gi < nx && nb >= 0 && nb < nx;
    wx[0][t][c] = ok ? L.kx[3 * gi + t] : 0.f;
    wx[1][t][c] = ok ? L.mx[3 * gi + t] : 0.f;
  }
  for (int q = tid; q < 3 * LZ_BH; q += LZ_NT) {
    const int c = q % LZ_BH, t = q / LZ_BH, gj = j0 - 1 + c, nb = gj + t - 1;
    const bool ok = gj >= 0 && gj < ny && nb >= 0 && nb < ny;
    wy[0][t][c] = ok ? L.ky[3 * gj + t] : 0.f;
    wy[1][t][c] = ok ? L.my[3 * gj + t] : 0.f;
  }
  // plane p of the box into its ring slot (zeros outside the domain)
  auto load_plane = [&](int p) {
    const int sl = p & (LZ_NS - 1);
    const bool pin = p >= 0 && p < nz;
    const bool second = MODE == LZ_RESID || a.want_m != 0;
    for (int q = tid; q < LZ_BC; q += LZ_NT) {
      const int gi = i0 - 1 + q % LZ_BW, gj = j0 - 1 + q / LZ_BW;
      const bool ok = pin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
      const size_t o = ok ? (size_t)p * plane + (size_t)gj * nx + gi : 0;
      cp_async4(&ring[sl][0][q], a.a0 + o, ok);
      cp_async4(&ring[sl][1][q], ok && second ? a.a1 + o : a.a0, ok && second);
    }
    cp_async_commit();
  };
  for (int p = ZC ? zs0 - 1 : zs0; p <= (ZC ? zs0 + 1 : zs0); ++p) load_plane(p);

  float srr = 0.f, sbb = 0.f;
  // the right-hand side pair of this thread's two x-stage cells, loaded a
  // step ahead of its use (RESID)
  constexpr int XQ = LZ_TX * LZ_TY / LZ_NT;
  static_assert(XQ * LZ_NT == LZ_TX * LZ_TY, "x-stage cells per thread");
  float bnh[XQ], bnl[XQ];
  auto load_b = [&](int k) {
#pragma unroll
    for (int u = 0; u < XQ; ++u) {
      const int q = tid + u * LZ_NT, gi = i0 + q % LZ_TX, gj = j0 + q / LZ_TX;
      bnh[u] = bnl[u] = 0.f;
      if (MODE == LZ_RESID && k < ze && gi < nx && gj < ny) {
        const size_t o = (size_t)k * plane + (size_t)gj * nx + gi;
        bnh[u] = a.bh[o];
        bnl[u] = a.bl[o];
      }
    }
  };
  load_b(zs0);
  for (int k = zs0; k < ze; ++k) {
    float bkh[XQ], bkl[XQ];
#pragma unroll
    for (int u = 0; u < XQ; ++u) {
      bkh[u] = bnh[u];
      bkl[u] = bnl[u];
    }
    load_b(k + 1);
    load_plane(ZC ? k + 2 : k + 1);
    cp_async_wait1();
    __syncthreads();
    // ---- z stage: Zm = Mz x and Zk = Kz x (RHS: Zm of a0 and of a1) ----
    const float mz1 = L.mz[3 * k + 1];
    float mz0 = 0.f, mz2 = 0.f, kz0 = 0.f, kz1 = 0.f, kz2 = 0.f;
    if (ZC) {
      kz1 = L.kz[3 * k + 1];
      if (k > 0) {
        mz0 = L.mz[3 * k];
        kz0 = L.kz[3 * k];
      }
      if (k < nz - 1) {
        mz2 = L.mz[3 * k + 2];
        kz2 = L.kz[3 * k + 2];
      }
    }
    const int sm = (k - 1) & (LZ_NS - 1), s0 = k & (LZ_NS - 1), sp = (k + 1) & (LZ_NS - 1);
    for (int q = tid; q < LZ_BC; q += LZ_NT) {
      DF zm = {0.f, 0.f}, z2 = {0.f, 0.f};
      if (MODE == LZ_RESID) {
        const float2 x0 = make_float2(ring[s0][0][q], ring[s0][1][q]);
        if (ZC) {
          const float2 xm = make_float2(ring[sm][0][q], ring[sm][1][q]);
          const float2 xp = make_float2(ring[sp][0][q], ring[sp][1][q]);
          zm = df_tap3(mz0, xm, mz1, x0, mz2, xp);
          if (y3) z2 = df_tap3(kz0, xm, kz1, x0, kz2, xp);
        } else {
          zm = DF{mz1 * x0.x, mz1 * x0.y};
        }
      } else {
        const float2 a0 = make_float2(ring[s0][0][q], 0.f), b0 = make_float2(ring[s0][1][q], 0.f);
        if (ZC) {
          zm = df_tap3(mz0, make_float2(ring[sm][0][q], 0.f), mz1, a0, mz2, make_float2(ring[sp][0][q], 0.f));
          if (y3) z2 = df_tap3(mz0, make_float2(ring[sm][1][q], 0.f), mz1, b0, mz2, make_float2(ring[sp][1][q], 0.f));
        } else {
          zm = DF{mz1 * a0.x, 0.f};
          if (y3) z2 = DF{mz1 * b0.x, 0.f};
        }
      }
      zst[0][q] = make_float2(zm.h, zm.l);
      zst[1][q] = make_float2(z2.h, z2.l);
    }
    __syncthreads();
    // ---- y stage: My Zm, Ky Zm and My Z2 ----
    for (int q = tid; q < LZ_YC; q += LZ_NT) {
      const int c = q % LZ_BW, by = q / LZ_BW + 1;
      const int o = by * LZ_BW + c;
      const float2 zu = zst[0][o - LZ_BW], zc0 = zst[0][o], zd = zst[0][o + LZ_BW];
      const DF ymm = df_tap3(wy[1][0][by], zu, wy[1][1][by], zc0, wy[1][2][by], zd);
      const DF ykm = df_tap3(wy[0][0][by], zu, wy[0][1][by], zc0, wy[0][2][by], zd);
      DF yz = {0.f, 0.f};
      if (y3) yz = df_tap3(wy[1][0][by], zst[1][o - LZ_BW], wy[1][1][by], zst[1][o], wy[1][2][by], zst[1][o + LZ_BW]);
      yst[0][q] = make_float2(ymm.h, ymm.l);
      yst[1][q] = make_float2(ykm.h, ykm.l);
      yst[2][q] = make_float2(yz.h, yz.l);
    }
    __syncthreads();
    // ---- x stage: Kx Ymm, Mx Ykm, Mx Y3 (and Mx Ymm), then the output ----
#pragma unroll
    for (int u = 0; u < XQ; ++u) {
      const int q = tid + u * LZ_NT;
      const int tx = q % LZ_TX, ty = q / LZ_TX, gi = i0 + tx, gj = j0 + ty;
      if (gi >= nx || gj >= ny) continue;
      const int bx = tx + 1, o0 = ty * LZ_BW + bx;
      const float kx0 = wx[0][0][bx], kx1 = wx[0][1][bx], kx2 = wx[0][2][bx];
      const float mx0 = wx[1][0][bx], mx1 = wx[1][1][bx], mx2 = wx[1][2][bx];
      const float2 m0 = yst[0][o0 - 1], m1 = yst[0][o0], m2 = yst[0][o0 + 1];
      const DF skx = df_tap3(kx0, m0, kx1, m1, kx2, m2);
      const DF sky = df_tap3(mx0, yst[1][o0 - 1], mx1, yst[1][o0], mx2, yst[1][o0 + 1]);
      DF s3 = {0.f, 0.f}, smm = {0.f, 0.f};
      if (y3) s3 = df_tap3(mx0, yst[2][o0 - 1], mx1, yst[2][o0], mx2, yst[2][o0 + 1]);
      if (MODE == LZ_RESID && a.want_m) smm = df_tap3(mx0, m0, mx1, m1, mx2, m2);
      DF v = {0.f, 0.f};
      df_wadd(v, a.wh[0], a.wl[0], skx);
      df_wadd(v, a.wh[1], a.wl[1], sky);
      const size_t o = (size_t)k * plane + (size_t)gj * nx + gi;
      if (MODE == LZ_RESID) {
        if (y3) df_wadd(v, a.wh[2], a.wl[2], s3);
        if (a.want_m) df_wadd(v, a.wh[3], a.wl[3], smm);
        // r = b - v in float-pair arithmetic, rounded once
        const float bhv = bkh[u], blv = bkl[u];
        const float t = bhv - v.h;
        const float bb = t - bhv;
        const float err = (bhv - (t - bb)) + (-v.h - bb);
        const float rv = t + (err + (blv - v.l));
        if (a.r) a.r[o] = rv;
        srr = fmaf(rv, rv, srr);
        const float bv = bhv + blv;
        sbb = fmaf(bv, bv, sbb);
      } else {
        if (y3) df_wadd(v, a.wh[2], a.wl[2], s3);
        const float sh = v.h + v.l;
        a.oh[o] = sh;
        a.ol[o] = v.l - (sh - v.h);
      }
    }
  }
  cp_async_wait0();  // the last plane's copies (past the chunk) land before exit
  if (MODE == LZ_RESID) {
    double dr = srr, db = sbb;
    for (int o = 16; o > 0; o >>= 1) {
      dr += __shfl_down_sync(0xffffffffu, dr, o);
      db += __shfl_down_sync(0xffffffffu, db, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = dr;
      red[1][tid >> 5] = db;
    }
    __syncthreads();
    if (tid == 0) {
      double s0 = 0.0, s1 = 0.0;
      for (int w = 0; w < LZ_NT / 32; ++w) {
        s0 += red[0][w];
        s1 += red[1][w];
      }
      const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      a.partials[blk * S_NUM + S_RR] = s0;
      a.partials[blk * S_NUM + S_BB] = s1;
    }
  }
}

// (h, l) += e in float-pair arithmetic (TwoSum, then renormalised: ~48 bits,
// against FP64's 53; GB300's narrow FP64 pipe would make this streaming pass
// several times slower than its bytes); block sums of the new iterate (slot
// S_X), accumulated per thread as a float pair
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__global__ void __launch_bounds__(HNT) k_l_update(long long n, const float *__restrict__ e, float *__restrict__ h,
                                                  float *__restrict__ l, double *__restrict__ partials) {
  float sxh = 0.f, sxl = 0.f;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    float s, t;
    two_sum(h[q], e[q], s, t);
    t += l[q];
    const float hv = s + t;
    const float lv = t - (hv - s);
    h[q] = hv;
    l[q] = lv;
    float u, err;
    two_sum(sxh, hv, u, err);
    sxh = u;
    sxl += err + lv;
  }
  block_sums((double)sxh + (double)sxl, 0.0, partials, S_X, -1);
}

// block sums of an array (slot)
__global__ void __launch_bounds__(HNT) k_l_sum(long long n, const float *__restrict__ a, double *__restrict__ partials,
                                               int slot) {
  double s = 0.0;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) s += a[q];
  block_sums(s, 0.0, partials, slot, -1);
}

// out = h + l + shift, rounded to float (the shift split as sh + sl)
__global__ void __launch_bounds__(HNT) k_l_final(long long n, const float *__restrict__ h, const float *__restrict__ l,
                                                 float sh, float sl, float *__restrict__ out) {
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    float s, e;
    two_sum(h[q], sh, s, e);
    out[q] = s + (e + (l[q] + sl));
  }
}

}  // namespace

int linear_grid(long long n) { return grid_of(n); }

namespace {
// z chunks of a k_lz launch: a launch lasts about ceil(CTAs / resident
// slots) CTA durations and a CTA's duration is its chunk plus the planes
// it loads beyond it, so the chunk count minimises that product
template <typename K>
dim3 lz_grid(K kernel, const HLevelDev &L, bool zc, int &zchunk) {
  static int slots_cache[2] = {0, 0};
  int &slots = slots_cache[zc ? 1 : 0];
  if (!slots) {
    int occ = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, LZ_NT, 0) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    slots = occ * (sms > 0 ? sms : 1);
  }
  const int gx = (L.nx + LZ_TX - 1) / LZ_TX, gy = (L.ny + LZ_TY - 1) / LZ_TY;
  const long tiles = (long)gx * gy;
  const int h = zc ? 3 : 1;
  long best = -1;
  zchunk = L.nz;
  for (int c = 1; c <= std::min(L.nz, LZ_MAX_CHUNKS); ++c) {
    const int zcq = (L.nz + c - 1) / c;
    const long gz = (L.nz + zcq - 1) / zcq;
    const long cost = ((tiles * gz + slots - 1) / slots) * (zcq + h);
    if (best < 0 || cost < best) {
      best = cost;
      zchunk = zcq;
    }
  }
  return dim3(gx, gy, (L.nz + zchunk - 1) / zchunk);
}
void split_w(double w, float &h, float &l) {
  h = (float)w;
  l = (float)(w - (double)h);
}
template <int MODE>
cudaError_t run_lz(const HLevelDev &L, LzArgs a, int *nblocks, cudaStream_t st) {
  const bool zc = L.wz != 0.f && L.nz > 1;
  dim3 g = zc ? lz_grid(k_lz<true, MODE>, L, true, a.zchunk) : lz_grid(k_lz<false, MODE>, L, false, a.zchunk);
  if (nblocks) *nblocks = (int)(g.x * g.y * g.z);
  if (zc)
    k_lz<true, MODE><<<g, LZ_NT, 0, st>>>(L, a);
  else
    k_lz<false, MODE><<<g, LZ_NT, 0, st>>>(L, a);
  return cudaGetLastError();
}
}  // namespace

int linear_zmax_blocks(const HLevelDev &L) {
  return ((L.nx + LZ_TX - 1) / LZ_TX) * ((L.ny + LZ_TY - 1) / LZ_TY) * std::min(L.nz, LZ_MAX_CHUNKS);
}

cudaError_t launch_l_rhs(const HLevelDev &L, const LinW &w, const float *I0, const float *I1, float *bh, float *bl,
                         cudaStream_t st) {
  LzArgs a{};
  a.a0 = I0;
  a.a1 = I1;
  a.oh = bh;
  a.ol = bl;
  split_w(w.gx, a.wh[0], a.wl[0]);
  split_w(w.gy, a.wh[1], a.wl[1]);
  split_w(w.gm, a.wh[2], a.wl[2]);
  a.want_m = (w.gm != 0.0 && I1) ? 1 : 0;
  return run_lz<LZ_RHS>(L, a, nullptr, st);
}

cudaError_t launch_l_resid(const HLevelDev &L, const LinW &w, const float *bh, const float *bl, const float *h,
                           const float *l, float *r, double *partials, int *nblocks, cudaStream_t st) {
  LzArgs a{};
  a.a0 = h;
  a.a1 = l;
  a.bh = bh;
  a.bl = bl;
  a.r = r;
  a.partials = partials;
  split_w(w.ax, a.wh[0], a.wl[0]);
  split_w(w.ay, a.wh[1], a.wl[1]);
  split_w(w.az, a.wh[2], a.wl[2]);
  split_w(w.am, a.wh[3], a.wl[3]);
  a.want_kz = w.az != 0.0 ? 1 : 0;
  a.want_m = w.am != 0.0 ? 1 : 0;
  return run_lz<LZ_RESID>(L, a, nblocks, st);
}

cudaError_t launch_l_update(long long n, const float *e, float *h, float *l, double *partials, int *nblocks,
                            cudaStream_t st) {
  const int g = grid_of(n);
  if (nblocks) *nblocks = g;
  k_l_update<<<g, HNT, 0, st>>>(n, e, h, l, partials);
  return cudaGetLastError();
}

cudaError_t launch_l_sum(long long n, const float *a, double *partials, int slot, int *nblocks, cudaStream_t st) {
  const int g = grid_of(n);
  if (nblocks) *nblocks = g;
  k_l_sum<<<g, HNT, 0, st>>>(n, a, partials, slot);
  return cudaGetLastError();
}

cudaError_t launch_l_final(long long n, const float *h, const float *l, double shift, float *out, cudaStream_t st) {
  const float sh = (float)shift, sl = (float)(shift - (double)sh);
  k_l_final<<<grid_of(n), HNT, 0, st>>>(n, h, l, sh, sl, out);
  return cudaGetLastError();
}
