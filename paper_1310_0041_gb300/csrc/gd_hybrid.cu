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
// parities of i, j and k; same-colour cells are never neighbours), one launch
// per colour, in place.
#include <cuda_runtime.h>

#include "gd_internal.h"

namespace {

constexpr int HNT = 256;

__device__ __forceinline__ long long cell(const HLevelDev &L, int i, int j, int k) {
  return ((long long)k * L.ny + j) * L.nx + i;
}

// A x at (i, j, k) without the diagonal term (off) and the diagonal (dg).
template <bool ZC, bool SIX>
__device__ __forceinline__ void apply_off(const HLevelDev &L, const float *__restrict__ x, int i, int j, int k,
                                          float &off, float &dg) {
  off = 0.f;
  dg = 0.f;
  if (SIX) {
    // fine level: K = 1D Neumann Laplacian, M = I
    float cnt = 0.f, s = 0.f;
    if (i > 0) { s += L.wx * x[cell(L, i - 1, j, k)]; cnt += L.wx; }
    if (i < L.nx - 1) { s += L.wx * x[cell(L, i + 1, j, k)]; cnt += L.wx; }
    if (j > 0) { s += L.wy * x[cell(L, i, j - 1, k)]; cnt += L.wy; }
    if (j < L.ny - 1) { s += L.wy * x[cell(L, i, j + 1, k)]; cnt += L.wy; }
    if (ZC) {
      if (k > 0) { s += L.wz * x[cell(L, i, j, k - 1)]; cnt += L.wz; }
      if (k < L.nz - 1) { s += L.wz * x[cell(L, i, j, k + 1)]; cnt += L.wz; }
    }
    off = -s;
    dg = cnt + L.wm;
    return;
  }
  if (i >= L.ilo[0] && i <= L.ihi[0] && j >= L.ilo[1] && j <= L.ihi[1] &&
      (!ZC || (k >= L.ilo[2] && k <= L.ihi[2]))) {
    // interior: constant coefficients, every neighbour exists
    const int c0 = ZC ? -1 : 0, c1 = ZC ? 1 : 0;
#pragma unroll
    for (int c = c0; c <= c1; ++c)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        const float *xr = x + cell(L, i, j + b, k + c);
#pragma unroll
        for (int a = -1; a <= 1; ++a) {
          if (a == 0 && b == 0 && c == 0) continue;
          off = fmaf(L.cst[(c + 1) * 9 + (b + 1) * 3 + (a + 1)], xr[a], off);
        }
      }
    dg = L.cst[13];
    return;
  }
  const float *kx = L.kx + 3 * i, *mx = L.mx + 3 * i;
  const float *ky = L.ky + 3 * j, *my = L.my + 3 * j;
  const float *kz = L.kz + 3 * k, *mz = L.mz + 3 * k;
  const int c0 = ZC ? -1 : 0, c1 = ZC ? 1 : 0;
  for (int c = c0; c <= c1; ++c) {
    const int kk = k + c;
    if (kk < 0 || kk >= L.nz) continue;
    const float mzc = mz[c + 1], kzc = ZC ? kz[c + 1] : 0.f;
    const float zterm = L.wz * kzc + L.wm * mzc;
    for (int b = -1; b <= 1; ++b) {
      const int jj = j + b;
      if (jj < 0 || jj >= L.ny) continue;
      const float myb = my[b + 1], kyb = ky[b + 1];
      const float yz = myb * zterm + L.wy * kyb * mzc;  // coefficient of mx
      const float xz = L.wx * myb * mzc;                // coefficient of kx
      const float *xr = x + cell(L, 0, jj, kk);
      for (int a = -1; a <= 1; ++a) {
        const int ii = i + a;
        if (ii < 0 || ii >= L.nx) continue;
        const float cf = mx[a + 1] * yz + kx[a + 1] * xz;
        if (a == 0 && b == 0 && c == 0)
          dg = cf;
        else
          off = fmaf(cf, xr[ii], off);
      }
    }
  }
}

// One colour of the eight-colour Gauss-Seidel sweep on a 27-point level.
template <bool ZC>
__global__ void __launch_bounds__(HNT) k_h_gs(HLevelDev L, int colour, float *__restrict__ x,
                                              const float *__restrict__ b) {
  const int px = colour & 1, py = (colour >> 1) & 1, pz = (colour >> 2) & 1;
  const int hx = (L.nx - px + 1) / 2, hy = (L.ny - py + 1) / 2, hz = (L.nz - pz + 1) / 2;
  const long long n = (long long)hx * hy * hz;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int ti = (int)(q % hx);
    const long long r = q / hx;
    const int tj = (int)(r % hy), tk = (int)(r / hy);
    const int i = 2 * ti + px, j = 2 * tj + py, k = 2 * tk + pz;
    float off, dg;
    apply_off<ZC, false>(L, x, i, j, k, off, dg);
    const long long o = cell(L, i, j, k);
    x[o] = (b[o] - off) / dg;
  }
}

// r = b - A x (SIX: the fine 6-point operator).
template <bool ZC, bool SIX>
__global__ void __launch_bounds__(HNT) k_h_resid(HLevelDev L, const float *__restrict__ x,
                                                 const float *__restrict__ b, float *__restrict__ r) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int i = (int)(q % L.nx);
    const long long t = q / L.nx;
    const int j = (int)(t % L.ny), k = (int)(t / L.ny);
    float off, dg;
    apply_off<ZC, SIX>(L, x, i, j, k, off, dg);
    r[q] = b[q] - (dg * x[q] + off);
  }
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

cudaError_t launch_h_gs(const HLevelDev &L, float *x, const float *b, cudaStream_t st) {
  const long long n8 = ((long long)L.nx * L.ny * L.nz + 7) / 8;
  const bool zc = L.wz != 0.f && L.nz > 1;
  for (int c = 0; c < 8; ++c) {
    if (zc)
      k_h_gs<true><<<grid_of(n8), HNT, 0, st>>>(L, c, x, b);
    else
      k_h_gs<false><<<grid_of(n8), HNT, 0, st>>>(L, c, x, b);
  }
  return cudaGetLastError();
}

cudaError_t launch_h_resid(const HLevelDev &L, bool six, const float *x, const float *b, float *r,
                           cudaStream_t st) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  const bool zc = L.wz != 0.f && L.nz > 1;
  if (six) {
    if (zc)
      k_h_resid<true, true><<<grid_of(n), HNT, 0, st>>>(L, x, b, r);
    else
      k_h_resid<false, true><<<grid_of(n), HNT, 0, st>>>(L, x, b, r);
  } else {
    if (zc)
      k_h_resid<true, false><<<grid_of(n), HNT, 0, st>>>(L, x, b, r);
    else
      k_h_resid<false, false><<<grid_of(n), HNT, 0, st>>>(L, x, b, r);
  }
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

// Integer-weighted neighbourhood sums, compensated.  With the fine factors
// scaled to integers (K_n as is, the P1 mass times 6), every product of
// three factor entries is a small integer, exact in FP32; each term p (h + l)
// enters a float pair by TwoProd and TwoSum, so the four sums
//   S_kx = sum (Kx My Mz) x, S_ky = sum (Mx Ky Mz) x,
//   S_kz = sum (Mx My Kz) x, S_m = sum (Mx My Mz) x
// come out exact to ~1e-12 of their terms, and the operator is their
// weighted sum, formed in FP64 (a few operations per cell).
struct Sums {
  float h[4], l[4];
};
__device__ __forceinline__ void acc_term(float P, float xh, float xl, float &sh, float &sl) {
  if (P == 0.f) return;
  const float p = P * xh;
  const float e = fmaf(P, xh, -p);
  const float s = sh + p;
  const float bb = s - sh;
  const float err = (sh - (s - bb)) + (p - bb);
  sh = s;
  sl += err + e + P * xl;
}
template <bool ZC, typename V>
__device__ __forceinline__ Sums kron_sums(const HLevelDev &L, bool want_kz, bool want_m, int i, int j, int k,
                                          V val) {
  Sums S;
#pragma unroll
  for (int q = 0; q < 4; ++q) S.h[q] = S.l[q] = 0.f;
  const float *kx = L.kx + 3 * i, *mx = L.mx + 3 * i;
  const float *ky = L.ky + 3 * j, *my = L.my + 3 * j;
  const float *kz = L.kz + 3 * k, *mz = L.mz + 3 * k;
  const int c0 = ZC ? -1 : 0, c1 = ZC ? 1 : 0;
  for (int c = c0; c <= c1; ++c) {
    const int kk = k + c;
    if (kk < 0 || kk >= L.nz) continue;
    const float mzc = mz[c + 1], kzc = ZC ? kz[c + 1] : 0.f;
    for (int b = -1; b <= 1; ++b) {
      const int jj = j + b;
      if (jj < 0 || jj >= L.ny) continue;
      const float myb = my[b + 1], kyb = ky[b + 1];
      for (int a = -1; a <= 1; ++a) {
        const int ii = i + a;
        if (ii < 0 || ii >= L.nx) continue;
        float xh, xl;
        val(((long long)kk * L.ny + jj) * L.nx + ii, xh, xl);
        const float mxa = mx[a + 1], kxa = kx[a + 1];
        acc_term(kxa * myb * mzc, xh, xl, S.h[0], S.l[0]);
        acc_term(mxa * kyb * mzc, xh, xl, S.h[1], S.l[1]);
        if (want_kz) acc_term(mxa * myb * kzc, xh, xl, S.h[2], S.l[2]);
        if (want_m) acc_term(mxa * myb * mzc, xh, xl, S.h[3], S.l[3]);
      }
    }
  }
  return S;
}
__device__ __forceinline__ double sum_of(const Sums &S, int q) { return (double)S.h[q] + (double)S.l[q]; }

// b = gx' S_kx(I0) + gy' S_ky(I0) + gm' S_m(I1) (weights already divided by
// the factor scales), stored as a float pair
template <bool ZC>
__global__ void __launch_bounds__(HNT) k_l_rhs(HLevelDev L, LinW w, const float *__restrict__ I0,
                                               const float *__restrict__ I1, float *__restrict__ bh,
                                               float *__restrict__ bl) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int i = (int)(q % L.nx);
    const long long t = q / L.nx;
    const int j = (int)(t % L.ny), k = (int)(t / L.ny);
    const Sums S0 = kron_sums<ZC>(L, false, false, i, j, k, [&](long long o, float &h, float &l) {
      h = I0[o];
      l = 0.f;
    });
    double v = w.gx * sum_of(S0, 0) + w.gy * sum_of(S0, 1);
    if (w.gm != 0.0) {
      const Sums S1 = kron_sums<ZC>(L, false, true, i, j, k, [&](long long o, float &h, float &l) {
        h = I1[o];
        l = 0.f;
      });
      v += w.gm * sum_of(S1, 3);
    }
    const float hv = (float)v;
    bh[q] = hv;
    bl[q] = (float)(v - (double)hv);
  }
}

// r = b - A (h + l) from the compensated sums (stored as float), and the
// block sums of r^2 (slot S_RR) and b^2 (slot S_BB)
template <bool ZC>
__global__ void __launch_bounds__(HNT) k_l_resid(HLevelDev L, LinW w, const float *__restrict__ bh,
                                                 const float *__restrict__ bl, const float *__restrict__ h,
                                                 const float *__restrict__ l, float *__restrict__ r,
                                                 double *__restrict__ partials) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  const bool want_kz = w.az != 0.0, want_m = w.am != 0.0;
  double srr = 0.0, sbb = 0.0;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const int i = (int)(q % L.nx);
    const long long t = q / L.nx;
    const int j = (int)(t % L.ny), k = (int)(t / L.ny);
    const Sums S = kron_sums<ZC>(L, want_kz, want_m, i, j, k, [&](long long o, float &xh, float &xl) {
      xh = h[o];
      xl = l[o];
    });
    double ax = w.ax * sum_of(S, 0) + w.ay * sum_of(S, 1);
    if (want_kz) ax += w.az * sum_of(S, 2);
    if (want_m) ax += w.am * sum_of(S, 3);
    const double b = (double)bh[q] + (double)bl[q];
    const double rv = b - ax;
    if (r) r[q] = (float)rv;
    srr += rv * rv;
    sbb += b * b;
  }
  block_sums(srr, sbb, partials, S_RR, S_BB);
}

// (h, l) += e exactly in FP64 and rounded back to a float pair; block sums
// of the new iterate (slot S_X)
__global__ void __launch_bounds__(HNT) k_l_update(long long n, const float *__restrict__ e, float *__restrict__ h,
                                                  float *__restrict__ l, double *__restrict__ partials) {
  double sx = 0.0;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) {
    const double v = (double)h[q] + (double)l[q] + (double)e[q];
    const float hv = (float)v;
    h[q] = hv;
    l[q] = (float)(v - (double)hv);
    sx += v;
  }
  block_sums(sx, 0.0, partials, S_X, -1);
}

// block sums of an array (slot)
__global__ void __launch_bounds__(HNT) k_l_sum(long long n, const float *__restrict__ a, double *__restrict__ partials,
                                               int slot) {
  double s = 0.0;
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT) s += a[q];
  block_sums(s, 0.0, partials, slot, -1);
}

// out = h + l + shift, rounded to float
__global__ void __launch_bounds__(HNT) k_l_final(long long n, const float *__restrict__ h, const float *__restrict__ l,
                                                 double shift, float *__restrict__ out) {
  for (long long q = blockIdx.x * (long long)HNT + threadIdx.x; q < n; q += (long long)gridDim.x * HNT)
    out[q] = (float)((double)h[q] + (double)l[q] + shift);
}

}  // namespace

int linear_grid(long long n) { return grid_of(n); }

cudaError_t launch_l_rhs(const HLevelDev &L, const LinW &w, const float *I0, const float *I1, float *bh, float *bl,
                         cudaStream_t st) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  if (L.wz != 0.f && L.nz > 1)
    k_l_rhs<true><<<grid_of(n), HNT, 0, st>>>(L, w, I0, I1, bh, bl);
  else
    k_l_rhs<false><<<grid_of(n), HNT, 0, st>>>(L, w, I0, I1, bh, bl);
  return cudaGetLastError();
}

cudaError_t launch_l_resid(const HLevelDev &L, const LinW &w, const float *bh, const float *bl, const float *h,
                           const float *l, float *r, double *partials, int *nblocks, cudaStream_t st) {
  const long long n = (long long)L.nx * L.ny * L.nz;
  const int g = grid_of(n);
  if (nblocks) *nblocks = g;
  if (L.wz != 0.f && L.nz > 1)
    k_l_resid<true><<<g, HNT, 0, st>>>(L, w, bh, bl, h, l, r, partials);
  else
    k_l_resid<false><<<g, HNT, 0, st>>>(L, w, bh, bl, h, l, r, partials);
  return cudaGetLastError();
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
  k_l_final<<<grid_of(n), HNT, 0, st>>>(n, h, l, shift, out);
  return cudaGetLastError();
}
