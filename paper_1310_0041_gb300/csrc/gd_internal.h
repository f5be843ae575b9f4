// gd_internal.h -- structures shared by the host driver and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

// One multigrid level.  The operator is the Kronecker form
//   A = wx Kx (x) My (x) Mz + wy Mx (x) Ky (x) Mz + wz Mx (x) My (x) Kz + wm Mx (x) My (x) Mz
// where K_n is the 1D Neumann Laplacian and M_d = diag(children counts of the
// level's cells along axis d, counted in fine cells).  Along axis d every cell
// has s_d children except the last, which has l_d (ragged sizes).
// At the fine level all M are identity and (wx, wy, wz, wm) = (bx, by, bz, alpha),
// the 6-point operator of Sec. 4.2.  Coarser levels (see the planner) scale
// the stiffness wd by 1/2 per coarsening of axis d, which is the 6-point
// stencil re-discretised at the coarse spacing.
struct LevelDev {
  int nx, ny, nz;
  int sx, sy, sz;
  int lx, ly, lz;
  float wx, wy, wz, wm;
};

// Slots of the per-block partial sums (FP64) and of the reduced scalars.
enum {
  S_RR = 0,   // sum r^2
  S_BB = 1,   // sum b^2
  S_X = 2,    // sum of the new iterate (hi + lo)
  S_I0 = 3,   // sum of I0
  S_E = 4,    // sum of the correction e
  S_NUM = 5
};
// scalars[S_RMAX] holds max |r| of the last outer pass (float bits in its
// first word); scalars[S_ERR] is set to 1 by a kernel whose bounded wait gave
// up
constexpr int S_RMAX = 6;
constexpr int S_ERR = 7;

enum RhsMode { RHS_EXPLICIT = 0, RHS_AD = 1, RHS_SP = 2 };

// Arguments of the fine-level outer pass (update + residual + norms).
struct OuterArgs {
  int nx, ny, nz;
  // operator weights (fine level) and rhs weights (b = ralpha*I1 + rbx*Kx I0 +
  // rby*Ky I0), each as a float pair (w, w_lo) with w + w_lo = the double weight
  float bx, by, bz, alpha;
  float bx_lo, by_lo, bz_lo, alpha_lo;
  float rbx, rby, ralpha;
  float rbx_lo, rby_lo, ralpha_lo;
  const float *b;               // explicit rhs (RHS_EXPLICIT)
  const float *I0, *I1;         // inputs (RHS_AD / RHS_SP)
  const float *xh_in;           // iterate, high part
  const float *xl_in;           // iterate, low part (nullable: zero)
  const void *e;                // correction to add (nullable: none); stored / e_scale
  float *xh_out, *xl_out;       // new iterate (nullable: not written)
  void *r_out;                  // residual (nullable: not written); stored * r_scale
  float e_scale, r_scale;       // 1 for float32 storage; powers of two for float16
  unsigned *rmax;               // nullable: atomic max of |r| (float bits)
  const double *scalars;        // reduced sums of the previous passes (mean fix)
  int mean_fix;                 // AD: shift the update so that sum x = sum I0
  int accurate;                 // residual by error-free transformations (else plain FP32)
  double inv_n;                 // 1 / (nx*ny*nz)
  double *partials;             // [gridDim.x][S_NUM]
};

// Arguments of the TMA z-march sweep (gd_zmarch.cu).
struct ZSweepArgs {
  LevelDev L;
  void *xout;           // relaxed iterate (a different array from the input)
  const void *xc;       // prolongation: coarse correction (next level's x)
  int ncx, ncy;         // next level's x, y sizes (prolongation / restriction)
  int fx, fy, fz;       // axes coarsened from this level to the next
  void *bc;             // restriction: next level's right-hand side
  int zchunk;           // set by the launcher
  int cpf;              // set by the launcher: prolongation prefetches the coarse level
  double *partials;     // SUM: per-block sums of the output, slot S_E
  double *err;          // set to 1 when a bounded wait gives up
};

// TMA z-march launchers (gd_zmarch.cu); cudaErrorNotSupported when the arrays
// do not meet TMA's alignment rules (nx % 4, 16-byte base) -- the caller then
// uses the plain kernels.
// esz: bytes per element of a level's arrays (4: float32, 2: float16); esz_c
// the same for the next coarser level
bool zmarch_usable(const LevelDev &L, int esz);
cudaError_t launch_zsweep(ZSweepArgs a, const void *xin, const void *b, bool zero_in, bool prolong,
                          bool sum, int esz, int esz_c, int *nblocks_out, cudaStream_t st);
// residual of (x, b) on level a.L summed into the next level's b (a.bc)
cudaError_t launch_zrestrict(ZSweepArgs a, const void *x, const void *b, int esz, int esz_c,
                             cudaStream_t st);
// esz_e: element size of the correction e read and the residual r written
cudaError_t launch_zouter(const OuterArgs &a, int rhs_mode, int esz_e, double *err, int *nblocks_out,
                          cudaStream_t st);
int zouter_max_blocks(int nx, int ny, int nz);
// self-test of the kernels' bounded mbarrier wait on a barrier nothing
// arrives at: 1 if the wait gave up after `limit` polls, 0 if it completed,
// -1 on a CUDA error
int zmarch_wait_selftest(unsigned limit, cudaStream_t st);

// Host-side launchers (gd_kernels.cu).  All enqueue on `st` and return the
// cudaGetLastError() of the launch.
cudaError_t launch_rb_sweep(const LevelDev &L, const float *xin, const float *b, float *xout,
                            bool zero_in, double *partials_sum, int *nblocks_out, cudaStream_t st);
cudaError_t launch_residual_restrict(const LevelDev &F, const float *x, const float *b, int fx,
                                     int fy, int fz, float *bc, cudaStream_t st);
cudaError_t launch_prolong_add(const LevelDev &F, int fx, int fy, int fz, const float *xc,
                               float *x, cudaStream_t st);
cudaError_t launch_outer(const OuterArgs &a, int rhs_mode, int *nblocks_out, cudaStream_t st);
cudaError_t launch_reduce(const double *partials, int nblocks, double *scalars, int slot_lo,
                          int slot_hi, int accumulate, cudaStream_t st);
// Coarsest solve by fast diagonalisation: x = V Dinv V^T b (V = Vx (x) Vy (x) Vz).
// batch_z: z is not transformed (independent slices; Dinv is nx*ny).
cudaError_t launch_fdm(int nx, int ny, int nz, const float *Vx, const float *Vy, const float *Vz,
                       const float *Dinv, int batch_z, const float *b, float *x, float *tmp,
                       cudaStream_t st);
cudaError_t launch_fill(float *p, size_t n, float v, cudaStream_t st);
cudaError_t launch_copy(float *dst, const float *src, size_t n, cudaStream_t st);
// the same copy in 16-byte pieces with several loads in flight per thread
// (falls back to launch_copy when a pointer is not 16-byte aligned)
cudaError_t launch_copy_wide(float *dst, const float *src, size_t n, cudaStream_t st);
// b = alpha I0 - div(W V) of the NPR gradient filter (gd_kernels.cu)
cudaError_t launch_npr_rhs(const float *I0, float *b, int nx, int ny, int nz, double alpha, double wx,
                           double wy, double wz, double lam, double sigma, cudaStream_t st);

// A level of the Hybrid discretisation (gd_hybrid.cu): the Kronecker form
// of the fine operator with per-axis tridiagonal factors, 3 floats per index
// (sub-diagonal, diagonal, super-diagonal), and the fine weights.
struct HLevelDev {
  int nx, ny, nz;
  float wx, wy, wz, wm;
  const float *kx, *mx, *ky, *my, *kz, *mz;
  // cells whose factor rows along every axis equal the uniform interior rows
  // (index range [ilo, ihi] per axis, empty when ilo > ihi) share the 27
  // coefficients cst[(c+1)*9 + (b+1)*3 + (a+1)] of offset (a, b, c)
  int ilo[3], ihi[3];
  float cst[27];
};
// eight-colour Gauss-Seidel sweep of a 27-point level with the in-plane
// colours fused, out of place: the result is in xout (two launches on a
// coupled level, one otherwise)
cudaError_t launch_h_gsf(const HLevelDev &L, const float *x, float *xout, const float *b, cudaStream_t st);
int h_gsf_launches(const HLevelDev &L);
// r = b - A x (six: the fine 6-point operator, factors unused)
cudaError_t launch_h_resid(const HLevelDev &L, bool six, const float *x, const float *b, float *r,
                           cudaStream_t st);
// A coupled level halved along z only: bc = P^T (b - A x) in one z-march
// (no r array); six: the fine 6-point operator
cudaError_t launch_h_resid_rz(const HLevelDev &L, bool six, const float *x, const float *b, float *bc, int ncz,
                              cudaStream_t st);
// bc = P^T r and x += P e with the first-order B-spline transfers along the
// halved axes (fx, fy, fz)
cudaError_t launch_h_restrict(int nx, int ny, int nz, int fx, int fy, int fz, int cnx, int cny, int cnz,
                              const float *r, float *bc, cudaStream_t st);
cudaError_t launch_h_prolong(int nx, int ny, int nz, int fx, int fy, int fz, int cnx, int cny, int cnz,
                             const float *e, float *x, cudaStream_t st);
// Weights of the Linear discretisation's fine operator (ax Kx(x)My(x)Mz +
// ay Mx(x)Ky(x)Mz + az Mx(x)My(x)Kz + am Mx(x)My(x)Mz) and right-hand side
// (gx Kx(x)My(x)Mz I0 + gy Mx(x)Ky(x)Mz I0 + gm Mx(x)My(x)Mz I1), given for
// the integer-scaled fine factors the kernels take (each weight divided by
// the scales of the mass factors in its term).
struct LinW {
  double ax, ay, az, am;
  double gx, gy, gm;
};
// upper bound of the blocks (partial-sum rows) of a launch_l_resid launch
int linear_zmax_blocks(const HLevelDev &L);
cudaError_t launch_l_rhs(const HLevelDev &L, const LinW &w, const float *I0, const float *I1, float *bh, float *bl,
                         cudaStream_t st);
// r = b - A (h + l) (r nullable) with FP64 sums of r^2, b^2 per block (S_RR, S_BB)
cudaError_t launch_l_resid(const HLevelDev &L, const LinW &w, const float *bh, const float *bl, const float *h,
                           const float *l, float *r, double *partials, int *nblocks, cudaStream_t st);
// (h, l) += e with per-block sums of the new iterate (S_X)
cudaError_t launch_l_update(long long n, const float *e, float *h, float *l, double *partials, int *nblocks,
                            cudaStream_t st);
cudaError_t launch_l_sum(long long n, const float *a, double *partials, int slot, int *nblocks, cudaStream_t st);
cudaError_t launch_l_final(long long n, const float *h, const float *l, double shift, float *out, cudaStream_t st);
int linear_grid(long long n);

// Host: the per-axis Galerkin product T_c = P^T T P of a tridiagonal T (n x 3)
// with the first-order B-spline prolongation from nc = ceil(n / 2) cells.
void galerkin_tri(int n, const std::vector<double> &T, std::vector<double> &Tc);
// Host: generalised eigen-decomposition of tridiagonal (K, M) (n x 3 each, M
// symmetric positive definite): V^T M V = I, V^T K V = diag(lam).
void axis_eig_tri(int n, const std::vector<double> &K, const std::vector<double> &M, std::vector<float> &V,
                  std::vector<double> &lam);

// Host: symmetric eigen-decomposition (cyclic Jacobi), FP64, row-major a[n*n].
// On return w holds the eigenvalues and v (row-major, column k = eigenvector k).
void jacobi_eigen(int n, double *a, double *w, double *v);
// Host: generalised eigen-decomposition of (K_n, M) with K_n the 1D Neumann
// Laplacian and M = diag(sfac, ..., sfac, last): V (row-major, n x n, column
// k = eigenvector k) with V^T M V = I and V^T K V = diag(lam).
void axis_eig(int n, int sfac, int last, std::vector<float> &V, std::vector<double> &lam);
