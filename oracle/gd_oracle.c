/*
 * gd_oracle.c -- plain, slow, FP64 CPU oracle for the gradient-domain solver.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the solver library calls this code;
 * only the tests, the entry point's smoke check and the benchmark's CPU
 * baseline do.  It shares no code with the CUDA path.
 *
 * Grid: nx*ny*nz voxels, x fastest: v[(k*ny + j)*nx + i].  Unit spacing.
 *
 * Discrete system (Kazhdan et al., "Gradient-Domain Processing for Large EM
 * Image Stacks"):
 *   general form, Sec. 4:   (alpha - div W grad) I = alpha I0 - div W G
 *   6-point "Constant" discretisation, Sec. 4.2: face-adjacent neighbours
 *   have coefficient -1, and (reading: homogeneous Neumann boundary, no
 *   ghost cells) the diagonal is the number of existing neighbours.  Along
 *   one axis this is the 1D matrix K_n = tridiag(-1, [1,2,...,2,1], -1).
 *     A = alpha I + bx Kx + by Ky + bz Kz          (Kd acts along axis d)
 *   anisotropic diffusion, Sec. 3.1 Eq. (anisotropic_diffusion):
 *     G = (dI0/dx, dI0/dy, 0) as forward differences on voxel faces, so
 *     div W G = -(bx Kx + by Ky) I0 and the system is
 *     (bx Kx + by Ky + bz Kz) I1 = (bx Kx + by Ky) I0,  alpha = 0
 *     (singular: constants are the null space; the oracle picks the
 *      solution with mean(I1) = mean(I0)).
 *   screened Poisson, Sec. 3.1 Eq. (screened_poisson), per slice:
 *     (alpha + Kx + Ky) I2 = alpha I1 + (Kx + Ky) I0.
 *
 * Solvers:
 *   gdo_cg     conjugate gradients to a relative residual tolerance
 *   gdo_dense  assembled dense matrix + Cholesky (small grids)
 *   gdo_mg     the paper's V-cycle (Sec. 4.1): Gauss-Seidel relaxation,
 *              residual, down-sampling by summing children, direct solve at
 *              the coarsest level, up-sampling by replication into the
 *              children (Constant transfers, Sec. 4.2), relaxation again.
 *              Coarse operators are Galerkin, P^T A P (Sec. 4.2 names the
 *              Galerkin formulation); with replication transfers they keep
 *              the Kronecker form  sum_d b_d K_d (x) M_others + alpha M,
 *              where M_d = P^T P = diag(children counts) and P^T K_n P is
 *              the coarse K_{n_c}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OK 0
#define ERR_ARG 1
#define ERR_OOM 3
#define ERR_NOT_CONVERGED 5

#define IDX(i, j, k) (((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i))

/* ------------------------------------------------------------------------ */
/* Operator with per-axis mass arrays (fine level: all masses 1).            */
/*   (A x)_p = cx(p) * sum_{x-nbrs n} (x_p - x_n)                             */
/*           + cy(p) * sum_{y-nbrs n} (x_p - x_n)                             */
/*           + cz(p) * sum_{z-nbrs n} (x_p - x_n) + alpha * m(p) * x_p        */
/*   cx(p) = bx * My[j] * Mz[k],  cy = by * Mx[i] * Mz[k],                    */
/*   cz = bz * Mx[i] * My[j],     m = Mx[i] * My[j] * Mz[k].                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nx, ny, nz;
  double alpha, bx, by, bz;
  double *Mx, *My, *Mz; /* per-axis children counts; NULL means all ones */
} op_t;

static inline double mval(const double *M, int i) { return M ? M[i] : 1.0; }

static inline double op_row(const op_t *A, const double *x, int i, int j, int k, double *diag) {
  const int nx = A->nx, ny = A->ny, nz = A->nz;
  double mx = mval(A->Mx, i), my = mval(A->My, j), mz = mval(A->Mz, k);
  double cx = A->bx * my * mz, cy = A->by * mx * mz, cz = A->bz * mx * my;
  double xp = x[IDX(i, j, k)];
  double s = A->alpha * mx * my * mz * xp;
  double d = A->alpha * mx * my * mz;
  if (i > 0) { s += cx * (xp - x[IDX(i - 1, j, k)]); d += cx; }
  if (i < nx - 1) { s += cx * (xp - x[IDX(i + 1, j, k)]); d += cx; }
  if (j > 0) { s += cy * (xp - x[IDX(i, j - 1, k)]); d += cy; }
  if (j < ny - 1) { s += cy * (xp - x[IDX(i, j + 1, k)]); d += cy; }
  if (k > 0) { s += cz * (xp - x[IDX(i, j, k - 1)]); d += cz; }
  if (k < nz - 1) { s += cz * (xp - x[IDX(i, j, k + 1)]); d += cz; }
  if (diag) *diag = d;
  return s;
}

static void op_apply(const op_t *A, const double *x, double *y) {
  const int nx = A->nx, ny = A->ny, nz = A->nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) y[IDX(i, j, k)] = op_row(A, x, i, j, k, NULL);
}

/* r = b - A x; returns ||r||_2 */
static double op_residual(const op_t *A, const double *b, const double *x, double *r) {
  const int nx = A->nx, ny = A->ny, nz = A->nz;
  double ss = 0.0;
#pragma omp parallel for collapse(2) schedule(static) reduction(+ : ss)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double v = b[IDX(i, j, k)] - op_row(A, x, i, j, k, NULL);
        if (r) r[IDX(i, j, k)] = v;
        ss += v * v;
      }
  return sqrt(ss);
}

static double norm2(const double *v, size_t n) {
  double ss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ss)
  for (size_t p = 0; p < n; ++p) ss += v[p] * v[p];
  return sqrt(ss);
}

/* One Gauss-Seidel update of voxel (i,j,k): x_p <- x_p + (b_p - (A x)_p)/a_pp,
   which equals x_p <- (b_p + sum_n a_pn x_n)/a_pp. */
static inline void gs_point(const op_t *A, const double *b, double *x, int i, int j, int k) {
  const int nx = A->nx, ny = A->ny;
  double d;
  double ax = op_row(A, x, i, j, k, &d);
  if (d > 0.0) x[IDX(i, j, k)] += (b[IDX(i, j, k)] - ax) / d;
}

/* order 0: lexicographic (x fastest, then y, then z); order 1: red-black,
   red = (i+j+k) even first, then black (Sec. 4.1 "multi-coloring"). */
static void gs_sweep(const op_t *A, const double *b, double *x, int order) {
  const int nx = A->nx, ny = A->ny, nz = A->nz;
  if (order == 0) {
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) gs_point(A, b, x, i, j, k);
    return;
  }
  for (int colour = 0; colour < 2; ++colour) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = (j + k + colour) & 1; i < nx; i += 2) gs_point(A, b, x, i, j, k);
  }
}

/* ------------------------------------------------------------------------ */
/* Public: right-hand sides and operator                                    */
/* ------------------------------------------------------------------------ */

/* Anisotropic diffusion RHS, Eq. (anisotropic_diffusion): b = (bx Kx + by Ky) I0 */
int gdo_rhs_ad(int nx, int ny, int nz, double bx, double by, const double *I0, double *b) {
  if (nx < 1 || ny < 1 || nz < 1 || !I0 || !b) return ERR_ARG;
  op_t A = {nx, ny, 1, 0.0, bx, by, 0.0, NULL, NULL, NULL};
  for (int k = 0; k < nz; ++k) op_apply(&A, I0 + (size_t)k * nx * ny, b + (size_t)k * nx * ny);
  return OK;
}

/* Screened-Poisson RHS, Eq. (screened_poisson): b = alpha I1 + (Kx + Ky) I0 */
int gdo_rhs_sp(int nx, int ny, int nz, double alpha, const double *I0, const double *I1, double *b) {
  if (nx < 1 || ny < 1 || nz < 1 || !I0 || !I1 || !b) return ERR_ARG;
  op_t A = {nx, ny, 1, 0.0, 1.0, 1.0, 0.0, NULL, NULL, NULL};
  for (int k = 0; k < nz; ++k) op_apply(&A, I0 + (size_t)k * nx * ny, b + (size_t)k * nx * ny);
  size_t n = (size_t)nx * ny * nz;
  for (size_t p = 0; p < n; ++p) b[p] += alpha * I1[p];
  return OK;
}

/* y = A x for the fine-level operator A = alpha I + bx Kx + by Ky + bz Kz */
int gdo_apply(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
              const double *x, double *y) {
  if (nx < 1 || ny < 1 || nz < 1 || !x || !y) return ERR_ARG;
  op_t A = {nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  op_apply(&A, x, y);
  return OK;
}

/* ||b - A x|| / ||b||  (returns ||b - A x|| if ||b|| == 0) */
double gdo_rel_residual(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
                        const double *b, const double *x) {
  op_t A = {nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  double rn = op_residual(&A, b, x, NULL);
  double bn = norm2(b, (size_t)nx * ny * nz);
  return bn > 0 ? rn / bn : rn;
}

/* nsweeps Gauss-Seidel sweeps on the fine-level system, in place. */
int gdo_gs_sweeps(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
                  const double *b, double *x, int order, int nsweeps) {
  if (nx < 1 || ny < 1 || nz < 1 || !b || !x || nsweeps < 0) return ERR_ARG;
  op_t A = {nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  for (int s = 0; s < nsweeps; ++s) gs_sweep(&A, b, x, order);
  return OK;
}

/* ------------------------------------------------------------------------ */
/* Conjugate gradients (Jacobi-preconditioned), FP64                        */
/* ------------------------------------------------------------------------ */
int gdo_cg(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
           const double *b, double *x, double tol, int maxit, int *iters, double *relres) {
  if (nx < 1 || ny < 1 || nz < 1 || !b || !x) return ERR_ARG;
  op_t A = {nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  size_t n = (size_t)nx * ny * nz;
  double *r = malloc(n * sizeof(double)), *z = malloc(n * sizeof(double));
  double *p = malloc(n * sizeof(double)), *q = malloc(n * sizeof(double));
  double *dinv = malloc(n * sizeof(double));
  if (!r || !z || !p || !q || !dinv) { free(r); free(z); free(p); free(q); free(dinv); return ERR_OOM; }
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double d;
        op_row(&A, x, i, j, k, &d);
        dinv[IDX(i, j, k)] = d > 0 ? 1.0 / d : 0.0;
      }
  double bn = norm2(b, n);
  if (bn == 0.0) bn = 1.0;
  op_residual(&A, b, x, r);
  double rz = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz)
  for (size_t t = 0; t < n; ++t) { z[t] = dinv[t] * r[t]; p[t] = z[t]; rz += r[t] * z[t]; }
  int it = 0;
  double rn = norm2(r, n);
  while (rn / bn > tol && it < maxit) {
    op_apply(&A, p, q);
    double pq = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : pq)
    for (size_t t = 0; t < n; ++t) pq += p[t] * q[t];
    if (pq <= 0.0) break;
    double a = rz / pq;
    double rz2 = 0.0, rr = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rz2, rr)
    for (size_t t = 0; t < n; ++t) {
      x[t] += a * p[t];
      r[t] -= a * q[t];
      z[t] = dinv[t] * r[t];
      rz2 += r[t] * z[t];
      rr += r[t] * r[t];
    }
    double beta = rz2 / rz;
    rz = rz2;
#pragma omp parallel for schedule(static)
    for (size_t t = 0; t < n; ++t) p[t] = z[t] + beta * p[t];
    rn = sqrt(rr);
    ++it;
    /* recompute the true residual now and then against drift */
    if (it % 200 == 0) rn = op_residual(&A, b, x, r);
  }
  rn = op_residual(&A, b, x, NULL);
  if (iters) *iters = it;
  if (relres) *relres = rn / bn;
  free(r); free(z); free(p); free(q); free(dinv);
  return rn / bn <= tol ? OK : ERR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------ */
/* Dense direct solve (assembled matrix, Cholesky).  For the singular        */
/* (alpha = 0) system the RHS is projected onto the range (the orthogonal    */
/* complement of the constants) and 1 1^T / n is added to the matrix, which  */
/* picks the zero-sum solution among all solutions.                          */
/* ------------------------------------------------------------------------ */
typedef struct { size_t n; int singular; double *L; } chol_t;

static void chol_free(chol_t *c) { free(c->L); c->L = NULL; }

static int chol_factor(const op_t *A, int singular, chol_t *c) {
  size_t n = (size_t)A->nx * A->ny * A->nz;
  c->n = n; c->singular = singular; c->L = NULL;
  if (n > 4096) return ERR_ARG;
  double *M = calloc(n * n, sizeof(double));
  double *e = calloc(n, sizeof(double)), *col = malloc(n * sizeof(double));
  if (!M || !e || !col) { free(M); free(e); free(col); return ERR_OOM; }
  for (size_t j = 0; j < n; ++j) { /* column j of the matrix = A e_j */
    e[j] = 1.0;
    op_apply(A, e, col);
    e[j] = 0.0;
    for (size_t i = 0; i < n; ++i) M[i * n + j] = col[i] + (singular ? 1.0 / (double)n : 0.0);
  }
  free(e); free(col);
  for (size_t j = 0; j < n; ++j) { /* M = L L^T, L in the lower triangle */
    double d = M[j * n + j];
    for (size_t k = 0; k < j; ++k) d -= M[j * n + k] * M[j * n + k];
    if (!(d > 0.0)) { free(M); return ERR_ARG; }
    d = sqrt(d);
    M[j * n + j] = d;
    for (size_t i = j + 1; i < n; ++i) {
      double s = M[i * n + j];
      for (size_t k = 0; k < j; ++k) s -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = s / d;
    }
  }
  c->L = M;
  return OK;
}

static void chol_solve(const chol_t *c, const double *b, double *x) {
  size_t n = c->n;
  const double *M = c->L;
  double mean = 0.0;
  if (c->singular) {
    for (size_t i = 0; i < n; ++i) mean += b[i];
    mean /= (double)n;
  }
  for (size_t i = 0; i < n; ++i) { /* L y = b */
    double s = b[i] - mean;
    for (size_t k = 0; k < i; ++k) s -= M[i * n + k] * x[k];
    x[i] = s / M[i * n + i];
  }
  for (size_t ii = n; ii-- > 0;) { /* L^T x = y */
    double s = x[ii];
    for (size_t k = ii + 1; k < n; ++k) s -= M[k * n + ii] * x[k];
    x[ii] = s / M[ii * n + ii];
  }
}

static int dense_solve_op(const op_t *A, const double *b, double *x, int singular) {
  chol_t c;
  int err = chol_factor(A, singular, &c);
  if (err != OK) return err;
  chol_solve(&c, b, x);
  chol_free(&c);
  return OK;
}

int gdo_dense(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
              const double *b, double *x) {
  if (nx < 1 || ny < 1 || nz < 1 || !b || !x) return ERR_ARG;
  op_t A = {nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  return dense_solve_op(&A, b, x, alpha == 0.0);
}

/* ------------------------------------------------------------------------ */
/* Transfers between levels (Constant discretisation, Sec. 4.2): coarse cell  */
/* c along a coarsened axis has children 2c and 2c+1 (if it exists).          */
/* Down-sampling sums the children ("accumulating", Sec. 4.1), i.e. P^T;      */
/* up-sampling replicates the coarse value into the children, i.e. P.        */
/* ------------------------------------------------------------------------ */
int gdo_restrict(int nx, int ny, int nz, int fx, int fy, int fz, const double *r, double *rc) {
  if (nx < 1 || ny < 1 || nz < 1 || !r || !rc) return ERR_ARG;
  int ncx = fx ? (nx + 1) / 2 : nx, ncy = fy ? (ny + 1) / 2 : ny, ncz = fz ? (nz + 1) / 2 : nz;
  memset(rc, 0, sizeof(double) * (size_t)ncx * ncy * ncz);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int I = fx ? i / 2 : i, J = fy ? j / 2 : j, K = fz ? k / 2 : k;
        rc[((size_t)K * ncy + J) * ncx + I] += r[IDX(i, j, k)];
      }
  return OK;
}

/* x += P ec */
int gdo_prolong_add(int nx, int ny, int nz, int fx, int fy, int fz, const double *ec, double *x) {
  if (nx < 1 || ny < 1 || nz < 1 || !ec || !x) return ERR_ARG;
  int ncx = fx ? (nx + 1) / 2 : nx, ncy = fy ? (ny + 1) / 2 : ny;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int I = fx ? i / 2 : i, J = fy ? j / 2 : j, K = fz ? k / 2 : k;
        x[IDX(i, j, k)] += ec[((size_t)K * ncy + J) * ncx + I];
      }
  return OK;
}

/* ------------------------------------------------------------------------ */
/* V-cycle multigrid (Sec. 4.1) with Galerkin coarse operators.               */
/* ------------------------------------------------------------------------ */
typedef struct {
  op_t A;
  int fx, fy, fz; /* axes coarsened to reach the next level */
  double *x, *b, *r;
} level_t;

static void coarsen_mass(const double *M, int n, double *Mc) {
  int nc = (n + 1) / 2;
  for (int c = 0; c < nc; ++c) Mc[c] = 0.0;
  for (int i = 0; i < n; ++i) Mc[i / 2] += M ? M[i] : 1.0;
}

static void vcycle(level_t *L, int l, int nlev, int order, int nu1, int nu2, const chol_t *coarsest) {
  level_t *F = &L[l];
  if (l == nlev - 1) {
    chol_solve(coarsest, F->b, F->x);
    return;
  }
  for (int s = 0; s < nu1; ++s) gs_sweep(&F->A, F->b, F->x, order);
  op_residual(&F->A, F->b, F->x, F->r);
  level_t *C = &L[l + 1];
  gdo_restrict(F->A.nx, F->A.ny, F->A.nz, F->fx, F->fy, F->fz, F->r, C->b);
  memset(C->x, 0, sizeof(double) * (size_t)C->A.nx * C->A.ny * C->A.nz);
  vcycle(L, l + 1, nlev, order, nu1, nu2, coarsest);
  gdo_prolong_add(F->A.nx, F->A.ny, F->A.nz, F->fx, F->fy, F->fz, C->x, F->x);
  for (int s = 0; s < nu2; ++s) gs_sweep(&F->A, F->b, F->x, order);
}

/*
 * Solve A x = b by V(nu1,nu2) cycles, starting from x, until
 * ||b - A x|| <= tol ||b|| or max_cycles.  Full coarsening of x and y while
 * the level has more than min_xy cells along them (n_c = ceil(n/2)); z is
 * coarsened alongside while nz > 1, except when bz == 0 (independent slices,
 * which stay separate problems).  The coarsest level (at most 4096 cells) is
 * solved directly (Cholesky, factored once).  hist (may be NULL) receives the relative residual before
 * the first cycle and after each cycle (max_cycles + 1 entries).
 */
int gdo_mg(int nx, int ny, int nz, double alpha, double bx, double by, double bz,
           const double *b, double *x, int order, int nu1, int nu2, int min_xy,
           double tol, int max_cycles, int *cycles, double *relres, double *hist) {
  if (nx < 1 || ny < 1 || nz < 1 || !b || !x || min_xy < 1) return ERR_ARG;
  level_t L[64];
  memset(L, 0, sizeof(L));
  int nlev = 0;
  L[0].A = (op_t){nx, ny, nz, alpha, bx, by, bz, NULL, NULL, NULL};
  L[0].x = x;
  L[0].b = (double *)b;
  int err = OK;
  for (;;) {
    level_t *F = &L[nlev];
    size_t nf = (size_t)F->A.nx * F->A.ny * F->A.nz;
    F->r = malloc(nf * sizeof(double));
    if (!F->r) { err = ERR_OOM; break; }
    ++nlev;
    int fx = F->A.nx > min_xy, fy = F->A.ny > min_xy;
    int fz = (bz != 0.0) && F->A.nz > 1 && (fx || fy);
    if ((!fx && !fy) || nf <= 512 || nlev == 64) break;
    F->fx = fx; F->fy = fy; F->fz = fz;
    level_t *C = &L[nlev];
    op_t *a = &C->A;
    *a = F->A;
    a->nx = fx ? (F->A.nx + 1) / 2 : F->A.nx;
    a->ny = fy ? (F->A.ny + 1) / 2 : F->A.ny;
    a->nz = fz ? (F->A.nz + 1) / 2 : F->A.nz;
    a->Mx = malloc(sizeof(double) * a->nx);
    a->My = malloc(sizeof(double) * a->ny);
    a->Mz = malloc(sizeof(double) * a->nz);
    size_t nc = (size_t)a->nx * a->ny * a->nz;
    C->x = malloc(nc * sizeof(double));
    C->b = malloc(nc * sizeof(double));
    if (!a->Mx || !a->My || !a->Mz || !C->x || !C->b) { err = ERR_OOM; ++nlev; break; }
    if (fx) coarsen_mass(F->A.Mx, F->A.nx, a->Mx);
    else for (int i = 0; i < a->nx; ++i) a->Mx[i] = mval(F->A.Mx, i);
    if (fy) coarsen_mass(F->A.My, F->A.ny, a->My);
    else for (int i = 0; i < a->ny; ++i) a->My[i] = mval(F->A.My, i);
    if (fz) coarsen_mass(F->A.Mz, F->A.nz, a->Mz);
    else for (int i = 0; i < a->nz; ++i) a->Mz[i] = mval(F->A.Mz, i);
  }
  chol_t coarsest = {0, 0, NULL};
  if (err == OK) err = chol_factor(&L[nlev - 1].A, alpha == 0.0, &coarsest);
  double bn = norm2(b, (size_t)nx * ny * nz);
  if (bn == 0.0) bn = 1.0;
  int c = 0;
  double rel = op_residual(&L[0].A, b, x, NULL) / bn;
  if (hist) hist[0] = rel;
  if (err == OK) {
    while (c < max_cycles && rel > tol) {
      vcycle(L, 0, nlev, order, nu1, nu2, &coarsest);
      ++c;
      rel = op_residual(&L[0].A, b, x, NULL) / bn;
      if (hist) hist[c] = rel;
    }
  }
  if (cycles) *cycles = c;
  if (relres) *relres = rel;
  chol_free(&coarsest);
  for (int l = 0; l < nlev; ++l) {
    free(L[l].r);
    if (l > 0) { free(L[l].x); free(L[l].b); free(L[l].A.Mx); free(L[l].A.My); free(L[l].A.Mz); }
  }
  if (err != OK) return err;
  return rel <= tol ? OK : ERR_NOT_CONVERGED;
}

int gdo_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
