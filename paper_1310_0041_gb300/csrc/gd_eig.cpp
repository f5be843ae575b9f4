// gd_eig.cpp -- small dense symmetric eigen-decomposition for the coarsest
// level's fast diagonalisation (host, FP64, matrices of at most a few hundred
// rows).  Cyclic Jacobi rotations (Jacobi 1846; Golub & Van Loan, "Matrix
// Computations", Sec. 8.5): each rotation zeroes one off-diagonal pair and the
// off-diagonal mass decreases monotonically.
#include <cmath>
#include <vector>

#include "gd_internal.h"

void jacobi_eigen(int n, double *a, double *w, double *v) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i * n + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a[i * n + i] * a[i * n + i];
      for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
    }
    if (off <= 1e-30 * (diag + 1e-300)) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[p * n + p], aqq = a[q * n + q];
        // rotation angle that zeroes a[p][q]: tan(2 theta) = 2 apq / (aqq - app)
        const double theta = 0.5 * std::atan2(2.0 * apq, aqq - app);
        const double c = std::cos(theta), s = std::sin(theta);
        for (int k = 0; k < n; ++k) {  // A <- A J  (columns p, q)
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A  (rows p, q)
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        a[p * n + q] = a[q * n + p] = 0.0;
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = v[k * n + p], vkq = v[k * n + q];
          v[k * n + p] = c * vkp - s * vkq;
          v[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

// Generalised eigen-decomposition of (K_n, M) with K_n the 1D Neumann
// Laplacian and M = diag(children counts): V^T M V = I, V^T K V = diag(lam).
void axis_eig(int n, int sfac, int last, std::vector<float> &V, std::vector<double> &lam) {
  std::vector<double> m(n), a((size_t)n * n, 0.0), v((size_t)n * n), w(n);
  for (int i = 0; i < n; ++i) m[i] = (i == n - 1) ? last : sfac;
  for (int i = 0; i + 1 < n; ++i) {  // K_n = sum over edges of e e^T, e = u_i - u_{i+1}
    a[i * n + i] += 1.0;
    a[(i + 1) * n + i + 1] += 1.0;
    a[i * n + i + 1] -= 1.0;
    a[(i + 1) * n + i] -= 1.0;
  }
  for (int i = 0; i < n; ++i)  // C = M^{-1/2} K M^{-1/2}
    for (int j = 0; j < n; ++j) a[i * n + j] /= std::sqrt(m[i] * m[j]);
  jacobi_eigen(n, a.data(), w.data(), v.data());
  V.assign((size_t)n * n, 0.f);
  lam.assign(n, 0.0);
  for (int k = 0; k < n; ++k) lam[k] = w[k] < 0 ? 0.0 : w[k];
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) V[(size_t)i * n + k] = (float)(v[i * n + k] / std::sqrt(m[i]));
}

// Rows of the first-order B-spline prolongation P (n fine x nc coarse cells,
// nc = ceil(n / 2)): fine 2I takes coarse I; fine 2I+1 takes half of coarse I
// and half of I+1, or all of I when it has no I+1 (the last cell of an even
// extent), so P 1 = 1.
static int prolong_row(int i, int nc, int *idx, double *w) {
  if ((i & 1) == 0) {
    idx[0] = i >> 1;
    w[0] = 1.0;
    return 1;
  }
  const int I = i >> 1;
  if (I + 1 < nc) {
    idx[0] = I;
    idx[1] = I + 1;
    w[0] = w[1] = 0.5;
    return 2;
  }
  idx[0] = I;
  w[0] = 1.0;
  return 1;
}

void galerkin_tri(int n, const std::vector<double> &T, std::vector<double> &Tc) {
  const int nc = (n + 1) / 2;
  Tc.assign((size_t)nc * 3, 0.0);
  // Tc = P^T T P, accumulated over the nonzeros T(i, j) and the rows of P
  for (int i = 0; i < n; ++i) {
    int pi[2], pj[2];
    double wi[2], wj[2];
    const int mi = prolong_row(i, nc, pi, wi);
    for (int d = -1; d <= 1; ++d) {
      const int j = i + d;
      if (j < 0 || j >= n) continue;
      const double t = T[(size_t)i * 3 + d + 1];
      if (t == 0.0) continue;
      const int mj = prolong_row(j, nc, pj, wj);
      for (int a = 0; a < mi; ++a)
        for (int b = 0; b < mj; ++b) {
          const int off = pj[b] - pi[a];  // |off| <= 1: Tc stays tridiagonal
          Tc[(size_t)pi[a] * 3 + off + 1] += wi[a] * t * wj[b];
        }
    }
  }
}

void axis_eig_tri(int n, const std::vector<double> &K, const std::vector<double> &M, std::vector<float> &V,
                  std::vector<double> &lam) {
  // dense copies; M = L L^T (Cholesky); C = L^-1 K L^-T = Q diag(lam) Q^T;
  // V = L^-T Q satisfies V^T M V = I and V^T K V = diag(lam)
  std::vector<double> Kd((size_t)n * n, 0.0), L((size_t)n * n, 0.0), Md((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int d = -1; d <= 1; ++d) {
      const int j = i + d;
      if (j < 0 || j >= n) continue;
      Kd[(size_t)i * n + j] = K[(size_t)i * 3 + d + 1];
      Md[(size_t)i * n + j] = M[(size_t)i * 3 + d + 1];
    }
  for (int j = 0; j < n; ++j) {
    double s = Md[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
    const double ljj = std::sqrt(s > 0.0 ? s : 1e-300);
    L[(size_t)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double t = Md[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
      L[(size_t)i * n + j] = t / ljj;
    }
  }
  // Y = L^-1 K (forward substitution per column), C = L^-1 Y^T (K symmetric)
  auto lower_solve = [&](std::vector<double> &B) {  // B <- L^-1 B, column by column
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) {
        double t = B[(size_t)i * n + c];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * B[(size_t)k * n + c];
        B[(size_t)i * n + c] = t / L[(size_t)i * n + i];
      }
  };
  std::vector<double> Y = Kd;
  lower_solve(Y);
  std::vector<double> C((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) C[(size_t)i * n + j] = Y[(size_t)j * n + i];
  lower_solve(C);
  for (int i = 0; i < n; ++i)  // symmetrise the rounding
    for (int j = i + 1; j < n; ++j) {
      const double a = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
      C[(size_t)i * n + j] = C[(size_t)j * n + i] = a;
    }
  std::vector<double> w(n), Q((size_t)n * n);
  jacobi_eigen(n, C.data(), w.data(), Q.data());
  // V = L^-T Q: back substitution with L^T, column by column
  std::vector<double> Vd = Q;
  for (int c = 0; c < n; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double t = Vd[(size_t)i * n + c];
      for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * Vd[(size_t)k * n + c];
      Vd[(size_t)i * n + c] = t / L[(size_t)i * n + i];
    }
  V.assign((size_t)n * n, 0.f);
  lam.assign(n, 0.0);
  for (int k = 0; k < n; ++k) lam[k] = w[k] < 0 ? 0.0 : w[k];
  for (size_t q = 0; q < Vd.size(); ++q) V[q] = (float)Vd[q];
}
