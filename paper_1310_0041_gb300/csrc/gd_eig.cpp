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
