// basis.cpp -- host FP64 construction of the 1D operators of the nodal
// Gauss-Legendre basis (Sec. 3) used by the kernels.
//
// Nodes and weights come from the Golub-Welsch method: the Gauss points of
// the Legendre weight are the eigenvalues of the symmetric tridiagonal
// Jacobi matrix with off-diagonal k / sqrt(4k^2 - 1), the weights are twice
// the squared first components of its unit eigenvectors.  The eigenproblem
// is solved with cyclic Jacobi rotations.  Derivatives and face values use
// the barycentric form of Lagrange interpolation (Berrut & Trefethen 2004).
#include "basis.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace aderdg {

static void jacobi_eigen(int n, std::vector<double> &A, std::vector<double> &V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J (columns p, q)
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A (rows p, q)
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

bool gauss_legendre01(int N, double *xi, double *w) {
  if (N < 0 || N > kBasisMaxN) return false;
  const int n = N + 1;
  std::vector<double> J(n * n, 0.0), V;
  for (int k = 1; k < n; ++k) {
    const double b = k / std::sqrt(4.0 * k * k - 1.0);
    J[(k - 1) * n + k] = J[k * n + (k - 1)] = b;
  }
  jacobi_eigen(n, J, V);
  std::vector<std::pair<double, double>> pw(n);
  for (int i = 0; i < n; ++i) pw[i] = {J[i * n + i], V[0 * n + i] * V[0 * n + i]};
  std::sort(pw.begin(), pw.end());
  for (int i = 0; i < n; ++i) {
    xi[i] = 0.5 * (1.0 + pw[i].first);
    w[i] = pw[i].second;  // 2 v0^2 on [-1,1], halved for [0,1]
  }
  return true;
}

// LU factorisation with partial pivoting, then inverse column by column.
static bool lu_inverse(int n, const double *A, double *Ainv) {
  std::vector<double> LU(A, A + n * n);
  std::vector<int> piv(n);
  for (int i = 0; i < n; ++i) piv[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(LU[i * n + k]) > std::fabs(LU[p * n + k])) p = i;
    if (LU[p * n + k] == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(LU[k * n + j], LU[p * n + j]);
      std::swap(piv[k], piv[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      LU[i * n + k] /= LU[k * n + k];
      for (int j = k + 1; j < n; ++j) LU[i * n + j] -= LU[i * n + k] * LU[k * n + j];
    }
  }
  for (int col = 0; col < n; ++col) {
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) {  // forward: L y = P e_col
      double s = (piv[i] == col) ? 1.0 : 0.0;
      for (int j = 0; j < i; ++j) s -= LU[i * n + j] * x[j];
      x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {  // back: U x = y
      double s = x[i];
      for (int j = i + 1; j < n; ++j) s -= LU[i * n + j] * x[j];
      x[i] = s / LU[i * n + i];
    }
    for (int i = 0; i < n; ++i) Ainv[i * n + col] = x[i];
  }
  return true;
}

void lagrange_values(const Basis1D &B, double x, double *phi) {
  const int n = B.n;
  double lam[kBasisMaxN + 1];
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (B.xi[j] - B.xi[k]);
    lam[j] = 1.0 / p;
  }
  for (int j = 0; j < n; ++j)
    if (x == B.xi[j]) {
      for (int k = 0; k < n; ++k) phi[k] = k == j ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int k = 0; k < n; ++k) den += lam[k] / (x - B.xi[k]);
  for (int j = 0; j < n; ++j) phi[j] = (lam[j] / (x - B.xi[j])) / den;
}

bool build_basis(int N, Basis1D &B) {
  if (N < 0 || N > kBasisMaxN) return false;
  const int n = B.n = N + 1;
  if (!gauss_legendre01(N, B.xi, B.w)) return false;
  double lam[kBasisMaxN + 1];  // barycentric weights
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) p *= (B.xi[j] - B.xi[k]);
    lam[j] = 1.0 / p;
  }
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      const double v = (lam[j] / lam[i]) / (B.xi[i] - B.xi[j]);
      B.Dm[i * n + j] = v;
      diag -= v;
    }
    B.Dm[i * n + i] = diag;
  }
  for (int side = 0; side < 2; ++side) {
    const double x = side;
    double den = 0.0;
    for (int k = 0; k < n; ++k) den += lam[k] / (x - B.xi[k]);
    for (int j = 0; j < n; ++j) (side ? B.FR : B.FL)[j] = (lam[j] / (x - B.xi[j])) / den;
  }
  double K1[(kBasisMaxN + 1) * (kBasisMaxN + 1)];
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) K1[k * n + l] = B.FR[k] * B.FR[l] - B.w[l] * B.Dm[l * n + k];
  if (!lu_inverse(n, K1, B.K1inv)) return false;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) B.Kvol[i * n + a] = B.w[a] * B.Dm[a * n + i] / B.w[i];
  // time-modal vectors c_s = (K1^-1 W)^s 1 and weights g_s = w . c_s
  std::vector<double> c(n, 1.0), t(n);
  for (int s = 0; s <= kBasisMaxPicard; ++s) {
    double g = 0.0;
    for (int k = 0; k < n; ++k) {
      B.cvec[s * n + k] = c[k];
      g += B.w[k] * c[k];
    }
    B.g[s] = g;
    for (int k = 0; k < n; ++k) {
      double acc = 0.0;
      for (int l = 0; l < n; ++l) acc += B.K1inv[k * n + l] * B.w[l] * c[l];
      t[k] = acc;
    }
    c = t;
  }
  return true;
}

}  // namespace aderdg
