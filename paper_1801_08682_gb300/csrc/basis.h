// basis.h -- host FP64 1D operators of the nodal Gauss-Legendre basis.
#pragma once

namespace aderdg {

constexpr int kBasisMaxN = 9;
constexpr int kBasisMaxPicard = 16;

struct Basis1D {
  int n;
  double xi[kBasisMaxN + 1], w[kBasisMaxN + 1];
  double Dm[(kBasisMaxN + 1) * (kBasisMaxN + 1)];    // Dm[i*n+a] = phi_a'(xi_i)
  double Kvol[(kBasisMaxN + 1) * (kBasisMaxN + 1)];  // w_a Dm[a][i] / w_i
  double K1inv[(kBasisMaxN + 1) * (kBasisMaxN + 1)];
  double FL[kBasisMaxN + 1], FR[kBasisMaxN + 1];
  double g[kBasisMaxPicard + 1];
  double cvec[(kBasisMaxPicard + 1) * (kBasisMaxN + 1)];
};

bool gauss_legendre01(int N, double *xi, double *w);
bool build_basis(int N, Basis1D &B);
// phi[a] = the Lagrange polynomial of node a at x (any real x: outside [0,1]
// it extrapolates), barycentric form.
void lagrange_values(const Basis1D &B, double x, double *phi);

}  // namespace aderdg
