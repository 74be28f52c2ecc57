// pde.cuh -- conservative fluxes of Eq. 1 (B = S = delta = 0) for the four
// PDE families, as device functors templated on dimension d and arithmetic
// type R.
//
// Interface of a PDE functor P<d, R>:
//   M                         number of variables m
//   LINEAR                    F_j(q) = A_j q with A_j constant inside a cell
//   struct Mat                per-cell constants (material)
//   load(Mat&, args, cell)    fill Mat from pde_const / per-cell material
//   flux(Mat, q, j, f)        f = F_j(q), the x_j column of the flux tensor
//   speed(Mat, q, j)          spectral radius of dF_j/dQ at q (>= 0)
//   flux_all(Mat, q, f)       f[j] = F_j(q) for every j (shared sub-expressions)
// Linear functors add
//   reads(j, c)               does A_j read component c (compile-time)
//   applyA(Mat, j, dq, out)   out = A_j dq, reading only components with reads(j, c)
//   accA(Mat, j, dq, acc)     acc += A_j dq, touching only the non-zero rows (FMAs)
//   scaleA(Mat&, s)           A_j <- s A_j for every j (fold dt / dx into the operator)
//   applyAT(Mat, j, x, out)   out = A_j^T x (adjoint step)
//   NMAT, dA(Mat, j, w, x, g) g[k] += <w, (dA_j/dtheta_k) x> for the NMAT material
//                             parameters theta the flux is linear in (adjoint
//                             material gradient); NMAT = 0 for no material
#pragma once
#include "common.cuh"

namespace aderdg {

// ---------------------------------------------------------------------------
template <int d, class R>
struct Advection {
  static constexpr int M = 1;
  static constexpr bool LINEAR = true;
  static constexpr bool OWNED = false;
  struct Mat { R a[3]; };
  __device__ static void load(Mat &mt, const double *cst, const float *, long long) {
    mt.a[0] = (R)cst[0]; mt.a[1] = (R)cst[1]; mt.a[2] = (R)cst[2];
  }
  __host__ __device__ static constexpr bool reads(int, int) { return true; }
  __device__ __forceinline__ static void applyA(const Mat &mt, int j, const R *dq, R *out) {
    out[0] = mt.a[j] * dq[0];
  }
  __device__ __forceinline__ static void accA(const Mat &mt, int j, const R *dq, R *acc) { acc[0] += mt.a[j] * dq[0]; }
  __device__ __forceinline__ static void scaleA(Mat &mt, R s) { mt.a[0] *= s; mt.a[1] *= s; mt.a[2] *= s; }
  __device__ __forceinline__ static void flux(const Mat &mt, const R *q, int j, R *f) { applyA(mt, j, q, f); }
  __device__ __forceinline__ static R speed(const Mat &mt, const R *, int j) { return fabs(mt.a[j]); }
  __device__ __forceinline__ static void flux_all(const Mat &mt, const R *q, R (*f)[M]) {
#pragma unroll
    for (int j = 0; j < d; ++j) flux(mt, q, j, f[j]);
  }
  __device__ __forceinline__ static void applyAT(const Mat &mt, int j, const R *x, R *out) { out[0] = mt.a[j] * x[0]; }
  static constexpr int NMAT = 0;
  __device__ __forceinline__ static void dA(const Mat &, int, const R *, const R *, R *) {}
};

// ---------------------------------------------------------------------------
// Linear acoustics: Q = (p, v_0..v_{d-1}), dp/dt + K div v = 0, dv/dt + grad p / rho = 0.
template <int d, class R>
struct Acoustics {
  static constexpr int M = d + 1;
  static constexpr bool LINEAR = true;
  // the line-owner predictor keeps p and v_x on x-lines and v_j on lines along
  // axis j: A_j reads and writes only p and v_j, so the derivatives of v_j along
  // j and the update of v_j stay with the owner of its line
  static constexpr bool OWNED = true;
  __host__ __device__ static constexpr int owner(int c) { return c == 0 ? 0 : c - 1; }
  __host__ __device__ static constexpr bool writes(int j, int c) { return c == 0 || c == 1 + j; }
  struct Mat { R K, irho, c; };
  __device__ static void load(Mat &mt, const double *cst, const float *, long long) {
    const double rho = cst[0], c = cst[1];
    mt.K = (R)(rho * c * c); mt.irho = (R)(1.0 / rho); mt.c = (R)c;
  }
  __host__ __device__ static constexpr bool reads(int j, int c) { return c == 0 || c == 1 + j; }
  __device__ __forceinline__ static void applyA(const Mat &mt, int j, const R *dq, R *out) {
    out[0] = mt.K * dq[1 + j];
#pragma unroll
    for (int a = 0; a < d; ++a) out[1 + a] = (a == j) ? mt.irho * dq[0] : R(0);
  }
  __device__ __forceinline__ static void accA(const Mat &mt, int j, const R *dq, R *acc) {
    acc[0] += mt.K * dq[1 + j];
    acc[1 + j] += mt.irho * dq[0];
  }
  __device__ __forceinline__ static void scaleA(Mat &mt, R s) { mt.K *= s; mt.irho *= s; }
  __device__ __forceinline__ static void flux(const Mat &mt, const R *q, int j, R *f) { applyA(mt, j, q, f); }
  __device__ __forceinline__ static R speed(const Mat &mt, const R *, int) { return mt.c; }
  __device__ __forceinline__ static void flux_all(const Mat &mt, const R *q, R (*f)[M]) {
#pragma unroll
    for (int j = 0; j < d; ++j) flux(mt, q, j, f[j]);
  }
  __device__ __forceinline__ static void applyAT(const Mat &mt, int j, const R *x, R *out) {
#pragma unroll
    for (int c = 0; c < M; ++c) out[c] = R(0);
    out[1 + j] = mt.K * x[0];
    out[0] = mt.irho * x[1 + j];
  }
  static constexpr int NMAT = 0;
  __device__ __forceinline__ static void dA(const Mat &, int, const R *, const R *, R *) {}
  // applyA on two nodes at once (FP32: packed two-lane multiplies)
  __device__ __forceinline__ static void applyA2(const Mat &mt, int j, const float2 *dq, float2 *out) {
    out[0] = __fmul2_rn(make_float2(mt.K, mt.K), dq[1 + j]);
#pragma unroll
    for (int a = 0; a < d; ++a)
      out[1 + a] = (a == j) ? __fmul2_rn(make_float2(mt.irho, mt.irho), dq[0]) : make_float2(0.f, 0.f);
  }
  // acc += A_j dq for dq non-zero in component c only (one line of n values)
  template <int n>
  __device__ __forceinline__ static void accA_comp(const Mat &mt, int j, int c, const R (&dl)[n], R (&acc)[M][n]) {
    if (c == 0) {
#pragma unroll
      for (int o = 0; o < n; ++o) acc[1 + j][o] += mt.irho * dl[o];
    } else if (c == 1 + j) {
#pragma unroll
      for (int o = 0; o < n; ++o) acc[0][o] += mt.K * dl[o];
    }
  }
  template <int n>
  __device__ __forceinline__ static void dA_comp(const Mat &, int, int, const R (&)[M][n], const R (&)[n], R *) {}
};

// ---------------------------------------------------------------------------
// Compressible Euler (Sec. 7): Q = (rho, j, E), p = (gamma-1)(E - |j|^2/(2 rho)).
template <int d, class R>
struct Euler {
  static constexpr int M = d + 2;
  static constexpr bool LINEAR = false;
  static constexpr bool OWNED = false;
  struct Mat { R gm1, gamma; };
  __device__ static void load(Mat &mt, const double *cst, const float *, long long) {
    mt.gamma = (R)cst[0]; mt.gm1 = (R)(cst[0] - 1.0);
  }
  __host__ __device__ static constexpr bool reads(int, int) { return true; }
  __device__ __forceinline__ static void flux(const Mat &mt, const R *q, int j, R *f) {
    const R irho = R(1) / q[0];
    R jj = R(0);
#pragma unroll
    for (int a = 0; a < d; ++a) jj += q[1 + a] * q[1 + a];
    const R p = mt.gm1 * (q[d + 1] - R(0.5) * jj * irho);
    const R vj = q[1 + j] * irho;
    f[0] = q[1 + j];
#pragma unroll
    for (int a = 0; a < d; ++a) f[1 + a] = vj * q[1 + a] + (a == j ? p : R(0));
    f[d + 1] = vj * (q[d + 1] + p);
  }
  // all d directions from one evaluation of 1/rho and p: F_j = (j_j, v_j j + p e_j, j_j (E + p) / rho)
  __device__ __forceinline__ static void flux_all(const Mat &mt, const R *q, R (*f)[M]) {
    const R irho = R(1) / q[0];
    R jj = R(0);
#pragma unroll
    for (int a = 0; a < d; ++a) jj += q[1 + a] * q[1 + a];
    const R p = mt.gm1 * (q[d + 1] - R(0.5) * jj * irho);
    const R hp = (q[d + 1] + p) * irho;
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const R vj = q[1 + j] * irho;
      f[j][0] = q[1 + j];
#pragma unroll
      for (int a = 0; a < d; ++a) f[j][1 + a] = vj * q[1 + a] + (a == j ? p : R(0));
      f[j][d + 1] = q[1 + j] * hp;
    }
  }
  __device__ __forceinline__ static R speed(const Mat &mt, const R *q, int j) {
    const R irho = R(1) / q[0];
    R jj = R(0);
#pragma unroll
    for (int a = 0; a < d; ++a) jj += q[1 + a] * q[1 + a];
    const R p = mt.gm1 * (q[d + 1] - R(0.5) * jj * irho);
    return fabs(q[1 + j] * irho) + sqrt(mt.gamma * p * irho);
  }
  __device__ __forceinline__ static void applyA(const Mat &, int, const R *, R *) {}
  __device__ __forceinline__ static void accA(const Mat &, int, const R *, R *) {}
  __device__ __forceinline__ static void scaleA(Mat &, R) {}
  __device__ __forceinline__ static void applyAT(const Mat &, int, const R *, R *) {}
  static constexpr int NMAT = 0;
  __device__ __forceinline__ static void dA(const Mat &, int, const R *, const R *, R *) {}
};

// ---------------------------------------------------------------------------
// Linear elasticity, velocity-stress form with per-cell material:
//   d sigma/dt = lambda (div v) I + mu (grad v + grad v^T),  rho dv/dt = div sigma
// written as dQ/dt + sum_j d(F_j)/dx_j = 0 with F_j = -A_j Q.
// 3D: Q = (sxx syy szz sxy syz sxz vx vy vz); 2D (plane strain): (sxx syy sxy vx vy).
template <int d, class R>
struct Elasticity {
  static constexpr int M = d == 3 ? 9 : 5;
  static constexpr int VO = d == 3 ? 6 : 3;   // offset of the velocities
  static constexpr bool LINEAR = true;
  static constexpr bool OWNED = false;
  struct Mat { R lam, mu, irho, cp; };
  __host__ __device__ static constexpr int sig(int a, int b) {
    return a == b ? a : (d == 2 ? 2 : ((a + b == 1) ? 3 : ((a + b == 3) ? 4 : 5)));
  }
  __device__ static void load(Mat &mt, const double *cst, const float *mat, long long cell) {
    double rho, cp, cs;
    if (mat) {
      rho = mat[3 * cell]; cp = mat[3 * cell + 1]; cs = mat[3 * cell + 2];
    } else {
      rho = cst[0]; cp = cst[1]; cs = cst[2];
    }
    const double mu = rho * cs * cs;
    mt.mu = (R)mu; mt.lam = (R)(rho * cp * cp - 2.0 * mu); mt.irho = (R)(1.0 / rho); mt.cp = (R)cp;
  }
  // A_j reads the velocities and the stresses sigma_{a j}.
  __host__ __device__ static constexpr bool reads(int j, int c) {
    return c >= VO || c == sig(0, j) || c == sig(1, j) || (d == 3 && c == sig(2, j));
  }
  __device__ __forceinline__ static void applyA(const Mat &mt, int j, const R *dq, R *out) {
#pragma unroll
    for (int a = 0; a < d; ++a)
#pragma unroll
      for (int b = a; b < d; ++b) {
        R v = (a == b) ? mt.lam * dq[VO + j] : R(0);
        if (b == j) v += mt.mu * dq[VO + a];
        if (a == j) v += mt.mu * dq[VO + b];
        out[sig(a, b)] = -v;
      }
#pragma unroll
    for (int a = 0; a < d; ++a) out[VO + a] = -mt.irho * dq[sig(a, j)];
  }
  __device__ __forceinline__ static void accA(const Mat &mt, int j, const R *dq, R *acc) {
#pragma unroll
    for (int a = 0; a < d; ++a)
#pragma unroll
      for (int b = a; b < d; ++b) {
        if (a == b) acc[sig(a, b)] -= mt.lam * dq[VO + j];
        if (b == j) acc[sig(a, b)] -= mt.mu * dq[VO + a];
        if (a == j) acc[sig(a, b)] -= mt.mu * dq[VO + b];
      }
#pragma unroll
    for (int a = 0; a < d; ++a) acc[VO + a] -= mt.irho * dq[sig(a, j)];
  }
  __device__ __forceinline__ static void scaleA(Mat &mt, R s) { mt.lam *= s; mt.mu *= s; mt.irho *= s; }
  // The operator is bipartite: the stress rows of A_j read only velocities and
  // the velocity rows only stresses (group(c): 0 stresses, 1 velocities).
  static constexpr bool BIPARTITE = true;
  __host__ __device__ static constexpr int group(int c) { return c >= VO ? 1 : 0; }
  // acc += A_j dq for dq non-zero in component c only, given as one line of n
  // values: the rows A_j feeds from component c (c, j compile-time after
  // unrolling, so only those rows are touched)
  template <int n>
  __device__ __forceinline__ static void accA_comp(const Mat &mt, int j, int c, const R (&dl)[n], R (&acc)[M][n]) {
    if (c >= VO) {
      const int vv = c - VO;
#pragma unroll
      for (int a = 0; a < d; ++a)
#pragma unroll
        for (int b = a; b < d; ++b) {
          R k = R(0);
          bool any = false;
          if (a == b && vv == j) { k += mt.lam; any = true; }
          if (b == j && a == vv) { k += mt.mu; any = true; }
          if (a == j && b == vv) { k += mt.mu; any = true; }
          if (any) {
#pragma unroll
            for (int o = 0; o < n; ++o) acc[sig(a, b)][o] -= k * dl[o];
          }
        }
    } else {
#pragma unroll
      for (int a = 0; a < d; ++a)
        if (sig(a, j) == c) {
#pragma unroll
          for (int o = 0; o < n; ++o) acc[VO + a][o] -= mt.irho * dl[o];
        }
    }
  }
  __device__ __forceinline__ static void flux(const Mat &mt, const R *q, int j, R *f) { applyA(mt, j, q, f); }
  __device__ __forceinline__ static R speed(const Mat &mt, const R *, int) { return mt.cp; }
  __device__ __forceinline__ static void flux_all(const Mat &mt, const R *q, R (*f)[M]) {
#pragma unroll
    for (int j = 0; j < d; ++j) flux(mt, q, j, f[j]);
  }
  // transpose of applyA, term by term
  __device__ __forceinline__ static void applyAT(const Mat &mt, int j, const R *x, R *out) {
#pragma unroll
    for (int c = 0; c < M; ++c) out[c] = R(0);
#pragma unroll
    for (int a = 0; a < d; ++a)
#pragma unroll
      for (int b = a; b < d; ++b) {
        const R xs = x[sig(a, b)];
        if (a == b) out[VO + j] -= mt.lam * xs;
        if (b == j) out[VO + a] -= mt.mu * xs;
        if (a == j) out[VO + b] -= mt.mu * xs;
      }
#pragma unroll
    for (int a = 0; a < d; ++a) out[sig(a, j)] -= mt.irho * x[VO + a];
  }
  // theta = (lambda, mu, 1/rho): A_j = lambda A^lam_j + mu A^mu_j + (1/rho) A^rho_j
  static constexpr int NMAT = 3;
  __device__ __forceinline__ static void dA(const Mat &, int j, const R *w, const R *x, R *g) {
#pragma unroll
    for (int a = 0; a < d; ++a)
#pragma unroll
      for (int b = a; b < d; ++b) {
        const R ws = w[sig(a, b)];
        if (a == b) g[0] -= ws * x[VO + j];
        R t = R(0);
        if (b == j) t += x[VO + a];
        if (a == j) t += x[VO + b];
        g[1] -= ws * t;
      }
#pragma unroll
    for (int a = 0; a < d; ++a) g[2] -= w[VO + a] * x[sig(a, j)];
  }
  // the same for x non-zero in component c only, summed over one line of n
  // nodes (w and x as lines; c, j compile-time after unrolling)
  template <int n>
  __device__ __forceinline__ static void dA_comp(const Mat &, int j, int c, const R (&w)[M][n], const R (&dl)[n],
                                                 R *g) {
    if (c >= VO) {
      const int vv = c - VO;
#pragma unroll
      for (int a = 0; a < d; ++a)
#pragma unroll
        for (int b = a; b < d; ++b) {
          const int s = sig(a, b);
          if (a == b && vv == j) {
#pragma unroll
            for (int o = 0; o < n; ++o) g[0] -= w[s][o] * dl[o];
          }
          const int k = (b == j && a == vv ? 1 : 0) + (a == j && b == vv ? 1 : 0);
          if (k > 0) {
            R acc = w[s][0] * dl[0];
#pragma unroll
            for (int o = 1; o < n; ++o) acc += w[s][o] * dl[o];
            g[1] -= k == 2 ? R(2) * acc : acc;
          }
        }
    } else {
#pragma unroll
      for (int a = 0; a < d; ++a)
        if (sig(a, j) == c) {
#pragma unroll
          for (int o = 0; o < n; ++o) g[2] -= w[VO + a][o] * dl[o];
        }
    }
  }
};

}  // namespace aderdg
