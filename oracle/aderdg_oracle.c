/*
 * aderdg_oracle.c -- plain, slow FP64 CPU oracle for nodal ADER-DG on a
 * regular periodic Cartesian grid (Charrier & Weinzierl, "Stop talking to
 * me -- a communication-avoiding ADER-DG realisation", arXiv:1801.08682).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. The CUDA product path
 * never calls it, and the two share no code, headers or tables.
 *
 * What it computes
 *   The PDE is Eq. 1 with B = S = delta = 0 (Sec. 3 drops them as well):
 *   dQ/dt + div F(Q) = 0, Q in R^m, d in {2,3}.
 *   Each cell holds m*(N+1)^d nodal values of a tensor-product Lagrange
 *   polynomial on Gauss-Legendre points (Sec. 3).  One time step is
 *   Eq. 6 executed in the straightforward three-sweep order of
 *   Algorithm 1 (left):
 *     sweep 1  predict (Eq. 3, Picard) + extrapolate, for every cell
 *     sweep 2  solveRiemann (Eq. 4, Rusanov), for every face
 *     sweep 3  integrateVolume + integrateFace + update (Eq. 2) and
 *              calcTimeStep, for every cell
 *   with the per-task data of Table 1 stored explicitly: the predictor
 *   writes the full space-time polynomial and its d fluxes, extrapolate
 *   writes space-time face data, solveRiemann writes a space-time F*.
 *   A second driver runs the same tasks in the shifted, optimistic order
 *   of Algorithm 2 (Techniques 3 and 5), including STP reruns.
 *
 * Discrete operators (the paper names the basis but prints no matrices;
 * this is the standard collocated derivation from Eqs. 2-3):
 *   xi_k, w_k   Gauss-Legendre nodes/weights on [0,1], sum w = 1
 *   phi_a       Lagrange polynomials on xi
 *   Dm[i][a]  = phi_a'(xi_i)
 *   FL[a]     = phi_a(0),  FR[a] = phi_a(1)
 *   K1[k][l]  = FR_k FR_l - w_l Dm[l][k]   (time part of Eq. 3 after one
 *               integration by parts, upwind value at tau = 0 is u)
 *   Kvol[i][a]= w_a Dm[a][i] / w_i          (volume term of Eq. 2)
 *   predict:  q^{r+1}_{.,k} = sum_l K1^{-1}[k][l] ( FL_l u
 *                 - w_l dt sum_j (1/dx_j) sum_a Dm[i_j][a] F_j(q^r_{i_j->a,l}) )
 *   Riemann:  F* = 1/2 (F_L + F_R) - 1/2 s (q_R - q_L), s = max over the
 *             face nodes and both sides of the spectral radius of dF_j/dQ
 *             at the time-averaged face state.
 *   update:   Q_i += dt sum_k w_k sum_j (1/dx_j) sum_a Kvol[i_j][a] F_j(q_k)(i_j->a)
 *                  - dt sum_j (1/dx_j)(1/w_{i_j}) sum_k w_k
 *                      [FR_{i_j} F*_{j,right,k} - FL_{i_j} F*_{j,left,k}]
 *   calcTimeStep: dt_adm = min_j dx_j / (d (2N+1) lambda_max), the used
 *             step is C_dT * dt_adm (Algorithm 1).
 *
 * Two terms of Eq. 1 beyond the conservative flux, both optional:
 *   Non-conservative products B_j(x) dQ/dx_j for heterogeneous elasticity
 *   (Sec. 1: the B_i model material parameter changes).  Inside a cell the
 *   material is constant and B_j = dF_j/dQ; across a face the material jumps.
 *   The volume term is then taken in strong form, -int phi_i B_j dq/dx_j,
 *   and each face contributes path-conservative fluctuations
 *     D- = 1/2 (A~ - s) (q_R - q_L)  to the cell on its left,
 *     D+ = 1/2 (A~ + s) (q_R - q_L)  to the cell on its right,
 *   A~ = int_0^1 B_j(theta_L + r (theta_R - theta_L)) dr along the straight
 *   path in the material theta = (lambda, mu, 1/rho), evaluated by two-point
 *   Gauss quadrature in r (exact: B_j is linear in theta).
 *   Point sources (the delta terms of Eq. 1): a_c s(t) delta(x - x_s),
 *   projected onto the cell containing x_s as the nodal values
 *   sigma_{c,i} = a_c prod_j phi_{i_j}(xi_s,j) / (w_{i_j} dx_j); they enter the
 *   predictor's right-hand side at every time node and the update as
 *   dt sum_k w_k s(t + xi_k dt) sigma.
 *
 * Layouts (shared with the CUDA library's public API only by convention):
 *   Q[cell][comp][node], cell = c0 + G0 (c1 + G1 c2), node = i0 + n (i1 + n i2)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_ADVECTION = 0, ORC_ACOUSTICS = 1, ORC_EULER = 2, ORC_ELASTICITY = 3 };
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 4 };

#define ORC_MAXN 9
#define ORC_MAXM 9

/* A point source a s(t) delta(x - pos) (the delta terms of Eq. 1). */
typedef struct {
  double pos[3];        /* physical position; outside the grid: the boundary cell */
  double amp[ORC_MAXM]; /* a_c for every variable */
  int kind;             /* 0: s(t) = sum_p coef[p] (t - t0)^p;
                           1: Ricker wavelet (1 - 2 a) exp(-a), a = (pi f0 (t - t0))^2 */
  int pad_;
  double t0, f0;
  double coef[8];
} orc_source;

typedef struct {
  int d, N, m, pde;
  int grid[3];
  double dx[3];
  double cst[8];      /* advection: a0,a1,a2 | acoustics: rho,c | Euler: gamma | elasticity: rho,cp,cs */
  const double *mat;  /* elasticity: per-cell (rho, cp, cs) [C][3]; NULL = uniform cst */
  int picard;         /* > 0: this many Picard iterations; <= 0: iterate to the fixed point */
  double cfl;         /* safety factor C_dT of Algorithm 1 */
  int ncp;            /* elasticity: 1 = material jumps in non-conservative form (B_j), 0 = per-cell flux */
  int nsrc;           /* point sources */
  const orc_source *src;
} orc_cfg;

/* ------------------------------------------------------------------------ */
/* Threads                                                                   */

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1D basis: Gauss-Legendre nodes and weights on [0,1] (Sec. 3)              */

/* Legendre P_n(t) and P_n'(t) by the three-term recurrence. */
static void legendre(int n, double t, double *p, double *dp) {
  double p0 = 1.0, p1 = t;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double pk = ((2.0 * k - 1.0) * t * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *p = p1;
  *dp = n * (t * p1 - p0) / (t * t - 1.0);
}

/* Roots of P_{N+1}(2x-1) in ascending order and their weights (sum = 1). */
int orc_gauss_legendre(int N, double *xi, double *w) {
  if (N < 0 || N > ORC_MAXN) return ORC_EINVAL;
  int n = N + 1;
  for (int k = 0; k < n; ++k) {
    double t = cos(M_PI * (k + 0.75) / (n + 0.5)), p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(n, t, &p, &dp);
      double step = p / dp;
      t -= step;
      if (fabs(step) < 1e-17) break;
    }
    legendre(n, t, &p, &dp);
    xi[n - 1 - k] = 0.5 * (1.0 + t);
    w[n - 1 - k] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
  return ORC_OK;
}

/* phi_a(x): Lagrange polynomial through the nodes xi. */
static double lagrange(int n, const double *xi, int a, double x) {
  double v = 1.0;
  for (int b = 0; b < n; ++b)
    if (b != a) v *= (x - xi[b]) / (xi[a] - xi[b]);
  return v;
}

/* phi_a'(x) by the product rule. */
static double lagrange_deriv(int n, const double *xi, int a, double x) {
  double s = 0.0;
  for (int b = 0; b < n; ++b) {
    if (b == a) continue;
    double t = 1.0 / (xi[a] - xi[b]);
    for (int c = 0; c < n; ++c)
      if (c != a && c != b) t *= (x - xi[c]) / (xi[a] - xi[c]);
    s += t;
  }
  return s;
}

int orc_lagrange_eval(int N, double x, double *phi) {
  double xi[ORC_MAXN + 1], w[ORC_MAXN + 1];
  int rc = orc_gauss_legendre(N, xi, w);
  if (rc) return rc;
  for (int a = 0; a <= N; ++a) phi[a] = lagrange(N + 1, xi, a, x);
  return ORC_OK;
}

/* Inverse of an n x n matrix by Gauss-Jordan elimination with partial pivoting. */
static int invert(int n, const double *A, double *Ainv) {
  double M[ORC_MAXN + 1][2 * (ORC_MAXN + 1)];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c)
      M[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return ORC_EINVAL;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) { double t = M[col][c]; M[col][c] = M[piv][c]; M[piv][c] = t; }
    double inv = 1.0 / M[col][col];
    for (int c = 0; c < 2 * n; ++c) M[col][c] *= inv;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = M[r][col];
      for (int c = 0; c < 2 * n; ++c) M[r][c] -= f * M[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = M[r][n + c];
  return ORC_OK;
}

typedef struct {
  int n;
  double xi[ORC_MAXN + 1], w[ORC_MAXN + 1];
  double Dm[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
  double FL[ORC_MAXN + 1], FR[ORC_MAXN + 1];
  double K1[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
  double K1inv[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
  double Kvol[(ORC_MAXN + 1) * (ORC_MAXN + 1)];
} orc_ops;

static int make_ops(int N, orc_ops *O) {
  int rc = orc_gauss_legendre(N, O->xi, O->w);
  if (rc) return rc;
  int n = O->n = N + 1;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) O->Dm[i * n + a] = lagrange_deriv(n, O->xi, a, O->xi[i]);
  for (int a = 0; a < n; ++a) {
    O->FL[a] = lagrange(n, O->xi, a, 0.0);
    O->FR[a] = lagrange(n, O->xi, a, 1.0);
  }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l)
      O->K1[k * n + l] = O->FR[k] * O->FR[l] - O->w[l] * O->Dm[l * n + k];
  rc = invert(n, O->K1, O->K1inv);
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < n; ++a) O->Kvol[i * n + a] = O->w[a] * O->Dm[a * n + i] / O->w[i];
  return ORC_OK;
}

/* Export of the 1D operators for the pins in the test suite. */
int orc_operators(int N, double *xi, double *w, double *Dm, double *FL, double *FR,
                  double *K1, double *K1inv, double *Kvol) {
  orc_ops O;
  int rc = make_ops(N, &O);
  if (rc) return rc;
  int n = N + 1;
  memcpy(xi, O.xi, n * sizeof(double));
  memcpy(w, O.w, n * sizeof(double));
  memcpy(Dm, O.Dm, n * n * sizeof(double));
  memcpy(FL, O.FL, n * sizeof(double));
  memcpy(FR, O.FR, n * sizeof(double));
  memcpy(K1, O.K1, n * n * sizeof(double));
  memcpy(K1inv, O.K1inv, n * n * sizeof(double));
  memcpy(Kvol, O.Kvol, n * n * sizeof(double));
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* PDEs: conservative fluxes F_j(Q) and spectral radii of dF_j/dQ            */

int orc_num_vars(int pde, int d) {
  switch (pde) {
    case ORC_ADVECTION: return 1;
    case ORC_ACOUSTICS: return d + 1;          /* p, v */
    case ORC_EULER: return d + 2;              /* rho, j, E  (Sec. 7) */
    case ORC_ELASTICITY: return d == 3 ? 9 : 5; /* stresses, velocities */
  }
  return -1;
}

/* Index of the stress component sigma_ab in the state vector. */
static int sig_index(int d, int a, int b) {
  if (a == b) return a;
  if (d == 2) return 2;
  int lo = a < b ? a : b, hi = a < b ? b : a;
  if (lo == 0 && hi == 1) return 3;
  if (lo == 1 && hi == 2) return 4;
  return 5; /* (0,2) */
}

static void material(const orc_cfg *P, long cell, double *rho, double *cp, double *cs) {
  if (P->mat) {
    *rho = P->mat[3 * cell + 0];
    *cp = P->mat[3 * cell + 1];
    *cs = P->mat[3 * cell + 2];
  } else {
    *rho = P->cst[0];
    *cp = P->cst[1];
    *cs = P->cst[2];
  }
}

/* Elastic flux F_j = -A_j q for the material theta = (lambda, mu, 1/rho). */
static void elastic_flux(int d, const double *theta, const double *q, int j, double *f) {
  double lam = theta[0], mu = theta[1], irho = theta[2];
  int vo = d == 3 ? 6 : 3; /* offset of the velocities */
  for (int a = 0; a < d; ++a)
    for (int b = a; b < d; ++b) {
      double val = (a == b ? lam * q[vo + j] : 0.0);
      val += mu * ((b == j ? q[vo + a] : 0.0) + (a == j ? q[vo + b] : 0.0));
      f[sig_index(d, a, b)] = -val;
    }
  for (int a = 0; a < d; ++a) f[vo + a] = -irho * q[sig_index(d, a, j)];
}

/* The material of a cell as theta = (lambda, mu, 1/rho). */
static void theta_of(const orc_cfg *P, long cell, double *theta) {
  double rho, cp, cs;
  material(P, cell, &rho, &cp, &cs);
  theta[1] = rho * cs * cs;
  theta[0] = rho * cp * cp - 2.0 * theta[1];
  theta[2] = 1.0 / rho;
}

/* F_j(q): the x_j column of the flux tensor. */
static void flux(const orc_cfg *P, long cell, const double *q, int j, double *f) {
  int d = P->d;
  switch (P->pde) {
    case ORC_ADVECTION:
      f[0] = P->cst[j] * q[0];
      break;
    case ORC_ACOUSTICS: {
      double rho = P->cst[0], c = P->cst[1], K = rho * c * c;
      f[0] = K * q[1 + j];
      for (int a = 0; a < d; ++a) f[1 + a] = (a == j) ? q[0] / rho : 0.0;
      break;
    }
    case ORC_EULER: {
      double g = P->cst[0], rho = q[0], E = q[d + 1], jj = 0.0;
      for (int a = 0; a < d; ++a) jj += q[1 + a] * q[1 + a];
      double p = (g - 1.0) * (E - 0.5 * jj / rho);
      double vj = q[1 + j] / rho;
      f[0] = q[1 + j];
      for (int a = 0; a < d; ++a) f[1 + a] = vj * q[1 + a] + (a == j ? p : 0.0);
      f[d + 1] = vj * (E + p);
      break;
    }
    case ORC_ELASTICITY: {
      double theta[3];
      theta_of(P, cell, theta);
      elastic_flux(d, theta, q, j, f);
      break;
    }
  }
}

/* Spectral radius of dF_j/dQ at q. */
static double speed(const orc_cfg *P, long cell, const double *q, int j) {
  int d = P->d;
  switch (P->pde) {
    case ORC_ADVECTION: return fabs(P->cst[j]);
    case ORC_ACOUSTICS: return P->cst[1];
    case ORC_EULER: {
      double g = P->cst[0], rho = q[0], E = q[d + 1], jj = 0.0;
      for (int a = 0; a < d; ++a) jj += q[1 + a] * q[1 + a];
      double p = (g - 1.0) * (E - 0.5 * jj / rho);
      return fabs(q[1 + j] / rho) + sqrt(g * p / rho);
    }
    case ORC_ELASTICITY: {
      double rho, cp, cs;
      material(P, cell, &rho, &cp, &cs);
      return cp;
    }
  }
  return 0.0;
}

/* Point evaluations for the tests (flux Jacobian eigenvalue pins). */
int orc_flux_point(const orc_cfg *P, long cell, const double *q, int j, double *f) {
  flux(P, cell, q, j, f);
  return ORC_OK;
}
double orc_speed_point(const orc_cfg *P, long cell, const double *q, int j) {
  return speed(P, cell, q, j);
}

/* A~ dq = int_0^1 B_j(theta_L + r (theta_R - theta_L)) dr dq on the straight
 * path between the materials of cells cl and cr, by two-point Gauss quadrature
 * in r (B_j is linear in theta, so the rule is exact). */
static void path_jacobian_times(const orc_cfg *P, long cl, long cr, const double *dq, int j, double *out) {
  double tl[3], tr[3], th[3], f[ORC_MAXM];
  theta_of(P, cl, tl);
  theta_of(P, cr, tr);
  const double g = 0.5 / sqrt(3.0);
  const double r[2] = {0.5 - g, 0.5 + g};
  for (int c = 0; c < P->m; ++c) out[c] = 0.0;
  for (int k = 0; k < 2; ++k) {
    for (int e = 0; e < 3; ++e) th[e] = tl[e] + r[k] * (tr[e] - tl[e]);
    elastic_flux(P->d, th, dq, j, f);
    for (int c = 0; c < P->m; ++c) out[c] += 0.5 * f[c];
  }
}

/* ------------------------------------------------------------------------ */
/* Point sources (the delta terms of Eq. 1)                                  */

static double src_time(const orc_source *S, double t) {
  double tau = t - S->t0;
  if (S->kind == 1) {
    double a = M_PI * S->f0 * tau;
    a *= a;
    return (1.0 - 2.0 * a) * exp(-a);
  }
  double v = 0.0;
  for (int p = 7; p >= 0; --p) v = v * tau + S->coef[p];
  return v;
}

/* Cell holding the source (positions outside the grid: the boundary cell)
 * and the nodal weights pw[i] = prod_j phi_{i_j}(xi_j) / (w_{i_j} dx_j), so
 * that sigma_{c,i} = amp_c pw[i] is the lumped-mass projection of the delta. */
static long src_weights(const orc_cfg *P, const orc_source *S, double *pw) {
  int n = P->N + 1, d = P->d;
  double xi[ORC_MAXN + 1], w[ORC_MAXN + 1], loc[3] = {0, 0, 0};
  orc_gauss_legendre(P->N, xi, w);
  long cell = 0, stride = 1;
  for (int a = 0; a < d; ++a) {
    double x = S->pos[a] / P->dx[a];
    long ci = (long)floor(x);
    if (ci < 0) ci = 0;
    if (ci >= P->grid[a]) ci = P->grid[a] - 1;
    loc[a] = x - ci;
    cell += ci * stride;
    stride *= P->grid[a];
  }
  int NS = 1;
  for (int a = 0; a < d; ++a) NS *= n;
  for (int i = 0; i < NS; ++i) {
    double v = 1.0;
    int r = i;
    for (int a = 0; a < d; ++a) {
      int ia = r % n;
      r /= n;
      v *= lagrange(n, xi, ia, loc[a]) / (w[ia] * P->dx[a]);
    }
    pw[i] = v;
  }
  return cell;
}

/* Exported for the pins: the cell and nodal weights of source k. */
long orc_source_weights(const orc_cfg *P, int k, double *pw) { return src_weights(P, &P->src[k], pw); }
double orc_source_time(const orc_cfg *P, int k, double t) { return src_time(&P->src[k], t); }

/* ------------------------------------------------------------------------ */
/* Index helpers                                                             */

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

static long num_cells(const orc_cfg *P) {
  long c = 1;
  for (int a = 0; a < P->d; ++a) c *= P->grid[a];
  return c;
}

/* Digit j of a node index in base n. */
static int digit(int i, int j, int n) { for (int k = 0; k < j; ++k) i /= n; return i % n; }

/* Node index with axis j replaced by a. */
static int with_axis(int i, int j, int a, int n) {
  int s = ipow(n, j);
  return i + (a - digit(i, j, n)) * s;
}

/* Node index of face node p (the other d-1 axes, ascending, lowest fastest)
 * on the line along axis j at position a. */
static int face_node_to_node(int d, int n, int j, int p, int a) {
  int idx = 0, s = 1, q = p;
  for (int k = 0; k < d; ++k) {
    int v;
    if (k == j) v = a;
    else { v = q % n; q /= n; }
    idx += v * s;
    s *= n;
  }
  return idx;
}

/* Face node index of a volume node for the face normal to axis j. */
static int node_to_face_node(int d, int n, int j, int i) {
  int p = 0, s = 1;
  for (int k = 0; k < d; ++k) {
    if (k == j) continue;
    p += digit(i, k, n) * s;
    s *= n;
  }
  return p;
}

/* Periodic neighbour of cell c along axis j (dir = +1 or -1). */
static long neighbour(const orc_cfg *P, long c, int j, int dir) {
  long co[3] = {0, 0, 0}, r = c;
  for (int a = 0; a < P->d; ++a) { co[a] = r % P->grid[a]; r /= P->grid[a]; }
  co[j] = (co[j] + dir + P->grid[j]) % P->grid[j];
  long idx = 0, s = 1;
  for (int a = 0; a < P->d; ++a) { idx += co[a] * s; s *= P->grid[a]; }
  return idx;
}

static int check_cfg(const orc_cfg *P) {
  if (P->d < 2 || P->d > 3 || P->N < 0 || P->N > ORC_MAXN) return ORC_EINVAL;
  if (P->pde < 0 || P->pde > 3) return ORC_EINVAL;
  if (P->m != orc_num_vars(P->pde, P->d)) return ORC_EINVAL;
  for (int a = 0; a < P->d; ++a)
    if (P->grid[a] < 1 || !(P->dx[a] > 0.0)) return ORC_EINVAL;
  if (P->ncp && P->pde != ORC_ELASTICITY) return ORC_EINVAL;
  if (P->nsrc < 0 || (P->nsrc > 0 && !P->src)) return ORC_EINVAL;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Task predict (Eq. 3): Picard iteration for one cell.                      */
/* st layout: [slot 0..d][k][comp][node]; slot 0 = q^, slot 1+j = F_j(q^).   */

typedef struct {
  int d, n, m, NS, NF;
  long C;
  size_t st_size;   /* doubles per cell of the space-time predictor output */
  size_t face_size; /* doubles per cell of the space-time face data */
} orc_dims;

static orc_dims dims_of(const orc_cfg *P) {
  orc_dims D;
  D.d = P->d;
  D.n = P->N + 1;
  D.m = P->m;
  D.NS = ipow(D.n, D.d);
  D.NF = ipow(D.n, D.d - 1);
  D.C = num_cells(P);
  D.st_size = (size_t)(D.d + 1) * D.n * D.m * D.NS;
  D.face_size = (size_t)(2 * D.d) * 2 * D.n * D.m * D.NF;
  return D;
}

/* Point sources of a cell at the n time nodes of the step [t0, t0 + dt]:
 * src[k][c][i] = sum over the cell's sources of amp_c pw[i] s(t0 + xi_k dt);
 * returns 0 if the cell holds no source (src untouched). */
static int cell_sources(const orc_cfg *P, const orc_ops *O, const orc_dims *D, long cell, double t0,
                        double dt, double *src) {
  int n = D->n, m = D->m, NS = D->NS, any = 0;
  double pw[(ORC_MAXN + 1) * (ORC_MAXN + 1) * (ORC_MAXN + 1)];
  for (int s = 0; s < P->nsrc; ++s) {
    if (src_weights(P, &P->src[s], pw) != cell) continue;
    if (!any) memset(src, 0, (size_t)n * m * NS * sizeof(double));
    any = 1;
    for (int k = 0; k < n; ++k) {
      double sv = src_time(&P->src[s], t0 + O->xi[k] * dt);
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < NS; ++i) src[((size_t)k * m + c) * NS + i] += P->src[s].amp[c] * pw[i] * sv;
    }
  }
  return any;
}

static int predict_cell(const orc_cfg *P, const orc_ops *O, const orc_dims *D, long cell,
                        const double *u, double dt, double t0, double *st, int *iters) {
  int n = D->n, m = D->m, NS = D->NS, d = D->d;
  size_t blk = (size_t)n * m * NS;
  double *qh = st;                               /* [k][comp][node] */
  double *Fb = st + blk;                         /* [j][k][comp][node] */
  double *rhs = (double *)malloc(3 * blk * sizeof(double));
  if (!rhs) return ORC_ENOMEM;
  double *qn = rhs + blk;
  double *src = rhs + 2 * blk;                   /* point sources at the time nodes */
  int has_src = cell_sources(P, O, D, cell, t0, dt, src);
  double q[ORC_MAXM], f[ORC_MAXM];

  for (int k = 0; k < n; ++k)
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < NS; ++i) qh[((size_t)k * m + c) * NS + i] = u[c * NS + i];

  int R = P->picard > 0 ? P->picard : 64, it;
  for (it = 0; it < R; ++it) {
    /* fluxes at every space-time node */
    for (int k = 0; k < n; ++k)
      for (int i = 0; i < NS; ++i) {
        for (int c = 0; c < m; ++c) q[c] = qh[((size_t)k * m + c) * NS + i];
        for (int j = 0; j < d; ++j) {
          flux(P, cell, q, j, f);
          for (int c = 0; c < m; ++c) Fb[(((size_t)j * n + k) * m + c) * NS + i] = f[c];
        }
      }
    /* right-hand side: FL_k u - w_k dt div F */
    for (int k = 0; k < n; ++k)
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < NS; ++i) {
          double div = 0.0;
          for (int j = 0; j < d; ++j) {
            int ij = digit(i, j, n);
            double s = 0.0;
            for (int a = 0; a < n; ++a)
              s += O->Dm[ij * n + a] * Fb[(((size_t)j * n + k) * m + c) * NS + with_axis(i, j, a, n)];
            div += s / P->dx[j];
          }
          double sk = has_src ? src[((size_t)k * m + c) * NS + i] : 0.0;
          rhs[((size_t)k * m + c) * NS + i] = O->FL[k] * u[c * NS + i] - O->w[k] * dt * (div - sk);
        }
    /* solve along time with K1 */
    double diff = 0.0, nrm = 0.0;
    for (int k = 0; k < n; ++k)
      for (int c = 0; c < m; ++c)
        for (int i = 0; i < NS; ++i) {
          double s = 0.0;
          for (int l = 0; l < n; ++l) s += O->K1inv[k * n + l] * rhs[((size_t)l * m + c) * NS + i];
          size_t at = ((size_t)k * m + c) * NS + i;
          qn[at] = s;
          diff = fmax(diff, fabs(s - qh[at]));
          nrm = fmax(nrm, fabs(s));
        }
    memcpy(qh, qn, blk * sizeof(double));
    if (P->picard <= 0 && diff <= 1e-14 * fmax(1.0, nrm)) { ++it; break; }
  }
  if (iters) *iters = it;
  /* fluxes of the final iterate (output of predict, Table 1) */
  for (int k = 0; k < n; ++k)
    for (int i = 0; i < NS; ++i) {
      for (int c = 0; c < m; ++c) q[c] = qh[((size_t)k * m + c) * NS + i];
      for (int j = 0; j < d; ++j) {
        flux(P, cell, q, j, f);
        for (int c = 0; c < m; ++c) Fb[(((size_t)j * n + k) * m + c) * NS + i] = f[c];
      }
    }
  free(rhs);
  return ORC_OK;
}

/* Task extrapolate: q^ and F_j(q^) onto the 2d faces at every time node.
 * face layout: [f = 2j+side][0 = q, 1 = F_j][k][comp][face node]. */
static void extrapolate_cell(const orc_ops *O, const orc_dims *D, const double *st, double *face) {
  int n = D->n, m = D->m, NS = D->NS, NF = D->NF, d = D->d;
  size_t blk = (size_t)n * m * NS;
  for (int j = 0; j < d; ++j)
    for (int side = 0; side < 2; ++side) {
      const double *phi = side ? O->FR : O->FL;
      for (int v = 0; v < 2; ++v) {
        const double *src = v == 0 ? st : st + blk * (1 + j);
        double *dst = face + ((size_t)(2 * j + side) * 2 + v) * n * m * NF;
        for (int k = 0; k < n; ++k)
          for (int c = 0; c < m; ++c)
            for (int p = 0; p < NF; ++p) {
              double s = 0.0;
              for (int a = 0; a < n; ++a)
                s += phi[a] * src[((size_t)k * m + c) * NS + face_node_to_node(d, n, j, p, a)];
              dst[((size_t)k * m + c) * NF + p] = s;
            }
      }
    }
}

/* Task solveRiemann (Eq. 4, Rusanov) on the face normal to axis j between
 * cell cl (left, its side-1 data) and cr (right, its side-0 data).
 * fstar layout: [k][comp][face node].  With P->ncp the face instead yields
 * the path-conservative fluctuations: fstar = D- (for cl), fplus = D+ (for cr). */
static void riemann_face(const orc_cfg *P, const orc_ops *O, const orc_dims *D, int j, long cl,
                         const double *faceL, long cr, const double *faceR, double *fstar,
                         double *fplus) {
  int n = D->n, m = D->m, NF = D->NF;
  size_t fb = (size_t)n * m * NF;
  const double *qL = faceL + ((size_t)(2 * j + 1) * 2 + 0) * fb;
  const double *FLx = faceL + ((size_t)(2 * j + 1) * 2 + 1) * fb;
  const double *qR = faceR + ((size_t)(2 * j + 0) * 2 + 0) * fb;
  const double *FRx = faceR + ((size_t)(2 * j + 0) * 2 + 1) * fb;
  /* s: max spectral radius over face nodes and both sides, at the
   * time-averaged face states */
  double s = 0.0, qa[ORC_MAXM], qb[ORC_MAXM];
  for (int p = 0; p < NF; ++p) {
    for (int c = 0; c < m; ++c) {
      qa[c] = qb[c] = 0.0;
      for (int k = 0; k < n; ++k) {
        qa[c] += O->w[k] * qL[((size_t)k * m + c) * NF + p];
        qb[c] += O->w[k] * qR[((size_t)k * m + c) * NF + p];
      }
    }
    s = fmax(s, speed(P, cl, qa, j));
    s = fmax(s, speed(P, cr, qb, j));
  }
  if (P->ncp) {
    double dq[ORC_MAXM], ad[ORC_MAXM];
    for (int k = 0; k < n; ++k)
      for (int p = 0; p < NF; ++p) {
        for (int c = 0; c < m; ++c) {
          size_t at = ((size_t)k * m + c) * NF + p;
          dq[c] = qR[at] - qL[at];
        }
        path_jacobian_times(P, cl, cr, dq, j, ad);
        for (int c = 0; c < m; ++c) {
          size_t at = ((size_t)k * m + c) * NF + p;
          fstar[at] = 0.5 * (ad[c] - s * dq[c]);
          fplus[at] = 0.5 * (ad[c] + s * dq[c]);
        }
      }
    return;
  }
  for (int k = 0; k < n; ++k)
    for (int c = 0; c < m; ++c)
      for (int p = 0; p < NF; ++p) {
        size_t at = ((size_t)k * m + c) * NF + p;
        fstar[at] = 0.5 * (FLx[at] + FRx[at]) - 0.5 * s * (qR[at] - qL[at]);
      }
}

/* Tasks integrateVolume + integrateFace + update (Eq. 2) and the cell's
 * spectral radius for calcTimeStep.  fs_right[j] / fs_left[j] are the
 * space-time F* on the cell's right / left face normal to axis j; with
 * P->ncp they are the fluctuations D- of the right face and D+ of the left
 * face, and the volume term is in strong form.  Point sources add
 * dt sum_k w_k s(t0 + xi_k dt) sigma. */
static double correct_cell(const orc_cfg *P, const orc_ops *O, const orc_dims *D, long cell,
                           const double *st, const double *const *fs_right,
                           const double *const *fs_left, double dt, double t0, double *Qc) {
  int n = D->n, m = D->m, NS = D->NS, NF = D->NF, d = D->d;
  size_t blk = (size_t)n * m * NS;
  if (P->nsrc > 0) {
    double *src = (double *)malloc(blk * sizeof(double));
    if (src && cell_sources(P, O, D, cell, t0, dt, src))
      for (int k = 0; k < n; ++k)
        for (int c = 0; c < m; ++c)
          for (int i = 0; i < NS; ++i) Qc[c * NS + i] += dt * O->w[k] * src[((size_t)k * m + c) * NS + i];
    free(src);
  }
  if (P->ncp) {
    /* strong volume term -int phi_i B_j dq/dx_j (collocated; exact by GL) and
     * the face fluctuations */
    double dq[ORC_MAXM], f[ORC_MAXM];
    double *upd = (double *)calloc((size_t)m * NS, sizeof(double));
    if (!upd) return NAN;
    for (int i = 0; i < NS; ++i)
      for (int j = 0; j < d; ++j) {
        int ij = digit(i, j, n), p = node_to_face_node(d, n, j, i);
        for (int k = 0; k < n; ++k) {
          for (int c = 0; c < m; ++c) {
            double sum = 0.0;
            for (int a = 0; a < n; ++a) sum += O->Dm[ij * n + a] * st[((size_t)k * m + c) * NS + with_axis(i, j, a, n)];
            dq[c] = sum;
          }
          flux(P, cell, dq, j, f);   /* B_j dq (the flux is linear) */
          for (int c = 0; c < m; ++c) upd[c * NS + i] -= O->w[k] * f[c] / P->dx[j];
        }
        for (int c = 0; c < m; ++c) {
          double fr = 0.0, fl = 0.0;
          for (int k = 0; k < n; ++k) {
            fr += O->w[k] * fs_right[j][((size_t)k * m + c) * NF + p];
            fl += O->w[k] * fs_left[j][((size_t)k * m + c) * NF + p];
          }
          upd[c * NS + i] -= (O->FR[ij] * fr + O->FL[ij] * fl) / O->w[ij] / P->dx[j];
        }
      }
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < NS; ++i) Qc[c * NS + i] += dt * upd[c * NS + i];
    free(upd);
  } else
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < NS; ++i) {
      double upd = 0.0;
      for (int j = 0; j < d; ++j) {
        const double *Fj = st + blk * (1 + j);
        int ij = digit(i, j, n);
        double vol = 0.0;
        for (int k = 0; k < n; ++k)
          for (int a = 0; a < n; ++a)
            vol += O->w[k] * O->Kvol[ij * n + a] * Fj[((size_t)k * m + c) * NS + with_axis(i, j, a, n)];
        int p = node_to_face_node(d, n, j, i);
        double fr = 0.0, fl = 0.0;
        for (int k = 0; k < n; ++k) {
          fr += O->w[k] * fs_right[j][((size_t)k * m + c) * NF + p];
          fl += O->w[k] * fs_left[j][((size_t)k * m + c) * NF + p];
        }
        double face = (O->FR[ij] * fr - O->FL[ij] * fl) / O->w[ij];
        upd += (vol - face) / P->dx[j];
      }
      Qc[c * NS + i] += dt * upd;
    }
  double lam = 0.0, q[ORC_MAXM];
  for (int i = 0; i < NS; ++i) {
    for (int c = 0; c < m; ++c) q[c] = Qc[c * NS + i];
    for (int j = 0; j < d; ++j) {
      double s = speed(P, cell, q, j);
      if (!(s == s)) return s; /* NaN propagates to the caller */
      lam = fmax(lam, s);
    }
  }
  return lam;
}

static double lambda_cell(const orc_cfg *P, const orc_dims *D, long cell, const double *Qc) {
  double lam = 0.0, q[ORC_MAXM];
  for (int i = 0; i < D->NS; ++i) {
    for (int c = 0; c < D->m; ++c) q[c] = Qc[c * D->NS + i];
    for (int j = 0; j < D->d; ++j) {
      double s = speed(P, cell, q, j);
      if (!(s == s)) return s;
      lam = fmax(lam, s);
    }
  }
  return lam;
}

static double dt_admissible(const orc_cfg *P, double lam) {
  double h = P->dx[0];
  for (int a = 1; a < P->d; ++a) h = fmin(h, P->dx[a]);
  return h / (P->d * (2.0 * P->N + 1.0) * lam);
}

/* Largest spectral radius over all cells, nodes and axes. */
int orc_lambda(const orc_cfg *P, const double *Q, double *lam_out) {
  int rc = check_cfg(P);
  if (rc) return rc;
  orc_dims D = dims_of(P);
  double lam = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : lam) reduction(| : bad) schedule(static)
  for (long c = 0; c < D.C; ++c) {
    double l = lambda_cell(P, &D, c, Q + (size_t)c * D.m * D.NS);
    if (!(l == l) || isinf(l)) bad = 1;
    else lam = fmax(lam, l);
  }
  *lam_out = lam;
  return bad ? ORC_ENONFINITE : ORC_OK;
}

double orc_dt_admissible(const orc_cfg *P, double lam) { return dt_admissible(P, lam); }

/* ------------------------------------------------------------------------ */
/* Workspace for a whole-grid sweep                                          */

typedef struct {
  orc_dims D;
  orc_ops O;
  double *st;    /* [C][st_size] */
  double *face;  /* [C][face_size] */
  double *fstar; /* [d][C][n][m][NF], face between c and c+e_j stored at c (ncp: D-) */
  double *fplus; /* ncp: D+ of the same faces */
} orc_ws;

static int ws_init(const orc_cfg *P, orc_ws *W) {
  memset(W, 0, sizeof(*W));
  int rc = check_cfg(P);
  if (rc) return rc;
  W->D = dims_of(P);
  rc = make_ops(P->N, &W->O);
  if (rc) return rc;
  size_t fsz = (size_t)W->D.n * W->D.m * W->D.NF;
  W->st = (double *)malloc((size_t)W->D.C * W->D.st_size * sizeof(double));
  W->face = (double *)malloc((size_t)W->D.C * W->D.face_size * sizeof(double));
  W->fstar = (double *)malloc((size_t)W->D.d * W->D.C * fsz * sizeof(double));
  W->fplus = P->ncp ? (double *)malloc((size_t)W->D.d * W->D.C * fsz * sizeof(double)) : NULL;
  if (!W->st || !W->face || !W->fstar || (P->ncp && !W->fplus)) return ORC_ENOMEM;
  return ORC_OK;
}

static void ws_free(orc_ws *W) {
  free(W->st);
  free(W->face);
  free(W->fstar);
  free(W->fplus);
}

/* STP sweep: predict + extrapolate for every cell (Algorithm 1, first loop). */
static int sweep_stp(const orc_cfg *P, orc_ws *W, const double *Q, double dt, double t0, int *max_iters) {
  orc_dims *D = &W->D;
  int err = 0, mi = 0;
#pragma omp parallel for reduction(| : err) reduction(max : mi) schedule(dynamic, 4)
  for (long c = 0; c < D->C; ++c) {
    int it = 0;
    double *st = W->st + (size_t)c * D->st_size;
    err |= predict_cell(P, &W->O, D, c, Q + (size_t)c * D->m * D->NS, dt, t0, st, &it);
    extrapolate_cell(&W->O, D, st, W->face + (size_t)c * D->face_size);
    if (it > mi) mi = it;
  }
  if (max_iters) *max_iters = mi;
  return err ? ORC_ENOMEM : ORC_OK;
}

/* Riemann sweep: every face once (Algorithm 1, second loop). */
static void sweep_riemann(const orc_cfg *P, orc_ws *W) {
  orc_dims *D = &W->D;
  size_t fsz = (size_t)D->n * D->m * D->NF;
#pragma omp parallel for collapse(2) schedule(static)
  for (int j = 0; j < D->d; ++j)
    for (long c = 0; c < D->C; ++c) {
      long cr = neighbour(P, c, j, +1);
      riemann_face(P, &W->O, D, j, c, W->face + (size_t)c * D->face_size, cr,
                   W->face + (size_t)cr * D->face_size, W->fstar + ((size_t)j * D->C + c) * fsz,
                   W->fplus ? W->fplus + ((size_t)j * D->C + c) * fsz : NULL);
    }
}

/* Corrector sweep (Algorithm 1, third loop); returns lambda_max. */
static int sweep_correct(const orc_cfg *P, orc_ws *W, double *Q, double dt, double t0, double *lam_out) {
  orc_dims *D = &W->D;
  size_t fsz = (size_t)D->n * D->m * D->NF;
  double lam = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : lam) reduction(| : bad) schedule(static)
  for (long c = 0; c < D->C; ++c) {
    const double *fr[3], *fl[3];
    for (int j = 0; j < D->d; ++j) {
      fr[j] = W->fstar + ((size_t)j * D->C + c) * fsz;
      fl[j] = (W->fplus ? W->fplus : W->fstar) + ((size_t)j * D->C + neighbour(P, c, j, -1)) * fsz;
    }
    double l = correct_cell(P, &W->O, D, c, W->st + (size_t)c * D->st_size, fr, fl, dt, t0,
                            Q + (size_t)c * D->m * D->NS);
    if (!(l == l) || isinf(l)) bad = 1;
    else lam = fmax(lam, l);
  }
  *lam_out = lam;
  return bad ? ORC_ENONFINITE : ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Drivers                                                                   */

/* Algorithm 1 (left): nsteps straightforward steps.  The step size of step
 * k is dt_seq[k] if given, else fixed_dt if > 0, else C_dT * dt_adm of the
 * current solution (the first from the initial data).  dt_used[k] (may be
 * NULL) records the sizes; *t_inout is advanced; *max_iters (may be NULL)
 * reports the largest Picard count used. */
int orc_run(const orc_cfg *P, double *Q, int nsteps, const double *dt_seq, double fixed_dt,
            double *dt_used, double *t_inout, int *max_iters) {
  orc_ws W;
  int rc = ws_init(P, &W);
  if (rc) { ws_free(&W); return rc; }
  double dt = fixed_dt, lam = 0.0;
  if (!dt_seq && !(fixed_dt > 0.0)) {
    rc = orc_lambda(P, Q, &lam);
    if (rc) { ws_free(&W); return rc; }
    dt = P->cfl * dt_admissible(P, lam);
  }
  int mi = 0;
  double t = t_inout ? *t_inout : 0.0;
  for (int k = 0; k < nsteps; ++k) {
    if (dt_seq) dt = dt_seq[k];
    int it = 0;
    rc = sweep_stp(P, &W, Q, dt, t, &it);
    if (rc) break;
    if (it > mi) mi = it;
    sweep_riemann(P, &W);
    rc = sweep_correct(P, &W, Q, dt, t, &lam);
    if (dt_used) dt_used[k] = dt;
    t += dt;
    if (t_inout) *t_inout = t;
    if (rc) break;
    if (!dt_seq && !(fixed_dt > 0.0)) dt = P->cfl * dt_admissible(P, lam);
  }
  if (max_iters) *max_iters = mi;
  ws_free(&W);
  return rc;
}

/* Algorithm 2: shifted, fused, optimistic time stepping, executed with the
 * same task bodies (the oracle does not fuse; it only reproduces the order
 * and the time-step control).  policy 0 = strict dt_new = C dt_adm,
 * policy 1 = creeping average dt_new = (dt_old + C dt_adm)/2.
 * fixed_dt > 0 switches the control off.  If inject_step >= 1, dt_adm
 * computed in step inject_step is multiplied by inject_factor (host-side
 * fault injection for the rerun path).  dt_used[k] = step size of step k,
 * *reruns = number of STP reruns. */
int orc_run_shifted(const orc_cfg *P, double *Q, int nsteps, int policy, double fixed_dt,
                    int inject_step, double inject_factor, double *dt_used, int *reruns,
                    double *t_inout) {
  orc_ws W;
  int rc = ws_init(P, &W);
  if (rc) { ws_free(&W); return rc; }
  int nre = 0;
  double C = P->cfl, lam = 0.0, dt_adm, dt_old, dt_new;
  if (fixed_dt > 0.0) {
    dt_adm = INFINITY; /* control off: never a rerun */
    dt_new = fixed_dt;
  } else {
    rc = orc_lambda(P, Q, &lam);
    if (rc) { ws_free(&W); return rc; }
    dt_adm = dt_admissible(P, lam);
    dt_new = C * dt_adm;
  }
  /* first sweep: dt_old = 0, so only STP runs (Technique 3) */
  double t = t_inout ? *t_inout : 0.0;
  rc = sweep_stp(P, &W, Q, dt_new, t, NULL);
  for (int k = 0; k < nsteps && !rc; ++k) {
    if (!(fixed_dt > 0.0) && dt_adm < dt_new) {
      dt_old = dt_new = C * dt_adm; /* optimistic guess was wrong: rerun STP */
      rc = sweep_stp(P, &W, Q, dt_new, t, NULL);
      if (rc) break;
      ++nre;
    }
    dt_old = dt_new;
    if (fixed_dt > 0.0) dt_new = fixed_dt;
    else dt_new = policy == 1 ? 0.5 * (dt_old + C * dt_adm) : C * dt_adm;
    /* timeStep(dt_old, dt_new): Riemann + corrector with dt_old, then STP */
    sweep_riemann(P, &W);
    rc = sweep_correct(P, &W, Q, dt_old, t, &lam);
    if (dt_used) dt_used[k] = dt_old;
    t += dt_old;
    if (t_inout) *t_inout = t;
    if (rc) break;
    if (!(fixed_dt > 0.0)) {
      dt_adm = dt_admissible(P, lam);
      if (k + 1 == inject_step) dt_adm *= inject_factor;
    }
    if (k + 1 < nsteps) rc = sweep_stp(P, &W, Q, dt_new, t, NULL);
  }
  if (reruns) *reruns = nre;
  ws_free(&W);
  return rc;
}

/* One straightforward step (Algorithm 1) evaluated only for the listed
 * cells: predicts each listed cell and its 2d face neighbours, solves its
 * 2d Riemann problems and corrects it.  Used to check sampled cells of
 * grids too large for a whole oracle run.  Qout is [ncells][m][NS]. */
int orc_step_cells(const orc_cfg *P, const double *Q, double dt, double t0, const long *cells,
                   long ncells, double *Qout) {
  int rc = check_cfg(P);
  if (rc) return rc;
  orc_dims D = dims_of(P);
  orc_ops O;
  rc = make_ops(P->N, &O);
  if (rc) return rc;
  int err = 0;
#pragma omp parallel for reduction(| : err) schedule(dynamic, 1)
  for (long s = 0; s < ncells; ++s) {
    long c = cells[s];
    int d = D.d;
    size_t fsz = (size_t)D.n * D.m * D.NF;
    /* cells: self, then left/right neighbours per axis */
    long who[7];
    who[0] = c;
    for (int j = 0; j < d; ++j) {
      who[1 + 2 * j] = neighbour(P, c, j, -1);
      who[2 + 2 * j] = neighbour(P, c, j, +1);
    }
    int nw = 1 + 2 * d;
    double *st = (double *)malloc((size_t)nw * D.st_size * sizeof(double));
    double *face = (double *)malloc((size_t)nw * D.face_size * sizeof(double));
    double *fs = (double *)malloc((size_t)4 * d * fsz * sizeof(double));
    if (!st || !face || !fs) { err = 1; free(st); free(face); free(fs); continue; }
    for (int w = 0; w < nw; ++w) {
      int e = predict_cell(P, &O, &D, who[w], Q + (size_t)who[w] * D.m * D.NS, dt, t0,
                           st + (size_t)w * D.st_size, NULL);
      if (e) err = 1;
      extrapolate_cell(&O, &D, st + (size_t)w * D.st_size, face + (size_t)w * D.face_size);
    }
    const double *fr[3], *fl[3];
    for (int j = 0; j < d; ++j) {
      /* left face: F* (ncp: D- for the neighbour, D+ for this cell); right face: F* (ncp: D-) */
      double *left = fs + (size_t)(4 * j) * fsz, *left_p = fs + (size_t)(4 * j + 1) * fsz;
      double *right = fs + (size_t)(4 * j + 2) * fsz, *right_p = fs + (size_t)(4 * j + 3) * fsz;
      riemann_face(P, &O, &D, j, who[1 + 2 * j], face + (size_t)(1 + 2 * j) * D.face_size, c,
                   face, left, left_p);
      riemann_face(P, &O, &D, j, c, face, who[2 + 2 * j], face + (size_t)(2 + 2 * j) * D.face_size,
                   right, right_p);
      fl[j] = P->ncp ? left_p : left;
      fr[j] = right;
    }
    double *Qc = Qout + (size_t)s * D.m * D.NS;
    memcpy(Qc, Q + (size_t)c * D.m * D.NS, (size_t)D.m * D.NS * sizeof(double));
    correct_cell(P, &O, &D, c, st, fr, fl, dt, t0, Qc);
    free(st);
    free(face);
    free(fs);
  }
  return err ? ORC_ENOMEM : ORC_OK;
}

/* predict for a single cell (test access to Eq. 3).  qhat is
 * [k][comp][node]; *iters receives the Picard count. */
int orc_predict(const orc_cfg *P, long cell, const double *u, double dt, double t0, double *qhat,
                int *iters) {
  int rc = check_cfg(P);
  if (rc) return rc;
  orc_dims D = dims_of(P);
  orc_ops O;
  rc = make_ops(P->N, &O);
  if (rc) return rc;
  double *st = (double *)malloc(D.st_size * sizeof(double));
  if (!st) return ORC_ENOMEM;
  rc = predict_cell(P, &O, &D, cell, u, dt, t0, st, iters);
  memcpy(qhat, st, (size_t)D.n * D.m * D.NS * sizeof(double));
  free(st);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Receivers: point values of the nodal polynomial (Sec. 3 basis) at given   */
/* physical positions, for the components comps[0..nc-1].                    */
/* out[r][k] = sum_i prod_a phi_{i_a}(xi_{r,a}) Q[cell_r][comps[k]][i]       */

int orc_receivers(const orc_cfg *P, const double *Q, const double *pos, int R, const int *comps,
                  int nc, double *out) {
  int rc = check_cfg(P);
  if (rc) return rc;
  orc_dims D = dims_of(P);
  double xi[ORC_MAXN + 1], w[ORC_MAXN + 1];
  orc_gauss_legendre(P->N, xi, w);
  int n = D.n, d = D.d;
  for (int r = 0; r < R; ++r) {
    long cell = 0, stride = 1;
    double loc[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) {
      double x = pos[r * d + a] / P->dx[a];
      long ci = (long)floor(x);
      if (ci < 0) ci = 0;
      if (ci >= P->grid[a]) ci = P->grid[a] - 1;
      loc[a] = x - ci;
      cell += ci * stride;
      stride *= P->grid[a];
    }
    for (int k = 0; k < nc; ++k) {
      double s = 0.0;
      for (int i = 0; i < D.NS; ++i) {
        double wgt = 1.0;
        for (int a = 0; a < d; ++a) wgt *= lagrange(n, xi, digit(i, a, n), loc[a]);
        s += wgt * Q[((size_t)cell * D.m + comps[k]) * D.NS + i];
      }
      out[r * nc + k] = s;
    }
  }
  return ORC_OK;
}
