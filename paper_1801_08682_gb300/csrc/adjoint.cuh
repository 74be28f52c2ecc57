// adjoint.cuh -- discrete adjoint of one ADER-DG step for linear fluxes.
//
// Forward step (fixed dt, F_j = A_j(theta_c) q in cell c, h_j = 1/dx_j):
//   qbar_c = P_c u_c,  P_c = sum_{s<=R} g_s Lt_c^s,  Lt_c = -dt sum_j h_j A_j D_j
//            (Horner: v_R = g_R u, v_s = g_s u + Lt v_{s+1}, qbar = v_0)
//   D_c    = dt sum_j h_j A_j Kvol_j qbar_c                       (integrateVolume)
//   q_f    = E_f qbar_c  on the 2d faces                           (extrapolate)
//   F*_j   = 1/2 A^L q_L + 1/2 A^R q_R - 1/2 s (q_R - q_L)         (Rusanov, s = max speed)
//   Q'_c   = u_c + D_c - dt sum_j h_j [W_R F*_{j,right} - W_L F*_{j,left}],
//            W_R = FR/w, W_L = FL/w spread along axis j             (integrateFace)
// Adjoint (lam = dJ/dQ'), term by term in reverse:
//   Phi_face = -dt h_j W_R^T lam_left-cell + dt h_j W_L^T lam_right-cell
//   q*_L = (1/2 A^L^T + s/2) Phi,   q*_R = (1/2 A^R^T - s/2) Phi
//   qbar*_c = sum_f E_f^T q*_f + dt sum_j h_j Kvol_j^T A_j^T lam_c
//   lam_c  <- lam_c + P_c^T qbar*_c,  P_c^T = sum_s g_s (Lt_c^T)^s
// Material gradient (the flux is linear in theta = (lambda, mu, 1/rho)):
//   <lam, dt sum_j h_j dA_j Kvol_j qbar>  +  sum_{s<R} <(Lt^T)^s qbar*, dLt v_{s+1}>
//   + sum_faces <Phi, 1/2 dA q_own>  - 1/2 ds/dcp <Phi, q_R - q_L>   (s = max(cp_L, cp_R),
//   the derivative goes to the side that attains the max, the left one on a tie)
// then chained to (rho, cp, cs).  adj_faces_kernel forms the per-cell halves of
// Phi (psi), adj_cell_kernel does the rest for one tile of cells.
#pragma once
#include "sweep.cuh"

namespace aderdg {

struct AdjArgs {
  const void *lam_in;    // R  [C][m][NS]  dJ/dQ after the step
  void *lam_out;         // R  [C][m][NS]  dJ/dQ before the step
  const void *Qk;        // QT [C][m][NS]  state before the step
  const void *hull;      // R  q_bar on the faces of Qk's predictor (line-owner layout, stride hsl)
  void *psi;             // R  [C][2d][m][NF]
  const float *mat;      // [C][3] or nullptr
  double *gmat;          // [C][3] += dJ/d(rho, cp, cs); nullptr = not wanted
  const void *tables;    // Tables<R> in global memory
  long long ncells;
  int grid[3];
  int picard;
  int hsl, fsz;
  double inv_dx[3];
  double cst[8];
  double dt;
  const void *htab;      // host copy of Tables<R> (passed to the cell kernel by value)
  const void *htabT;     // the same built from Dm^T and Kvol^T
  void *zs;              // R scratch of the forward powers: zs_blocks blocks x (picard - 1) levels
  long long zs_blocks;
  const void *matp;      // MatBox<PDE::Mat> per cell (mat set) or one entry, or nullptr
};

// cells per block of adj_faces_kernel: about 256 face items
template <class K>
constexpr int adj_faces_cells() {
  return cmax(1, 256 / (2 * K::d * K::m * K::NF));
}

// psi[c][f][comp][p] = (side ? -1 : +1) dt h_j sum_a (side ? FR_a : FL_a)/w_a lam_c(node(p, j, a))
template <class K>
__global__ void __launch_bounds__(256) adj_faces_kernel(const AdjArgs a) {
  using R = typename K::R;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  __shared__ R wl[kMaxn], wr[kMaxn];
  const Tables<R> *T = reinterpret_cast<const Tables<R> *>(a.tables);
  if (threadIdx.x < n) {
    wl[threadIdx.x] = T->FL[threadIdx.x] * T->iw[threadIdx.x];
    wr[threadIdx.x] = T->FR[threadIdx.x] * T->iw[threadIdx.x];
  }
  __syncthreads();
  const R *lam = reinterpret_cast<const R *>(a.lam_in);
  R *psi = reinterpret_cast<R *>(a.psi);
  R sc[3];   // dt / dx_j, once (FP64 arithmetic is slow on this part)
#pragma unroll
  for (int j = 0; j < 3; ++j) sc[j] = (R)(a.dt * a.inv_dx[j]);
  // a block per FCPB cells (grid-stride over cell groups), its threads over
  // (cell, face, comp, face node): 32-bit index arithmetic by compile-time
  // constants
  constexpr int PER_CELL = 2 * d * m * NF;
  constexpr int FCPB = adj_faces_cells<K>();
  for (long long c0 = (long long)blockIdx.x * FCPB; c0 < a.ncells; c0 += (long long)gridDim.x * FCPB) {
    for (int it = threadIdx.x; it < FCPB * PER_CELL; it += blockDim.x) {
      const int lc = it / PER_CELL, r = it - lc * PER_CELL;
      const long long cell = c0 + lc;
      if (cell >= a.ncells) break;
      const int f = r / (m * NF), c = (r / NF) % m, p = r % NF;
      const int j = f >> 1, side = f & 1;
      const R *src = lam + (cell * m + c) * NS;
      R s = R(0);
#pragma unroll
      for (int b = 0; b < n; ++b) s += (side ? wr[b] : wl[b]) * src[I::node_of_face(p, j, b)];
      const R scj = j == 0 ? sc[0] : (j == 1 ? sc[1] : sc[2]);
      psi[cell * PER_CELL + r] = (side ? R(-1) : R(1)) * scj * s;
    }
  }
}

// Shared elements per cell: lambda, w, the face adjoints and, for the material
// gradient only, the forward Horner states v_0..v_R.
template <class K>
constexpr int adj_cell_elems(int picard, bool with_vh = true) {
  return (with_vh ? (picard + 1) * K::m * K::NS : 0) + 2 * K::m * K::NS + 2 * K::d * K::m * K::NF;
}

template <class K>
size_t adj_cell_smem(int picard, bool with_vh) {
  return tables_bytes<typename K::R>() + 4 * K::CPB * sizeof(double) +
         (size_t)K::CPB * adj_cell_elems<K>(picard, with_vh) * sizeof(typename K::R);
}

template <class K>
__global__ void __launch_bounds__(K::THREADS) adj_cell_kernel(const AdjArgs a) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, CPB = K::CPB;
  constexpr int THREADS = K::THREADS;
  constexpr int NMAT = PDE::NMAT;
  extern __shared__ __align__(16) unsigned char smem[];
  Tables<R> &T = *reinterpret_cast<Tables<R> *>(smem);
  double *red = reinterpret_cast<double *>(smem + tables_bytes<R>());  // [CPB][4]
  R *base = reinterpret_cast<R *>(red + 4 * CPB);
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.tables);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(Tables<R>) / 4); i += THREADS) dst[i] = src[i];
    for (int i = threadIdx.x; i < 4 * CPB; i += THREADS) red[i] = 0.0;
  }
  const int Rp = a.picard;
  // the forward Horner states enter only the material gradient
  const bool gm = NMAT && a.gmat;
  const int cell_elems = adj_cell_elems<K>(Rp, gm);
  const R dt = (R)a.dt;
  R h[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) h[j] = (R)a.inv_dx[j];
  const int tid = threadIdx.x;
  const int lc = tid / NS, node = tid - lc * NS;
  const int lcs = lc < CPB ? lc : CPB - 1;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool active = lc < CPB && cell < a.ncells;
  R *LAM = base + lcs * cell_elems;       // [m][NS]
  R *W = LAM + m * NS;                    // [m][NS]
  R *QSF = W + m * NS;                    // [2d][m][NF]
  R *VH = QSF + 2 * d * m * NF;           // [R+1][m][NS]
  const QT *Qk = reinterpret_cast<const QT *>(a.Qk);
  const R *lam_in = reinterpret_cast<const R *>(a.lam_in);
  R *lam_out = reinterpret_cast<R *>(a.lam_out);
  const R *psi = reinterpret_cast<const R *>(a.psi);
  const R *hull = reinterpret_cast<const R *>(a.hull);
  __syncthreads();

  typename PDE::Mat mt;
  PDE::load(mt, a.cst, a.mat, active ? cell : 0);
  R u[m], lamv[m];
  R g[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int c = 0; c < m; ++c) {
    u[c] = active && gm ? (R)Qk[(cell * m + c) * NS + node] : R(0);
    lamv[c] = active ? lam_in[(cell * m + c) * NS + node] : R(0);
    if (active) LAM[c * NS + node] = lamv[c];
  }

  // ---- forward Horner intermediates of this cell's predictor (material gradient)
  if (gm) {
    R v[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      v[c] = T.g[Rp] * u[c];
      if (active) VH[(Rp * m + c) * NS + node] = v[c];
    }
  }
  __syncthreads();
  for (int s = gm ? Rp - 1 : -1; s >= 0; --s) {
    if (active) {
      const R *Vn = VH + (s + 1) * m * NS;
      R Lv[m];
#pragma unroll
      for (int c = 0; c < m; ++c) Lv[c] = R(0);
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int ij = I::digit(node, j);
        R dv[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          dv[c] = R(0);
          if (PDE::reads(j, c)) {
#pragma unroll
            for (int b = 0; b < n; ++b) dv[c] += T.Dm[ij * n + b] * Vn[c * NS + I::with_axis(node, j, b)];
          }
        }
        PDE::applyA(mt, j, dv, out);
#pragma unroll
        for (int c = 0; c < m; ++c) Lv[c] += h[j] * out[c];
      }
#pragma unroll
      for (int c = 0; c < m; ++c) VH[(s * m + c) * NS + node] = T.g[s] * u[c] - dt * Lv[c];
    }
    __syncthreads();
  }

  // ---- face adjoints: Phi on each face of the tile's cells, q* of the own side
  for (int it = tid; it < CPB * 2 * d * NF; it += THREADS) {
    const int lc2 = it / (2 * d * NF);
    const int f = (it / NF) % (2 * d);
    const int p = it % NF;
    const long long cell2 = (long long)blockIdx.x * CPB + lc2;
    if (cell2 >= a.ncells) continue;
    const int j = f >> 1, side = f & 1;
    const long long nb = neighbour(cell2, j, side ? 1 : -1, a.grid);
    typename PDE::Mat m2, mn;
    PDE::load(m2, a.cst, a.mat, cell2);
    PDE::load(mn, a.cst, a.mat, nb);
    R phi[m], qc[m], at[m];
#pragma unroll
    for (int c = 0; c < m; ++c)
      phi[c] = psi[((cell2 * 2 * d + f) * m + c) * NF + p] + psi[((nb * 2 * d + (f ^ 1)) * m + c) * NF + p];
    const R s2 = PDE::speed(m2, phi, j), sn = PDE::speed(mn, phi, j);  // linear: state-independent
    const R s = s2 > sn ? s2 : sn;
    PDE::applyAT(m2, j, phi, at);
    R *dst = base + lc2 * cell_elems + 2 * m * NS;  // QSF of cell lc2
#pragma unroll
    for (int c = 0; c < m; ++c) dst[(f * m + c) * NF + p] = R(0.5) * at[c] + (side ? R(0.5) : R(-0.5)) * s * phi[c];
    if (NMAT && a.gmat) {
      R qn[m], gl[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
      for (int c = 0; c < m; ++c) {
        qc[c] = hull[cell2 * a.hsl + f * a.fsz + c * NF + p];
        qn[c] = hull[nb * a.hsl + (f ^ 1) * a.fsz + c * NF + p];
      }
      PDE::dA(m2, j, phi, qc, gl);
      const bool selected = side ? (s2 >= sn) : (s2 > sn);
      R gs = R(0);
      if (selected) {
#pragma unroll
        for (int c = 0; c < m; ++c) gs += phi[c] * (side ? (qn[c] - qc[c]) : (qc[c] - qn[c]));
      }
      atomicAdd(&red[lc2 * 4 + 0], (double)(R(0.5) * gl[0]));
      atomicAdd(&red[lc2 * 4 + 1], (double)(R(0.5) * gl[1]));
      atomicAdd(&red[lc2 * 4 + 2], (double)(R(0.5) * gl[2]));
      atomicAdd(&red[lc2 * 4 + 3], (double)(R(-0.5) * gs));
    }
  }
  __syncthreads();

  // ---- qbar* at this node: E^T of the face adjoints + Kvol^T A^T lam
  R qbs[m];
#pragma unroll
  for (int c = 0; c < m; ++c) qbs[c] = R(0);
  if (active) {
#pragma unroll
    for (int j = 0; j < d; ++j) {
      const int ij = I::digit(node, j), p = I::face_node(node, j);
#pragma unroll
      for (int c = 0; c < m; ++c)
        qbs[c] += T.FL[ij] * QSF[((2 * j) * m + c) * NF + p] + T.FR[ij] * QSF[((2 * j + 1) * m + c) * NF + p];
      R kt[m], out[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R sacc = R(0);
#pragma unroll
        for (int b = 0; b < n; ++b) sacc += T.Kvol[b * n + ij] * LAM[c * NS + I::with_axis(node, j, b)];
        kt[c] = sacc;
      }
      PDE::applyAT(mt, j, kt, out);
#pragma unroll
      for (int c = 0; c < m; ++c) qbs[c] += dt * h[j] * out[c];
      if (NMAT && a.gmat) {  // volume term: <lam, dt h_j dA_j Kvol_j qbar>
        R kq[m], gl[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R sacc = R(0);
#pragma unroll
          for (int b = 0; b < n; ++b) sacc += T.Kvol[ij * n + b] * VH[c * NS + I::with_axis(node, j, b)];
          kq[c] = sacc;
        }
        PDE::dA(mt, j, lamv, kq, gl);
#pragma unroll
        for (int k = 0; k < 3; ++k) g[k] += dt * h[j] * gl[k];
      }
    }
  }

  // ---- adjoint Horner: w_0 = qbar*, w_{s+1} = Lt^T w_s, lam += sum_s g_s w_s
  R acc[m];
#pragma unroll
  for (int c = 0; c < m; ++c) {
    acc[c] = T.g[0] * qbs[c];
    if (active) W[c * NS + node] = qbs[c];
  }
  __syncthreads();
  for (int s = 0; s < Rp; ++s) {
    R wn[m];
#pragma unroll
    for (int c = 0; c < m; ++c) wn[c] = R(0);
    if (active) {
      R ws[m];
#pragma unroll
      for (int c = 0; c < m; ++c) ws[c] = W[c * NS + node];
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int ij = I::digit(node, j);
        R dtw[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R sacc = R(0);
#pragma unroll
          for (int b = 0; b < n; ++b) sacc += T.Dm[b * n + ij] * W[c * NS + I::with_axis(node, j, b)];
          dtw[c] = sacc;
        }
        PDE::applyAT(mt, j, dtw, out);
#pragma unroll
        for (int c = 0; c < m; ++c) wn[c] -= dt * h[j] * out[c];
        if (NMAT && a.gmat) {  // <w_s, dLt v_{s+1}>, dLt = -dt h_j dA_j D_j
          const R *Vn = VH + (s + 1) * m * NS;
          R dv[m], gl[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
          for (int c = 0; c < m; ++c) {
            R sacc = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) sacc += T.Dm[ij * n + b] * Vn[c * NS + I::with_axis(node, j, b)];
            dv[c] = sacc;
          }
          PDE::dA(mt, j, ws, dv, gl);
#pragma unroll
          for (int k = 0; k < 3; ++k) g[k] -= dt * h[j] * gl[k];
        }
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c) W[c * NS + node] = wn[c];
    }
#pragma unroll
    for (int c = 0; c < m; ++c) acc[c] += T.g[s + 1] * wn[c];
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int c = 0; c < m; ++c) lam_out[(cell * m + c) * NS + node] = lamv[c] + acc[c];
  }

  // ---- material gradient of the tile's cells, chained to (rho, cp, cs)
  if (NMAT && a.gmat) {
    if (active) {
#pragma unroll
      for (int k = 0; k < 3; ++k) atomicAdd(&red[lc * 4 + k], (double)g[k]);
    }
    __syncthreads();
    if (tid < CPB) {
      const long long c2 = (long long)blockIdx.x * CPB + tid;
      if (c2 < a.ncells && a.mat) {
        const double rho = a.mat[3 * c2], cp = a.mat[3 * c2 + 1], cs = a.mat[3 * c2 + 2];
        const double gl = red[tid * 4 + 0], gm = red[tid * 4 + 1], gi = red[tid * 4 + 2], gs = red[tid * 4 + 3];
        a.gmat[3 * c2 + 0] += gl * (cp * cp - 2.0 * cs * cs) + gm * cs * cs - gi / (rho * rho);
        a.gmat[3 * c2 + 1] += gl * 2.0 * rho * cp + gs;
        a.gmat[3 * c2 + 2] += -4.0 * rho * cs * gl + 2.0 * rho * cs * gm;
      }
    }
  }
}

}  // namespace aderdg
