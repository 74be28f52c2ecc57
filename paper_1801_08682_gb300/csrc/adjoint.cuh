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
// then chained to (rho, cp, cs).  adj_faces_lin_kernel forms the per-cell halves
// of Phi (psi); adj_lin_kernel does the rest for one tile of cells (both in
// adj_lin.cuh).
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
  float scf[3];          // dt / dx_j rounded to FP32 (the FP32 kernels' operator scale)
};

// dt / dx_j in the kernel type R (FP32 kernels take the host-rounded copy: FP64
// arithmetic is slow on this part)
template <class R>
__device__ __forceinline__ R adj_scale(const AdjArgs &a, int j) {
  if constexpr (sizeof(R) == 4) return a.scf[j];
  else return (R)(a.dt * a.inv_dx[j]);
}

}  // namespace aderdg
