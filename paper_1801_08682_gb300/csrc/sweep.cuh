// sweep.cuh -- the cell sweep of the single-touch ADER-DG step (Alg. 2,
// function timeStep) and its bookends, as one kernel template.
//
// A block owns a tile of CPB consecutive cells, one thread per (cell, node).
// Stages (compile-time):
//   kCorrect   solveRiemann on the cell's 2d faces from the time-averaged
//              hull (each face is solved by both neighbours, the GPU form of
//              Technique 2), integrateFace + update (Eq. 2) with dt_old,
//              calcTimeStep as a block max folded into one atomic.
//   kPredict   predict (Eq. 3) with dt_new, integrateVolume into D
//              (Technique 1), extrapolate the time-averaged q and F_j to the
//              2d faces of the cell.
//   kFused     kCorrect then kPredict on the same registers (Technique 4):
//              the corrected Q never leaves the chip before the predictor.
//   kCorrectFs integrateFace + update from a stored F* (three-sweep form).
// Two predictor forms:
//   kSpaceTime the Picard iteration of Eq. 3 on the full space-time
//              polynomial: fluxes at all (N+1)^{d+1} nodes, d derivative
//              contractions, the K1^{-1} solve along time.
//   kTimeModal linear fluxes only.  With F_j(q) = A_j q and K1^{-1} FL = 1,
//              R Picard iterations started from q^0 = u give exactly
//                q^R = sum_{s=0}^{R} (-dt)^s c_s (x) L^s u,
//                c_s = (K1^{-1} W)^s 1,  L = sum_j (1/dx_j) A_j D_j,
//              so the time average is q_bar = sum_s (-dt)^s g_s L^s u with
//              g_s = w . c_s (Horner form below) and F_bar_j = A_j q_bar.
//              Same iterates, but the derivative contractions act on the
//              (N+1)^d spatial nodes instead of (N+1)^{d+1} space-time nodes.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "pde.cuh"
#include "sweep_lin.cuh"
#include "tc.cuh"

namespace aderdg {

template <template <int, class> class PDEt, int d_, int N_, class R_, class QT_, int PRED_>
struct Cfg {
  using R = R_;
  using QT = typename QStore<QT_>::T;         // element type of the state
  static constexpr bool PAIR = QStore<QT_>::PAIR;  // a low-word plane follows the states
  using PDE = PDEt<d_, R_>;
  using Lin = LinCfg<PDEt, d_, N_, R_, QT_>;  // line-owner kernel of the same configuration
  static constexpr int d = d_, N = N_, n = N_ + 1, m = PDE::M, PRED = PRED_;
  static constexpr int NS = ipow(n, d), NF = ipow(n, d - 1);
  static constexpr int CPB = cmax(1, 256 / NS);              // cells per block
  static constexpr int THREADS = round_up(CPB * NS, 32);
  static constexpr int HS = round_up(2 * d * 2 * m * NF, 4); // hull stride per cell
  static constexpr int FB = 2 * m * NF;                      // one face-side block
  static constexpr int FITEMS = CPB * 2 * d * NF;            // face items per tile
  static constexpr int FPT = (FITEMS + THREADS - 1) / THREADS;
  static constexpr int SMAX = round_up(CPB * 2 * d, 4);
  // work area (elements of R): max of F* (corrector) and the predictor buffers
  static constexpr int FS_ELEMS = CPB * 2 * d * m * NF;
  static constexpr int PRED_ELEMS =
      CPB * m * NS + (PRED != kTimeModal ? CPB * d * n * m * NS : 0);
  static constexpr int WORK = cmax(FS_ELEMS, PRED_ELEMS);
  // space-time predictor: dt K1^{-1} diag(w) and its row sums, for the launch
  static constexpr int DTM = PRED != kTimeModal ? round_up(n * n + n, 4) : 0;
  static_assert(THREADS >= n * n, "one thread per entry of dt K1^{-1} diag(w)");
  static constexpr size_t SMEM =
      tables_bytes<R>() + 32 * sizeof(unsigned long long) + (size_t)(SMAX + DTM + WORK) * sizeof(R);
  // nonlinear PDEs: ask for three blocks per SM where the shared memory allows it
  static constexpr int MINB = (!PDE::LINEAR && 3 * (SMEM + 1024) <= 227 * 1024) ? 3 : 1;
};

template <class K, int STAGES>
__device__ __forceinline__ void sweep_body(const SweepArgs &a) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, CPB = K::CPB;
  constexpr int THREADS = K::THREADS;

  extern __shared__ __align__(16) unsigned char smem[];
  Tables<R> &T = *reinterpret_cast<Tables<R> *>(smem);
  unsigned long long *sred = reinterpret_cast<unsigned long long *>(smem + tables_bytes<R>());
  R *smax = reinterpret_cast<R *>(sred + 32);
  R *dtM = smax + K::SMAX;  // [n][n] dt K1^{-1}[k][l] w_l, then [n] row sums
  R *work = dtM + K::DTM;

  DevCtl *ctl = a.ctl;
  if (STAGES == kPredict && a.gate) {
    if (*(volatile int *)&ctl->rerun == 0) return;  // uniform for the whole grid
  }
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.tables);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(Tables<R>) / 4); i += THREADS) dst[i] = src[i];
  }
  const R dt_old = (R)ctl->dt_old;
  const R dt_pred = (R)(a.pred_dt_old ? ctl->dt_old : ctl->dt_new);
  if constexpr (K::PRED != kTimeModal) {
    // K1 1 = FL (FR sums to one; GL integrates phi_k' exactly), so K1^{-1} FL = 1
    // and a Picard iterate is q_hat_k = u - sum_l dt K1^{-1}[k][l] w_l div_l
    const Tables<R> *Tg = reinterpret_cast<const Tables<R> *>(a.tables);
    const int t = threadIdx.x;
    if (t < n * n) dtM[t] = dt_pred * Tg->K1inv[t] * Tg->w[t % n];
    if (t < n) {
      R sum = R(0);
      for (int l = 0; l < n; ++l) sum += dt_pred * Tg->K1inv[t * n + l] * Tg->w[l];
      dtM[n * n + t] = sum;
    }
  }
  const QT *Qin = reinterpret_cast<const QT *>(a.Q_in);
  QT *Qout = reinterpret_cast<QT *>(a.Q_out);
  R *Dbuf = reinterpret_cast<R *>(a.Dbuf);
  const R *hin = reinterpret_cast<const R *>(a.hull_in);
  R *hout = reinterpret_cast<R *>(a.hull_out);
  R inv_dx[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) inv_dx[j] = (R)a.inv_dx[j];
  __syncthreads();

  const int tid = threadIdx.x;
  const int lc = tid / NS;
  const int node = tid - lc * NS;
  const int lcs = lc < CPB ? lc : CPB - 1;  // padding threads read in-bounds shared memory

  for (long long tile = a.tile_lo + blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
    const long long cell = tile * CPB + lc;
    const bool active = lc < CPB && cell < a.ncells;
    typename PDE::Mat mt;
    load_mat<PDE>(mt, a.matp, a.cst, a.mat, active ? cell : 0);
    R u[m];
    QT qold[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      qold[c] = active ? Qin[(cell * m + c) * NS + node] : QT(0);
      u[c] = (R)qold[c];
    }

    // ------------------------------------------------------------ corrector
    if (STAGES == kCorrect || STAGES == kFused || STAGES == kCorrectFs) {
      R *Fs = work;  // [CPB][2d][m][NF]
      if (STAGES == kCorrectFs) {
        const R *fst = reinterpret_cast<const R *>(a.fstar);
        for (int it = tid; it < CPB * 2 * d * m * NF; it += THREADS) {
          const int lc2 = it / (2 * d * m * NF);
          const int f = (it / (m * NF)) % (2 * d);
          const int cp = it % (m * NF);
          const long long cell2 = tile * CPB + lc2;
          if (cell2 >= a.ncells) continue;
          const int j = f >> 1;
          const long long owner = (f & 1) ? cell2 : neighbour(cell2, j, -1, a.grid);
          Fs[it] = fst[((long long)j * a.ncells + owner) * (m * NF) + cp];
        }
      } else {
        for (int i = tid; i < CPB * 2 * d; i += THREADS) smax[i] = R(0);
        __syncthreads();
        R qL[K::FPT][m], qR[K::FPT][m], fL[K::FPT][m], fR[K::FPT][m];
#pragma unroll
        for (int r = 0; r < K::FPT; ++r) {
          const int it = tid + r * THREADS;
          const int lc2 = it / (2 * d * NF);
          const int f = (it / NF) % (2 * d);
          const int p = it % NF;
          const long long cell2 = tile * CPB + lc2;
          if (it < K::FITEMS && cell2 < a.ncells) {
            const int j = f >> 1, side = f & 1;
            const long long nb = neighbour(cell2, j, side ? 1 : -1, a.grid);
            const R *own = hin + cell2 * K::HS + f * K::FB;
            const R *nbr = hin + nb * K::HS + (f ^ 1) * K::FB;
            const R *Lp = side ? own : nbr;
            const R *Rp = side ? nbr : own;
#pragma unroll
            for (int c = 0; c < m; ++c) {
              qL[r][c] = ldg(Lp + c * NF + p);
              fL[r][c] = ldg(Lp + (m + c) * NF + p);
              qR[r][c] = ldg(Rp + c * NF + p);
              fR[r][c] = ldg(Rp + (m + c) * NF + p);
            }
            typename PDE::Mat mL, mR;
            load_mat<PDE>(mL, a.matp, a.cst, a.mat, side ? cell2 : nb);
            load_mat<PDE>(mR, a.matp, a.cst, a.mat, side ? nb : cell2);
            const R s = nanmax(PDE::speed(mL, qL[r], j), PDE::speed(mR, qR[r], j));
            smem_max(&smax[lc2 * 2 * d + f], s);
          }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < K::FPT; ++r) {
          const int it = tid + r * THREADS;
          const int lc2 = it / (2 * d * NF);
          const int f = (it / NF) % (2 * d);
          const int p = it % NF;
          const long long cell2 = tile * CPB + lc2;
          if (it < K::FITEMS && cell2 < a.ncells) {
            const R s = smax[lc2 * 2 * d + f];
#pragma unroll
            for (int c = 0; c < m; ++c)
              Fs[((lc2 * 2 * d + f) * m + c) * NF + p] =
                  R(0.5) * (fL[r][c] + fR[r][c]) - R(0.5) * s * (qR[r][c] - qL[r][c]);
          }
        }
      }
      __syncthreads();

      R lam = R(0);
      if (active) {
        R acc[m];
#pragma unroll
        for (int c = 0; c < m; ++c) acc[c] = Dbuf[(cell * m + c) * NS + node];
#pragma unroll
        for (int j = 0; j < d; ++j) {
          const int ij = I::digit(node, j), p = I::face_node(node, j);
          const R cr = dt_old * inv_dx[j] * T.FR[ij] * T.iw[ij];
          const R cl = dt_old * inv_dx[j] * T.FL[ij] * T.iw[ij];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            const R fr = Fs[((lc * 2 * d + 2 * j + 1) * m + c) * NF + p];
            const R fl = Fs[((lc * 2 * d + 2 * j) * m + c) * NF + p];
            acc[c] -= cr * fr - cl * fl;
          }
        }
        R chk = R(0);
#pragma unroll
        for (int c = 0; c < m; ++c) {
          QT qn;
          if constexpr (K::PAIR) {
            // compensated FP32 pair: the low words sit one state plane further on
            QT *lop = Qout + (a.ncells + cell) * m * NS + c * NS + node;
            QT lo = *lop;
            qn = qold[c];
            pair_add(qn, lo, acc[c]);
            *lop = lo;
          } else {
            qn = qold[c] + (QT)acc[c];
          }
          Qout[(cell * m + c) * NS + node] = qn;
          u[c] = (R)qn;
          chk += u[c] * R(0);  // NaN/Inf in any variable survives
        }
#pragma unroll
        for (int j = 0; j < d; ++j) lam = nanmax(lam, PDE::speed(mt, u, j));
        lam += chk;
      }
      block_lambda_max<THREADS>(lam_bits(lam), sred, ctl);
      __syncthreads();  // F* consumed; the work area is free for the predictor
    }

    // ------------------------------------------------------------ predictor
    if (STAGES == kPredict || STAGES == kFused) {
      R *V = work;  // [CPB][m][NS] time-averaged q
      R qb[m];
      if (K::PRED == kTimeModal) {
        // Horner form of q_bar = sum_s g_s (-dt L)^s u
        const int Rp = a.picard;
#pragma unroll
        for (int c = 0; c < m; ++c) qb[c] = T.g[Rp] * u[c];
        for (int s = Rp - 1; s >= 0; --s) {
          if (active) {
#pragma unroll
            for (int c = 0; c < m; ++c) V[(lc * m + c) * NS + node] = qb[c];
          }
          __syncthreads();
          R Lv[m];
#pragma unroll
          for (int c = 0; c < m; ++c) Lv[c] = R(0);
          if (active) {
#pragma unroll
            for (int j = 0; j < d; ++j) {
              const int ij = I::digit(node, j);
              R dv[m], out[m];
#pragma unroll
              for (int c = 0; c < m; ++c) {
                dv[c] = R(0);
                if (PDE::reads(j, c)) {
#pragma unroll
                  for (int b = 0; b < n; ++b)
                    dv[c] += T.Dm[ij * n + b] * V[(lc * m + c) * NS + I::with_axis(node, j, b)];
                }
              }
              PDE::applyA(mt, j, dv, out);
#pragma unroll
              for (int c = 0; c < m; ++c) Lv[c] += inv_dx[j] * out[c];
            }
          }
          __syncthreads();
#pragma unroll
          for (int c = 0; c < m; ++c) qb[c] = T.g[s] * u[c] - dt_pred * Lv[c];
        }
        if (active) {
#pragma unroll
          for (int c = 0; c < m; ++c) V[(lc * m + c) * NS + node] = qb[c];
        }
        __syncthreads();
        // integrateVolume: D = dt sum_j (1/dx_j) A_j (Kvol_j q_bar)
        R Dacc[m];
#pragma unroll
        for (int c = 0; c < m; ++c) Dacc[c] = R(0);
#pragma unroll
        for (int j = 0; j < d; ++j) {
          const int ij = I::digit(node, j);
          R kv[m], out[m];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            kv[c] = R(0);
            if (PDE::reads(j, c)) {
#pragma unroll
              for (int b = 0; b < n; ++b)
                kv[c] += T.Kvol[ij * n + b] * V[(lcs * m + c) * NS + I::with_axis(node, j, b)];
            }
          }
          PDE::applyA(mt, j, kv, out);
#pragma unroll
          for (int c = 0; c < m; ++c) Dacc[c] += inv_dx[j] * out[c];
        }
        if (active) {
#pragma unroll
          for (int c = 0; c < m; ++c) Dbuf[(cell * m + c) * NS + node] = dt_pred * Dacc[c];
        }
        // extrapolate q_bar; F_bar_j . e_j = A_j q_bar on the face
        for (int it = tid; it < K::FITEMS; it += THREADS) {
          const int lc2 = it / (2 * d * NF);
          const int f = (it / NF) % (2 * d);
          const int p = it % NF;
          const long long cell2 = tile * CPB + lc2;
          if (cell2 >= a.ncells) continue;
          const int j = f >> 1;
          const R *phi = (f & 1) ? T.FR : T.FL;
          R qf[m], Fn[m];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            R s = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) s += phi[b] * V[(lc2 * m + c) * NS + I::node_of_face(p, j, b)];
            qf[c] = s;
          }
          typename PDE::Mat m2;
          load_mat<PDE>(m2, a.matp, a.cst, a.mat, cell2);
          PDE::flux(m2, qf, j, Fn);
          R *dst = hout + cell2 * K::HS + f * K::FB;
#pragma unroll
          for (int c = 0; c < m; ++c) {
            dst[c * NF + p] = qf[c];
            dst[(m + c) * NF + p] = Fn[c];
          }
        }
      } else {
        // ------------------------------------------ space-time Picard (Eq. 3)
        R *Fst = work + CPB * m * NS;  // [CPB][d][n][m][NS]
        R qh[n][m];
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int c = 0; c < m; ++c) qh[k][c] = u[c];
        // tensor-core packed layout (n divides 8): the flux of axis j stored
        // with axis j fastest, 16 rows of whole lines per tensor-core step
        constexpr bool PACKED = K::PRED == kSpaceTimeTC && TcPacked<n>::value;
        int fpos[d];
#pragma unroll
        for (int j = 0; j < d; ++j) fpos[j] = PACKED ? tc_pos<n, d>(node, j) : node;
        // tensor cores: every flux value is stored minus the flux of a state that
        // is constant over the cell (the cell's first node, corrected); Dm maps
        // constants to zero, so the derivatives are unchanged while the TF32
        // operands (10-bit mantissa) carry only the variation over the cell
        // this node's rows of Dm, scaled by 1/dx_j (registers; reused by every
        // variable, time node and iteration)
        R dmr[d][n];
        if constexpr (K::PRED != kSpaceTimeTC) {
#pragma unroll
          for (int j = 0; j < d; ++j) {
            const int ij = I::digit(node, j);
#pragma unroll
            for (int b = 0; b < n; ++b) dmr[j][b] = inv_dx[j] * T.Dm[ij * n + b];
          }
        }
        R fref[d][m];
        if constexpr (K::PRED == kSpaceTimeTC) {
          R *uref = work;  // [CPB][m], free until the time averages
          if (active && node == 0) {
#pragma unroll
            for (int c = 0; c < m; ++c) uref[lc * m + c] = u[c];
          }
          __syncthreads();
          R ur[m];
#pragma unroll
          for (int c = 0; c < m; ++c) ur[c] = uref[lcs * m + c];
          PDE::flux_all(mt, ur, fref);
        } else {
#pragma unroll
          for (int j = 0; j < d; ++j)
#pragma unroll
            for (int c = 0; c < m; ++c) fref[j][c] = R(0);
        }
        // One Picard iteration.  The first iterate is constant in time (q_hat = u
        // at every time node), so on the CUDA cores its flux and flux divergence
        // are those of one time node, reused for all n (the same values).
        auto picard_step = [&](auto first_t) {
          constexpr bool ONE = decltype(first_t)::value && K::PRED == kSpaceTime;
          constexpr int NK = ONE ? 1 : n;
          if (active) {
#pragma unroll
            for (int k = 0; k < NK; ++k)
              {
                R f[d][m];
                PDE::flux_all(mt, qh[k], f);
#pragma unroll
                for (int j = 0; j < d; ++j)
#pragma unroll
                  for (int c = 0; c < m; ++c)
                    Fst[(((lc * d + j) * n + k) * m + c) * NS + fpos[j]] = f[j][c] - fref[j][c];
              }
          }
          __syncthreads();
          if constexpr (K::PRED == kSpaceTimeTC) {
            // (1/dx_j) Dm_j F_j on the tensor cores, in place; then each node
            // sums its d directions
            if constexpr (PACKED) tc_flux_divergence_packed<K>(Fst, T, inv_dx);
            else tc_flux_divergence<K>(Fst, T, inv_dx);
            __syncthreads();
          }
          // one variable at a time: its n flux divergences along time, then
          // q_hat_k = u - sum_l (dt K1^{-1} W)[k][l] div_l (registers only, so
          // before the barrier); the first iterate's divergence is one value
#pragma unroll
          for (int c = 0; c < m; ++c) {
            R dv[n];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
              R div = R(0);
              if constexpr (K::PRED == kSpaceTimeTC) {
#pragma unroll
                for (int j = 0; j < d; ++j) div += Fst[(((lcs * d + j) * n + k) * m + c) * NS + fpos[j]];
              } else {
#pragma unroll
                for (int j = 0; j < d; ++j) {
#pragma unroll
                  for (int b = 0; b < n; ++b)
                    div += dmr[j][b] * Fst[(((lcs * d + j) * n + k) * m + c) * NS + I::with_axis(node, j, b)];
                }
              }
              dv[k] = div;
            }
#pragma unroll
            for (int k = 0; k < n; ++k) {
              R s = u[c];
              if constexpr (ONE) {
                s -= dtM[n * n + k] * dv[0];
              } else {
#pragma unroll
                for (int l = 0; l < n; ++l) s -= dtM[k * n + l] * dv[l];
              }
              qh[k][c] = s;
            }
          }
          __syncthreads();  // F_st is rewritten by the next iteration
        };
        if (a.picard > 0) {
          picard_step(std::true_type{});
          for (int r = 1; r < a.picard; ++r) picard_step(std::false_type{});
        }
        // time averages of q and of the fluxes
        R *Fb = Fst;  // [CPB][d][m][NS]
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R s = R(0);
#pragma unroll
          for (int k = 0; k < n; ++k) s += T.w[k] * qh[k][c];
          qb[c] = s;
        }
        R fbar[d][m];
#pragma unroll
        for (int j = 0; j < d; ++j)
#pragma unroll
          for (int c = 0; c < m; ++c) fbar[j][c] = R(0);
#pragma unroll
        for (int k = 0; k < n; ++k)
          {
            R f[d][m];
            PDE::flux_all(mt, qh[k], f);
#pragma unroll
            for (int j = 0; j < d; ++j)
#pragma unroll
              for (int c = 0; c < m; ++c) fbar[j][c] += T.w[k] * f[j][c];
          }
        if (active) {
#pragma unroll
          for (int c = 0; c < m; ++c) V[(lc * m + c) * NS + node] = qb[c];
#pragma unroll
          for (int j = 0; j < d; ++j)
#pragma unroll
            for (int c = 0; c < m; ++c) Fb[((lc * d + j) * m + c) * NS + node] = fbar[j][c];
        }
        __syncthreads();
        // integrateVolume
        R Dacc[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R s = R(0);
#pragma unroll
          for (int j = 0; j < d; ++j) {
            const int ij = I::digit(node, j);
            R sj = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b)
              sj += T.Kvol[ij * n + b] * Fb[((lcs * d + j) * m + c) * NS + I::with_axis(node, j, b)];
            s += inv_dx[j] * sj;
          }
          Dacc[c] = s;
        }
        if (active) {
#pragma unroll
          for (int c = 0; c < m; ++c) Dbuf[(cell * m + c) * NS + node] = dt_pred * Dacc[c];
        }
        // extrapolate q_bar and F_bar_j to the faces
        for (int it = tid; it < K::FITEMS; it += THREADS) {
          const int lc2 = it / (2 * d * NF);
          const int f = (it / NF) % (2 * d);
          const int p = it % NF;
          const long long cell2 = tile * CPB + lc2;
          if (cell2 >= a.ncells) continue;
          const int j = f >> 1;
          const R *phi = (f & 1) ? T.FR : T.FL;
          R *dst = hout + cell2 * K::HS + f * K::FB;
#pragma unroll
          for (int c = 0; c < m; ++c) {
            R sq = R(0), sf = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) {
              const int nd = I::node_of_face(p, j, b);
              sq += phi[b] * V[(lc2 * m + c) * NS + nd];
              sf += phi[b] * Fb[((lc2 * d + j) * m + c) * NS + nd];
            }
            dst[c * NF + p] = sq;
            dst[(m + c) * NF + p] = sf;
          }
        }
      }
    }
    __syncthreads();
  }
}

// The kernel: linear PDEs keep the compiler's own register choice (a minimum
// of one block per SM in the launch bounds lets it spend registers freely and
// costs occupancy); nonlinear PDEs ask for three blocks per SM (Cfg::MINB).
template <class K, int STAGES>
__global__ void __launch_bounds__(K::THREADS) sweep_kernel(const SweepArgs a) {
  sweep_body<K, STAGES>(a);
}
template <class K, int STAGES>
__global__ void __launch_bounds__(K::THREADS, 3) sweep_kernel_nl3(const SweepArgs a) {
  sweep_body<K, STAGES>(a);
}
template <class K, int STAGES>
constexpr auto sweep_kernel_of() {
  if constexpr (K::MINB == 3) return &sweep_kernel_nl3<K, STAGES>;
  else return &sweep_kernel<K, STAGES>;
}

// Riemann sweep of the three-sweep form: every face once, F* stored.
// A block handles RFPB faces of one axis.
template <class K>
__global__ void __launch_bounds__(256) riemann_kernel(const SweepArgs a) {
  using R = typename K::R;
  using PDE = typename K::PDE;
  constexpr int d = K::d, m = K::m, NF = K::NF;
  constexpr int RFPB = cmax(1, 256 / NF);
  __shared__ R smax[RFPB];
  const R *hin = reinterpret_cast<const R *>(a.hull_in);
  R *fst = reinterpret_cast<R *>(a.fstar);
  const long long nfaces = (long long)d * a.ncells;
  for (long long base = (long long)blockIdx.x * RFPB; base < nfaces; base += (long long)gridDim.x * RFPB) {
    for (int i = threadIdx.x; i < RFPB; i += blockDim.x) smax[i] = R(0);
    __syncthreads();
    const int lf = threadIdx.x / NF, p = threadIdx.x % NF;
    const long long face = base + lf;
    const bool ok = lf < RFPB && face < nfaces;
    R qL[m], qR[m], fL[m], fR[m];
    int j = 0;
    long long cl = 0;
    if (ok) {
      j = (int)(face / a.ncells);
      cl = face % a.ncells;
      const long long cr = neighbour(cl, j, 1, a.grid);
      const R *Lp = hin + cl * K::HS + (2 * j + 1) * K::FB;
      const R *Rp = hin + cr * K::HS + (2 * j) * K::FB;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        qL[c] = ldg(Lp + c * NF + p);
        fL[c] = ldg(Lp + (m + c) * NF + p);
        qR[c] = ldg(Rp + c * NF + p);
        fR[c] = ldg(Rp + (m + c) * NF + p);
      }
      typename PDE::Mat mL, mR;
      load_mat<PDE>(mL, a.matp, a.cst, a.mat, cl);
      load_mat<PDE>(mR, a.matp, a.cst, a.mat, cr);
      smem_max(&smax[lf], nanmax(PDE::speed(mL, qL, j), PDE::speed(mR, qR, j)));
    }
    __syncthreads();
    if (ok) {
      const R s = smax[lf];
      R *dst = fst + ((long long)j * a.ncells + cl) * (m * NF);
#pragma unroll
      for (int c = 0; c < m; ++c) dst[c * NF + p] = R(0.5) * (fL[c] + fR[c]) - R(0.5) * s * (qR[c] - qL[c]);
    }
    __syncthreads();
  }
}

// Largest spectral radius of Q over cells, nodes and axes (initial dt_adm).
template <class K>
__global__ void __launch_bounds__(256) lambda_kernel(const SweepArgs a) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  constexpr int d = K::d, m = K::m, NS = K::NS;
  __shared__ unsigned long long sred[32];
  const QT *Q = reinterpret_cast<const QT *>(a.Q_in);
  R lam = R(0);
  const long long total = a.ncells * NS;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / NS;
    const int node = (int)(t % NS);
    typename PDE::Mat mt;
    load_mat<PDE>(mt, a.matp, a.cst, a.mat, cell);
    R u[m];
    R chk = R(0);
#pragma unroll
    for (int c = 0; c < m; ++c) {
      u[c] = (R)Q[(cell * m + c) * NS + node];
      chk += u[c] * R(0);
    }
#pragma unroll
    for (int j = 0; j < d; ++j) lam = nanmax(lam, PDE::speed(mt, u, j));
    lam += chk;
  }
  block_lambda_max<256>(lam_bits(lam), sred, a.ctl);
}

// Largest wave speed of a linear PDE from the material alone (it does not
// depend on the state), so that Delta t can be set before the state arrives.
template <class K>
__global__ void __launch_bounds__(256) lambda_mat_kernel(const SweepArgs a) {
  using R = typename K::R;
  using PDE = typename K::PDE;
  constexpr int d = K::d, m = K::m;
  __shared__ unsigned long long sred[32];
  R lam = R(0);
  R q0[m];
#pragma unroll
  for (int c = 0; c < m; ++c) q0[c] = R(0);
  const long long ncell = a.mat ? a.ncells : 1;  // uniform material: one cell says it all
  for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    typename PDE::Mat mt;
    load_mat<PDE>(mt, a.matp, a.cst, a.mat, cell);
#pragma unroll
    for (int j = 0; j < d; ++j) lam = nanmax(lam, PDE::speed(mt, q0, j));
  }
  block_lambda_max<256>(lam_bits(lam), sred, a.ctl);
}

}  // namespace aderdg
