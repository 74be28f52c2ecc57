// sweep_lin.cuh -- fused single-touch sweep for linear fluxes F_j = A_j q
// (advection, acoustics, elasticity), line-owner layout.
//
// Same arithmetic as sweep_kernel with the time-modal predictor, organised
// for the GB300 memory hierarchy:
//   * one thread owns one x-line of a cell (n nodes x m variables in
//     registers): x-derivatives, x-face Riemann problems and x-face
//     extrapolation never touch shared memory;
//   * y- and z-contractions are done by the owner of the y- (z-) line after
//     one transpose through shared memory, with all n outputs of a line per
//     thread (n^2 FMAs per n loads);
//   * the 1D operators arrive as a kernel parameter, so every coefficient of
//     an unrolled contraction is a uniform constant-bank operand;
//   * the face hull keeps only the time-averaged q on each face: the normal
//     flux of a linear PDE is A_j q (the own-side A_j of each cell), so
//     storing F_j . n as well would double the face traffic for no
//     information (Rusanov stays affine in (q, F) for the fixed wave speed).
// Stages as in sweep.cuh: kCorrect, kPredict (gate / pred_dt_old honoured),
// kFused.
#pragma once
#include "common.cuh"
#include "pde.cuh"

namespace aderdg {

template <class PDE, int d>
struct LinSlots {
  __host__ __device__ static constexpr bool inY(int c) { return PDE::reads(1, c); }
  __host__ __device__ static constexpr bool inZ(int c) { return d == 3 && PDE::reads(d == 3 ? 2 : 1, c); }
  __host__ __device__ static constexpr int slotY(int c) {
    int s = 0;
    for (int k = 0; k < c; ++k) s += inY(k) ? 1 : 0;
    return s;
  }
  __host__ __device__ static constexpr int slotZ(int c) {
    int s = 0;
    for (int k = 0; k < c; ++k) s += inZ(k) ? 1 : 0;
    return s;
  }
  static constexpr int NY = slotY(PDE::M);
  static constexpr int NZ = slotZ(PDE::M);
};

template <template <int, class> class PDEt, int d_, int N_, class R_, class QT_>
struct LinCfg {
  using R = R_;
  using QT = QT_;
  using PDE = PDEt<d_, R_>;
  using S = LinSlots<PDE, d_>;
  static constexpr int d = d_, N = N_, n = N_ + 1, m = PDE::M;
  static constexpr int NS = ipow(n, d), NF = ipow(n, d - 1), NL = NF;  // x-lines per cell
  // u (the corrected state, reused by every Horner step) stays in registers
  // for short lines and moves to shared memory for long ones (m n > 30)
  static constexpr bool U_SMEM = m * n > 30;
  static constexpr int FSZ = round_up(m * NF, 4);       // q on one face side, padded to 16 B
  static constexpr int HSL = 2 * d * FSZ;               // hull stride per cell
  static constexpr int CELL = round_up(((U_SMEM ? 2 : 1) * m + S::NY + S::NZ) * NS, 4);  // shared elements per cell
  // cells per block: about 256 threads, and at most ~72 KB of shared memory so
  // that three blocks fit on an SM
  static constexpr int CPB = cmax(1, cmin(256 / NL, (72 * 1024) / (CELL * (int)sizeof(R_))));
  static constexpr int THREADS = round_up(CPB * NL, 32);
  // blocks per SM the register allocation must allow (3 fit the shared memory
  // budget); lines of more than 24 words keep more registers per thread
  static constexpr int LINE_WORDS = m * n * (int)(sizeof(R_) / 4);
  static constexpr int MINB = (LINE_WORDS <= 24 && m <= 4) ? 3 : (LINE_WORDS <= 36 ? 2 : (THREADS <= 128 ? 3 : 1));
  static constexpr int FS_CELL = (2 * d - 2) * m * NF;  // y/z face F* per cell
  static_assert(FS_CELL <= CELL, "F* exchange must fit the cell's work area");
  static constexpr size_t SMEM = 32 * sizeof(unsigned long long) + (size_t)CPB * CELL * sizeof(R);
};

// Vector width (elements) for a line of n elements of T.
template <class T, int n>
struct LineVec {
  static constexpr int V = (n % 4 == 0 && 4 * sizeof(T) <= 16) ? 4 : ((n % 2 == 0 && 2 * sizeof(T) <= 16) ? 2 : 1);
};

template <class T, int n>
__device__ __forceinline__ void load_line(const T *p, T (&x)[n]) {
  constexpr int V = LineVec<T, n>::V;
  if constexpr (V == 4 && sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(p + i);
      x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
    }
  } else if constexpr (V == 2 && sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 2) {
      const float2 v = *reinterpret_cast<const float2 *>(p + i);
      x[i] = v.x; x[i + 1] = v.y;
    }
  } else if constexpr (V == 2 && sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < n; i += 2) {
      const double2 v = *reinterpret_cast<const double2 *>(p + i);
      x[i] = v.x; x[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) x[i] = p[i];
  }
}

template <class T, int n>
__device__ __forceinline__ void store_line(T *p, const T (&x)[n]) {
  constexpr int V = LineVec<T, n>::V;
  if constexpr (V == 4 && sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 4) *reinterpret_cast<float4 *>(p + i) = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
  } else if constexpr (V == 2 && sizeof(T) == 4) {
#pragma unroll
    for (int i = 0; i < n; i += 2) *reinterpret_cast<float2 *>(p + i) = make_float2(x[i], x[i + 1]);
  } else if constexpr (V == 2 && sizeof(T) == 8) {
#pragma unroll
    for (int i = 0; i < n; i += 2) *reinterpret_cast<double2 *>(p + i) = make_double2(x[i], x[i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < n; ++i) p[i] = x[i];
  }
}

// Rusanov flux of a linear PDE on the face normal to j from the two
// time-averaged face states; each side applies its own A_j.
template <class PDE, class R>
__device__ __forceinline__ void rusanov_lin(const typename PDE::Mat &mL, const typename PDE::Mat &mR, int j,
                                            const R *qL, const R *qR, R *fs) {
  constexpr int m = PDE::M;
  R fl[m], fr[m];
  PDE::flux(mL, qL, j, fl);
  PDE::flux(mR, qR, j, fr);
  const R sL = PDE::speed(mL, qL, j), sR = PDE::speed(mR, qR, j);
  const R s = sL > sR ? sL : sR;
#pragma unroll
  for (int c = 0; c < m; ++c) fs[c] = R(0.5) * (fl[c] + fr[c]) - R(0.5) * s * (qR[c] - qL[c]);
}

// One application of sum_j (1/dx_j) A_j C_j to the line-distributed state v,
// C = Dm (a Horner step of the predictor) or C = Kvol (integrateVolume, VOL).
// Result in Lv (this thread's x-line).  With VOL the y/z line owners also
// extrapolate v to the y/z faces into the hull.  Two block barriers.
template <class K, bool VOL>
struct LinPass {
  using R = typename K::R;
  using PDE = typename K::PDE;
  using S = typename K::S;
  static constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  __device__ __forceinline__ static R coef(const Tables<R> &T, int o, int b) {
    return VOL ? T.Kvol[o * n + b] : T.Dm[o * n + b];
  }
  __device__ __forceinline__ static void run(const Tables<R> &T, const typename PDE::Mat &mt, const R (&v)[m][n],
                                             R (&Lv)[m][n], R *VS, R *DYS, R *DZS, R *hout, long long cell,
                                             int t, bool active, R idx0, R idx1, R idx2) {
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (VOL || PDE::reads(0, c) || S::inY(c) || S::inZ(c)) store_line<R, n>(VS + c * NS + t * n, v[c]);
    }
    __syncthreads();
    if (active) {
      // y-line owner (i0 = t % n, i2 = t / n); z-line owner (i0 = t % n, i1 = t / n)
      const int y0 = (t % n) + n * n * (t / n);
      const int z0 = t;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (S::inY(c) || VOL) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + y0 + n * b];
          if (S::inY(c)) {
#pragma unroll
            for (int o = 0; o < n; ++o) {
              R acc = R(0);
#pragma unroll
              for (int b = 0; b < n; ++b) acc += coef(T, o, b) * line[b];
              DYS[S::slotY(c) * NS + y0 + n * o] = acc;
            }
          }
          if (VOL) {  // extrapolate to the two y faces, face node p = t
            R sl = R(0), sr = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) {
              sl += T.FL[b] * line[b];
              sr += T.FR[b] * line[b];
            }
            hout[cell * K::HSL + 2 * K::FSZ + c * NF + t] = sl;
            hout[cell * K::HSL + 3 * K::FSZ + c * NF + t] = sr;
          }
        }
        if (d == 3 && (S::inZ(c) || VOL)) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + z0 + n * n * b];
          if (S::inZ(c)) {
#pragma unroll
            for (int o = 0; o < n; ++o) {
              R acc = R(0);
#pragma unroll
              for (int b = 0; b < n; ++b) acc += coef(T, o, b) * line[b];
              DZS[S::slotZ(c) * NS + z0 + n * n * o] = acc;
            }
          }
          if (VOL) {
            R sl = R(0), sr = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) {
              sl += T.FL[b] * line[b];
              sr += T.FR[b] * line[b];
            }
            hout[cell * K::HSL + 4 * K::FSZ + c * NF + t] = sl;
            hout[cell * K::HSL + 5 * K::FSZ + c * NF + t] = sr;
          }
        }
      }
    }
    __syncthreads();
    if (VOL && active) {  // extrapolate to the two x faces, face node p = t
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R line[n];
        load_line<R, n>(VS + c * NS + t * n, line);
        R sl = R(0), sr = R(0);
#pragma unroll
        for (int b = 0; b < n; ++b) {
          sl += T.FL[b] * line[b];
          sr += T.FR[b] * line[b];
        }
        hout[cell * K::HSL + 0 * K::FSZ + c * NF + t] = sl;
        hout[cell * K::HSL + 1 * K::FSZ + c * NF + t] = sr;
      }
    }
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) Lv[c][i] = R(0);
    if (active) {
      // x-derivatives of the components A_x reads, from this thread's line in VS
      R dx[m][n];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (PDE::reads(0, c)) {
          R line[n];
          load_line<R, n>(VS + c * NS + t * n, line);
#pragma unroll
          for (int o = 0; o < n; ++o) {
            R acc = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b) acc += coef(T, o, b) * line[b];
            dx[c][o] = acc;
          }
        }
      }
#pragma unroll
      for (int o = 0; o < n; ++o) {
        R dv[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) dv[c] = PDE::reads(0, c) ? dx[c][o] : R(0);
        PDE::applyA(mt, 0, dv, out);
#pragma unroll
        for (int c = 0; c < m; ++c) Lv[c][o] += idx0 * out[c];
      }
      // y (z) derivatives of this thread's line, vector loads of the whole line
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (S::inY(c)) load_line<R, n>(DYS + S::slotY(c) * NS + t * n, dx[c]);
#pragma unroll
      for (int o = 0; o < n; ++o) {
        R dv[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) dv[c] = S::inY(c) ? dx[c][o] : R(0);
        PDE::applyA(mt, 1, dv, out);
#pragma unroll
        for (int c = 0; c < m; ++c) Lv[c][o] += idx1 * out[c];
      }
      if (d == 3) {
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (S::inZ(c)) load_line<R, n>(DZS + S::slotZ(c) * NS + t * n, dx[c]);
#pragma unroll
        for (int o = 0; o < n; ++o) {
          R dv[m], out[m];
#pragma unroll
          for (int c = 0; c < m; ++c) dv[c] = S::inZ(c) ? dx[c][o] : R(0);
          PDE::applyA(mt, 2, dv, out);
#pragma unroll
          for (int c = 0; c < m; ++c) Lv[c][o] += idx2 * out[c];
        }
      }
    }
    __syncthreads();  // the work area is reused by the next pass or tile
  }
};

// One tile (K::CPB consecutive cells) of the sweep; every thread of the block
// must call it (it contains block barriers).  TAB is Tables<R> in the
// parameter or constant space, so that unrolled coefficients are uniform
// constant-bank operands.
template <class K, int STAGES, class TAB>
__device__ __forceinline__ void lin_tile(const SweepArgs &a, const TAB &T, long long tile, unsigned char *smem) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using S = typename K::S;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, NL = K::NL, CPB = K::CPB;
  constexpr int THREADS = K::THREADS;

  unsigned long long *sred = reinterpret_cast<unsigned long long *>(smem);
  R *work = reinterpret_cast<R *>(smem + 32 * sizeof(unsigned long long));

  DevCtl *ctl = a.ctl;
  const R dt_old = (R)ctl->dt_old;
  const R dt_pred = (R)(a.pred_dt_old ? ctl->dt_old : ctl->dt_new);
  const QT *Qin = reinterpret_cast<const QT *>(a.Q_in);
  QT *Qout = reinterpret_cast<QT *>(a.Q_out);
  R *Dbuf = reinterpret_cast<R *>(a.Dbuf);
  const R *hin = reinterpret_cast<const R *>(a.hull_in);
  R *hout = reinterpret_cast<R *>(a.hull_out);
  const R idx0 = (R)a.inv_dx[0], idx1 = (R)a.inv_dx[1], idx2 = (R)a.inv_dx[2];

  const int tid = threadIdx.x;
  const int lc = tid / NL;
  const int t = tid - lc * NL;                 // x-line index = i1 + n i2
  const int lcs = lc < CPB ? lc : CPB - 1;
  const int i1 = t % n, i2 = t / n;            // (d = 2: i2 = 0)
  R *VS = work + lcs * K::CELL;                // [m][NS]  line layout: node = i0 + n t
  R *US = VS + m * NS;                         // [m][NS]  u, if K::U_SMEM
  R *DYS = US + (K::U_SMEM ? m * NS : 0);      // [NY][NS]
  R *DZS = DYS + S::NY * NS;                   // [NZ][NS]
  R *FS = VS;                                  // corrector: [2d-2][m][NF]

  // face weights of this thread's line position along y and z
  const R wyR = T.FR[i1] * T.iw[i1], wyL = T.FL[i1] * T.iw[i1];
  const R wzR = d == 3 ? T.FR[i2] * T.iw[i2] : R(0), wzL = d == 3 ? T.FL[i2] * T.iw[i2] : R(0);

  {
  const long long cell = tile * CPB + lc;
  const bool active = lc < CPB && cell < a.ncells;
  const long long cs = active ? cell : 0;
  typename PDE::Mat mt;
  PDE::load(mt, a.cst, a.mat, cs);
  R u[m][n];
  if (STAGES == kPredict) {
#pragma unroll
    for (int c = 0; c < m; ++c) {
      QT q[n];
      if (active) load_line<QT, n>(Qin + (cell * m + c) * NS + t * n, q);
      else {
#pragma unroll
        for (int i = 0; i < n; ++i) q[i] = QT(0);
      }
#pragma unroll
      for (int i = 0; i < n; ++i) u[c][i] = (R)q[i];
    }
  }

  // ------------------------------------------------------------ corrector
  if (STAGES == kCorrect || STAGES == kFused) {
    // face terms first; D and the old state are read only at the update
    R acc[m][n];
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) acc[c][i] = R(0);
    if (active) {
      // x faces: face node p = t, F* in registers
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const long long nb = neighbour(cell, 0, side ? 1 : -1, a.grid);
        const R *own = hin + cell * K::HSL + side * K::FSZ;
        const R *nbr = hin + nb * K::HSL + (side ^ 1) * K::FSZ;
        R qo[m], qn[m], fs[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          qo[c] = ldg(own + c * NF + t);
          qn[c] = ldg(nbr + c * NF + t);
        }
        typename PDE::Mat mn;
        PDE::load(mn, a.cst, a.mat, nb);
        if (side) rusanov_lin<PDE, R>(mt, mn, 0, qo, qn, fs);
        else rusanov_lin<PDE, R>(mn, mt, 0, qn, qo, fs);
        const R sg = side ? R(1) : R(-1);
#pragma unroll
        for (int i = 0; i < n; ++i) {
          const R wgt = dt_old * idx0 * sg * (side ? T.FR[i] : T.FL[i]) * T.iw[i];
#pragma unroll
          for (int c = 0; c < m; ++c) acc[c][i] -= wgt * fs[c];
        }
      }
      // y (z) faces: this thread solves face node p = t of faces 2..2d-1
#pragma unroll
      for (int f = 2; f < 2 * d; ++f) {
        const int j = f >> 1, side = f & 1;
        const long long nb = neighbour(cell, j, side ? 1 : -1, a.grid);
        const R *own = hin + cell * K::HSL + f * K::FSZ;
        const R *nbr = hin + nb * K::HSL + (f ^ 1) * K::FSZ;
        R qo[m], qn[m], fs[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          qo[c] = ldg(own + c * NF + t);
          qn[c] = ldg(nbr + c * NF + t);
        }
        typename PDE::Mat mn;
        PDE::load(mn, a.cst, a.mat, nb);
        if (side) rusanov_lin<PDE, R>(mt, mn, j, qo, qn, fs);
        else rusanov_lin<PDE, R>(mn, mt, j, qn, qo, fs);
#pragma unroll
        for (int c = 0; c < m; ++c) FS[((f - 2) * m + c) * NF + t] = fs[c];
      }
    }
    __syncthreads();
    R lam = R(0);
    if (active) {
      // y faces: face node p = i0 + n i2 ; z faces: p = i0 + n i1
      const int py = n * i2, pz = n * i1;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R yl[n], yr[n];
        load_line<R, n>(FS + (0 * m + c) * NF + py, yl);
        load_line<R, n>(FS + (1 * m + c) * NF + py, yr);
#pragma unroll
        for (int i = 0; i < n; ++i) acc[c][i] -= dt_old * idx1 * (wyR * yr[i] - wyL * yl[i]);
        if (d == 3) {
          R zl[n], zr[n];
          load_line<R, n>(FS + (2 * m + c) * NF + pz, zl);
          load_line<R, n>(FS + (3 * m + c) * NF + pz, zr);
#pragma unroll
          for (int i = 0; i < n; ++i) acc[c][i] -= dt_old * idx2 * (wzR * zr[i] - wzL * zl[i]);
        }
      }
      R chk = R(0);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        QT q[n];
        R dl[n];
        load_line<QT, n>(Qin + (cell * m + c) * NS + t * n, q);
        load_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, dl);
#pragma unroll
        for (int i = 0; i < n; ++i) {
          q[i] = q[i] + (QT)(dl[i] + acc[c][i]);
          u[c][i] = (R)q[i];
          chk += u[c][i] * R(0);   // NaN/Inf anywhere in the line survives
        }
        store_line<QT, n>(Qout + (cell * m + c) * NS + t * n, q);
      }
      R uq[m];
#pragma unroll
      for (int c = 0; c < m; ++c) uq[c] = u[c][0];
#pragma unroll
      for (int j = 0; j < d; ++j) lam = nanmax(lam, PDE::speed(mt, uq, j));
      lam += chk;
    }
    block_lambda_max<THREADS>(lam_bits(lam), sred, ctl);
    __syncthreads();  // F* consumed
  }

  // ------------------------------------------------------------ predictor
  if (STAGES == kPredict || STAGES == kFused) {
    // Horner form of q_bar = sum_s g_s (-dt L)^s u, then integrateVolume
    R v[m][n], Lv[m][n];
    if (K::U_SMEM && active) {
#pragma unroll
      for (int c = 0; c < m; ++c) store_line<R, n>(US + c * NS + t * n, u[c]);
    }
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) v[c][i] = T.g[a.picard] * u[c][i];
    for (int s = a.picard - 1; s >= 0; --s) {
      LinPass<K, false>::run(T, mt, v, Lv, VS, DYS, DZS, hout, cell, t, active, idx0, idx1, idx2);
      const R gs = T.g[s];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R uc[n];
        if (K::U_SMEM) {
          if (active) load_line<R, n>(US + c * NS + t * n, uc);
          else {
#pragma unroll
            for (int i = 0; i < n; ++i) uc[i] = R(0);
          }
        } else {
#pragma unroll
          for (int i = 0; i < n; ++i) uc[i] = u[c][i];
        }
#pragma unroll
        for (int i = 0; i < n; ++i) v[c][i] = gs * uc[i] - dt_pred * Lv[c][i];
      }
    }
    LinPass<K, true>::run(T, mt, v, Lv, VS, DYS, DZS, hout, cell, t, active, idx0, idx1, idx2);
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R dl[n];
#pragma unroll
        for (int i = 0; i < n; ++i) dl[i] = dt_pred * Lv[c][i];
        store_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, dl);
      }
    }
  }
  }
}

template <class K, int STAGES>
__global__ void __launch_bounds__(K::THREADS, K::MINB) lin_sweep_kernel(const SweepArgs a, const Tables<typename K::R> T) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (STAGES == kPredict && a.gate) {
    if (*(volatile int *)&a.ctl->rerun == 0) return;  // uniform for the whole grid
  }
  for (long long tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) lin_tile<K, STAGES>(a, T, tile, smem);
}

}  // namespace aderdg
