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
#include <type_traits>
#include "common.cuh"
#include "pde.cuh"
#include "tma.cuh"

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

// PDEs whose operator is bipartite (PDE::BIPARTITE: rows of one group read
// only the other group's components), detected without requiring the trait.
template <class PDE, class = void>
struct Bipartite {
  static constexpr bool value = false;
};
template <class PDE>
struct Bipartite<PDE, decltype(void(PDE::BIPARTITE))> {
  static constexpr bool value = PDE::BIPARTITE;
};

// PDEs whose predictor state is split over line orientations (PDE::OWNED):
// component c lives on lines along axis PDE::owner(c).  Axis j's pass writes
// the components A_j updates but does not own into one buffer each
// (contribution slots, [slot][NS] in node layout).
template <class PDE, int d, bool OWN = PDE::OWNED>
struct OwnSlots {
  static constexpr int NCB = 0;
};
template <class PDE, int d>
struct OwnSlots<PDE, d, true> {
  __host__ __device__ static constexpr bool cross(int j, int c) { return PDE::writes(j, c) && PDE::owner(c) != j; }
  __host__ __device__ static constexpr int slot(int j, int c) {
    int s = 0;
    for (int jj = 0; jj < d; ++jj)
      for (int k = 0; k < PDE::M; ++k) {
        if (jj == j && k == c) return s;
        s += cross(jj, k) ? 1 : 0;
      }
    return s;
  }
  static constexpr int NCB = slot(d, 0);
  // read along an axis other than its owner's: goes through shared memory each pass
  __host__ __device__ static constexpr bool shared(int c) {
    for (int j = 0; j < d; ++j)
      if (j != PDE::owner(c) && PDE::reads(j, c)) return true;
    return false;
  }
};

// CPB_ > 0 fixes the cells per block (the ensemble kernel, whose block is
// always 256 threads, fills it with whole cells of every configuration).
template <template <int, class> class PDEt, int d_, int N_, class R_, class QT_, int CPB_ = 0>
struct LinCfg {
  using R = R_;
  using QT = typename QStore<QT_>::T;         // element type of the state rows
  static constexpr bool PAIR = QStore<QT_>::PAIR;  // a low-word plane follows the states
  using PDE = PDEt<d_, R_>;
  using S = LinSlots<PDE, d_>;
  static constexpr int d = d_, N = N_, n = N_ + 1, m = PDE::M;
  static constexpr int NS = ipow(n, d), NF = ipow(n, d - 1), NL = NF;  // x-lines per cell
  // u (the corrected state, reused by every Horner step) stays in registers
  // for short lines; long lines (m n > 30) read it back from the state row
  // each step (just written by this thread: an L1/L2 hit), which keeps the
  // shared memory per cell, and so the cells per block, as for short lines
  // Bipartite operators (elasticity) update the Horner state in place group by
  // group (LinPassBip) and keep u in registers however long the line is.
  static constexpr bool BIP = Bipartite<PDE>::value;
  static constexpr bool U_SMEM = !BIP && m * n > 30;
  static constexpr int FSZ = round_up(m * NF, 4);       // q on one face side, padded to 16 B
  static constexpr int HSL = 2 * d * FSZ;               // hull stride per cell
  // shared elements per cell, padded so that CELL = NL (mod 32): lanes of a
  // warp that straddles two cells then hit consecutive banks in the z-line
  // pattern (node i0 + n i1 + n^2 b) instead of two overlapping ranges
  static constexpr bool OWN = PDE::OWNED;
  using O = OwnSlots<PDE, d_>;
  static constexpr int CELL0 = round_up((m + (OWN ? O::NCB : S::NY + S::NZ)) * NS, 4);
  // (bipartite elasticity, 25 lines per cell: residue 29, which a model of the
  // pass's x-line, y-column and z-column accesses puts 18 % fewer wavefronts on)
  static constexpr int CELL_RES = (BIP && NL == 25) ? 29 : NL % 32;
  static constexpr int CELL = CELL0 + ((CELL_RES - CELL0 % 32) % 32 + 32) % 32;
  // cells per block: about 256 threads, and at most ~72 KB of shared memory so
  // that three blocks fit on an SM
  static constexpr int CPB = CPB_ > 0 ? CPB_ : cmax(1, cmin(256 / NL, (72 * 1024) / (CELL * (int)sizeof(R_))));
  static constexpr int THREADS = round_up(CPB * NL, 32);
  // blocks per SM the register allocation must allow (3 fit the shared memory
  // budget); lines of more than 24 words keep more registers per thread
  static constexpr int LINE_WORDS = m * n * (int)(sizeof(R_) / 4);
  static constexpr int MINB = (LINE_WORDS <= 24 && m <= 4) ? 3 : (LINE_WORDS <= 36 ? 2 : (THREADS <= 160 ? 3 : 1));
  static constexpr int FS_CELL = (2 * d - 2) * m * NF;  // y/z face F* per cell
  static constexpr int FSC = round_up(FS_CELL, 4);        // its slot, 16-byte multiple
  static_assert(FSC <= CELL, "F* exchange must fit the cell's work area");
  static_assert(!(OWN && U_SMEM), "split ownership keeps u in registers");
  // Q and D of a tile staged in shared memory by the bulk copy engine during
  // the corrector (its F* slots first, then Q, then D); needs 16-byte rows
  static constexpr bool TMA_QD = (m * NS * sizeof(QT)) % 16 == 0 && (m * NS * sizeof(R_)) % 16 == 0;
  static constexpr size_t WORK_BYTES = (size_t)CPB * CELL * sizeof(R_);
  static constexpr size_t STAGE_BYTES = (size_t)CPB * FSC * sizeof(R_) + (size_t)CPB * m * NS * (sizeof(QT) + sizeof(R_));
  static constexpr size_t SMEM_NOTMA = 32 * sizeof(unsigned long long) + WORK_BYTES;
  static constexpr size_t SMEM =
      32 * sizeof(unsigned long long) + (TMA_QD && STAGE_BYTES > WORK_BYTES ? STAGE_BYTES : WORK_BYTES);
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

// Material jump in non-conservative form (the products B_j(x) dQ/dx_j of
// Eq. 1, B_j = dF_j/dQ constant inside a cell).  Along the straight path in
// (lambda, mu, 1/rho), in which B_j is linear, the path-conservative
// fluctuations D- = (A~ - s)(q_R - q_L)/2 and D+ = (A~ + s)(q_R - q_L)/2 with
// A~ = (B_L + B_R)/2 turn the cell's weak-form update into an own-side flux
//   F*_own = F* + (B_own - B_nb)(q_L + q_R)/4,
// F* the conservative Rusanov flux: fs += (F_j(mo, qo + qn) - F_j(mn, qo + qn))/4.
template <class PDE, class R>
__device__ __forceinline__ void ncp_own_side(const typename PDE::Mat &mo, const typename PDE::Mat &mn, int j,
                                             const R *qo, const R *qn, R *fs) {
  constexpr int m = PDE::M;
  R qs[m], fo[m], fb[m];
#pragma unroll
  for (int c = 0; c < m; ++c) qs[c] = qo[c] + qn[c];
  PDE::flux(mo, qs, j, fo);
  PDE::flux(mn, qs, j, fb);
#pragma unroll
  for (int c = 0; c < m; ++c) fs[c] += R(0.25) * (fo[c] - fb[c]);
}

// Point sources of a cell (bit k of mask: source k) added to one line of
// component c: x[b] += co_k amp_k[c] prod_j e_k[j][i_j] along the line of
// orientation o that thread t owns (OwnLine's layout; o = 0: x-line t), with
// co_k = srcco[k][coi].  Taken by the threads of source cells only.
template <int n, int d, class R>
__device__ __forceinline__ void src_add_line(const SweepArgs &a, unsigned long long mask, int coi, int c, int o,
                                             int t, R (&x)[n]) {
  int f0 = 0, f1 = 0, f2 = 0;  // the digits of the axes the line does not run along
  if (o == 0) {
    f1 = t % n;
    f2 = t / n;
  } else if (o == 1) {
    f0 = d == 3 ? t / n : t;
    f2 = d == 3 ? t % n : 0;
  } else {
    f0 = t % n;
    f1 = t / n;
  }
  while (mask) {
    const int k = __ffsll((long long)mask) - 1;
    mask &= mask - 1;
    const SrcDev &S = a.src[k];
    const double wk = a.srcco[(long long)k * kSrcCo + coi] * S.amp[c];
#pragma unroll
    for (int b = 0; b < n; ++b) {
      const int i0 = o == 0 ? b : f0, i1 = o == 1 ? b : f1, i2 = o == 2 ? b : f2;
      double v = wk * S.e[0][i0] * S.e[1][i1];
      if (d == 3) v *= S.e[2][i2];
      x[b] += (R)v;
    }
  }
}

// out[o] = sum_b C[o][b] x[b] along one line, C = Dm (VOL false) or Kvol (VOL
// true).  For n >= 5 through the even/odd halves of the centro-antisymmetric C
// (Tables::DmE/DmO/DmM, KvE/KvO/KvM): with e_b = x_b + x_{n-1-b} and
// d_b = x_b - x_{n-1-b}, S_o = sum_b E[o][b] e_b (+ M[o] x_h for odd n) and
// T_o = sum_b O[o][b] d_b give out[o] = S_o + T_o, out[n-1-o] = T_o - S_o,
// and for odd n out[h] = sum_b O[h][b] d_b: n^2/2 + 2n operations instead of n^2.
template <int n, bool VOL, class TAB, class R>
__device__ __forceinline__ void contract_line(const TAB &T, const R (&x)[n], R (&out)[n]) {
  if constexpr (std::is_same<R, float>::value && n % 2 == 0 && n >= 4) {
    // FP32, even n: two rows at once with packed two-lane FMAs (row pairs
    // DmP/KvP), n^2/2 of them
    const float2 *P = reinterpret_cast<const float2 *>(VOL ? T.KvP : T.DmP);
    float2 acc[n / 2];
    const float2 x0 = make_float2(x[0], x[0]);
#pragma unroll
    for (int k = 0; k < n / 2; ++k) acc[k] = __fmul2_rn(P[k * kMaxn], x0);
#pragma unroll
    for (int b = 1; b < n; ++b) {
      const float2 xb = make_float2(x[b], x[b]);
#pragma unroll
      for (int k = 0; k < n / 2; ++k) acc[k] = __ffma2_rn(P[k * kMaxn + b], xb, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < n / 2; ++k) {
      out[2 * k] = acc[k].x;
      out[2 * k + 1] = acc[k].y;
    }
  } else if constexpr (n < 5) {
#pragma unroll
    for (int o = 0; o < n; ++o) {
      R acc = (VOL ? T.Kvol[o * n] : T.Dm[o * n]) * x[0];
#pragma unroll
      for (int b = 1; b < n; ++b) acc += (VOL ? T.Kvol[o * n + b] : T.Dm[o * n + b]) * x[b];
      out[o] = acc;
    }
  } else {
    constexpr int h = n / 2;
    R e[h], dd[h];
#pragma unroll
    for (int b = 0; b < h; ++b) {
      e[b] = x[b] + x[n - 1 - b];
      dd[b] = x[b] - x[n - 1 - b];
    }
#pragma unroll
    for (int o = 0; o < h; ++o) {
      R S = (VOL ? T.KvE[o * kMaxH] : T.DmE[o * kMaxH]) * e[0];
      R Tt = (VOL ? T.KvO[o * kMaxH] : T.DmO[o * kMaxH]) * dd[0];
#pragma unroll
      for (int b = 1; b < h; ++b) {
        S += (VOL ? T.KvE[o * kMaxH + b] : T.DmE[o * kMaxH + b]) * e[b];
        Tt += (VOL ? T.KvO[o * kMaxH + b] : T.DmO[o * kMaxH + b]) * dd[b];
      }
      if (n % 2) S += (VOL ? T.KvM[o] : T.DmM[o]) * x[h];
      out[o] = S + Tt;
      out[n - 1 - o] = Tt - S;
    }
    if (n % 2) {
      R Tm = (VOL ? T.KvO[h * kMaxH] : T.DmO[h * kMaxH]) * dd[0];
#pragma unroll
      for (int b = 1; b < h; ++b) Tm += (VOL ? T.KvO[h * kMaxH + b] : T.DmO[h * kMaxH + b]) * dd[b];
      out[h] = Tm;
    }
  }
}

// One application of sum_j A'_j C_j to the line-distributed state v, where
// A'_j = (dt / dx_j) A_j is folded into the per-direction material ms[j]
// (PDE::scaleA), C = Dm (a Horner step of the predictor) or C = Kvol
// (integrateVolume, VOL).  Result in Lv (this thread's x-line).  With VOL the
// y/z line owners also extrapolate v to the y/z faces into the hull.  Two
// block barriers.
template <class K, bool VOL>
struct LinPass {
  using R = typename K::R;
  using PDE = typename K::PDE;
  using S = typename K::S;
  using Mat = typename PDE::Mat;
  static constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  template <class TAB>
  __device__ __forceinline__ static void run(const TAB &T, const Mat &mt, const R (&sc)[d], const R (&v)[m][n],
                                             R (&Lv)[m][n], R *VS, R *DYS, R *DZS, R *hout, long long cell,
                                             int t, bool active) {
    if (active) {
      // only what the y/z line owners read goes through shared memory (x-derivatives
      // and x-face values come from the registers)
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (VOL || S::inY(c) || S::inZ(c)) store_line<R, n>(VS + c * NS + t * n, v[c]);
    }
    __syncthreads();
    if (active) {
      // y-line owner (3D: i0 = t / n, i2 = t % n); z-line owner (i0 = t % n, i1 = t / n)
      const int yi0 = d == 3 ? t / n : t, yi2 = d == 3 ? t % n : 0;
      const int y0 = yi0 + n * n * yi2, py = yi0 + n * yi2;
      const int z0 = t;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (S::inY(c) || VOL) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + y0 + n * b];
          if (S::inY(c)) {
            R dl[n];
            contract_line<n, VOL>(T, line, dl);
#pragma unroll
            for (int o = 0; o < n; ++o) DYS[S::slotY(c) * NS + y0 + n * o] = dl[o];
          }
          if (VOL) {  // extrapolate to the two y faces, face node p = t
            R sl = T.FL[0] * line[0], sr = T.FR[0] * line[0];
#pragma unroll
            for (int b = 1; b < n; ++b) {
              sl += T.FL[b] * line[b];
              sr += T.FR[b] * line[b];
            }
            hout[cell * K::HSL + 2 * K::FSZ + c * NF + py] = sl;
            hout[cell * K::HSL + 3 * K::FSZ + c * NF + py] = sr;
          }
        }
        if (d == 3 && (S::inZ(c) || VOL)) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + z0 + n * n * b];
          if (S::inZ(c)) {
            R dl[n];
            contract_line<n, VOL>(T, line, dl);
#pragma unroll
            for (int o = 0; o < n; ++o) DZS[S::slotZ(c) * NS + z0 + n * n * o] = dl[o];
          }
          if (VOL) {
            R sl = T.FL[0] * line[0], sr = T.FR[0] * line[0];
#pragma unroll
            for (int b = 1; b < n; ++b) {
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
        R sl = T.FL[0] * v[c][0], sr = T.FR[0] * v[c][0];
#pragma unroll
        for (int b = 1; b < n; ++b) {
          sl += T.FL[b] * v[c][b];
          sr += T.FR[b] * v[c][b];
        }
        hout[cell * K::HSL + 0 * K::FSZ + c * NF + t] = sl;
        hout[cell * K::HSL + 1 * K::FSZ + c * NF + t] = sr;
      }
    }
    if (active) {
      // x-derivatives of the components A_x reads, from this thread's own line
      // (registers); A'_x sets Lv, A'_y and A'_z accumulate into it (FMAs on
      // the non-zero rows)
      R dx[m][n];
      Mat mj = mt;
      PDE::scaleA(mj, sc[0]);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (PDE::reads(0, c)) contract_line<n, VOL>(T, v[c], dx[c]);
      }
#pragma unroll
      for (int o = 0; o < n; ++o) {
        R dv[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) dv[c] = PDE::reads(0, c) ? dx[c][o] : R(0);
        PDE::applyA(mj, 0, dv, out);
#pragma unroll
        for (int c = 0; c < m; ++c) Lv[c][o] = out[c];
      }
      // y (z) derivatives of this thread's line, vector loads of the whole line
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (S::inY(c)) load_line<R, n>(DYS + S::slotY(c) * NS + t * n, dx[c]);
      mj = mt;
      PDE::scaleA(mj, sc[1]);
#pragma unroll
      for (int o = 0; o < n; ++o) {
        R dv[m], acc[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          dv[c] = S::inY(c) ? dx[c][o] : R(0);
          acc[c] = Lv[c][o];
        }
        PDE::accA(mj, 1, dv, acc);
#pragma unroll
        for (int c = 0; c < m; ++c) Lv[c][o] = acc[c];
      }
      if (d == 3) {
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (S::inZ(c)) load_line<R, n>(DZS + S::slotZ(c) * NS + t * n, dx[c]);
        mj = mt;
        PDE::scaleA(mj, sc[d - 1]);
#pragma unroll
        for (int o = 0; o < n; ++o) {
          R dv[m], acc[m];
#pragma unroll
          for (int c = 0; c < m; ++c) {
            dv[c] = S::inZ(c) ? dx[c][o] : R(0);
            acc[c] = Lv[c][o];
          }
          PDE::accA(mj, d - 1, dv, acc);
#pragma unroll
          for (int c = 0; c < m; ++c) Lv[c][o] = acc[c];
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < m; ++c)
#pragma unroll
        for (int i = 0; i < n; ++i) Lv[c][i] = R(0);
    }
    // No barrier here within the Horner loop: the next pass first stores each
    // thread's own x-line (read by others only before this pass's second
    // barrier) and writes DY/DZ only after its own first barrier.  The caller
    // synchronises before the work area is reused as the corrector's F* space.
  }
};

// LinPass for bipartite operators (PDE::BIPARTITE; elasticity: the stress rows
// of A_j read only velocities, the velocity rows only stresses).  The shared-
// memory exchange is LinPass's; then the update is in place, group by group:
//   L1 = sum_j A'_j C_j v[group 0]          (rows of group 1, from old group-0 lines)
//   v[group 0] <- g u - sum_j A'_j C_j v[group 1]   (group-0 lines no longer read)
//   v[group 1] <- g u - L1
// (VOL: v <- L v, C = Kvol, with the face extrapolation first), so no separate
// L v lines are kept and u stays in registers.  Two block barriers.
template <class K, bool VOL>
struct LinPassBip {
  using R = typename K::R;
  using PDE = typename K::PDE;
  using S = typename K::S;
  using Mat = typename PDE::Mat;
  static constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  template <class TAB>
  __device__ __forceinline__ static void run(const TAB &T, const Mat &mt, const R (&sc)[d], R (&v)[m][n],
                                             const R (&u)[m][n], R gs, R *VS, R *DYS, R *DZS, R *hout,
                                             long long cell, int t, bool active) {
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (VOL || S::inY(c) || S::inZ(c)) store_line<R, n>(VS + c * NS + t * n, v[c]);
    }
    __syncthreads();
    if (active) {
      const int yi0 = d == 3 ? t / n : t, yi2 = d == 3 ? t % n : 0;
      const int y0 = yi0 + n * n * yi2, py = yi0 + n * yi2;
      const int z0 = t;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (S::inY(c) || VOL) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + y0 + n * b];
          if (S::inY(c)) {
            R dl[n];
            contract_line<n, VOL>(T, line, dl);
#pragma unroll
            for (int o = 0; o < n; ++o) DYS[S::slotY(c) * NS + y0 + n * o] = dl[o];
          }
          if (VOL) {
            R sl = T.FL[0] * line[0], sr = T.FR[0] * line[0];
#pragma unroll
            for (int b = 1; b < n; ++b) {
              sl += T.FL[b] * line[b];
              sr += T.FR[b] * line[b];
            }
            hout[cell * K::HSL + 2 * K::FSZ + c * NF + py] = sl;
            hout[cell * K::HSL + 3 * K::FSZ + c * NF + py] = sr;
          }
        }
        if (d == 3 && (S::inZ(c) || VOL)) {
          R line[n];
#pragma unroll
          for (int b = 0; b < n; ++b) line[b] = VS[c * NS + z0 + n * n * b];
          if (S::inZ(c)) {
            R dl[n];
            contract_line<n, VOL>(T, line, dl);
#pragma unroll
            for (int o = 0; o < n; ++o) DZS[S::slotZ(c) * NS + z0 + n * n * o] = dl[o];
          }
          if (VOL) {
            R sl = T.FL[0] * line[0], sr = T.FR[0] * line[0];
#pragma unroll
            for (int b = 1; b < n; ++b) {
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
    if (!active) {
#pragma unroll
      for (int c = 0; c < m; ++c)
#pragma unroll
        for (int i = 0; i < n; ++i) v[c][i] = R(0);
      return;
    }
    if (VOL) {  // extrapolate to the two x faces, face node p = t, before v is overwritten
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R sl = T.FL[0] * v[c][0], sr = T.FR[0] * v[c][0];
#pragma unroll
        for (int b = 1; b < n; ++b) {
          sl += T.FL[b] * v[c][b];
          sr += T.FR[b] * v[c][b];
        }
        hout[cell * K::HSL + 0 * K::FSZ + c * NF + t] = sl;
        hout[cell * K::HSL + 1 * K::FSZ + c * NF + t] = sr;
      }
    }
    // the operator of direction j carries dt/dx_j and the sign of the Horner
    // step (v <- g u - L v), so every contribution is an accumulation
    const R sgn = VOL ? R(1) : R(-1);
    R L1[m][n];   // only the group-1 rows are used
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) L1[c][i] = R(0);
    // the derivative line of component c along j: x from this thread's own
    // line, y and z from the owners' results in shared memory
    auto deriv = [&](int j, int c, R (&dl)[n]) {
      if (j == 0) contract_line<n, VOL>(T, v[c], dl);
      else if (j == 1) load_line<R, n>(DYS + S::slotY(c) * NS + t * n, dl);
      else load_line<R, n>(DZS + S::slotZ(c) * NS + t * n, dl);
    };
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Mat mj = mt;
      PDE::scaleA(mj, sgn * sc[j]);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (PDE::group(c) != 0 || !PDE::reads(j, c)) continue;
        R dl[n];
        deriv(j, c, dl);
        PDE::template accA_comp<n>(mj, j, c, dl, L1);
      }
    }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (PDE::group(c) != 0) continue;
#pragma unroll
      for (int i = 0; i < n; ++i) v[c][i] = VOL ? R(0) : gs * u[c][i];
    }
#pragma unroll
    for (int j = 0; j < d; ++j) {
      Mat mj = mt;
      PDE::scaleA(mj, sgn * sc[j]);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (PDE::group(c) != 1 || !PDE::reads(j, c)) continue;
        R dl[n];
        deriv(j, c, dl);
        PDE::template accA_comp<n>(mj, j, c, dl, v);
      }
    }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (PDE::group(c) != 1) continue;
#pragma unroll
      for (int i = 0; i < n; ++i) v[c][i] = (VOL ? R(0) : gs * u[c][i]) + L1[c][i];
    }
    // No barrier at the end, as in LinPass.
  }
};

// The line along axis o that thread t of a cell owns: first node and node
// stride.  x: nodes n t + i; y (3D, owned transposed): i0 = t / n, i2 = t mod n;
// z: i0 = t mod n, i1 = t / n.  face() is the node of the line's end faces.
template <int n, int d>
struct OwnLine {
  __device__ __forceinline__ static int base(int o, int t) {
    return o == 0 ? n * t : (o == 1 ? (d == 3 ? t / n + n * n * (t % n) : t) : t);
  }
  __host__ __device__ static constexpr int stride(int o) { return o == 0 ? 1 : (o == 1 ? n : n * n); }
  __device__ __forceinline__ static int face(int o, int t) {
    return o == 1 && d == 3 ? t / n + n * (t % n) : t;
  }
  template <class R>
  __device__ __forceinline__ static void load(const R *p, int o, R (&x)[n]) {
    if (o == 0) {
      load_line<R, n>(p, x);
    } else {
#pragma unroll
      for (int b = 0; b < n; ++b) x[b] = p[stride(o) * b];
    }
  }
  template <class R>
  __device__ __forceinline__ static void store(R *p, int o, const R (&x)[n]) {
    if (o == 0) {
      store_line<R, n>(p, x);
    } else {
#pragma unroll
      for (int b = 0; b < n; ++b) p[stride(o) * b] = x[b];
    }
  }
};

// LinPass for PDEs whose components live on lines of their own axis
// (PDE::OWNED; v holds component c on this thread's line along
// PDE::owner(c)).  Each thread works the line of every orientation it owns:
// along axis j it differentiates the components A'_j reads (its own lines from
// registers, the others' from the shared copy), keeps the part of A'_j C_j v
// that falls on components it owns along j and hands the rest to their owners
// through the contribution slots.  For 3D acoustics a pass moves p to the y-
// and z-line owners and brings back two lines of p updates: 7 line transfers
// instead of 15.  The update is in place (a line's registers are dead once its
// own axis has read it): a Horner step leaves v <- g_s u - L v, VOL leaves
// v <- L v (C = Kvol) and extrapolates every component to the faces of every
// axis into the hull.  Two block barriers.
template <class K, bool VOL>
struct LinPassOwn {
  using R = typename K::R;
  using PDE = typename K::PDE;
  using O = typename K::O;
  using Mat = typename PDE::Mat;
  using L = OwnLine<K::n, K::d>;
  static constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  // FP32 with even n: packed two-lane FMAs along the line
  static constexpr bool kPacked = std::is_same<R, float>::value && n % 2 == 0;
  template <class TAB>
  __device__ __forceinline__ static void run(const TAB &T, const Mat &mt, const R (&sc)[d], R (&v)[m][n],
                                             const R (&u)[m][n], R gs, R *VS, R *CB, R *hout, long long cell,
                                             int t, bool active) {
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c)
        if (VOL || O::shared(c)) L::store(VS + c * NS + L::base(PDE::owner(c), t), PDE::owner(c), v[c]);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int lb = L::base(j, t);
        R D[m][n];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          if (PDE::reads(j, c) || VOL) {
            R line[n];
            if (PDE::owner(c) == j) {
#pragma unroll
              for (int b = 0; b < n; ++b) line[b] = v[c][b];
            } else {
              L::load(VS + c * NS + lb, j, line);
            }
            if (PDE::reads(j, c)) contract_line<n, VOL>(T, line, D[c]);
            if (VOL) {  // the two faces normal to j at this line's face node
              R sl, sr;
              if constexpr (kPacked) {
                const float2 *P = reinterpret_cast<const float2 *>(T.FLR);
                float2 lr = __fmul2_rn(P[0], make_float2(line[0], line[0]));
#pragma unroll
                for (int b = 1; b < n; ++b) lr = __ffma2_rn(P[b], make_float2(line[b], line[b]), lr);
                sl = lr.x;
                sr = lr.y;
              } else {
                sl = T.FL[0] * line[0];
                sr = T.FR[0] * line[0];
#pragma unroll
                for (int b = 1; b < n; ++b) {
                  sl += T.FL[b] * line[b];
                  sr += T.FR[b] * line[b];
                }
              }
              const int pf = L::face(j, t);
              hout[cell * K::HSL + (2 * j) * K::FSZ + c * NF + pf] = sl;
              hout[cell * K::HSL + (2 * j + 1) * K::FSZ + c * NF + pf] = sr;
            }
          }
        }
        // the lines owned along j have been read: overwrite them
        Mat mj = mt;
        PDE::scaleA(mj, sc[j]);
        R cb[m][n];
        if constexpr (kPacked) {
          // two nodes at a time on packed two-lane multiplies; each lane
          // rounds as the scalar form below does
#pragma unroll
          for (int k = 0; k < n / 2; ++k) {
            float2 dv[m], out[m];
#pragma unroll
            for (int c = 0; c < m; ++c)
              dv[c] = PDE::reads(j, c) ? make_float2(D[c][2 * k], D[c][2 * k + 1]) : make_float2(0.f, 0.f);
            PDE::applyA2(mj, j, dv, out);
#pragma unroll
            for (int c = 0; c < m; ++c) {
              if (PDE::owner(c) == j) {
                const float2 w = PDE::writes(j, c) ? out[c] : make_float2(0.f, 0.f);
                const float2 r = VOL ? w
                                     : __ffma2_rn(make_float2(gs, gs), make_float2(u[c][2 * k], u[c][2 * k + 1]),
                                                  make_float2(-w.x, -w.y));
                v[c][2 * k] = r.x;
                v[c][2 * k + 1] = r.y;
              } else if (PDE::writes(j, c)) {
                cb[c][2 * k] = out[c].x;
                cb[c][2 * k + 1] = out[c].y;
              }
            }
          }
        } else {
#pragma unroll
          for (int o = 0; o < n; ++o) {
            R dv[m], out[m];
#pragma unroll
            for (int c = 0; c < m; ++c) dv[c] = PDE::reads(j, c) ? D[c][o] : R(0);
            PDE::applyA(mj, j, dv, out);
#pragma unroll
            for (int c = 0; c < m; ++c) {
              if (PDE::owner(c) == j) {
                const R w = PDE::writes(j, c) ? out[c] : R(0);
                v[c][o] = VOL ? w : gs * u[c][o] - w;
              } else if (PDE::writes(j, c)) {
                cb[c][o] = out[c];
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (O::cross(j, c)) L::store(CB + O::slot(j, c) * NS + lb, j, cb[c]);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const int oc = PDE::owner(c);
#pragma unroll
        for (int j = 0; j < d; ++j) {
          if (!O::cross(j, c)) continue;
          R x[n];
          L::load(CB + O::slot(j, c) * NS + L::base(oc, t), oc, x);
#pragma unroll
          for (int i = 0; i < n; ++i) v[c][i] = VOL ? v[c][i] + x[i] : v[c][i] - x[i];
        }
      }
    }
    // No barrier at the end, as in LinPass: VS is rewritten by the next pass
    // before its first barrier only at the entries read before this pass's
    // second barrier, and the contribution slots after the next first barrier.
  }
};

// Integer coordinates of a cell (axis 0 fastest) and its periodic neighbours.
struct CellPos {
  long long cell;
  int x[3];
  __device__ __forceinline__ void set(long long c, const int *g, int d) {
    cell = c;
    const long long q = c / g[0];
    x[0] = (int)(c - q * g[0]);
    if (d == 3) {
      const long long r = q / g[1];
      x[1] = (int)(q - r * g[1]);
      x[2] = (int)r;
    } else {
      x[1] = (int)q;
      x[2] = 0;
    }
  }
  // neighbour across face (j, side): side 1 = +x_j
  __device__ __forceinline__ long long nb(int j, int side, const int *g) const {
    const long long stride = j == 0 ? 1 : (j == 1 ? (long long)g[0] : (long long)g[0] * g[1]);
    if (side) return x[j] + 1 == g[j] ? cell - (long long)(g[j] - 1) * stride : cell + stride;
    return x[j] == 0 ? cell + (long long)(g[j] - 1) * stride : cell - stride;
  }
};

// One tile (K::CPB consecutive cells) of the sweep; every thread of the block
// must call it (it contains block barriers).  TAB is Tables<R> in the
// parameter or constant space, so that unrolled coefficients are uniform
// constant-bank operands.  With bar (an initialised mbarrier, K::TMA_QD) the
// corrector's Q and D rows of the tile are brought into shared memory by two
// bulk copies issued at the start of the tile and awaited (phase `parity`)
// only at the update, after the face Riemann problems.  EXT compiles in the
// terms of Eq. 1 beyond the conservative flux (point sources, material jumps
// in non-conservative form); the kernels without them carry none of their
// code or registers.
template <class K, int STAGES, class TAB, bool EXT = false>
__device__ __forceinline__ void lin_tile(const SweepArgs &a, const TAB &T, long long tile, unsigned char *smem,
                                         unsigned long long *bar = nullptr, unsigned parity = 0) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using S = typename K::S;
  using Mat = typename PDE::Mat;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, NL = K::NL, CPB = K::CPB;
  constexpr int THREADS = K::THREADS;
  // Plain FP32 state with even n: the corrector's element-wise work two nodes
  // at a time on packed two-lane FP32 instructions.  Not for the compensated
  // pair (its sweep measured slower with it: 1.764 against 1.716 ms at 64^3,
  // acoustics N = 5) and not for the FP64 state, whose increments must stay
  // those of the pair bit for bit.
  constexpr bool kPk = std::is_same<R, float>::value && std::is_same<QT, float>::value && n % 2 == 0 && !K::PAIR;

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
  const bool uniform = a.mat == nullptr;
  const bool ncp = EXT && a.ncp && !uniform;   // material jumps in non-conservative form

  const int tid = threadIdx.x;
  const int lc = tid / NL;
  const int t = tid - lc * NL;                 // x-line index = i1 + n i2
  const int lcs = lc < CPB ? lc : CPB - 1;
  const int i1 = t % n, i2 = t / n;            // (d = 2: i2 = 0)
  R *VS = work + lcs * K::CELL;                // [m][NS]  line layout: node = i0 + n t
  R *DYS = VS + m * NS;                        // [NY][NS]
  R *DZS = DYS + S::NY * NS;                   // [NZ][NS]
  R *FS = work + lcs * K::FSC;                 // corrector: [2d-2][m][NF]
  const bool tma = K::TMA_QD && bar != nullptr && STAGES != kPredict;
  QT *QS = reinterpret_cast<QT *>(work + CPB * K::FSC);  // staged Q rows [cell][comp][node]
  R *DS = reinterpret_cast<R *>(QS + (size_t)CPB * m * NS);

  // face weights of this thread's line position along y and z
  const R wyR = T.FR[i1] * T.iw[i1], wyL = T.FL[i1] * T.iw[i1];
  const R wzR = d == 3 ? T.FR[i2] * T.iw[i2] : R(0), wzL = d == 3 ? T.FL[i2] * T.iw[i2] : R(0);

  {
  const long long cell = tile * CPB + lc;
  const bool active = lc < CPB && cell < a.ncells;
  const long long cs = active ? cell : 0;
  Mat mt;
  load_mat<PDE>(mt, a.matp, a.cst, a.mat, cs);
  unsigned long long smask = 0ull;  // point sources in this cell
  if (EXT && a.nsrc > 0 && active)
    for (int k = 0; k < a.nsrc; ++k)
      if (a.src[k].cell == cell) smask |= 1ull << k;
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
    if (tma && tid == 0) {
      // the previous tile ended with a block barrier: no generic access to the
      // staging area is outstanding
      const long long c0 = tile * CPB;
      const long long nc = a.ncells - c0 < CPB ? a.ncells - c0 : CPB;
      const unsigned bq = (unsigned)(nc * m * NS * sizeof(QT)), bd = (unsigned)(nc * m * NS * sizeof(R));
      fence_proxy_async();
      mbar_expect_tx(bar, bq + bd);
      tma_load_1d(QS, Qin + c0 * m * NS, bq, bar);
      tma_load_1d(DS, Dbuf + c0 * m * NS, bd, bar);
      // the compensated pair's low words are read straight from global memory
      // at the update: bring the tile's rows into L2 now
      if constexpr (K::PAIR) l2_prefetch_bulk(Qout + (a.ncells + c0) * m * NS, bq);
      // the tile's own face-hull rows (the neighbours' facing sides mostly hit L2)
      if constexpr ((K::HSL * sizeof(R)) % 16 == 0) l2_prefetch_bulk(hin + c0 * K::HSL, (unsigned)(nc * K::HSL * sizeof(R)));
    }
    if (!tma && tid == 0) {
      // no staging (rows that are not 16-byte multiples): bring the tile's Q, D
      // and face-hull rows into L2 ahead of their plain loads
      const long long c0 = tile * CPB;
      const long long nc = a.ncells - c0 < CPB ? a.ncells - c0 : CPB;
      l2_prefetch_range(Qin + c0 * m * NS, (size_t)nc * m * NS * sizeof(QT));
      l2_prefetch_range(Dbuf + c0 * m * NS, (size_t)nc * m * NS * sizeof(R));
      l2_prefetch_range(hin + c0 * K::HSL, (size_t)nc * K::HSL * sizeof(R));
      if constexpr (K::PAIR) l2_prefetch_range(Qout + (a.ncells + c0) * m * NS, (size_t)nc * m * NS * sizeof(QT));
    }
    // face terms first; D and the old state are read only at the update
    R acc[m][n];
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) acc[c][i] = R(0);
    if (active) {
      CellPos pos;
      pos.set(cell, a.grid, d);
      // x faces: face node p = t, F* in registers
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const long long nb = pos.nb(0, side, a.grid);
        const R *own = hin + cell * K::HSL + side * K::FSZ;
        const R *nbr = hin + nb * K::HSL + (side ^ 1) * K::FSZ;
        R qo[m], qn[m], fs[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          qo[c] = ldg(own + c * NF + t);
          qn[c] = ldg(nbr + c * NF + t);
        }
        Mat mn = mt;
        if (!uniform) load_mat<PDE>(mn, a.matp, a.cst, a.mat, nb);
        if (side) rusanov_lin<PDE, R>(mt, mn, 0, qo, qn, fs);
        else rusanov_lin<PDE, R>(mn, mt, 0, qn, qo, fs);
        if constexpr (EXT) {
          if (ncp) ncp_own_side<PDE, R>(mt, mn, 0, qo, qn, fs);
        }
        const R sg = side ? R(1) : R(-1);
        if constexpr (kPk) {
#pragma unroll
          for (int k = 0; k < n / 2; ++k) {
            const float2 nw = make_float2(-(dt_old * idx0 * sg * (side ? T.FR[2 * k] : T.FL[2 * k]) * T.iw[2 * k]),
                                          -(dt_old * idx0 * sg * (side ? T.FR[2 * k + 1] : T.FL[2 * k + 1]) *
                                            T.iw[2 * k + 1]));
#pragma unroll
            for (int c = 0; c < m; ++c) {
              const float2 a2 = __ffma2_rn(nw, make_float2(fs[c], fs[c]), make_float2(acc[c][2 * k], acc[c][2 * k + 1]));
              acc[c][2 * k] = a2.x;
              acc[c][2 * k + 1] = a2.y;
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < n; ++i) {
            const R wgt = dt_old * idx0 * sg * (side ? T.FR[i] : T.FL[i]) * T.iw[i];
#pragma unroll
            for (int c = 0; c < m; ++c) acc[c][i] -= wgt * fs[c];
          }
        }
      }
      // y (z) faces: this thread solves face node p = t of faces 2..2d-1
#pragma unroll
      for (int f = 2; f < 2 * d; ++f) {
        const int j = f >> 1, side = f & 1;
        const long long nb = pos.nb(j, side, a.grid);
        const R *own = hin + cell * K::HSL + f * K::FSZ;
        const R *nbr = hin + nb * K::HSL + (f ^ 1) * K::FSZ;
        R qo[m], qn[m], fs[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          qo[c] = ldg(own + c * NF + t);
          qn[c] = ldg(nbr + c * NF + t);
        }
        Mat mn = mt;
        if (!uniform) load_mat<PDE>(mn, a.matp, a.cst, a.mat, nb);
        if (side) rusanov_lin<PDE, R>(mt, mn, j, qo, qn, fs);
        else rusanov_lin<PDE, R>(mn, mt, j, qn, qo, fs);
        if constexpr (EXT) {
          if (ncp) ncp_own_side<PDE, R>(mt, mn, j, qo, qn, fs);
        }
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
        if constexpr (kPk) {
          const float cy = dt_old * idx1;
#pragma unroll
          for (int k = 0; k < n / 2; ++k) {
            float2 t2 = __fmul2_rn(make_float2(wyR, wyR), make_float2(yr[2 * k], yr[2 * k + 1]));
            t2 = __ffma2_rn(make_float2(-wyL, -wyL), make_float2(yl[2 * k], yl[2 * k + 1]), t2);
            const float2 a2 = __ffma2_rn(make_float2(-cy, -cy), t2, make_float2(acc[c][2 * k], acc[c][2 * k + 1]));
            acc[c][2 * k] = a2.x;
            acc[c][2 * k + 1] = a2.y;
          }
        } else {
#pragma unroll
          for (int i = 0; i < n; ++i) acc[c][i] -= dt_old * idx1 * (wyR * yr[i] - wyL * yl[i]);
        }
        if (d == 3) {
          R zl[n], zr[n];
          load_line<R, n>(FS + (2 * m + c) * NF + pz, zl);
          load_line<R, n>(FS + (3 * m + c) * NF + pz, zr);
          if constexpr (kPk) {
            const float cz = dt_old * idx2;
#pragma unroll
            for (int k = 0; k < n / 2; ++k) {
              float2 t2 = __fmul2_rn(make_float2(wzR, wzR), make_float2(zr[2 * k], zr[2 * k + 1]));
              t2 = __ffma2_rn(make_float2(-wzL, -wzL), make_float2(zl[2 * k], zl[2 * k + 1]), t2);
              const float2 a2 = __ffma2_rn(make_float2(-cz, -cz), t2, make_float2(acc[c][2 * k], acc[c][2 * k + 1]));
              acc[c][2 * k] = a2.x;
              acc[c][2 * k + 1] = a2.y;
            }
          } else {
#pragma unroll
            for (int i = 0; i < n; ++i) acc[c][i] -= dt_old * idx2 * (wzR * zr[i] - wzL * zl[i]);
          }
        }
      }
      if constexpr (EXT) {
        if (smask) {  // point sources: dt_old sum_k w_k s(t_k) sigma
#pragma unroll
          for (int c = 0; c < m; ++c) src_add_line<n, d, R>(a, smask, 0, c, 0, t, acc[c]);
        }
      }
      R chk = R(0);
      if (tma) mbar_wait(bar, parity, ctl);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        QT q[n];
        R dl[n];
        if (tma) {
          load_line<QT, n>(QS + (lc * m + c) * NS + t * n, q);
          load_line<R, n>(DS + (lc * m + c) * NS + t * n, dl);
        } else {
          load_line<QT, n>(Qin + (cell * m + c) * NS + t * n, q);
          load_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, dl);
        }
        if constexpr (K::PAIR) {
          // compensated FP32 pair: the low words sit one state plane further on
          QT *lop = Qout + (a.ncells + cell) * m * NS + c * NS + t * n;
          QT lo[n];
          load_line<QT, n>(lop, lo);
#pragma unroll
          for (int i = 0; i < n; ++i) {
            pair_add(q[i], lo[i], dl[i] + acc[c][i]);
            u[c][i] = q[i];
            chk += u[c][i] * R(0);
          }
          store_line<QT, n>(lop, lo);
        } else if constexpr (kPk && std::is_same<QT, float>::value) {
#pragma unroll
          for (int k = 0; k < n / 2; ++k) {
            const float2 q2 = __fadd2_rn(make_float2(q[2 * k], q[2 * k + 1]),
                                         __fadd2_rn(make_float2(dl[2 * k], dl[2 * k + 1]),
                                                    make_float2(acc[c][2 * k], acc[c][2 * k + 1])));
            q[2 * k] = q2.x;
            q[2 * k + 1] = q2.y;
            u[c][2 * k] = q2.x;
            u[c][2 * k + 1] = q2.y;
            chk += q2.x * R(0);
            chk += q2.y * R(0);
          }
        } else {
#pragma unroll
          for (int i = 0; i < n; ++i) {
            q[i] = q[i] + (QT)(dl[i] + acc[c][i]);
            u[c][i] = (R)q[i];
            chk += u[c][i] * R(0);   // NaN/Inf anywhere in the line survives
          }
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
    // Horner form of q_bar = sum_s g_s (-dt L)^s u, then integrateVolume; the
    // operator of direction j carries dt / dx_j, so a Horner step is one FMA
    R sc[d];
#pragma unroll
    for (int j = 0; j < d; ++j) sc[j] = dt_pred * (j == 0 ? idx0 : (j == 1 ? idx1 : idx2));
    // the point-source coefficients of this predictor (fused, first or rerun sweep)
    const int coi0 = STAGES == kFused ? 1 : (a.pred_dt_old ? 1 + 2 * kMaxPicard : 1 + kMaxPicard);
    R v[m][n], Lv[m][n];
    using L = OwnLine<n, d>;
    if constexpr (K::OWN) {
      // u onto the lines of each component's owner (the corrector and the
      // state rows work on x-lines); the previous barrier ended all use of VS
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (PDE::owner(c) != 0) store_line<R, n>(VS + c * NS + t * n, u[c]);
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (PDE::owner(c) != 0) L::load(VS + c * NS + L::base(PDE::owner(c), t), PDE::owner(c), u[c]);
      }
    }

#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) v[c][i] = T.g[a.picard] * u[c][i];
    for (int s = a.picard - 1; s >= 0; --s) {
      if constexpr (K::OWN) {
        LinPassOwn<K, false>::run(T, mt, sc, v, u, T.g[s], VS, DYS, hout, cell, t, active);
        if constexpr (EXT) {
          if (smask) {  // Horner level s gains dt h_s sigma
#pragma unroll
            for (int c = 0; c < m; ++c) src_add_line<n, d, R>(a, smask, coi0 + s, c, PDE::owner(c), t, v[c]);
          }
        }
      } else if constexpr (K::BIP) {
        LinPassBip<K, false>::run(T, mt, sc, v, u, T.g[s], VS, DYS, DZS, hout, cell, t, active);
        if constexpr (EXT) {
          if (smask) {  // Horner level s gains dt h_s sigma
#pragma unroll
            for (int c = 0; c < m; ++c) src_add_line<n, d, R>(a, smask, coi0 + s, c, 0, t, v[c]);
          }
        }
      } else {
        LinPass<K, false>::run(T, mt, sc, v, Lv, VS, DYS, DZS, hout, cell, t, active);
        const R gs = T.g[s];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R uc[n];
          if (K::U_SMEM) {
            if (active) {
              QT qq[n];
              load_line<QT, n>((STAGES == kPredict ? Qin : Qout) + (cell * m + c) * NS + t * n, qq);
#pragma unroll
              for (int i = 0; i < n; ++i) uc[i] = (R)qq[i];
            } else {
#pragma unroll
              for (int i = 0; i < n; ++i) uc[i] = R(0);
            }
          } else {
#pragma unroll
            for (int i = 0; i < n; ++i) uc[i] = u[c][i];
          }
#pragma unroll
          for (int i = 0; i < n; ++i) v[c][i] = gs * uc[i] - Lv[c][i];
        }
        if constexpr (EXT) {
          if (smask) {  // Horner level s gains dt h_s sigma
#pragma unroll
            for (int c = 0; c < m; ++c) src_add_line<n, d, R>(a, smask, coi0 + s, c, 0, t, v[c]);
          }
        }
      }
    }
    if constexpr (K::OWN) {
      LinPassOwn<K, true>::run(T, mt, sc, v, u, R(0), VS, DYS, hout, cell, t, active);
      // L v back onto x-lines for the coalesced D rows (VS was last read before
      // the pass's second barrier)
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (PDE::owner(c) != 0) L::store(VS + c * NS + L::base(PDE::owner(c), t), PDE::owner(c), v[c]);
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c) {
          if (PDE::owner(c) != 0) {
            R x[n];
            load_line<R, n>(VS + c * NS + t * n, x);
            store_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, x);
          } else {
            store_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, v[c]);
          }
        }
      }
    } else if constexpr (K::BIP) {
      LinPassBip<K, true>::run(T, mt, sc, v, u, R(0), VS, DYS, DZS, hout, cell, t, active);
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c) store_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, v[c]);
      }
    } else {
      LinPass<K, true>::run(T, mt, sc, v, Lv, VS, DYS, DZS, hout, cell, t, active);
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c) store_line<R, n>(Dbuf + (cell * m + c) * NS + t * n, Lv[c]);
      }
    }
    __syncthreads();  // the work area is reused by the next tile
  }
  }
}

template <class K, int STAGES, bool EXT = false>
__global__ void __launch_bounds__(K::THREADS, K::MINB) lin_sweep_kernel(const SweepArgs a, const Tables<typename K::R> T) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bar;
  if (STAGES == kPredict && a.gate) {
    if (*(volatile int *)&a.ctl->rerun == 0) return;  // uniform for the whole grid
  }
  constexpr bool TMA = K::TMA_QD && STAGES != kPredict;
  if (TMA) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  unsigned k = 0;
  for (long long tile = a.tile_lo + blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++k)
    lin_tile<K, STAGES, Tables<typename K::R>, EXT>(a, T, tile, smem, TMA ? &bar : nullptr, k & 1u);
}

}  // namespace aderdg
