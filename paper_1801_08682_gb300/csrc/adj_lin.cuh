// adj_lin.cuh -- the adjoint cell kernel of the step (see adjoint.cuh for the
// formulas) in the line-owner layout of the forward sweep (sweep_lin.cuh):
// one thread per x-line of a cell, all components of the line in registers,
// y- and z-contractions by the owners of the y- and z-columns through shared
// memory, every coefficient a kernel-parameter (constant-bank) operand.
//
// Per tile of CPB cells (Alg. 2's step run backwards, term by term):
//   (gm) forward powers z_s = Lt^s u, s = 0..R-1, of the cell's predictor and
//        its time average qbar = sum_s g_s z_s; z_1..z_{R-1} go to a scratch
//        slot private to the block (the kernel loops over tiles, so the
//        scratch is sized by the grid of blocks, not by the mesh)
//   (gm) volume term  sum_j sc_j <lam, dA_j Kvol_j qbar>
//   face adjoints q*_f from psi (Rusanov transpose, face material terms)
//   qbar* = sum_f E_f^T q*_f + sum_j sc_j A_j^T Kvol_j^T lam
//   adjoint Horner  y_R = g_R qbar*,  y_s = g_s qbar* + Lt^T y_{s+1}
//   (gm) Horner term  sum_{s<R} <y_{s+1}, dLt z_s>, dLt = -sum_j sc_j dA_j D_j
//   lam_out = lam + y_0
// with sc_j = dt / dx_j and Lt = -sum_j sc_j A_j D_j.  A_j and the 1D
// contraction C_j act on different indices, so A_j C_j = C_j A_j and the
// transposed operator is sum_j sc_j C_j^T A_j^T: the transposed passes apply
// A_j^T at each node first and contract with C^T (tables built from Dm^T and
// Kvol^T) after the exchange.  The operators are bipartite (acoustics: p <->
// v; elasticity: stresses <-> velocities), so each pass updates its lines in
// place, group by group.
#pragma once
#include "adjoint.cuh"

namespace aderdg {

// Groups of a bipartite operator: A_j[r][c] != 0 only if group(r) != group(c).
template <class PDE>
struct AdjGroups;
template <int d, class R>
struct AdjGroups<Acoustics<d, R>> {
  __host__ __device__ static constexpr int group(int c) { return c == 0 ? 0 : 1; }
};
template <int d, class R>
struct AdjGroups<Elasticity<d, R>> {
  __host__ __device__ static constexpr int group(int c) { return Elasticity<d, R>::group(c); }
};

// Layout and launch shape.  Per cell: one exchange set of the components
// A_y and A_z read (y slots, then z slots), and the face adjoints
// q*[2d][m][NF] over the start of the same area.
template <class K>
struct AdjLinCfg {
  using R = typename K::R;
  using PDE = typename K::PDE;
  using G = AdjGroups<PDE>;
  static constexpr int d = K::d, N = K::N, n = K::n, m = K::m, NS = K::NS, NF = K::NF, NL = NF;
  __host__ __device__ static constexpr int nread(int j) {
    int k = 0;
    for (int c = 0; c < m; ++c) k += PDE::reads(j, c) ? 1 : 0;
    return k;
  }
  __host__ __device__ static constexpr int slot(int j, int c) {
    int k = 0;
    for (int cc = 0; cc < c; ++cc) k += PDE::reads(j, cc) ? 1 : 0;
    return k;
  }
  static constexpr int NRY = nread(1), NRZ = d == 3 ? nread(2) : 0;
  static constexpr int XS = (NRY + NRZ) * NS;   // one exchange set
  static constexpr int CELL0 = round_up(cmax(XS, 2 * d * m * NF), 4);
  // 25-line cells (3D, N = 4: scalar lines) straddle warps; a bank model of the
  // x-line, y- and z-column and face accesses puts 21 % fewer wavefronts on a
  // stride of 29 (mod 32) than on the 16-byte multiple
  static constexpr int CELL = NL == 25 ? CELL0 + ((29 - CELL0 % 32) % 32 + 32) % 32 : CELL0;
  static constexpr int CPB = cmax(1, cmin(256 / NL, (72 * 1024) / (CELL * (int)sizeof(R))));
  static constexpr int THREADS = round_up(CPB * NL, 32);
  static constexpr int MINB = THREADS <= 160 ? 3 : 2;
  static constexpr size_t SMEM = (size_t)CPB * 4 * sizeof(double) + (size_t)CPB * CELL * sizeof(R);
  static constexpr int ZLEVEL = CPB * m * NS;     // scratch elements of one level of one block
};

template <class C>
struct AdjLin {
  using R = typename C::R;
  using PDE = typename C::PDE;
  using G = typename C::G;
  using Mat = typename PDE::Mat;
  static constexpr int d = C::d, n = C::n, m = C::m, NS = C::NS;

  __device__ __forceinline__ static R *slot_ptr(R *set, int j, int c) {
    return set + (j == 1 ? C::slot(1, c) : C::NRY + C::slot(2, c)) * NS;
  }

  // The exchange of one pass.  Before the first barrier each x-line owner has
  // written its lines into the set; between the barriers the owner of y-column
  // t (3D: i0 = t / n, i2 = t mod n) and of z-column t (i0 = t mod n,
  // i1 = t / n) contracts every slot along its column in place (no other
  // thread touches that column); after the second barrier the x-line owners
  // read their lines back.
  template <bool VOL, class TAB>
  __device__ __forceinline__ static void contract_columns(const TAB &T, R *set, int t) {
    const int y0 = d == 3 ? t / n + n * n * (t % n) : t;
#pragma unroll
    for (int k = 0; k < C::NRY; ++k) {
      R col[n], out[n];
      R *p = set + k * NS + y0;
#pragma unroll
      for (int b = 0; b < n; ++b) col[b] = p[n * b];
      contract_line<n, VOL>(T, col, out);
#pragma unroll
      for (int o = 0; o < n; ++o) p[n * o] = out[o];
    }
    if constexpr (d == 3) {
#pragma unroll
      for (int k = 0; k < C::NRZ; ++k) {
        R col[n], out[n];
        R *p = set + (C::NRY + k) * NS + t;
#pragma unroll
        for (int b = 0; b < n; ++b) col[b] = p[n * n * b];
        contract_line<n, VOL>(T, col, out);
#pragma unroll
        for (int o = 0; o < n; ++o) p[n * n * o] = out[o];
      }
    }
  }

  // Forward pass: x <- sgn sum_j sc_j A_j C_j x (+ gs base), C = Dm or Kvol
  // (VOL), T the forward tables.  In place: the rows of group 1 from the old
  // group-0 lines into L1, then group 0 from the old group-1 lines, then
  // group 1 from L1.  Two block barriers.
  template <bool VOL, bool BASE, class TAB>
  __device__ __forceinline__ static void fwd(const TAB &T, const Mat &mt, const R (&sc)[d], R sgn, R (&x)[m][n],
                                             const R (&base)[m][n], R gs, R *set, int t, bool active) {
    if (active) {
#pragma unroll
      for (int j = 1; j < d; ++j)
#pragma unroll
        for (int c = 0; c < m; ++c)
          if (PDE::reads(j, c)) store_line<R, n>(slot_ptr(set, j, c) + t * n, x[c]);
    }
    __syncthreads();
    if (active) contract_columns<VOL>(T, set, t);
    __syncthreads();
    if (!active) return;
    Mat ms[d];
#pragma unroll
    for (int j = 0; j < d; ++j) {
      ms[j] = mt;
      PDE::scaleA(ms[j], sgn * sc[j]);
    }
    auto deriv = [&](int j, int c, R (&dl)[n]) {
      if (j == 0) contract_line<n, VOL>(T, x[c], dl);
      else load_line<R, n>(slot_ptr(set, j, c) + t * n, dl);
    };
    R L1[m][n];
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) L1[c][i] = R(0);
#pragma unroll
    for (int j = 0; j < d; ++j)
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (G::group(c) != 0 || !PDE::reads(j, c)) continue;
        R dl[n];
        deriv(j, c, dl);
        PDE::template accA_comp<n>(ms[j], j, c, dl, L1);
      }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (G::group(c) != 0) continue;
#pragma unroll
      for (int i = 0; i < n; ++i) x[c][i] = BASE ? gs * base[c][i] : R(0);
    }
#pragma unroll
    for (int j = 0; j < d; ++j)
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (G::group(c) != 1 || !PDE::reads(j, c)) continue;
        R dl[n];
        deriv(j, c, dl);
        PDE::template accA_comp<n>(ms[j], j, c, dl, x);
      }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (G::group(c) != 1) continue;
#pragma unroll
      for (int i = 0; i < n; ++i) x[c][i] = (BASE ? gs * base[c][i] : R(0)) + L1[c][i];
    }
  }

  // (A'_0^T x)_c along this thread's x-line (node by node; only the terms of
  // row c survive), A'_0 = ms0.
  __device__ __forceinline__ static void at_line(const Mat &ms0, int c, const R (&x)[m][n], R (&out)[n]) {
#pragma unroll
    for (int o = 0; o < n; ++o) {
      R xn[m], on[m];
#pragma unroll
      for (int k = 0; k < m; ++k) xn[k] = x[k][o];
      PDE::applyAT(ms0, 0, xn, on);
      out[o] = on[c];
    }
  }

  // Transposed pass: x <- sgn sum_j sc_j C_j^T A_j^T x (+ gs base), TT the
  // transposed tables (C^T = Dm^T or Kvol^T, VOL).  A_j^T is applied at each
  // node before the exchange, so the y/z owners only contract.  In place,
  // group by group as in fwd.  Two block barriers.
  template <bool VOL, bool BASE, class TAB>
  __device__ __forceinline__ static void adj(const TAB &TT, const Mat &mt, const R (&sc)[d], R sgn, R (&x)[m][n],
                                             const R (&base)[m][n], R gs, R *set, int t, bool active) {
    Mat ms[d];
#pragma unroll
    for (int j = 0; j < d; ++j) {
      ms[j] = mt;
      PDE::scaleA(ms[j], sgn * sc[j]);
    }
    if (active) {
#pragma unroll
      for (int j = 1; j < d; ++j)
#pragma unroll
        for (int o = 0; o < n; ++o) {
          R xn[m], on[m];
#pragma unroll
          for (int k = 0; k < m; ++k) xn[k] = x[k][o];
          PDE::applyAT(ms[j], j, xn, on);
#pragma unroll
          for (int c = 0; c < m; ++c)
            if (PDE::reads(j, c)) slot_ptr(set, j, c)[t * n + o] = on[c];
        }
    }
    __syncthreads();
    if (active) contract_columns<VOL>(TT, set, t);
    __syncthreads();
    if (!active) return;
    // rows of group 1 (from the old group-0 lines)
    R L1[m][n];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (G::group(c) != 1) continue;
      R acc[n];
      if (PDE::reads(0, c)) {
        R pre[n];
        at_line(ms[0], c, x, pre);
        contract_line<n, VOL>(TT, pre, acc);
      } else {
#pragma unroll
        for (int i = 0; i < n; ++i) acc[i] = R(0);
      }
#pragma unroll
      for (int j = 1; j < d; ++j) {
        if (!PDE::reads(j, c)) continue;
        R dl[n];
        load_line<R, n>(slot_ptr(set, j, c) + t * n, dl);
#pragma unroll
        for (int i = 0; i < n; ++i) acc[i] += dl[i];
      }
#pragma unroll
      for (int i = 0; i < n; ++i) L1[c][i] = acc[i];
    }
    // rows of group 0 in place (they read only the group-1 lines, still old)
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (G::group(c) != 0) continue;
      R acc[n];
      if (PDE::reads(0, c)) {
        R pre[n];
        at_line(ms[0], c, x, pre);
        contract_line<n, VOL>(TT, pre, acc);
      } else {
#pragma unroll
        for (int i = 0; i < n; ++i) acc[i] = R(0);
      }
#pragma unroll
      for (int j = 1; j < d; ++j) {
        if (!PDE::reads(j, c)) continue;
        R dl[n];
        load_line<R, n>(slot_ptr(set, j, c) + t * n, dl);
#pragma unroll
        for (int i = 0; i < n; ++i) acc[i] += dl[i];
      }
#pragma unroll
      for (int i = 0; i < n; ++i) x[c][i] = (BASE ? gs * base[c][i] : R(0)) + acc[i];
    }
#pragma unroll
    for (int c = 0; c < m; ++c) {
      if (G::group(c) != 1) continue;
#pragma unroll
      for (int i = 0; i < n; ++i) x[c][i] = (BASE ? gs * base[c][i] : R(0)) + L1[c][i];
    }
  }

  // Material terms: g[k] += sgn sum_j sc_j <w, dA_j^(k) C_j x> summed over
  // this thread's line, C = Dm or Kvol (VOL), T the forward tables; loadx(c,
  // line) yields this thread's x-line of component c, read once: the x
  // contraction and its term are done before the exchange.  Two block barriers.
  template <bool VOL, class TAB, class LOADX>
  __device__ __forceinline__ static void dots(const TAB &T, const Mat &mt, const R (&sc)[d], R sgn,
                                              const R (&w)[m][n], LOADX &&loadx, R *set, int t, bool active,
                                              R (&g)[3]) {
    R gl[3] = {R(0), R(0), R(0)};
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const bool ry = d > 1 && PDE::reads(1, c), rz = d > 2 && PDE::reads(2, c);
        if (!PDE::reads(0, c) && !ry && !rz) continue;
        R xl[n];
        loadx(c, xl);
        if (ry) store_line<R, n>(slot_ptr(set, 1, c) + t * n, xl);
        if (rz) store_line<R, n>(slot_ptr(set, 2, c) + t * n, xl);
        if (PDE::reads(0, c)) {
          R dl[n];
          contract_line<n, VOL>(T, xl, dl);
          PDE::template dA_comp<n>(mt, 0, c, w, dl, gl);
        }
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] += sgn * sc[0] * gl[k];
    }
    __syncthreads();
    if (active) contract_columns<VOL>(T, set, t);
    __syncthreads();
    if (!active) return;
#pragma unroll
    for (int j = 1; j < d; ++j) {
#pragma unroll
      for (int k = 0; k < 3; ++k) gl[k] = R(0);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (!PDE::reads(j, c)) continue;
        R dl[n];
        load_line<R, n>(slot_ptr(set, j, c) + t * n, dl);
        PDE::template dA_comp<n>(mt, j, c, w, dl, gl);
      }
      const R f = sgn * sc[j];
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] += f * gl[k];
    }
  }
};

// The per-cell halves of Phi on the faces:
//   psi[c][f][comp][p] = (side ? -1 : +1) dt h_j sum_a (side ? FR_a : FL_a)/w_a lam_c(node(p, j, a)).
// Thread t of a cell takes face node p = t of all 2d faces: the lines through
// it along x (nodes n t + a), y (i0 + n a + n^2 i2 with p = i0 + n i2) and z
// (t + n^2 a), two weighted sums each.
template <class C>
__global__ void __launch_bounds__(256) adj_faces_lin_kernel(const AdjArgs a) {
  using R = typename C::R;
  constexpr int d = C::d, n = C::n, m = C::m, NS = C::NS, NF = C::NF;
  constexpr int FC = cmax(1, 256 / NF);  // cells per block
  const int lc = threadIdx.x / NF, t = threadIdx.x - lc * NF;
  if (lc >= FC) return;
  const Tables<R> *T = reinterpret_cast<const Tables<R> *>(a.tables);
  R wl[n], wr[n], sc[d];
#pragma unroll
  for (int b = 0; b < n; ++b) {
    wl[b] = T->FL[b] * T->iw[b];
    wr[b] = T->FR[b] * T->iw[b];
  }
#pragma unroll
  for (int j = 0; j < d; ++j) sc[j] = adj_scale<R>(a, j);
  int base[3];
  base[0] = n * t;
  base[1] = d == 3 ? t % n + n * n * (t / n) : t;
  base[2] = t;
  const R *lam = reinterpret_cast<const R *>(a.lam_in);
  R *psi = reinterpret_cast<R *>(a.psi);
  for (long long cell = (long long)blockIdx.x * FC + lc; cell < a.ncells; cell += (long long)gridDim.x * FC) {
#pragma unroll
    for (int c = 0; c < m; ++c) {
      const R *src = lam + (cell * m + c) * NS;
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int st = j == 0 ? 1 : (j == 1 ? n : n * n);
        R sl = R(0), sr = R(0);
#pragma unroll
        for (int b = 0; b < n; ++b) {
          const R x = src[base[j] + st * b];
          sl += wl[b] * x;
          sr += wr[b] * x;
        }
        psi[((cell * 2 * d + 2 * j) * m + c) * NF + t] = sc[j] * sl;
        psi[((cell * 2 * d + 2 * j + 1) * m + c) * NF + t] = -sc[j] * sr;
      }
    }
  }
}

// One adjoint step for the cells of a grid-stride set of tiles.  T holds the
// forward operator tables, TT the same tables built from Dm^T and Kvol^T.
template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    adj_lin_kernel(const AdjArgs a, const Tables<typename C::R> T, const Tables<typename C::R> TT) {
  using R = typename C::R;
  using PDE = typename C::PDE;
  using Mat = typename PDE::Mat;
  using L = AdjLin<C>;
  constexpr int d = C::d, n = C::n, m = C::m, NS = C::NS, NF = C::NF, NL = C::NL, CPB = C::CPB;
  constexpr int THREADS = C::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  double *red = reinterpret_cast<double *>(smem);  // [CPB][4] material sums of the tile's cells
  R *work = reinterpret_cast<R *>(smem + CPB * 4 * sizeof(double));
  const int tid = threadIdx.x;
  const int lc = tid / NL, t = tid - lc * NL;
  const int lcs = lc < CPB ? lc : CPB - 1;
  const int i1 = t % n, i2 = t / n;  // digits of the x-line (d = 2: i2 = 0)
  R *set = work + lcs * C::CELL;
  const int Rp = a.picard;
  const bool gm = PDE::NMAT > 0 && a.gmat != nullptr;
  R sc[d];
#pragma unroll
  for (int j = 0; j < d; ++j) sc[j] = adj_scale<R>(a, j);
  const R *lam_in = reinterpret_cast<const R *>(a.lam_in);
  R *lam_out = reinterpret_cast<R *>(a.lam_out);
  const R *Qk = reinterpret_cast<const R *>(a.Qk);
  const R *psi = reinterpret_cast<const R *>(a.psi);
  const R *hull = reinterpret_cast<const R *>(a.hull);
  R *zs = reinterpret_cast<R *>(a.zs);
  const long long ntiles = (a.ncells + CPB - 1) / CPB;

  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long cell = tile * CPB + lc;
    const bool active = lc < CPB && cell < a.ncells;
    const long long cs = active ? cell : 0;
    for (int i = tid; i < 4 * CPB; i += THREADS) red[i] = 0.0;
    Mat mt;
    load_mat<PDE>(mt, a.matp, a.cst, a.mat, cs);
    R y[m][n], qs[m][n];
    R g3[3] = {R(0), R(0), R(0)};
    // this block's scratch line of component c at forward power s (1 <= s < R)
    auto zline = [&](int s, int c) -> R * {
      return zs + (((long long)blockIdx.x * (Rp - 1) + (s - 1)) * CPB + lcs) * m * NS + c * NS + t * n;
    };
    auto load_rows = [&](const R *src, R (&x)[m][n]) {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        if (active) load_line<R, n>(src + (cs * m + c) * NS + t * n, x[c]);
        else {
#pragma unroll
          for (int i = 0; i < n; ++i) x[c][i] = R(0);
        }
      }
    };

    if (gm) {
      // ---- forward powers z_s = Lt^s u and the time average qbar (in qs)
      load_rows(Qk, y);
#pragma unroll
      for (int c = 0; c < m; ++c)
#pragma unroll
        for (int i = 0; i < n; ++i) qs[c][i] = T.g[0] * y[c][i];
      for (int s = 0; s < Rp; ++s) {
        if (s >= 1 && active) {
#pragma unroll
          for (int c = 0; c < m; ++c) store_line<R, n>(zline(s, c), y[c]);
        }
        L::template fwd<false, false>(T, mt, sc, R(-1), y, y, R(0), set, t, active);
        const R gs = T.g[s + 1];
#pragma unroll
        for (int c = 0; c < m; ++c)
#pragma unroll
          for (int i = 0; i < n; ++i) qs[c][i] += gs * y[c][i];
      }
      // ---- volume term <lam, dt h_j dA_j Kvol_j qbar>
      load_rows(lam_in, y);
      L::template dots<true>(T, mt, sc, R(1), y,
                             [&](int c, R (&xl)[n]) {
#pragma unroll
                               for (int i = 0; i < n; ++i) xl[i] = qs[c][i];
                             },
                             set, t, active, g3);
    } else {
      load_rows(lam_in, y);
    }
    __syncthreads();  // the exchange sets are read: the area takes the face adjoints

    // ---- face adjoints: this thread takes face node p = t of its cell's 2d
    // faces (Phi = psi of both sides, q* of the own side, the face material
    // terms)
    R gsp = R(0);
    if (active) {
      R *dst = work + lc * C::CELL;
      CellPos pos;
      pos.set(cell, a.grid, d);
#pragma unroll
      for (int f = 0; f < 2 * d; ++f) {
        const int j = f >> 1, side = f & 1;
        const long long nb = pos.nb(j, side, a.grid);
        Mat mn;
        load_mat<PDE>(mn, a.matp, a.cst, a.mat, nb);
        R phi[m], at[m];
#pragma unroll
        for (int c = 0; c < m; ++c)
          phi[c] = psi[((cell * 2 * d + f) * m + c) * NF + t] + psi[((nb * 2 * d + (f ^ 1)) * m + c) * NF + t];
        const R s2 = PDE::speed(mt, phi, j), sn = PDE::speed(mn, phi, j);  // linear: state-independent
        const R s = s2 > sn ? s2 : sn;
        PDE::applyAT(mt, j, phi, at);
#pragma unroll
        for (int c = 0; c < m; ++c)
          dst[(f * m + c) * NF + t] = R(0.5) * at[c] + (side ? R(0.5) : R(-0.5)) * s * phi[c];
        if (gm) {
          R qc[m], qn[m], gl[4] = {R(0), R(0), R(0), R(0)};
#pragma unroll
          for (int c = 0; c < m; ++c) {
            qc[c] = hull[cell * a.hsl + f * a.fsz + c * NF + t];
            qn[c] = hull[nb * a.hsl + (f ^ 1) * a.fsz + c * NF + t];
          }
          PDE::dA(mt, j, phi, qc, gl);
#pragma unroll
          for (int k = 0; k < 3; ++k) g3[k] += R(0.5) * gl[k];
          const bool selected = side ? (s2 >= sn) : (s2 > sn);
          if (selected) {
            R gs = R(0);
#pragma unroll
            for (int c = 0; c < m; ++c) gs += phi[c] * (side ? (qn[c] - qc[c]) : (qc[c] - qn[c]));
            gsp -= R(0.5) * gs;
          }
        }
      }
    }
    __syncthreads();

    // ---- qbar* = sum_f E_f^T q*_f along this thread's x-line
    if (active) {
      const R *qf = work + lc * C::CELL;
#pragma unroll
      for (int c = 0; c < m; ++c) {
        const R xl = qf[(0 * m + c) * NF + t], xr = qf[(1 * m + c) * NF + t];
#pragma unroll
        for (int i0 = 0; i0 < n; ++i0) {
          R v = T.FL[i0] * xl + T.FR[i0] * xr;
          v += T.FL[i1] * qf[(2 * m + c) * NF + i0 + n * i2] + T.FR[i1] * qf[(3 * m + c) * NF + i0 + n * i2];
          if constexpr (d == 3)
            v += T.FL[i2] * qf[(4 * m + c) * NF + i0 + n * i1] + T.FR[i2] * qf[(5 * m + c) * NF + i0 + n * i1];
          qs[c][i0] = v;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < m; ++c)
#pragma unroll
        for (int i = 0; i < n; ++i) qs[c][i] = R(0);
    }
    __syncthreads();  // the face adjoints are read: the area is an exchange set again

    // ---- + sum_j sc_j Kvol_j^T A_j^T lam (in place on the lam lines)
    L::template adj<true, false>(TT, mt, sc, R(1), y, y, R(0), set, t, active);
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) qs[c][i] += y[c][i];

    // ---- adjoint Horner y_s = g_s qbar* + Lt^T y_{s+1}, with the material
    // term <y_{s+1}, dLt z_s> of each level
#pragma unroll
    for (int c = 0; c < m; ++c)
#pragma unroll
      for (int i = 0; i < n; ++i) y[c][i] = T.g[Rp] * qs[c][i];
    for (int s = Rp - 1; s >= 0; --s) {
      if (gm) {
        L::template dots<false>(T, mt, sc, R(-1), y,
                                [&](int c, R (&xl)[n]) {
                                  if (!active) {
#pragma unroll
                                    for (int i = 0; i < n; ++i) xl[i] = R(0);
                                  } else if (s == 0) {
                                    load_line<R, n>(Qk + (cs * m + c) * NS + t * n, xl);
                                  } else {
                                    load_line<R, n>(zline(s, c), xl);
                                  }
                                },
                                set, t, active, g3);
      }
      L::template adj<false, true>(TT, mt, sc, R(-1), y, qs, T.g[s], set, t, active);
    }
    if (active) {
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R l[n];
        load_line<R, n>(lam_in + (cell * m + c) * NS + t * n, l);
#pragma unroll
        for (int i = 0; i < n; ++i) l[i] += y[c][i];
        store_line<R, n>(lam_out + (cell * m + c) * NS + t * n, l);
      }
    }

    // ---- material gradient of the tile's cells, chained to (rho, cp, cs)
    if (gm) {
      if (active) {
#pragma unroll
        for (int k = 0; k < 3; ++k) atomicAdd(&red[lc * 4 + k], (double)g3[k]);
        atomicAdd(&red[lc * 4 + 3], (double)gsp);
      }
      __syncthreads();
      if (tid < CPB) {
        const long long c2 = tile * CPB + tid;
        if (c2 < a.ncells && a.mat) {
          const double rho = a.mat[3 * c2], cp = a.mat[3 * c2 + 1], csh = a.mat[3 * c2 + 2];
          const double gl = red[tid * 4 + 0], gmu = red[tid * 4 + 1], gi = red[tid * 4 + 2], gsv = red[tid * 4 + 3];
          a.gmat[3 * c2 + 0] += gl * (cp * cp - 2.0 * csh * csh) + gmu * csh * csh - gi / (rho * rho);
          a.gmat[3 * c2 + 1] += gl * 2.0 * rho * cp + gsv;
          a.gmat[3 * c2 + 2] += -4.0 * rho * csh * gl + 2.0 * rho * csh * gmu;
        }
      }
    }
    __syncthreads();  // red and the work area are reused by the next tile
  }
}

}  // namespace aderdg
