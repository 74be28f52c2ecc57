// multipass.cuh -- the plain multi-pass form of one ADER-DG step
// (Algorithm 1, left) with the task outputs of Table 1 stored explicitly:
//   phase 0 predict      Q -> st = (q^, F_0(q^), .., F_{d-1}(q^)) over space-time,
//                        (d+1) m (N+1)^{d+1} values per cell
//   phase 1 extrapolate  st -> space-time face data, 4d m (N+1)^d per cell
//   phase 2 solveRiemann face data of both sides -> F* integrated over the
//                        step (global time stepping needs no space-time F*)
//   phase 3 corrector    integrateVolume over the space-time fluxes,
//                        integrateFace, update, calcTimeStep
// Every phase uses dt_old of the control block (Alg. 1: one dt per step).
#pragma once
#include "sweep.cuh"

namespace aderdg {

// phase 0: the predictor of the fused path, writing the space-time result.
template <class K>
__global__ void __launch_bounds__(K::THREADS) t1_predict_kernel(const MultiArgs a) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, CPB = K::CPB, THREADS = K::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  Tables<R> &T = *reinterpret_cast<Tables<R> *>(smem);
  R *work = reinterpret_cast<R *>(smem + tables_bytes<R>());
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.tables);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(Tables<R>) / 4); i += THREADS) dst[i] = src[i];
  }
  const R dt = (R)a.ctl->dt_old;
  const QT *Q = reinterpret_cast<const QT *>(a.Q_in);
  R *st = reinterpret_cast<R *>(a.st);
  R inv_dx[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) inv_dx[j] = (R)a.inv_dx[j];
  __syncthreads();
  const int lc = threadIdx.x / NS, node = threadIdx.x - lc * NS;
  const int lcs = lc < CPB ? lc : CPB - 1;  // padding threads read in-bounds shared memory
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool active = lc < CPB && cell < a.ncells;
  typename PDE::Mat mt;
  PDE::load(mt, a.cst, a.mat, active ? cell : 0);
  R u[m];
#pragma unroll
  for (int c = 0; c < m; ++c) u[c] = active ? (R)Q[(cell * m + c) * NS + node] : R(0);
  R qh[n][m];
  if (K::PRED == kTimeModal) {
    // q^_k = sum_s (-dt)^s c_s[k] L^s u, accumulated term by term
    R *V = work;
    R w[m];
#pragma unroll
    for (int c = 0; c < m; ++c) w[c] = u[c];
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) qh[k][c] = u[c];  // c_0 = 1
    R fac = R(1);
    for (int s = 1; s <= a.picard; ++s) {
      if (active) {
#pragma unroll
        for (int c = 0; c < m; ++c) V[(lc * m + c) * NS + node] = w[c];
      }
      __syncthreads();
      R Lw[m];
#pragma unroll
      for (int c = 0; c < m; ++c) Lw[c] = R(0);
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int ij = I::digit(node, j);
        R dv[m], out[m];
#pragma unroll
        for (int c = 0; c < m; ++c) {
          dv[c] = R(0);
          if (PDE::reads(j, c)) {
#pragma unroll
            for (int b = 0; b < n; ++b) dv[c] += T.Dm[ij * n + b] * V[(lcs * m + c) * NS + I::with_axis(node, j, b)];
          }
        }
        PDE::applyA(mt, j, dv, out);
#pragma unroll
        for (int c = 0; c < m; ++c) Lw[c] += inv_dx[j] * out[c];
      }
      __syncthreads();
      fac *= -dt;
#pragma unroll
      for (int c = 0; c < m; ++c) w[c] = Lw[c];
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int c = 0; c < m; ++c) qh[k][c] += fac * T.cvec[s * n + k] * w[c];
    }
  } else {
    R *Fst = work;  // [CPB][d][n][m][NS]
#pragma unroll
    for (int k = 0; k < n; ++k)
#pragma unroll
      for (int c = 0; c < m; ++c) qh[k][c] = u[c];
    for (int r = 0; r < a.picard; ++r) {
      if (active) {
#pragma unroll
        for (int k = 0; k < n; ++k)
#pragma unroll
          for (int j = 0; j < d; ++j) {
            R f[m];
            PDE::flux(mt, qh[k], j, f);
#pragma unroll
            for (int c = 0; c < m; ++c) Fst[(((lc * d + j) * n + k) * m + c) * NS + node] = f[c];
          }
      }
      __syncthreads();
      R rhs[n][m];
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R div = R(0);
#pragma unroll
          for (int j = 0; j < d; ++j) {
            const int ij = I::digit(node, j);
            R sj = R(0);
#pragma unroll
            for (int b = 0; b < n; ++b)
              sj += T.Dm[ij * n + b] * Fst[(((lcs * d + j) * n + k) * m + c) * NS + I::with_axis(node, j, b)];
            div += inv_dx[j] * sj;
          }
          rhs[k][c] = T.FL[k] * u[c] - T.w[k] * dt * div;
        }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < n; ++k)
#pragma unroll
        for (int c = 0; c < m; ++c) {
          R s = R(0);
#pragma unroll
          for (int l = 0; l < n; ++l) s += T.K1inv[k * n + l] * rhs[l][c];
          qh[k][c] = s;
        }
    }
  }
  if (!active) return;
  const long long blk = (long long)n * m * NS;
  R *dst = st + cell * (d + 1) * blk;
#pragma unroll
  for (int k = 0; k < n; ++k) {
#pragma unroll
    for (int c = 0; c < m; ++c) dst[(k * m + c) * NS + node] = qh[k][c];
#pragma unroll
    for (int j = 0; j < d; ++j) {
      R f[m];
      PDE::flux(mt, qh[k], j, f);
#pragma unroll
      for (int c = 0; c < m; ++c) dst[(1 + j) * blk + (k * m + c) * NS + node] = f[c];
    }
  }
}

// phase 1: extrapolate q^ and F_j(q^) to the faces at every time node.
// face_st layout [cell][f][v][k][comp][fnode].
template <class K>
__global__ void __launch_bounds__(256) t1_extrapolate_kernel(const MultiArgs a) {
  using R = typename K::R;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF;
  __shared__ R phi[2][kMaxn];
  const Tables<R> *T = reinterpret_cast<const Tables<R> *>(a.tables);
  if (threadIdx.x < n) { phi[0][threadIdx.x] = T->FL[threadIdx.x]; phi[1][threadIdx.x] = T->FR[threadIdx.x]; }
  __syncthreads();
  const R *st = reinterpret_cast<const R *>(a.st);
  R *fo = reinterpret_cast<R *>(a.face_st);
  const long long per_cell = (long long)2 * d * 2 * n * m * NF;
  const long long total = a.ncells * per_cell;
  const long long blk = (long long)n * m * NS;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long cell = t / per_cell;
    int r = (int)(t % per_cell);
    const int p = r % NF; r /= NF;
    const int c = r % m; r /= m;
    const int k = r % n; r /= n;
    const int v = r % 2; r /= 2;
    const int f = r;
    const int j = f >> 1;
    const R *src = st + cell * (d + 1) * blk + (v == 0 ? 0 : (1 + j)) * blk + (k * m + c) * NS;
    R s = R(0);
#pragma unroll
    for (int b = 0; b < n; ++b) s += phi[f & 1][b] * src[I::node_of_face(p, j, b)];
    fo[t] = s;
  }
}

// phase 2: Rusanov on every face once; s from the time-averaged face states.
template <class K>
__global__ void __launch_bounds__(256) t1_riemann_kernel(const MultiArgs a) {
  using R = typename K::R;
  using PDE = typename K::PDE;
  constexpr int d = K::d, n = K::n, m = K::m, NF = K::NF;
  constexpr int RFPB = cmax(1, 256 / NF);
  __shared__ R smax[RFPB];
  __shared__ R wk[kMaxn];
  const Tables<R> *T = reinterpret_cast<const Tables<R> *>(a.tables);
  if (threadIdx.x < n) wk[threadIdx.x] = T->w[threadIdx.x];
  const R *fi = reinterpret_cast<const R *>(a.face_st);
  R *fst = reinterpret_cast<R *>(a.fstar);
  const long long per_cell = (long long)2 * d * 2 * n * m * NF;
  const long long fb = (long long)2 * n * m * NF;  // one face-side (q and F, all k)
  const long long nfaces = (long long)d * a.ncells;
  for (long long base = (long long)blockIdx.x * RFPB; base < nfaces; base += (long long)gridDim.x * RFPB) {
    for (int i = threadIdx.x; i < RFPB; i += blockDim.x) smax[i] = R(0);
    __syncthreads();
    const int lf = threadIdx.x / NF, p = threadIdx.x % NF;
    const long long face = base + lf;
    const bool ok = lf < RFPB && face < nfaces;
    int j = 0;
    long long cl = 0;
    const R *Lq = nullptr, *Rq = nullptr;
    if (ok) {
      j = (int)(face / a.ncells);
      cl = face % a.ncells;
      const long long cr = neighbour(cl, j, 1, a.grid);
      Lq = fi + cl * per_cell + (2 * j + 1) * fb;
      Rq = fi + cr * per_cell + (2 * j) * fb;
      R qa[m], qb[m];
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R sa = R(0), sb = R(0);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          sa += wk[k] * Lq[(k * m + c) * NF + p];
          sb += wk[k] * Rq[(k * m + c) * NF + p];
        }
        qa[c] = sa;
        qb[c] = sb;
      }
      typename PDE::Mat mL, mR;
      PDE::load(mL, a.cst, a.mat, cl);
      PDE::load(mR, a.cst, a.mat, cr);
      smem_max(&smax[lf], nanmax(PDE::speed(mL, qa, j), PDE::speed(mR, qb, j)));
    }
    __syncthreads();
    if (ok) {
      const R s = smax[lf];
      const long long fo = (long long)n * m * NF;  // offset of the F block
      R *dst = fst + ((long long)j * a.ncells + cl) * (m * NF);
#pragma unroll
      for (int c = 0; c < m; ++c) {
        R acc = R(0);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          const int at = (k * m + c) * NF + p;
          acc += wk[k] * (R(0.5) * (Lq[fo + at] + Rq[fo + at]) - R(0.5) * s * (Rq[at] - Lq[at]));
        }
        dst[c * NF + p] = acc;
      }
    }
    __syncthreads();
  }
}

// phase 3: integrateVolume (space-time quadrature of the stored fluxes),
// integrateFace, update, calcTimeStep.
template <class K>
__global__ void __launch_bounds__(K::THREADS) t1_correct_kernel(const MultiArgs a) {
  using R = typename K::R;
  using QT = typename K::QT;
  using PDE = typename K::PDE;
  using I = Idx<K::n, K::d>;
  constexpr int d = K::d, n = K::n, m = K::m, NS = K::NS, NF = K::NF, CPB = K::CPB, THREADS = K::THREADS;
  extern __shared__ __align__(16) unsigned char smem[];
  Tables<R> &T = *reinterpret_cast<Tables<R> *>(smem);
  unsigned long long *sred = reinterpret_cast<unsigned long long *>(smem + tables_bytes<R>());
  {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.tables);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(Tables<R>) / 4); i += THREADS) dst[i] = src[i];
  }
  const R dt = (R)a.ctl->dt_old;
  const QT *Qin = reinterpret_cast<const QT *>(a.Q_in);
  QT *Qout = reinterpret_cast<QT *>(a.Q_out);
  const R *st = reinterpret_cast<const R *>(a.st);
  const R *fst = reinterpret_cast<const R *>(a.fstar);
  R inv_dx[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) inv_dx[j] = (R)a.inv_dx[j];
  __syncthreads();
  const int lc = threadIdx.x / NS, node = threadIdx.x - lc * NS;
  const long long cell = (long long)blockIdx.x * CPB + lc;
  const bool active = lc < CPB && cell < a.ncells;
  R lam = R(0);
  if (active) {
    typename PDE::Mat mt;
    PDE::load(mt, a.cst, a.mat, cell);
    const long long blk = (long long)n * m * NS;
    const R *base = st + cell * (d + 1) * blk;
    R u[m];
#pragma unroll
    for (int c = 0; c < m; ++c) {
      R acc = R(0);
#pragma unroll
      for (int j = 0; j < d; ++j) {
        const int ij = I::digit(node, j), p = I::face_node(node, j);
        R vol = R(0);
#pragma unroll
        for (int k = 0; k < n; ++k) {
          R sk = R(0);
#pragma unroll
          for (int b = 0; b < n; ++b)
            sk += T.Kvol[ij * n + b] * base[(1 + j) * blk + (k * m + c) * NS + I::with_axis(node, j, b)];
          vol += T.w[k] * sk;
        }
        const R fr = fst[((long long)j * a.ncells + cell) * (m * NF) + c * NF + p];
        const R fl = fst[((long long)j * a.ncells + neighbour(cell, j, -1, a.grid)) * (m * NF) + c * NF + p];
        acc += inv_dx[j] * (vol - T.iw[ij] * (T.FR[ij] * fr - T.FL[ij] * fl));
      }
      const QT qn = Qin[(cell * m + c) * NS + node] + (QT)(dt * acc);
      Qout[(cell * m + c) * NS + node] = qn;
      u[c] = (R)qn;
    }
    R chk = R(0);
#pragma unroll
    for (int c = 0; c < m; ++c) chk += u[c] * R(0);
#pragma unroll
    for (int j = 0; j < d; ++j) lam = nanmax(lam, PDE::speed(mt, u, j));
    lam += chk;
  }
  block_lambda_max<THREADS>(lam_bits(lam), sred, a.ctl);
}

}  // namespace aderdg
