// common.cuh -- shared device-side definitions of libaderdg (sm_103a).
//
// Layouts (per cell, C-contiguous):
//   Q    [cell][comp][node]                      QT = float or double; with
//        the compensated pair (Pair32) Q is two float planes [2][cell][comp][node]:
//        the FP32 state, then the low-order word of every DoF
//   D    [cell][comp][node]                      R  (integrateVolume output, Technique 1)
//   hull [cell][face f = 2j+side][2][comp][fnode] R, padded per cell to HS
//        slot 0 = time-averaged q on the face, slot 1 = time-averaged F_j.
//        (global time stepping: Rusanov is affine in (q, F) for a fixed
//        wave speed, so the time-averaged hull carries the whole space-time
//        face data of Table 1 into the Riemann solve)
//   F*   [j][cell][comp][fnode]  face between cell and cell+e_j (hull3 form)
// node = i0 + n (i1 + n i2); face node of the face normal to axis j lists
// the other axes in ascending order, lowest fastest.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace aderdg {

constexpr int kMaxN = 6;            // highest polynomial order compiled
constexpr int kMaxn = kMaxN + 1;
constexpr int kMaxH = (kMaxn + 1) / 2;
constexpr int kMaxPicard = 16;      // highest Picard count

__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int round_up(int v, int q) { return (v + q - 1) / q * q; }
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

enum Stage : int {
  kCorrect = 1,      // Riemann + integrateFace + update + calcTimeStep
  kPredict = 2,      // predict + integrateVolume + extrapolate
  kFused = 3,        // both, in this order (Technique 4)
  kCorrectFs = 4     // integrateFace from stored F* + update + calcTimeStep (hull3)
};

// kSpaceTimeTC: the space-time Picard iteration with the flux-divergence
// contractions on the tensor cores (TF32 operands, FP32 accumulation)
enum Pred : int { kTimeModal = 0, kSpaceTime = 1, kSpaceTimeTC = 2 };

// State storage of a configuration.  Pair32 tags the compensated FP32 pair:
// the state is float and every DoF keeps a second float, its low-order word,
// in a plane that follows the C m NS states (hi + lo carries about 48 bits).
struct Pair32 {};
template <class QT>
struct QStore {
  using T = QT;
  static constexpr bool PAIR = false;
};
template <>
struct QStore<Pair32> {
  using T = float;
  static constexpr bool PAIR = true;
};

// (hi, lo) += x for a normalised pair (hi = fl(hi + lo)): the rounding error
// of hi + x by TwoSum (Knuth), added to the low word, then renormalised by
// Fast2Sum (Dekker).  Round-to-nearest intrinsics keep the compiler from
// contracting or reassociating the error terms.
__device__ __forceinline__ void pair_add(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  const float l = __fadd_rn(lo, err);
  const float h = __fadd_rn(s, l);
  lo = __fsub_rn(l, __fsub_rn(h, s));
  hi = h;
}

// 1D operator tables of one order, compact with stride n, in the kernel's
// arithmetic type.
template <class R>
struct Tables {
  R Dm[kMaxn * kMaxn];                 // Dm[i*n+a] = phi_a'(xi_i)
  R Kvol[kMaxn * kMaxn];               // Kvol[i*n+a] = w_a Dm[a][i] / w_i
  R K1inv[kMaxn * kMaxn];              // inverse of K1[k][l] = FR_k FR_l - w_l Dm[l][k]
  R FL[kMaxn], FR[kMaxn], w[kMaxn], iw[kMaxn];
  R g[kMaxPicard + 1];                 // w . (K1^-1 W)^s 1
  R cvec[(kMaxPicard + 1) * kMaxn];    // (K1^-1 W)^s 1, s-major
  // Even/odd halves of the centro-antisymmetric Dm and Kvol (symmetric
  // nodes: C[n-1-o][n-1-b] = -C[o][b]), h = n/2, o < (n+1)/2, b < h:
  //   E[o][b] = (C[o][b] + C[o][n-1-b]) / 2, O[o][b] = (C[o][b] - C[o][n-1-b]) / 2,
  //   M[o] = C[o][h] (odd n, middle column)
  R DmE[kMaxH * kMaxH], DmO[kMaxH * kMaxH], DmM[kMaxH];
  R KvE[kMaxH * kMaxH], KvO[kMaxH * kMaxH], KvM[kMaxH];
  // Row pairs of Dm and Kvol for packed two-lane FMAs (even n): element
  // [(k kMaxn + b) 2 + l] = C[2k + l][b]
  alignas(8) R DmP[kMaxH * kMaxn * 2];
  alignas(8) R KvP[kMaxH * kMaxn * 2];
  alignas(8) R FLR[kMaxn * 2];          // (FL[b], FR[b]) pairs
};

// Bytes of a Tables<R> copy in shared memory, rounded so that what follows
// it is 16-byte aligned.
template <class R>
__host__ __device__ constexpr size_t tables_bytes() { return (sizeof(Tables<R>) + 15) / 16 * 16; }

// Device-resident time-step control block (Alg. 1/2 scalars, FP64).
struct DevCtl {
  double dt_old, dt_new, dt_adm, t;
  double lam_last;
  unsigned long long lam_bits;  // running max of lambda (bits of a non-negative double)
  long long step, reruns;
  int rerun;                    // the pending STP rerun flag (Technique 5)
  int error;                    // aderdg_status of the first device-side failure
  int hist_cap, pad_;
  double *hist;                 // dt used by each corrector
};

// Constant control parameters, passed by value to the control kernels.
struct CtlParams {
  double cfl;         // C_dT
  double dt_scale;    // min_j dx_j / (d (2N+1)); dt_adm = dt_scale / lambda_max
  double fixed_dt;    // > 0: control off
  double inject_factor;
  int policy;         // 0 strict, 1 creeping
  int inject_step;
};

// Point sources a s(t) delta(x - x_s) (the delta terms of Eq. 1).  On the
// device a source is its cell, its amplitudes and the 1D factors of its
// lumped-mass projection e[j][a] = phi_a(xi_j) / (w_a dx_j), so that the nodal
// source of component c is amp[c] prod_j e[j][i_j].
constexpr int kMaxSources = 64;
struct SrcDev {
  long long cell;
  double amp[9];
  double e[3][kMaxn];
};
// Time function: kind 0 polynomial sum_p coef[p] (t - t0)^p, 1 Ricker wavelet.
struct SrcTime {
  int kind, pad_;
  double t0, f0;
  double coef[8];
};
// Per-sweep coefficients of each source, computed on the device from the
// control block before the sweep (double [nsrc][kSrcCo]):
//   [0]                       dt_old sum_k w_k s(t + xi_k dt_old)  (corrector)
//   [1 + s]                   dt h_s of the Horner level s for the predictor of
//                             the fused sweep (step [t + dt_old, + dt_new])
//   [1 + kMaxPicard + s]      ... of a first STP sweep (step [t, t + dt_new])
//   [1 + 2 kMaxPicard + s]    ... of a rerun STP sweep (step [t, t + dt_old])
// with h_s = w . (K1^-1 W)^(s+1) svec, svec_l = s(t_p + xi_l dt).
constexpr int kSrcCo = 1 + 3 * kMaxPicard;

struct SweepArgs {
  const void *Q_in;
  void *Q_out;
  void *Dbuf;
  const void *hull_in;
  void *hull_out;
  void *fstar;            // hull3: Riemann sweep output, corrector input
  const float *mat;       // [C][3] (rho, cp, cs) or nullptr
  DevCtl *ctl;
  const void *tables;     // Tables<R> in global memory
  const void *htab;       // the same Tables<R> in host memory (passed by value to
                          // the kernels that take the tables as a parameter)
  long long ncells;
  long long ntiles;       // the sweep covers tiles [tile_lo, ntiles)
  long long tile_lo;
  int grid[3];
  int picard;
  int gate;               // kPredict only: exit unless ctl->rerun (Technique 5 rerun sweep)
  int pred_dt_old;        // kPredict only: predict with dt_old instead of dt_new
  int ncp;                // per-cell material: jumps in non-conservative form (B_j of Eq. 1)
  int nsrc;               // point sources (line-owner kernel)
  const SrcDev *src;
  const double *srcco;    // [nsrc][kSrcCo]
  const void *matp;       // MatBox<PDE::Mat>: [C] (per-cell material) or [1] (uniform), or nullptr
  double inv_dx[3];
  double cst[8];
};

// A cell's PDE constants (PDE::Mat) as the kernels use them, computed once
// from pde_const or the per-cell material (FP64, then rounded to the kernel
// type: the values PDE::load gives) and kept 16-byte aligned for one vector
// load.  The sweeps would otherwise redo that FP64 arithmetic for their own
// cell and every neighbour in every step.
template <class Mat>
struct alignas(16) MatBox {
  Mat m;
};

template <class PDE>
__device__ __forceinline__ void load_mat(typename PDE::Mat &mt, const void *matp, const double *cst, const float *mat,
                                         long long cell) {
  if (matp) mt = reinterpret_cast<const MatBox<typename PDE::Mat> *>(matp)[mat ? cell : 0].m;
  else PDE::load(mt, cst, mat, cell);
}

// Multi-pass (Table 1) buffers.
struct MultiArgs {
  const void *Q_in;
  void *Q_out;
  void *st;               // [cell][slot 0..d][k][comp][node] space-time q^ and F_j(q^)
  void *face_st;          // [cell][f][2][k][comp][fnode] space-time face data
  void *fstar;            // [j][cell][comp][fnode] time-integrated F*
  const float *mat;
  DevCtl *ctl;
  const void *tables;
  long long ncells;
  int grid[3];
  int picard;
  double inv_dx[3];
  double cst[8];
};

// ---------------------------------------------------------------------------
// Index helpers (n, d compile-time)

template <int n, int d>
struct Idx {
  static constexpr int NS = ipow(n, d);
  static constexpr int NF = ipow(n, d - 1);
  __device__ __forceinline__ static int digit(int i, int j) {
    return (i / ipow_rt(j)) % n;
  }
  __device__ __forceinline__ static int ipow_rt(int j) {
    return j == 0 ? 1 : (j == 1 ? n : n * n);
  }
  // node with axis j set to a
  __device__ __forceinline__ static int with_axis(int i, int j, int a) {
    const int s = ipow_rt(j);
    return i + (a - (i / s) % n) * s;
  }
  // face node of volume node i on the face normal to j
  __device__ __forceinline__ static int face_node(int i, int j) {
    const int s = ipow_rt(j);
    return i % s + (i / (s * n)) * s;
  }
  // volume node at position a along axis j of face node p
  __device__ __forceinline__ static int node_of_face(int p, int j, int a) {
    const int s = ipow_rt(j);
    return p % s + a * s + (p / s) * (s * n);
  }
};

__device__ __forceinline__ long long neighbour(long long cell, int j, int dir, const int *grid) {
  long long stride = 1;
  for (int a = 0; a < j; ++a) stride *= grid[a];
  const long long cj = (cell / stride) % grid[j];
  long long nj = cj + dir;
  if (nj < 0) nj += grid[j];
  if (nj >= grid[j]) nj -= grid[j];
  return cell + (nj - cj) * stride;
}

// Non-negative max on IEEE bits: NaN (positive payload) and +Inf win, so a
// non-finite wave speed survives every reduction level.
__device__ __forceinline__ unsigned long long lam_bits(float v) {
  return (unsigned long long)__double_as_longlong((double)v);
}
__device__ __forceinline__ unsigned long long lam_bits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// Block max of per-thread lambda bits; thread 0 folds it into ctl->lam_bits.
template <int THREADS>
__device__ __forceinline__ void block_lambda_max(unsigned long long v, unsigned long long *sred,
                                                 DevCtl *ctl) {
  v = warp_max_u64(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sred[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long u = lane < THREADS / 32 ? sred[lane] : 0ull;
    u = warp_max_u64(u);
    if (lane == 0 && u) atomicMax(&ctl->lam_bits, u);
  }
}

__device__ __forceinline__ void smem_max(float *p, float v) {
  atomicMax(reinterpret_cast<int *>(p), __float_as_int(v));  // v >= 0 or NaN
}
__device__ __forceinline__ void smem_max(double *p, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

template <class T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// max that lets a NaN through (a non-finite wave speed must reach the host)
template <class T>
__device__ __forceinline__ T nanmax(T acc, T v) { return (v > acc || v != v) ? v : acc; }

}  // namespace aderdg
