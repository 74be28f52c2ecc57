// kernels.cuh -- launch wrappers of one kernel configuration and its
// registration.  Included only by the generated instantiation units.
#pragma once
#include "adj_lin.cuh"
#include "adjoint.cuh"
#include "multipass.cuh"
#include "registry.h"

namespace aderdg {

template <class K, int ST>
cudaError_t launch_sweep_st(const SweepArgs &a, int grid, cudaStream_t s) {
  sweep_kernel_of<K, ST>()<<<grid, K::THREADS, K::SMEM, s>>>(a);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_sweep(int stage, const SweepArgs &a, int grid, cudaStream_t s) {
  switch (stage) {
    case kCorrect: return launch_sweep_st<K, kCorrect>(a, grid, s);
    case kPredict: return launch_sweep_st<K, kPredict>(a, grid, s);
    case kFused: return launch_sweep_st<K, kFused>(a, grid, s);
    case kCorrectFs: return launch_sweep_st<K, kCorrectFs>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <class K>
int blocks_per_sm(int stage) {
  int nb = 0;
  const void *f = nullptr;
  switch (stage) {
    case kCorrect: f = (const void *)sweep_kernel_of<K, kCorrect>(); break;
    case kPredict: f = (const void *)sweep_kernel_of<K, kPredict>(); break;
    case kFused: f = (const void *)sweep_kernel_of<K, kFused>(); break;
    case kCorrectFs: f = (const void *)sweep_kernel_of<K, kCorrectFs>(); break;
    default: return 0;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, K::THREADS, K::SMEM) != cudaSuccess) return 0;
  return nb;
}

template <class K>
constexpr size_t t1_predict_smem() {
  return tables_bytes<typename K::R>() +
         (size_t)(K::PRED != kTimeModal ? K::CPB * K::d * K::n * K::m * K::NS : K::CPB * K::m * K::NS) *
             sizeof(typename K::R);
}
template <class K>
constexpr size_t t1_correct_smem() {
  return tables_bytes<typename K::R>() + 32 * sizeof(unsigned long long);
}

template <class K, bool WITH_T1, bool WITH_EXT = false>
cudaError_t prepare() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void *f, size_t bytes) {
    if (e == cudaSuccess && bytes > 48 * 1024)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  };
  set((const void *)sweep_kernel_of<K, kCorrect>(), K::SMEM);
  set((const void *)sweep_kernel_of<K, kPredict>(), K::SMEM);
  set((const void *)sweep_kernel_of<K, kFused>(), K::SMEM);
  set((const void *)sweep_kernel_of<K, kCorrectFs>(), K::SMEM);
  if constexpr (WITH_T1) {
    set((const void *)t1_predict_kernel<K>, t1_predict_smem<K>());
    set((const void *)t1_correct_kernel<K>, t1_correct_smem<K>());
  }
  if constexpr (K::PRED == kTimeModal && K::PDE::LINEAR) {
    using L = typename K::Lin;
    set((const void *)lin_sweep_kernel<L, kCorrect>, L::SMEM);
    set((const void *)lin_sweep_kernel<L, kPredict>, L::SMEM_NOTMA);
    set((const void *)lin_sweep_kernel<L, kFused>, L::SMEM);
    if constexpr (WITH_EXT) {
      set((const void *)lin_sweep_kernel<L, kCorrect, true>, L::SMEM);
      set((const void *)lin_sweep_kernel<L, kPredict, true>, L::SMEM_NOTMA);
      set((const void *)lin_sweep_kernel<L, kFused, true>, L::SMEM);
    }
  }
  return e;
}

template <class L, int ST, bool EXT = false>
cudaError_t launch_lin_st(const SweepArgs &a, int grid, cudaStream_t s) {
  constexpr size_t smem = ST == kPredict ? L::SMEM_NOTMA : L::SMEM;  // the STP-only sweep stages nothing
  lin_sweep_kernel<L, ST, EXT><<<grid, L::THREADS, smem, s>>>(a, *reinterpret_cast<const Tables<typename L::R> *>(a.htab));
  return cudaGetLastError();
}

template <class L, bool EXT = false>
cudaError_t launch_lin(int stage, const SweepArgs &a, int grid, cudaStream_t s) {
  switch (stage) {
    case kCorrect: return launch_lin_st<L, kCorrect, EXT>(a, grid, s);
    case kPredict: return launch_lin_st<L, kPredict, EXT>(a, grid, s);
    case kFused: return launch_lin_st<L, kFused, EXT>(a, grid, s);
  }
  return cudaErrorInvalidValue;
}

template <class L>
int lin_blocks_per_sm(int stage) {
  int nb = 0;
  const void *f = stage == kCorrect ? (const void *)lin_sweep_kernel<L, kCorrect>
                  : stage == kPredict ? (const void *)lin_sweep_kernel<L, kPredict>
                                      : (const void *)lin_sweep_kernel<L, kFused>;
  const size_t smem = stage == kPredict ? L::SMEM_NOTMA : L::SMEM;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, L::THREADS, smem) != cudaSuccess) return 0;
  return nb;
}

template <class K>
cudaError_t launch_riemann(const SweepArgs &a, int grid, cudaStream_t s) {
  riemann_kernel<K><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_lambda_mat(const SweepArgs &a, int grid, cudaStream_t s) {
  lambda_mat_kernel<K><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_lambda(const SweepArgs &a, int grid, cudaStream_t s) {
  lambda_kernel<K><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_table1(int phase, const MultiArgs &a, cudaStream_t s) {
  const long long tiles = (a.ncells + K::CPB - 1) / K::CPB;
  switch (phase) {
    case 0:
      t1_predict_kernel<K><<<(unsigned)tiles, K::THREADS, t1_predict_smem<K>(), s>>>(a);
      break;
    case 1: {
      const long long total = a.ncells * 2 * K::d * 2 * K::n * K::m * K::NF;
      long long g = (total + 255) / 256;
      if (g > (1ll << 30)) g = 1ll << 30;
      t1_extrapolate_kernel<K><<<(unsigned)g, 256, 0, s>>>(a);
      break;
    }
    case 2: {
      constexpr int RFPB = cmax(1, 256 / K::NF);
      long long g = ((long long)K::d * a.ncells + RFPB - 1) / RFPB;
      if (g > (1ll << 30)) g = 1ll << 30;
      t1_riemann_kernel<K><<<(unsigned)g, 256, 0, s>>>(a);
      break;
    }
    case 3:
      t1_correct_kernel<K><<<(unsigned)tiles, K::THREADS, t1_correct_smem<K>(), s>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class K>
cudaError_t launch_adj_faces(const AdjArgs &a, cudaStream_t s) {
  constexpr int FC = cmax(1, 256 / K::NF);
  long long g = (a.ncells + FC - 1) / FC;   // grid-stride beyond the cap
  if (g > 8192) g = 8192;
  adj_faces_lin_kernel<AdjLinCfg<K>><<<(unsigned)g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

struct MatPreArgs {
  double cst[8];
};

template <class PDE>
__global__ void mat_pre_kernel(const MatPreArgs p, const float *mat, long long C, MatBox<typename PDE::Mat> *out) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C; c += (long long)gridDim.x * blockDim.x)
    PDE::load(out[c].m, p.cst, mat, c);
}

template <class K>
cudaError_t launch_mat_pre(const double *cst, const float *mat, long long C, void *out, cudaStream_t s) {
  using PDE = typename K::PDE;
  MatPreArgs p;
  for (int i = 0; i < 8; ++i) p.cst[i] = cst[i];
  long long g = (C + 255) / 256;
  if (g > 4096) g = 4096;
  mat_pre_kernel<PDE><<<(unsigned)g, 256, 0, s>>>(p, mat, C, reinterpret_cast<MatBox<typename PDE::Mat> *>(out));
  return cudaGetLastError();
}

// The line-owner adjoint cell kernel: a grid-stride loop over tiles, at most
// a.zs_blocks blocks when the forward powers need the scratch (one slot per
// block).
template <class K>
cudaError_t launch_adj_lin(const AdjArgs &a, cudaStream_t s) {
  using C = AdjLinCfg<K>;
  using R = typename K::R;
  if (!a.htab || !a.htabT) return cudaErrorInvalidValue;
  const bool gm = K::PDE::NMAT > 0 && a.gmat != nullptr;
  if (gm && a.picard > 1 && (!a.zs || a.zs_blocks < 1)) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute((const void *)adj_lin_kernel<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  long long grid = (a.ncells + C::CPB - 1) / C::CPB;
  if (gm && grid > a.zs_blocks) grid = a.zs_blocks;
  if (grid > (1ll << 30)) grid = 1ll << 30;
  adj_lin_kernel<C><<<(unsigned)grid, C::THREADS, C::SMEM, s>>>(a, *reinterpret_cast<const Tables<R> *>(a.htab),
                                                                *reinterpret_cast<const Tables<R> *>(a.htabT));
  return cudaGetLastError();
}

template <class K, bool WITH_T1, bool WITH_ADJ = false, bool WITH_EXT = false>
KernelSet make_set(int pde, int prec) {
  KernelSet ks{};
  ks.pde = pde;
  ks.d = K::d;
  ks.N = K::N;
  ks.prec = prec;
  ks.pred = K::PRED;
  ks.m = K::m;
  ks.NS = K::NS;
  ks.NF = K::NF;
  ks.HS = K::HS;
  ks.CPB = K::CPB;
  ks.THREADS = K::THREADS;
  ks.real_bytes = sizeof(typename K::R);
  ks.q_bytes = sizeof(typename K::QT);
  ks.linear = K::PDE::LINEAR;
  ks.pair = K::PAIR;
  ks.mat_pre = &launch_mat_pre<K>;
  ks.mat_bytes = (int)sizeof(MatBox<typename K::PDE::Mat>);
  static_assert(!(K::PAIR && (WITH_T1 || WITH_ADJ)), "the Table 1 form and the adjoint keep no low words");
  ks.prepare = &prepare<K, WITH_T1, WITH_EXT && K::PRED == kTimeModal && K::PDE::LINEAR>;
  ks.sweep = &launch_sweep<K>;
  ks.blocks_per_sm = &blocks_per_sm<K>;
  ks.riemann = &launch_riemann<K>;
  ks.lambda = &launch_lambda<K>;
  if constexpr (K::PDE::LINEAR) ks.lambda_mat = &launch_lambda_mat<K>;
  else ks.lambda_mat = nullptr;
  if constexpr (WITH_T1) ks.table1 = &launch_table1<K>;
  else ks.table1 = nullptr;
  if constexpr (K::PRED == kTimeModal && K::PDE::LINEAR) {
    using L = typename K::Lin;
    ks.lin_sweep = &launch_lin<L>;
    if constexpr (WITH_EXT) ks.lin_sweep_ext = &launch_lin<L, true>;
    else ks.lin_sweep_ext = nullptr;
    ks.lin_blocks_per_sm = &lin_blocks_per_sm<L>;
    ks.HSL = L::HSL;
    ks.LIN_CPB = L::CPB;
  } else {
    ks.lin_sweep = nullptr;
    ks.lin_sweep_ext = nullptr;
    ks.lin_blocks_per_sm = nullptr;
    ks.HSL = 0;
    ks.LIN_CPB = 0;
  }
  if constexpr (WITH_ADJ && K::PRED == kTimeModal && K::PDE::LINEAR) {
    ks.adj_faces = &launch_adj_faces<K>;
    ks.adj_cell = &launch_adj_lin<K>;
    ks.adj_cpb = AdjLinCfg<K>::CPB;
    ks.adj_zlevel = AdjLinCfg<K>::ZLEVEL;
  } else {
    ks.adj_faces = nullptr;
    ks.adj_cell = nullptr;
    ks.adj_cpb = 0;
    ks.adj_zlevel = 0;
  }
  return ks;
}

}  // namespace aderdg
