// registry.h -- host-side table of compiled kernel configurations.
// Each generated translation unit registers the configurations it
// instantiates when the shared library is loaded.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include "common.cuh"

namespace aderdg {
struct AdjArgs;
}

namespace aderdg {

enum Prec : int { kFP32 = 0, kFP64 = 1, kACC64 = 2, kPAIR = 3 };

struct KernelSet {
  int pde, d, N, prec, pred;
  int m, NS, NF, HS, CPB, THREADS;
  int real_bytes, q_bytes;  // q_bytes: one state element (a float of each plane for the pair)
  bool linear;
  bool pair;                // compensated FP32 pair: a low-word plane follows the states
  cudaError_t (*prepare)();                                    // smem attributes, current device
  cudaError_t (*sweep)(int stage, const SweepArgs &, int grid, cudaStream_t);
  int (*blocks_per_sm)(int stage);
  cudaError_t (*riemann)(const SweepArgs &, int grid, cudaStream_t);
  cudaError_t (*lambda)(const SweepArgs &, int grid, cudaStream_t);
  // linear PDEs: the wave-speed maximum from the material alone; null otherwise
  cudaError_t (*lambda_mat)(const SweepArgs &, int grid, cudaStream_t);
  // Table 1 multi-pass form: phase 0 predict, 1 extrapolate, 2 Riemann, 3 correct
  cudaError_t (*table1)(int phase, const MultiArgs &, cudaStream_t);
  // line-owner fused sweep of linear PDEs (stages kCorrect, kPredict, kFused)
  // with the q-only hull of stride HSL; null if not compiled
  cudaError_t (*lin_sweep)(int stage, const SweepArgs &, int grid, cudaStream_t);
  // the same kernel with point sources and material jumps in non-conservative
  // form compiled in (SweepArgs::nsrc, ::ncp); null if not compiled
  cudaError_t (*lin_sweep_ext)(int stage, const SweepArgs &, int grid, cudaStream_t);
  int (*lin_blocks_per_sm)(int stage);
  int HSL, LIN_CPB;
  // discrete adjoint of the step (linear fluxes); null if not compiled
  cudaError_t (*adj_faces)(const AdjArgs &, cudaStream_t);
  cudaError_t (*adj_cell)(const AdjArgs &, cudaStream_t);
  // PDE constants per cell (MatBox<PDE::Mat>, mat_bytes each) from pde_const
  // (mat null: one entry) or the per-cell material, into out
  cudaError_t (*mat_pre)(const double *cst, const float *mat, long long C, void *out, cudaStream_t);
  int mat_bytes;
  // the cell kernel's cells per block and scratch elements per block and level
  // of the forward powers (material gradient)
  int adj_cpb;
  long long adj_zlevel;
};

void register_set(const KernelSet &ks);
const KernelSet *find_set(int pde, int d, int N, int prec, int pred);
int registered_count();
const KernelSet *registered_at(int i);

struct Registrar {
  explicit Registrar(const KernelSet &ks) { register_set(ks); }
};

}  // namespace aderdg
