// batch.cu -- many independent scenarios of uneven size and order advanced
// together: one persistent launch per sweep, the steady state captured in a
// CUDA graph, the work granularity and grid picked by an autotuner.
//
// Scenarios are 2D acoustics or elasticity, N = 2..6, FP32, fused form.  The
// states are packed in one buffer (offsets from aderdg_batch_offsets, each a
// multiple of 32 elements so that every scenario starts 128-byte aligned).  A
// work item is (scenario, first tile, tile count); items are ordered by cost,
// largest first, and handed to persistent blocks through a device counter.
// Each item runs the line-owner tile body of its (PDE, N), the same device
// function the single-scenario kernel runs, with the operator tables of its
// order in __constant__ memory.  Every scenario keeps its own time-step
// control block (its own dt); one thread per scenario runs the control rule.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "aderdg.h"
#include "basis.h"
#include "control.cuh"
#include "registry.h"
#include "sweep_lin.cuh"

namespace aderdg {

cudaError_t launch_control(int which, DevCtl *c, const CtlParams &p, int arg, cudaStream_t s);
template <class R>
void fill_tables(const Basis1D &B, Tables<R> &T);

namespace {

constexpr int kBNmin = 2, kBNmax = 6, kBOrders = kBNmax - kBNmin + 1;
constexpr int kBThreads = 256;

constexpr int kBMatStride = 32;  // bytes per scenario in the PDE-constant buffer

template <int N>
using BA = LinCfg<Acoustics, 2, N, float, float>;
template <int N>
using BE = LinCfg<Elasticity, 2, N, float, float>;

__constant__ Tables<float> c_btab[kBOrders];

constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kBSmem =
    smax(smax(smax(smax(BA<2>::SMEM_NOTMA, BA<3>::SMEM_NOTMA), smax(BA<4>::SMEM_NOTMA, BA<5>::SMEM_NOTMA)),
              smax(smax(BA<6>::SMEM_NOTMA, BE<2>::SMEM_NOTMA), smax(BE<3>::SMEM_NOTMA, BE<4>::SMEM_NOTMA))),
         smax(BE<5>::SMEM_NOTMA, BE<6>::SMEM_NOTMA));

int cfg_index(int pde, int N) { return (pde == ADERDG_ACOUSTICS ? 0 : kBOrders) + (N - kBNmin); }

int cfg_cpb(int cfg) {
  switch (cfg) {
    case 0: return BA<2>::CPB; case 1: return BA<3>::CPB; case 2: return BA<4>::CPB;
    case 3: return BA<5>::CPB; case 4: return BA<6>::CPB;
    case 5: return BE<2>::CPB; case 6: return BE<3>::CPB; case 7: return BE<4>::CPB;
    case 8: return BE<5>::CPB; default: return BE<6>::CPB;
  }
}

struct BItem {
  int scen, cfg, ntiles, pad_;
  long long tile0;
};

// One configuration's tile body as its own function: it is register-allocated
// on its own (the bodies differ a lot in register need) and addresses its
// order's tables in constant memory directly.
// MINB is part of the body's signature so that every kernel variant gets its
// own copy compiled under its own register budget.
template <class K, int ST, int ORD, int MINB>
__device__ __noinline__ void batch_body(const SweepArgs &a, long long tile, unsigned char *smem) {
  lin_tile<K, ST>(a, c_btab[ORD], tile, smem);
}

template <int ST, int MINB>
__device__ __forceinline__ void dispatch(int cfg, const SweepArgs &a, long long tile, unsigned char *smem) {
  switch (cfg) {
    case 0: batch_body<BA<2>, ST, 0, MINB>(a, tile, smem); break;
    case 1: batch_body<BA<3>, ST, 1, MINB>(a, tile, smem); break;
    case 2: batch_body<BA<4>, ST, 2, MINB>(a, tile, smem); break;
    case 3: batch_body<BA<5>, ST, 3, MINB>(a, tile, smem); break;
    case 4: batch_body<BA<6>, ST, 4, MINB>(a, tile, smem); break;
    case 5: batch_body<BE<2>, ST, 0, MINB>(a, tile, smem); break;
    case 6: batch_body<BE<3>, ST, 1, MINB>(a, tile, smem); break;
    case 7: batch_body<BE<4>, ST, 2, MINB>(a, tile, smem); break;
    case 8: batch_body<BE<5>, ST, 3, MINB>(a, tile, smem); break;
    default: batch_body<BE<6>, ST, 4, MINB>(a, tile, smem); break;
  }
}

// Persistent sweep over the work list.  scen[p * count + s] are the sweep
// arguments of scenario s for hull parity p (read face hull p, write 1 - p).
// Three register budgets, one per CTAs-per-SM setting: MINB = 1 (up to 255
// registers: the large elasticity bodies do not spill), 2 (128) and 3 (85:
// the small bodies at the occupancy of their own kernels); the autotuner picks.
template <int ST, int MINB>
__global__ void __launch_bounds__(kBThreads, MINB) batch_kernel(const SweepArgs *scen, int count,
                                                                const BItem *items, int nitems, int *counter,
                                                                int parity) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    __syncthreads();
    if (it >= nitems) return;  // uniform: every thread read the same item
    const BItem w = items[it];
    const SweepArgs &a = scen[parity * count + w.scen];
    for (int t = 0; t < w.ntiles; ++t) dispatch<ST, MINB>(w.cfg, a, w.tile0 + t, smem);
  }
}

// Largest wave speed over the item's cells (Eq. 5), NaN/Inf in Q included.
template <class K>
__device__ __forceinline__ void batch_lambda_body(const SweepArgs &a, long long tile0, int ntiles,
                                                  unsigned long long *sred) {
  using R = typename K::R;
  using PDE = typename K::PDE;
  constexpr int m = K::m, NS = K::NS;
  const float *Q = reinterpret_cast<const float *>(a.Q_in);
  const long long c0 = tile0 * K::CPB;
  const long long c1 = c0 + (long long)ntiles * K::CPB < a.ncells ? c0 + (long long)ntiles * K::CPB : a.ncells;
  R lam = R(0);
  for (long long t = c0 * NS + threadIdx.x; t < c1 * NS; t += blockDim.x) {
    const long long cell = t / NS;
    const int node = (int)(t - cell * NS);
    typename PDE::Mat mt;
    PDE::load(mt, a.cst, a.mat, cell);
    R u[m];
    R chk = R(0);
#pragma unroll
    for (int c = 0; c < m; ++c) {
      u[c] = (R)Q[(cell * m + c) * NS + node];
      chk += u[c] * R(0);
    }
#pragma unroll
    for (int j = 0; j < K::d; ++j) lam = nanmax(lam, PDE::speed(mt, u, j));
    lam += chk;
  }
  block_lambda_max<kBThreads>(lam_bits(lam), sred, a.ctl);
  __syncthreads();  // sred reused by the next item
}

__global__ void __launch_bounds__(kBThreads) batch_lambda_kernel(const SweepArgs *scen, const BItem *items,
                                                                 int nitems, int *counter) {
  __shared__ unsigned long long sred[32];
  __shared__ int cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
    __syncthreads();
    const int it = cur;
    __syncthreads();
    if (it >= nitems) return;
    const BItem w = items[it];
    const SweepArgs &a = scen[w.scen];
    switch (w.cfg) {
      case 0: batch_lambda_body<BA<2>>(a, w.tile0, w.ntiles, sred); break;
      case 1: batch_lambda_body<BA<3>>(a, w.tile0, w.ntiles, sred); break;
      case 2: batch_lambda_body<BA<4>>(a, w.tile0, w.ntiles, sred); break;
      case 3: batch_lambda_body<BA<5>>(a, w.tile0, w.ntiles, sred); break;
      case 4: batch_lambda_body<BA<6>>(a, w.tile0, w.ntiles, sred); break;
      case 5: batch_lambda_body<BE<2>>(a, w.tile0, w.ntiles, sred); break;
      case 6: batch_lambda_body<BE<3>>(a, w.tile0, w.ntiles, sred); break;
      case 7: batch_lambda_body<BE<4>>(a, w.tile0, w.ntiles, sred); break;
      case 8: batch_lambda_body<BE<5>>(a, w.tile0, w.ntiles, sred); break;
      default: batch_lambda_body<BE<6>>(a, w.tile0, w.ntiles, sred); break;
    }
  }
}

// Control rule of every scenario, one thread each; thread 0 also resets the
// work counter of the next sweep.
__global__ void batch_control_kernel(DevCtl *ctl, const CtlParams *cp, int count, int which, int *counter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0 && counter) *counter = 0;
  if (i >= count) return;
  switch (which) {
    case 0: ctl_reset(&ctl[i]); break;
    case 1: ctl_begin(&ctl[i], cp[i], 0); break;
    case 2: ctl_pre(&ctl[i], cp[i]); break;
    default: ctl_post(&ctl[i], cp[i], 0); break;
  }
}

}  // namespace
}  // namespace aderdg

using namespace aderdg;

struct aderdg_batch_ctx {
  int count;
  std::vector<aderdg_scenario> scen;
  std::vector<const KernelSet *> ks;
  std::vector<int> cfg;
  std::vector<long long> cells, offs, ntiles;
  long long total;
  int nsm, max_bps;
  int bps, tpi;  // tuning: blocks per SM, tiles per work item
  cudaStream_t is;
  cudaEvent_t ev_in, ev_out;
  // device
  float *D;
  DevCtl *ctl;
  double *hist;
  CtlParams *cp;
  SweepArgs *args;
  unsigned char *matbuf;  // each scenario's PDE constants (MatBox, kBMatStride bytes apart)
  BItem *items;
  int nitems;
  int *counter;
  std::vector<void *> hull_bufs;
  std::vector<SweepArgs> hargs;
  std::vector<CtlParams> hcp;
  const float *bound_Q;
  cudaGraphExec_t graph;
  long long launches;
  // profile: events around each persistent fused sweep launched directly
  bool prof;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  size_t prof_used;
  Tables<float> htab[kBOrders];  // host copies for the per-scenario kernels
};

static void batch_free(aderdg_batch_t b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void *ptrs[] = {b->D, b->ctl, b->hist, b->cp, b->args, b->matbuf, b->items, b->counter};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (void *p : b->hull_bufs)
    if (p) cudaFree(p);
  for (auto &pe : b->prof_ev) {
    cudaEventDestroy(pe.first);
    cudaEventDestroy(pe.second);
  }
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->is) cudaStreamDestroy(b->is);
}

// Work list: every scenario's tiles in items of b->tpi tiles, largest cost first.
static cudaError_t batch_items(aderdg_batch_t b) {
  std::vector<std::pair<double, BItem>> v;
  for (int s = 0; s < b->count; ++s) {
    const int N = b->scen[s].N, m = b->scen[s].m;
    const double cost_tile = (double)cfg_cpb(b->cfg[s]) * m * (N + 1) * (N + 1) * (N + 2);
    for (long long t = 0; t < b->ntiles[s]; t += b->tpi) {
      BItem it{};
      it.scen = s;
      it.cfg = b->cfg[s];
      it.tile0 = t;
      it.ntiles = (int)std::min<long long>(b->tpi, b->ntiles[s] - t);
      v.push_back({cost_tile * it.ntiles, it});
    }
  }
  std::stable_sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
  std::vector<BItem> items(v.size());
  for (size_t i = 0; i < v.size(); ++i) items[i] = v[i].second;
  if (b->items) cudaFree(b->items);
  b->items = nullptr;
  cudaError_t e = cudaMalloc(&b->items, sizeof(BItem) * std::max<size_t>(1, items.size()));
  if (e == cudaSuccess) e = cudaMemcpy(b->items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice);
  b->nitems = (int)items.size();
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return e;
}

// A scenario the ensemble kernels accept: 2D, N in [2, 6], acoustics (rho, c
// > 0) or elasticity (rho, cp > 0, cs >= 0) with the matching m, a grid of at
// least one cell, positive cell sizes, a CFL number in (0, 1] or 0 (default).
static aderdg_status scenario_status(const aderdg_scenario &c) {
  const double *k = c.pde_const;
  const bool mat_ok = c.pde == ADERDG_ACOUSTICS ? (k[0] > 0.0 && k[1] > 0.0)
                                                : (k[0] > 0.0 && k[1] > 0.0 && k[2] >= 0.0);
  const bool ok = c.d == 2 && c.N >= kBNmin && c.N <= kBNmax &&
                  ((c.pde == ADERDG_ACOUSTICS && c.m == 3) || (c.pde == ADERDG_ELASTICITY && c.m == 5)) &&
                  mat_ok && c.grid[0] >= 1 && c.grid[1] >= 1 && c.dx[0] > 0 && c.dx[1] > 0 &&
                  std::isfinite(c.dx[0]) && std::isfinite(c.dx[1]) && (c.cfl == 0.0 || (c.cfl > 0.0 && c.cfl <= 1.0));
  if (!ok) return ADERDG_EINVAL;
  const KernelSet *ks = find_set(c.pde, 2, c.N, ADERDG_FP32, kTimeModal);
  return ks && ks->lin_sweep ? ADERDG_OK : ADERDG_EUNSUPPORTED;
}

extern "C" aderdg_status aderdg_batch_create(int count, const aderdg_scenario *scen, aderdg_batch_t *out) {
  if (!out || !scen || count < 1) return ADERDG_EINVAL;
  *out = nullptr;
  for (int s = 0; s < count; ++s) {  // every scenario checked before any device call
    const aderdg_status st = scenario_status(scen[s]);
    if (st) return st;
  }
  aderdg_batch_t b = new aderdg_batch_ctx();
  b->count = count;
  b->scen.assign(scen, scen + count);
  b->bps = 2;
  b->tpi = 2;
  long long total = 0;
  for (int s = 0; s < count; ++s) {
    const aderdg_scenario &c = scen[s];
    const KernelSet *ks = find_set(c.pde, 2, c.N, ADERDG_FP32, kTimeModal);
    b->ks.push_back(ks);
    const bool seen = std::find(b->ks.begin(), b->ks.end() - 1, ks) != b->ks.end() - 1;
    if (!seen && ks->prepare() != cudaSuccess) {  // shared-memory limits of the per-scenario kernels
      delete b;
      return ADERDG_ECUDA;
    }
    b->cfg.push_back(cfg_index(c.pde, c.N));
    const long long C = (long long)c.grid[0] * c.grid[1];
    b->cells.push_back(C);
    b->offs.push_back(total);
    b->ntiles.push_back((C + cfg_cpb(b->cfg.back()) - 1) / cfg_cpb(b->cfg.back()));
    // 128-byte aligned starts: the line loads of the tile body are float4/float2
    total += (C * c.m * (c.N + 1) * (c.N + 1) + 31) / 32 * 32;
  }
  b->offs.push_back(total);
  b->total = total;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  // tables of every order into constant memory
  Tables<float> tabs[kBOrders];
  for (int N = kBNmin; N <= kBNmax; ++N) {
    Basis1D B;
    build_basis(N, B);
    fill_tables(B, tabs[N - kBNmin]);
  }
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_btab, tabs, sizeof(tabs));
  std::memcpy(b->htab, tabs, sizeof(tabs));
  const void *kf[9] = {(const void *)batch_kernel<kPredict, 1>, (const void *)batch_kernel<kFused, 1>,
                       (const void *)batch_kernel<kCorrect, 1>,  (const void *)batch_kernel<kPredict, 2>,
                       (const void *)batch_kernel<kFused, 2>,    (const void *)batch_kernel<kCorrect, 2>,
                       (const void *)batch_kernel<kPredict, 3>,  (const void *)batch_kernel<kFused, 3>,
                       (const void *)batch_kernel<kCorrect, 3>};
  for (int i = 0; i < 9 && e == cudaSuccess; ++i)
    e = cudaFuncSetAttribute(kf[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem);
  // largest CTAs per SM whose build actually reaches that occupancy
  b->max_bps = 1;
  for (int v = 2; v <= 3 && e == cudaSuccess; ++v) {
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kf[3 * (v - 1) + 1], kBThreads, kBSmem);
    if (e == cudaSuccess && occ >= v) b->max_bps = v;
  }
  b->bps = std::min(b->bps, b->max_bps);
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes ? bytes : 16);
  };
  alloc((void **)&b->D, sizeof(float) * total);
  alloc((void **)&b->ctl, sizeof(DevCtl) * count);
  alloc((void **)&b->hist, sizeof(double) * 16 * count);
  alloc((void **)&b->cp, sizeof(CtlParams) * count);
  alloc((void **)&b->args, sizeof(SweepArgs) * 2 * count);
  // the PDE constants of each scenario, once (FP64 arithmetic, rounded to FP32),
  // instead of in every thread of every tile
  alloc((void **)&b->matbuf, (size_t)kBMatStride * count);
  for (int s = 0; s < count && e == cudaSuccess; ++s) {
    if (b->ks[s]->mat_bytes > kBMatStride) e = cudaErrorInvalidValue;
    else e = b->ks[s]->mat_pre(scen[s].pde_const, nullptr, 1, b->matbuf + (size_t)kBMatStride * s, nullptr);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  alloc((void **)&b->counter, sizeof(int));
  b->hull_bufs.assign(2 * count, nullptr);
  for (int s = 0; s < count && e == cudaSuccess; ++s)
    for (int k = 0; k < 2; ++k) alloc(&b->hull_bufs[2 * s + k], sizeof(float) * b->cells[s] * b->ks[s]->HSL);
  // control blocks and parameters
  std::vector<DevCtl> hc(count);
  b->hcp.resize(count);
  for (int s = 0; s < count; ++s) {
    std::memset(&hc[s], 0, sizeof(DevCtl));
    hc[s].hist = b->hist + 16 * s;
    hc[s].hist_cap = 16;
    const aderdg_scenario &c = scen[s];
    CtlParams &p = b->hcp[s];
    std::memset(&p, 0, sizeof p);
    p.cfl = c.cfl > 0 ? c.cfl : std::max(0.3, std::min(0.9, 0.9 - 0.1 * c.N));
    p.dt_scale = std::min(c.dx[0], c.dx[1]) / (2 * (2.0 * c.N + 1.0));
    p.inject_factor = 1.0;
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->ctl, hc.data(), sizeof(DevCtl) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->cp, b->hcp.data(), sizeof(CtlParams) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->is, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = batch_items(b);
  if (e != cudaSuccess) {
    batch_free(b);
    delete b;
    return e == cudaErrorMemoryAllocation ? ADERDG_ENOMEM : ADERDG_ECUDA;
  }
  *out = b;
  return ADERDG_OK;
}

// Per-scenario sweep arguments for the packed state Q.
static cudaError_t batch_bind(aderdg_batch_t b, float *Q) {
  if (b->bound_Q == Q) return cudaSuccess;
  b->hargs.assign(b->count, SweepArgs{});
  for (int s = 0; s < b->count; ++s) {
    const aderdg_scenario &c = b->scen[s];
    SweepArgs &a = b->hargs[s];
    a.Q_in = Q + b->offs[s];
    a.Q_out = Q + b->offs[s];
    a.Dbuf = b->D + b->offs[s];
    a.ctl = b->ctl + s;
    a.ncells = b->cells[s];
    a.ntiles = b->ntiles[s];
    a.grid[0] = c.grid[0];
    a.grid[1] = c.grid[1];
    a.grid[2] = 1;
    a.inv_dx[0] = 1.0 / c.dx[0];
    a.inv_dx[1] = 1.0 / c.dx[1];
    a.inv_dx[2] = 1.0;
    a.picard = c.N + 1;
    for (int i = 0; i < 8; ++i) a.cst[i] = c.pde_const[i];
    a.matp = b->matbuf + (size_t)kBMatStride * s;
  }
  std::vector<SweepArgs> both(2 * b->count);
  for (int p = 0; p < 2; ++p)
    for (int s = 0; s < b->count; ++s) {
      both[p * b->count + s] = b->hargs[s];
      both[p * b->count + s].hull_in = b->hull_bufs[2 * s + p];
      both[p * b->count + s].hull_out = b->hull_bufs[2 * s + (p ^ 1)];
    }
  cudaError_t e = cudaMemcpy(b->args, both.data(), sizeof(SweepArgs) * 2 * b->count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) b->bound_Q = Q;
  return e;
}

static cudaError_t batch_ctl(aderdg_batch_t b, int which, cudaStream_t s) {
  batch_control_kernel<<<(b->count + 127) / 128, 128, 0, s>>>(b->ctl, b->cp, b->count, which, b->counter);
  b->launches += 1;
  return cudaGetLastError();
}

static cudaError_t batch_sweep_launch(aderdg_batch_t b, int stage, int parity, int grid, cudaStream_t s);

static cudaError_t batch_sweep(aderdg_batch_t b, int stage, int parity, cudaStream_t s, bool timed = false) {
  const int grid = b->nsm * b->bps;
  b->launches += 1;
  cudaEvent_t pe1 = nullptr;
  if (timed && b->prof) {
    if (b->prof_used == b->prof_ev.size()) {
      std::pair<cudaEvent_t, cudaEvent_t> pe{nullptr, nullptr};
      if (cudaEventCreate(&pe.first) != cudaSuccess || cudaEventCreate(&pe.second) != cudaSuccess)
        return cudaErrorMemoryAllocation;
      b->prof_ev.push_back(pe);
    }
    cudaEventRecord(b->prof_ev[b->prof_used].first, s);
    pe1 = b->prof_ev[b->prof_used].second;
    b->prof_used += 1;
  }
  cudaError_t e = batch_sweep_launch(b, stage, parity, grid, s);
  if (pe1) cudaEventRecord(pe1, s);
  return e;
}

template <int MINB>
static void batch_sweep_launch_v(aderdg_batch_t b, int stage, int parity, int grid, cudaStream_t s) {
  switch (stage) {
    case kPredict:
      batch_kernel<kPredict, MINB><<<grid, kBThreads, kBSmem, s>>>(b->args, b->count, b->items, b->nitems, b->counter,
                                                                  parity);
      break;
    case kFused:
      batch_kernel<kFused, MINB><<<grid, kBThreads, kBSmem, s>>>(b->args, b->count, b->items, b->nitems, b->counter,
                                                                parity);
      break;
    default:
      batch_kernel<kCorrect, MINB><<<grid, kBThreads, kBSmem, s>>>(b->args, b->count, b->items, b->nitems, b->counter,
                                                                  parity);
  }
}

// k CTAs per SM run the build with the register budget of k CTAs per SM.
static cudaError_t batch_sweep_launch(aderdg_batch_t b, int stage, int parity, int grid, cudaStream_t s) {
  if (b->bps == 1) batch_sweep_launch_v<1>(b, stage, parity, grid, s);
  else if (b->bps == 2) batch_sweep_launch_v<2>(b, stage, parity, grid, s);
  else batch_sweep_launch_v<3>(b, stage, parity, grid, s);
  return cudaGetLastError();
}

// Arguments of scenario i for its own single-scenario kernel, whose tiles may
// hold fewer cells than the ensemble kernel's.
static SweepArgs single_args(aderdg_batch_t b, int i) {
  SweepArgs a = b->hargs[i];
  a.htab = &b->htab[b->scen[i].N - kBNmin];
  a.ntiles = (b->cells[i] + b->ks[i]->LIN_CPB - 1) / b->ks[i]->LIN_CPB;
  return a;
}

// One fused step of every scenario with its own launches (the comparison form).
static cudaError_t per_scenario_step(aderdg_batch_t b, int stage, int parity, cudaStream_t s) {
  for (int i = 0; i < b->count; ++i) {
    cudaError_t e = launch_control(2, b->ctl + i, b->hcp[i], 0, s);
    if (e != cudaSuccess) return e;
    SweepArgs a = single_args(b, i);
    a.hull_in = b->hull_bufs[2 * i + parity];
    a.hull_out = b->hull_bufs[2 * i + (parity ^ 1)];
    e = b->ks[i]->lin_sweep(stage, a, (int)a.ntiles, s);
    if (e != cudaSuccess) return e;
    e = launch_control(3, b->ctl + i, b->hcp[i], 0, s);
    if (e != cudaSuccess) return e;
    b->launches += 3;
  }
  return cudaSuccess;
}

extern "C" aderdg_status aderdg_batch_offsets(aderdg_batch_t b, long long *elem_offsets) {
  if (!b || !elem_offsets) return ADERDG_EINVAL;
  for (int s = 0; s <= b->count; ++s) elem_offsets[s] = b->offs[s];
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_batch_step(aderdg_batch_t b, float *dev_Q, int nsteps, int mode, void *stream) {
  if (!b || !dev_Q || nsteps < 0 || mode < 0 || mode > 2) return ADERDG_EINVAL;
  if (((uintptr_t)dev_Q) % 16) return ADERDG_EINVAL;
  if (nsteps == 0) return ADERDG_OK;
  cudaStream_t us = (cudaStream_t)stream, s = b->is;
#define BK(call)                                 \
  do {                                           \
    if ((call) != cudaSuccess) return ADERDG_ECUDA; \
  } while (0)
  BK(batch_bind(b, dev_Q));
  BK(cudaEventRecord(b->ev_in, us));
  BK(cudaStreamWaitEvent(s, b->ev_in, 0));
  // first sweep: Delta t of every scenario from its state, STP only (writes hull 0)
  BK(batch_ctl(b, 0, s));
  if (mode == 2) {
    for (int i = 0; i < b->count; ++i) {
      SweepArgs a = b->hargs[i];
      const long long nodes = b->cells[i] * (b->scen[i].N + 1) * (b->scen[i].N + 1);
      BK(b->ks[i]->lambda(a, (int)std::min<long long>((nodes + 255) / 256, 1024), s));
      b->launches += 1;
    }
  } else {
    batch_lambda_kernel<<<b->nsm * b->bps, kBThreads, 0, s>>>(b->args, b->items, b->nitems, b->counter);
    b->launches += 1;
    BK(cudaGetLastError());
  }
  BK(batch_ctl(b, 1, s));
  if (mode == 2) {
    for (int i = 0; i < b->count; ++i) {
      SweepArgs a = single_args(b, i);
      a.hull_out = b->hull_bufs[2 * i];
      BK(b->ks[i]->lin_sweep(kPredict, a, (int)a.ntiles, s));
    }
  } else {
    BK(batch_sweep(b, kPredict, 1, s));
  }
  int parity = 0;
  int fused = nsteps - 1;
  if (mode == 0 && fused >= 2) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      BK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      const long long l0 = b->launches;
      for (int p = 0; p < 2; ++p) {
        batch_ctl(b, 2, s);
        batch_sweep(b, kFused, p, s);
        batch_ctl(b, 3, s);
      }
      b->launches = l0;
      BK(cudaStreamEndCapture(s, &g));
      const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
      cudaGraphDestroy(g);
      BK(e);
    }
    for (; fused >= 2; fused -= 2) {
      BK(cudaGraphLaunch(b->graph, s));
      b->launches += 6;
    }
  }
  for (; fused > 0; --fused) {
    if (mode == 2) {
      BK(per_scenario_step(b, kFused, parity, s));
    } else {
      BK(batch_ctl(b, 2, s));
      BK(batch_sweep(b, kFused, parity, s, true));
      BK(batch_ctl(b, 3, s));
    }
    parity ^= 1;
  }
  if (mode == 2) {
    BK(per_scenario_step(b, kCorrect, parity, s));
  } else {
    BK(batch_ctl(b, 2, s));
    BK(batch_sweep(b, kCorrect, parity, s));
    BK(batch_ctl(b, 3, s));
  }
  BK(cudaEventRecord(b->ev_out, s));
  BK(cudaStreamWaitEvent(us, b->ev_out, 0));
  // device errors of any scenario
  std::vector<DevCtl> hc(b->count);
  BK(cudaMemcpyAsync(hc.data(), b->ctl, sizeof(DevCtl) * b->count, cudaMemcpyDeviceToHost, s));
  BK(cudaStreamSynchronize(s));
#undef BK
  for (const DevCtl &c : hc)
    if (c.error) return (aderdg_status)c.error;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_batch_autotune(aderdg_batch_t b, float *dev_Q, int steps, void *stream) {
  if (!b || !dev_Q) return ADERDG_EINVAL;
  float *work = nullptr;
  if (cudaMalloc(&work, sizeof(float) * b->total) != cudaSuccess) return ADERDG_ENOMEM;
  const int tpis[4] = {1, 2, 4, 8};
  double best = 1e300;
  int bb = b->bps, bt = b->tpi;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  aderdg_status st = ADERDG_OK;
  for (int bps = 1; bps <= b->max_bps && !st; ++bps)
    for (int ti = 0; ti < 4 && !st; ++ti) {
      b->bps = bps;
      b->tpi = tpis[ti];
      if (batch_items(b) != cudaSuccess) {
        st = ADERDG_ECUDA;
        break;
      }
      if (cudaMemcpy(work, dev_Q, sizeof(float) * b->total, cudaMemcpyDeviceToDevice) != cudaSuccess) {
        st = ADERDG_ECUDA;
        break;
      }
      b->bound_Q = nullptr;
      cudaEventRecord(e0, b->is);
      st = aderdg_batch_step(b, work, std::max(3, steps), 1, stream);
      cudaEventRecord(e1, b->is);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!st && ms < best) {
        best = ms;
        bb = bps;
        bt = tpis[ti];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(work);
  b->bound_Q = nullptr;
  b->bps = bb;
  b->tpi = bt;
  if (batch_items(b) != cudaSuccess) return ADERDG_ECUDA;
  return st;
}

extern "C" aderdg_status aderdg_batch_profile(aderdg_batch_t b, int enable) {
  if (!b) return ADERDG_EINVAL;
  b->prof = enable != 0;
  b->prof_used = 0;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_batch_profile_read(aderdg_batch_t b, double *ms_total, long long *count) {
  if (!b || !ms_total || !count) return ADERDG_EINVAL;
  double tot = 0.0;
  for (size_t i = 0; i < b->prof_used; ++i) {
    if (cudaEventSynchronize(b->prof_ev[i].second) != cudaSuccess) return ADERDG_ECUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->prof_ev[i].first, b->prof_ev[i].second) != cudaSuccess) return ADERDG_ECUDA;
    tot += ms;
  }
  *ms_total = tot;
  *count = (long long)b->prof_used;
  b->prof_used = 0;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_batch_get_tuning(aderdg_batch_t b, int *blocks_per_sm, int *tiles_per_item,
                                                 long long *launches) {
  if (!b) return ADERDG_EINVAL;
  if (blocks_per_sm) *blocks_per_sm = b->bps;
  if (tiles_per_item) *tiles_per_item = b->tpi;
  if (launches) *launches = b->launches;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_batch_destroy(aderdg_batch_t b) {
  if (!b) return ADERDG_OK;
  cudaDeviceSynchronize();
  batch_free(b);
  delete b;
  return ADERDG_OK;
}
