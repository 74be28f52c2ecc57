// noalloc.cu -- aderdg_step_noalloc: the fused ADER-DG step for callers that
// cannot allocate device memory.
//
// Who needs it: code that may not call cudaMalloc or cudaFree while it runs --
// a plugin whose host application owns the device memory budget (all of it is
// handed out by the host's own pool) or forbids allocations after start-up, or
// a time-critical loop that must not add the device-wide synchronisation that
// cudaFree performs.  aderdg_create allocates the step's scratch (the
// integrateVolume buffer D, two face-hull buffers, the time-step control block
// and the operator tables) on the device; this entry point instead carves that
// scratch out of one file-scope device array of fixed size, kScratchBytes,
// that every GPU loading the library holds until the process exits.
//
// Rules for callers:
//   * The first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (once per device, with that device current).  Make
//     that first call before any stream capture begins.
//   * Every call is synchronous: it enqueues the step on `stream`, then waits
//     for that stream (not for the whole device) before it returns.
//   * Every call on a device shares the one array and leaves the last call's
//     contents in it.  Calls whose work overlaps on the GPU (different streams,
//     or different host threads on the same device) race on it: serialise them.
//   * Every argument is checked before any CUDA call; a problem whose scratch
//     does not fit is rejected with ADERDG_EINVAL and nothing is launched.
// The paper has no counterpart of this entry point; it reuses the kernels of
// the fused form unchanged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "aderdg.h"
#include "basis.h"
#include "registry.h"
#include "validate.h"

namespace aderdg {

cudaError_t launch_control(int which, DevCtl *c, const CtlParams &p, int arg, cudaStream_t s);
template <class R>
void fill_tables(const Basis1D &B, Tables<R> &T);

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kHistCap = 1024;                      // dt history entries kept
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char *g_dev_scratch[kMaxDevices];  // device address of g_scratch per device
Basis1D g_basis[kMaxN + 1];
bool g_basis_ok[kMaxN + 1];

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int pde_vars(int pde, int d) {
  switch (pde) {
    case ADERDG_ADVECTION: return 1;
    case ADERDG_ACOUSTICS: return d + 1;
    case ADERDG_EULER: return d + 2;
    case ADERDG_ELASTICITY: return d == 3 ? 9 : 5;
  }
  return -1;
}

}  // namespace
}  // namespace aderdg

using namespace aderdg;

extern "C" aderdg_status aderdg_step_noalloc(int d, int N, int m, aderdg_pde pde, const int grid[3],
                                             const double dx[3], const aderdg_params *params,
                                             const float *dev_mat, void *dev_Q, int nsteps,
                                             double fixed_dt, double *t_inout, void *stream) {
  // ---- arguments: every check comes before any CUDA call, so nothing is
  // launched on failure
  if (d < 2 || d > 3 || N < 0 || N > kMaxN || (int)pde < 0 || (int)pde > 3) return ADERDG_EINVAL;
  if (m != pde_vars(pde, d) || !grid || !dx || !dev_Q || nsteps < 0) return ADERDG_EINVAL;
  if (((uintptr_t)dev_Q) % 16) return ADERDG_EINVAL;
  if (!(fixed_dt >= 0.0) || !std::isfinite(fixed_dt)) return ADERDG_EINVAL;
  // Cells, bounded while they are multiplied up: no problem with more cells
  // than bytes of scratch can fit, and the running product stays below 2^55.
  long long C = 1;
  int g3[3] = {1, 1, 1};
  double dx3[3] = {1.0, 1.0, 1.0};
  for (int a = 0; a < d; ++a) {
    if (grid[a] < 1 || !(dx[a] > 0.0) || !std::isfinite(dx[a])) return ADERDG_EINVAL;
    g3[a] = grid[a];
    dx3[a] = dx[a];
    C *= grid[a];
    if (C > (long long)kScratchBytes) return ADERDG_EINVAL;
  }
  aderdg_params prm{};
  if (params) prm = *params;
  if (prm.cfl == 0.0) prm.cfl = std::fmax(0.3, std::fmin(0.9, 0.9 - 0.1 * N));
  if (!(prm.cfl > 0.0 && prm.cfl <= 1.0) || prm.picard_iters < 0 || prm.picard_iters > kMaxPicard)
    return ADERDG_EINVAL;
  if (prm.precision < 0 || prm.precision > 3 || prm.form != ADERDG_FORM_FUSED) return ADERDG_EINVAL;
  if (prm.dt_policy < 0 || prm.dt_policy > 1 || prm.predictor < 0 || prm.predictor > 2) return ADERDG_EINVAL;
  if (check_pde_const(pde, prm.pde_const)) return ADERDG_EINVAL;  // the same constants aderdg_create accepts
  if (check_material_jumps(prm.material_jumps, pde, prm.form, prm.predictor)) return ADERDG_EINVAL;
  if (dev_mat && pde != ADERDG_ELASTICITY) return ADERDG_EINVAL;
  const bool linear = pde != ADERDG_EULER;
  const int pred = prm.predictor == ADERDG_PREDICT_SPACETIME_TF32 ? kSpaceTimeTC
                   : (prm.predictor == ADERDG_PREDICT_SPACETIME || !linear) ? kSpaceTime : kTimeModal;
  const KernelSet *ks = find_set(pde, d, N, prm.precision, pred);
  if (!ks) return ADERDG_EUNSUPPORTED;
  const bool lin = ks->lin_sweep != nullptr;
  if (prm.material_jumps && !ks->lin_sweep_ext) return ADERDG_EUNSUPPORTED;

  // ---- scratch layout inside the static array
  const size_t rb = ks->real_bytes;
  const size_t tab_bytes = rb == 4 ? sizeof(Tables<float>) : sizeof(Tables<double>);
  const size_t hs = lin ? (size_t)ks->HSL : (size_t)ks->HS;
  const size_t off_ctl = 0;
  const size_t off_hist = align256(off_ctl + sizeof(DevCtl));
  const size_t off_tab = align256(off_hist + sizeof(double) * kHistCap);
  const size_t off_D = align256(off_tab + tab_bytes);
  // bytes per cell first: C is bounded before the region sizes are formed
  // (the three 256-byte alignments add at most 768 bytes)
  const size_t per_cell = ((size_t)m * ks->NS + 2 * hs) * rb;
  if (off_D + 768 > kScratchBytes || (size_t)C > (kScratchBytes - off_D - 768) / per_cell)
    return ADERDG_EINVAL;  // problem larger than the static scratch
  const size_t off_h0 = align256(off_D + (size_t)C * m * ks->NS * rb);
  const size_t off_h1 = align256(off_h0 + (size_t)C * hs * rb);
  const size_t need = align256(off_h1 + (size_t)C * hs * rb);
  if (need > kScratchBytes) return ADERDG_EINVAL;
  if (nsteps == 0) return ADERDG_OK;  // a valid no-op

  // ---- once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ADERDG_ECUDA;
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_scratch[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return ADERDG_ECUDA;
      g_dev_scratch[dev] = static_cast<unsigned char *>(p);
    }
    base = g_dev_scratch[dev];
    if (!g_basis_ok[N]) {
      if (!build_basis(N, g_basis[N])) return ADERDG_EINVAL;
      g_basis_ok[N] = true;
    }
  }
  if (ks->prepare() != cudaSuccess) return ADERDG_ECUDA;  // kernel attributes, no allocation
  cudaStream_t s = (cudaStream_t)stream;
  DevCtl *ctl = reinterpret_cast<DevCtl *>(base + off_ctl);

  // ---- per call: the control block starts from zero, the tables are rewritten
  union {
    Tables<float> f;
    Tables<double> d;
  } htab;
  if (rb == 4) fill_tables(g_basis[N], htab.f);
  else fill_tables(g_basis[N], htab.d);
  DevCtl c0;
  std::memset(&c0, 0, sizeof c0);
  c0.hist = reinterpret_cast<double *>(base + off_hist);
  c0.hist_cap = kHistCap;
  if (cudaMemcpyAsync(ctl, &c0, sizeof c0, cudaMemcpyHostToDevice, s) != cudaSuccess) return ADERDG_ECUDA;
  if (cudaMemcpyAsync(base + off_tab, &htab, tab_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return ADERDG_ECUDA;

  CtlParams cp{};
  double hmin = dx3[0];
  for (int a = 1; a < d; ++a) hmin = std::fmin(hmin, dx3[a]);
  cp.cfl = prm.cfl;
  cp.dt_scale = hmin / (d * (2.0 * N + 1.0));
  cp.fixed_dt = fixed_dt;
  cp.inject_factor = prm.inject_factor;
  cp.policy = prm.dt_policy;
  cp.inject_step = prm.inject_step;
  const bool gate = (!linear || prm.inject_step > 0) && !(fixed_dt > 0.0);

  SweepArgs a{};
  a.Q_in = dev_Q;
  a.Q_out = dev_Q;
  a.Dbuf = base + off_D;
  a.mat = dev_mat;
  a.ctl = ctl;
  a.tables = base + off_tab;
  a.htab = &htab;
  a.ncells = C;
  const int cpb = lin ? ks->LIN_CPB : ks->CPB;
  a.ntiles = (C + cpb - 1) / cpb;
  for (int i = 0; i < 3; ++i) {
    a.grid[i] = g3[i];
    a.inv_dx[i] = 1.0 / dx3[i];
  }
  a.picard = prm.picard_iters ? prm.picard_iters : N + 1;
  a.ncp = prm.material_jumps;
  for (int i = 0; i < 8; ++i) a.cst[i] = prm.pde_const[i];
  void *hull[2] = {base + off_h0, base + off_h1};
  const int grid_main = (int)a.ntiles;
  int bps = lin ? ks->lin_blocks_per_sm(kPredict) : ks->blocks_per_sm(kPredict);
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ADERDG_ECUDA;
  const int grid_gate = (int)std::min<long long>(a.ntiles, (long long)nsm * (bps > 0 ? bps : 1));
  const int grid_lambda = (int)std::min<long long>((C * ks->NS + 255) / 256, (long long)nsm * 8);
  auto sweep = [&](int stage, const SweepArgs &x, int g) {
    if (lin && prm.material_jumps) return ks->lin_sweep_ext(stage, x, g, s);
    return lin ? ks->lin_sweep(stage, x, g, s) : ks->sweep(stage, x, g, s);
  };
#define NA_CK(call)                         \
  do {                                      \
    if ((call) != cudaSuccess) return ADERDG_ECUDA; \
  } while (0)

  // ---- Algorithm 2: first sweep STP only, nsteps - 1 fused sweeps, last corrector
  int cur = 0;
  NA_CK(launch_control(0, ctl, cp, 0, s));
  NA_CK(ks->lambda(a, grid_lambda, s));
  NA_CK(launch_control(1, ctl, cp, 0, s));
  a.hull_out = hull[0];
  NA_CK(sweep(kPredict, a, grid_main));
  for (int k = 0; k < nsteps; ++k) {
    const int stage = k + 1 < nsteps ? kFused : kCorrect;
    NA_CK(launch_control(2, ctl, cp, 0, s));
    if (gate) {
      SweepArgs g = a;
      g.gate = 1;
      g.pred_dt_old = 1;
      g.hull_out = hull[cur];
      NA_CK(sweep(kPredict, g, grid_gate));
    }
    a.hull_in = hull[cur];
    a.hull_out = hull[cur ^ 1];
    NA_CK(sweep(stage, a, grid_main));
    if (stage == kFused) cur ^= 1;
    NA_CK(launch_control(3, ctl, cp, 0, s));
  }
#undef NA_CK
  DevCtl out;
  if (cudaMemcpyAsync(&out, ctl, sizeof out, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ADERDG_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return ADERDG_ECUDA;
  if (t_inout) *t_inout += out.t;
  if (out.error) return (aderdg_status)out.error;
  return ADERDG_OK;
}
