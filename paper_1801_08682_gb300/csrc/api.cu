// api.cu -- host orchestration and the C ABI of libaderdg (include/aderdg.h).
//
// Time-step control lives on the device (DevCtl, FP64) so a step needs no
// host round trip: the corrector sweep folds its spectral radius into one
// word, a one-thread control kernel turns it into dt_adm and, for the fused
// form, applies the optimistic rule of Algorithm 2 (Technique 5):
//   before sweep k:  rerun = dt_adm < dt_new
//                    dt_old = rerun ? C dt_adm : dt_new
//                    dt_new = C dt_adm  (strict)  or  (dt_old + C dt_adm)/2 (creeping)
//   a grid-capped STP sweep then runs only if rerun is set (it reads the
//   flag on the device), so the launch sequence is fixed and capturable.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "aderdg.h"
#include "adjoint.cuh"
#include "basis.h"
#include "control.cuh"
#include "registry.h"
#include "validate.h"

namespace aderdg {

static std::vector<KernelSet> &registry() {
  static std::vector<KernelSet> v;
  return v;
}
void register_set(const KernelSet &ks) { registry().push_back(ks); }
const KernelSet *find_set(int pde, int d, int N, int prec, int pred) {
  for (const KernelSet &k : registry())
    if (k.pde == pde && k.d == d && k.N == N && k.prec == prec && k.pred == pred) return &k;
  return nullptr;
}
int registered_count() { return (int)registry().size(); }
const KernelSet *registered_at(int i) { return &registry()[i]; }

// ---------------------------------------------------------------------------
// Control kernels (one thread)

__global__ void ctl_reset_kernel(DevCtl *c) { ctl_reset(c); }

__global__ void ctl_begin_kernel(DevCtl *c, CtlParams p, int multipass) { ctl_begin(c, p, multipass); }

__global__ void ctl_pre_kernel(DevCtl *c, CtlParams p) { ctl_pre(c, p); }

__global__ void ctl_post_kernel(DevCtl *c, CtlParams p, int multipass) { ctl_post(c, p, multipass); }

// The point-source coefficients of the coming sweep (one thread per source).
__global__ void src_coef_kernel(const DevCtl *c, const SrcTime *st, SrcCoefParams p, double *co) {
  const int k = threadIdx.x;
  if (k < p.nsrc) src_coef(c, st[k], p, co + (long long)k * kSrcCo);
}

// Host launcher of the control kernels for other translation units.
// which: 0 reset, 1 begin (arg = multipass), 2 pre, 3 post (arg = multipass).
cudaError_t launch_control(int which, DevCtl *c, const CtlParams &p, int arg, cudaStream_t s) {
  switch (which) {
    case 0: ctl_reset_kernel<<<1, 1, 0, s>>>(c); break;
    case 1: ctl_begin_kernel<<<1, 1, 0, s>>>(c, p, arg); break;
    case 2: ctl_pre_kernel<<<1, 1, 0, s>>>(c, p); break;
    case 3: ctl_post_kernel<<<1, 1, 0, s>>>(c, p, arg); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class R>
void fill_tables(const Basis1D &B, Tables<R> &T) {
  std::memset(&T, 0, sizeof(T));
  const int n = B.n;
  for (int i = 0; i < n * n; ++i) {
    T.Dm[i] = (R)B.Dm[i];
    T.Kvol[i] = (R)B.Kvol[i];
    T.K1inv[i] = (R)B.K1inv[i];
  }
  for (int i = 0; i < n; ++i) {
    T.FL[i] = (R)B.FL[i];
    T.FR[i] = (R)B.FR[i];
    T.w[i] = (R)B.w[i];
    T.iw[i] = (R)(1.0 / B.w[i]);
  }
  for (int s = 0; s <= kMaxPicard; ++s) {
    T.g[s] = (R)B.g[s];
    for (int k = 0; k < n; ++k) T.cvec[s * n + k] = (R)B.cvec[s * n + k];
  }
  const int h = n / 2, hc = (n + 1) / 2;
  for (int o = 0; o < hc; ++o) {
    for (int b = 0; b < h; ++b) {
      T.DmE[o * kMaxH + b] = (R)(0.5 * (B.Dm[o * n + b] + B.Dm[o * n + n - 1 - b]));
      T.DmO[o * kMaxH + b] = (R)(0.5 * (B.Dm[o * n + b] - B.Dm[o * n + n - 1 - b]));
      T.KvE[o * kMaxH + b] = (R)(0.5 * (B.Kvol[o * n + b] + B.Kvol[o * n + n - 1 - b]));
      T.KvO[o * kMaxH + b] = (R)(0.5 * (B.Kvol[o * n + b] - B.Kvol[o * n + n - 1 - b]));
    }
    if (n % 2) {
      T.DmM[o] = (R)B.Dm[o * n + h];
      T.KvM[o] = (R)B.Kvol[o * n + h];
    }
  }
  for (int b = 0; b < n; ++b) {
    T.FLR[2 * b] = (R)B.FL[b];
    T.FLR[2 * b + 1] = (R)B.FR[b];
  }
  for (int k = 0; 2 * k + 1 < n; ++k)
    for (int b = 0; b < n; ++b)
      for (int l = 0; l < 2; ++l) {
        T.DmP[(k * kMaxn + b) * 2 + l] = (R)B.Dm[(2 * k + l) * n + b];
        T.KvP[(k * kMaxn + b) * 2 + l] = (R)B.Kvol[(2 * k + l) * n + b];
      }
}

// Receivers: out[r][k] = sum_i w[r][i] Q[cell_r][comps[k]][i] (one block per receiver)
template <class T>
__global__ void rec_sample_kernel(const T *Q, const long long *rcell, const double *rw, int R, int NS, int m,
                                  const int *comps, int nc, double *out) {
  __shared__ double part[256];
  const int r = blockIdx.x;
  if (r >= R) return;
  for (int k = 0; k < nc; ++k) {
    double s = 0.0;
    const T *src = Q + (rcell[r] * m + comps[k]) * NS;
    for (int i = threadIdx.x; i < NS; i += blockDim.x) s += (double)rw[(long long)r * NS + i] * (double)src[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[r * nc + k] = part[0];
    __syncthreads();
  }
}

// Adjoint of the receivers: lam[cell_r][comps[k]][i] += res[r][k] w[r][i]
template <class T>
__global__ void rec_adjoint_kernel(T *lam, const long long *rcell, const double *rw, int R, int NS, int m,
                                   const int *comps, int nc, const double *res) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)R * NS) return;
  const int r = (int)(t / NS), i = (int)(t % NS);
  for (int k = 0; k < nc; ++k)
    atomicAdd(&lam[(rcell[r] * m + comps[k]) * NS + i], (T)(res[r * nc + k] * rw[t]));
}

__global__ void d2f_kernel(const double *src, float *dst, long long n) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}

template void fill_tables<float>(const Basis1D &, Tables<float> &);
template void fill_tables<double>(const Basis1D &, Tables<double> &);

}  // namespace aderdg

using namespace aderdg;

// chunks of the host-resident step (aderdg_step_host)
static constexpr int kHostChunks = 32;

struct aderdg_ctx {
  int d, N, m, pde, prec, pred, form, picard;
  int grid[3];
  double dx[3];
  aderdg_params prm;
  long long C;
  const KernelSet *ks;
  int device, nsm;
  void *tables;
  void *D;
  void *hull[2];
  int cur;
  void *fstar, *st, *face_st;
  float *mat;
  void *matp;                      // MatBox<PDE::Mat>: one entry (uniform) or C (per-cell material)
  long long matp_cap;              // entries allocated at matp
  int ncp;                         // material jumps in non-conservative form
  int nsrc;                        // point sources
  SrcDev *d_src;
  SrcTime *d_srct;
  double *d_srcco;                 // [kMaxSources][kSrcCo]
  SrcCoefParams scp;
  DevCtl *ctl;
  double *hist;
  int hist_cap;
  void *stage_Q;
  size_t stage_bytes;
  std::string err;
  long long launches;
  bool begun;
  void *begun_Q;
  bool gate_needed;
  int grid_gate, grid_lambda, grid_riemann;
  CtlParams cp;
  cudaStream_t last_stream;
  size_t persistent_bytes;
  struct Prof {
    int tag;
    cudaEvent_t a, b;
  };
  bool prof_on;
  std::vector<Prof> prof;
  bool use_lin;                    // fused form through the line-owner kernel
  std::vector<unsigned char> htab; // host copy of the operator tables
  // aderdg_step_host: copy streams (host to device, device to host) and
  // per-chunk events (created on first use)
  cudaStream_t copy_stream, copy_stream_out;
  cudaEvent_t host_ev[2 * kHostChunks + 1];
};

enum ProfTag { kTagFused = 0, kTagStp = 1, kTagCorrect = 2, kTagRiemann = 3, kTagT1 = 4 };

// Launch `fn` on stream s, bracketed by CUDA events when profiling is on.
template <class F>
static cudaError_t timed(aderdg_t h, int tag, cudaStream_t s, F fn) {
  if (!h->prof_on) return fn();
  aderdg_ctx::Prof p{tag, nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&p.a);
  if (e == cudaSuccess) e = cudaEventCreate(&p.b);
  if (e == cudaSuccess) e = cudaEventRecord(p.a, s);
  if (e != cudaSuccess) return e;
  e = fn();
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(p.b, s);
  h->prof.push_back(p);
  return e;
}

static thread_local std::string g_create_error;

static aderdg_status fail(aderdg_t h, aderdg_status st, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_error = msg;
  return st;
}

static aderdg_status cuda_fail(aderdg_t h, cudaError_t e, const char *what) {
  return fail(h, e == cudaErrorMemoryAllocation ? ADERDG_ENOMEM : ADERDG_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call, what)                          \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
  } while (0)

static int pde_vars(int pde, int d) {
  switch (pde) {
    case ADERDG_ADVECTION: return 1;
    case ADERDG_ACOUSTICS: return d + 1;
    case ADERDG_EULER: return d + 2;
    case ADERDG_ELASTICITY: return d == 3 ? 9 : 5;
  }
  return -1;
}

static void free_all(aderdg_t h) {
  void *ptrs[] = {h->tables, h->D, h->hull[0], h->hull[1], h->fstar, h->st, h->face_st,
                  h->mat, h->matp, h->ctl, h->hist, h->stage_Q, h->d_src, h->d_srct, h->d_srcco};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (cudaEvent_t e : h->host_ev)
    if (e) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  if (h->copy_stream_out) cudaStreamDestroy(h->copy_stream_out);
}

extern "C" aderdg_status aderdg_create(int d, int N, int m, aderdg_pde pde, const int grid[3],
                                       const double dx[3], const aderdg_params *params,
                                       aderdg_t *out) {
  if (!out) return fail(nullptr, ADERDG_EINVAL, "out is NULL");
  *out = nullptr;
  if (d < 2 || d > 3) return fail(nullptr, ADERDG_EINVAL, "d must be 2 or 3");
  if (N < 0 || N > kMaxN) return fail(nullptr, ADERDG_EINVAL, "N must be in [0, 6]");
  if ((int)pde < 0 || (int)pde > 3) return fail(nullptr, ADERDG_EINVAL, "unknown pde");
  if (m != pde_vars(pde, d)) return fail(nullptr, ADERDG_EINVAL, "m does not match the PDE");
  if (!grid || !dx) return fail(nullptr, ADERDG_EINVAL, "grid/dx is NULL");
  long long C = 1;
  for (int a = 0; a < d; ++a) {
    if (grid[a] < 1) return fail(nullptr, ADERDG_EINVAL, "grid sizes must be >= 1");
    if (!(dx[a] > 0.0) || !std::isfinite(dx[a])) return fail(nullptr, ADERDG_EINVAL, "dx must be > 0");
    C *= grid[a];
  }
  aderdg_params prm{};
  if (params) prm = *params;
  if (prm.cfl == 0.0) prm.cfl = std::max(0.3, std::min(0.9, 0.9 - 0.1 * N));
  if (!(prm.cfl > 0.0 && prm.cfl <= 1.0)) return fail(nullptr, ADERDG_EINVAL, "cfl must be in (0, 1]");
  if (prm.picard_iters < 0 || prm.picard_iters > kMaxPicard)
    return fail(nullptr, ADERDG_EINVAL, "picard_iters must be in [0, 16]");
  if (prm.precision < 0 || prm.precision > 3) return fail(nullptr, ADERDG_EINVAL, "bad precision");
  if (prm.form < 0 || prm.form > 2) return fail(nullptr, ADERDG_EINVAL, "bad form");
  if (prm.dt_policy < 0 || prm.dt_policy > 1) return fail(nullptr, ADERDG_EINVAL, "bad dt_policy");
  if (prm.predictor < 0 || prm.predictor > 2) return fail(nullptr, ADERDG_EINVAL, "bad predictor");
  if (const char *why = check_material_jumps(prm.material_jumps, pde, prm.form, prm.predictor))
    return fail(nullptr, ADERDG_EINVAL, why);
  if (const char *why = check_pde_const(pde, prm.pde_const)) return fail(nullptr, ADERDG_EINVAL, why);
  const bool linear = pde != ADERDG_EULER;
  const int pred = prm.predictor == ADERDG_PREDICT_SPACETIME_TF32 ? kSpaceTimeTC
                   : (prm.predictor == ADERDG_PREDICT_SPACETIME || !linear) ? kSpaceTime : kTimeModal;
  const KernelSet *ks = find_set(pde, d, N, prm.precision, pred);
  if (!ks) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "configuration not compiled: pde=%d d=%d N=%d precision=%d predictor=%d",
                  (int)pde, d, N, prm.precision, pred);
    return fail(nullptr, ADERDG_EUNSUPPORTED, buf);
  }
  if (prm.form == ADERDG_FORM_TABLE1 && !ks->table1)
    return fail(nullptr, ADERDG_EUNSUPPORTED, "Table 1 multi-pass form not compiled for this configuration");
  if (prm.material_jumps && !ks->lin_sweep_ext)
    return fail(nullptr, ADERDG_EUNSUPPORTED, "non-conservative material jumps not compiled for this configuration");
  if (prm.form == ADERDG_FORM_TABLE1 && ks->pair)
    return fail(nullptr, ADERDG_EUNSUPPORTED, "the Table 1 form keeps no low words (FP32_PAIR)");

  aderdg_t h = new aderdg_ctx();
  std::memset(h->grid, 0, sizeof h->grid);
  h->d = d;
  h->N = N;
  h->m = m;
  h->pde = pde;
  h->prec = prm.precision;
  h->pred = pred;
  h->form = prm.form;
  h->picard = prm.picard_iters ? prm.picard_iters : N + 1;
  for (int a = 0; a < 3; ++a) {
    h->grid[a] = a < d ? grid[a] : 1;
    h->dx[a] = a < d ? dx[a] : 1.0;
  }
  h->prm = prm;
  h->C = C;
  h->ks = ks;
  h->ncp = prm.material_jumps;
  h->last_stream = nullptr;

  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess) e = ks->prepare();
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA setup: ") + cudaGetErrorString(e);
    delete h;
    return ADERDG_ECUDA;
  }

  Basis1D B;
  if (!build_basis(N, B)) {
    delete h;
    return fail(nullptr, ADERDG_EINVAL, "basis construction failed");
  }
  {  // point sources: the time operator M = K1^-1 diag(w) of the predictor
    SrcCoefParams &sp = h->scp;
    std::memset(&sp, 0, sizeof sp);
    sp.n = N + 1;
    sp.R = h->picard;
    for (int k = 0; k <= N; ++k) {
      sp.xi[k] = B.xi[k];
      sp.w[k] = B.w[k];
      for (int l = 0; l <= N; ++l) sp.M[k * (N + 1) + l] = B.K1inv[k * (N + 1) + l] * B.w[l];
    }
  }
  const size_t rb = ks->real_bytes;
  const long long S = (long long)m * ks->NS;
  size_t tab_bytes = rb == 4 ? sizeof(Tables<float>) : sizeof(Tables<double>);
  std::vector<unsigned char> tab(tab_bytes);
  if (rb == 4) fill_tables(B, *reinterpret_cast<Tables<float> *>(tab.data()));
  else fill_tables(B, *reinterpret_cast<Tables<double> *>(tab.data()));

  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes ? bytes : 16);
  };
  alloc(&h->tables, tab_bytes);
  if (e == cudaSuccess) e = cudaMemcpy(h->tables, tab.data(), tab_bytes, cudaMemcpyHostToDevice);
  h->persistent_bytes = 0;
  h->use_lin = h->form == ADERDG_FORM_FUSED && ks->lin_sweep != nullptr;
  h->htab = tab;
  const size_t hs = h->use_lin ? (size_t)ks->HSL : (size_t)ks->HS;
  if (h->form == ADERDG_FORM_FUSED || h->form == ADERDG_FORM_HULL3) {
    alloc(&h->D, (size_t)C * S * rb);
    alloc(&h->hull[0], (size_t)C * hs * rb);
    h->persistent_bytes += (size_t)S * rb + hs * rb;
    if (h->form == ADERDG_FORM_FUSED) {
      alloc(&h->hull[1], (size_t)C * hs * rb);
      h->persistent_bytes += hs * rb;
    }
  }
  if (h->form != ADERDG_FORM_FUSED) {
    alloc(&h->fstar, (size_t)d * C * m * ks->NF * rb);
    h->persistent_bytes += (size_t)d * m * ks->NF * rb;
  }
  if (h->form == ADERDG_FORM_TABLE1) {
    const size_t n = N + 1;
    alloc(&h->st, (size_t)C * (d + 1) * n * S * rb);
    alloc(&h->face_st, (size_t)C * 2 * d * 2 * n * m * ks->NF * rb);
    h->persistent_bytes += (size_t)(d + 1) * n * S * rb + (size_t)2 * d * 2 * n * m * ks->NF * rb;
  }
  h->hist_cap = 1 << 16;
  alloc((void **)&h->hist, sizeof(double) * h->hist_cap);
  alloc((void **)&h->ctl, sizeof(DevCtl));
  if (e == cudaSuccess) {
    DevCtl c{};
    c.hist = h->hist;
    c.hist_cap = h->hist_cap;
    e = cudaMemcpy(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice);
  }
  // the PDE constants of the uniform material, once (FP64 arithmetic, rounded
  // to the kernel type)
  alloc(&h->matp, ks->mat_bytes);
  h->matp_cap = 1;
  if (e == cudaSuccess) e = ks->mat_pre(prm.pde_const, nullptr, 1, h->matp, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_create_error = std::string("allocation: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? ADERDG_ENOMEM : ADERDG_ECUDA;
  }
  double hmin = h->dx[0];
  for (int a = 1; a < d; ++a) hmin = std::fmin(hmin, h->dx[a]);
  h->cp.cfl = prm.cfl;
  h->cp.dt_scale = hmin / (d * (2.0 * N + 1.0));
  h->cp.fixed_dt = 0.0;
  h->cp.inject_factor = prm.inject_factor;
  h->cp.policy = prm.dt_policy;
  h->cp.inject_step = prm.inject_step;
  h->gate_needed = !linear || prm.inject_step > 0;
  const int bps = h->use_lin ? ks->lin_blocks_per_sm(kPredict) : ks->blocks_per_sm(kPredict);
  const long long ntiles = (C + (h->use_lin ? ks->LIN_CPB : ks->CPB) - 1) / (h->use_lin ? ks->LIN_CPB : ks->CPB);
  h->grid_gate = (int)std::min<long long>(ntiles, (long long)h->nsm * (bps > 0 ? bps : 1));
  h->grid_lambda = (int)std::min<long long>((C * ks->NS + 255) / 256, (long long)h->nsm * 8);
  const int rfpb = std::max(1, 256 / ks->NF);
  h->grid_riemann = (int)std::min<long long>((d * C + rfpb - 1) / rfpb, 1ll << 30);
  *out = h;
  return ADERDG_OK;
}

static SweepArgs sweep_args(aderdg_t h, void *Q) {
  SweepArgs a{};
  a.Q_in = Q;
  a.Q_out = Q;
  a.Dbuf = h->D;
  a.hull_in = h->hull[h->cur];
  a.hull_out = h->hull[h->cur ^ 1];
  a.fstar = h->fstar;
  a.mat = h->mat;
  a.ctl = h->ctl;
  a.tables = h->tables;
  a.htab = h->htab.data();
  a.ncells = h->C;
  const int cpb = h->use_lin ? h->ks->LIN_CPB : h->ks->CPB;
  a.ntiles = (h->C + cpb - 1) / cpb;
  for (int i = 0; i < 3; ++i) {
    a.grid[i] = h->grid[i];
    a.inv_dx[i] = 1.0 / h->dx[i];
  }
  a.picard = h->picard;
  for (int i = 0; i < 8; ++i) a.cst[i] = h->prm.pde_const[i];
  a.ncp = h->ncp;
  a.nsrc = h->nsrc;
  a.src = h->d_src;
  a.srcco = h->d_srcco;
  a.matp = h->matp;
  return a;
}

static MultiArgs multi_args(aderdg_t h, void *Q) {
  MultiArgs a{};
  a.Q_in = Q;
  a.Q_out = Q;
  a.st = h->st;
  a.face_st = h->face_st;
  a.fstar = h->fstar;
  a.mat = h->mat;
  a.ctl = h->ctl;
  a.tables = h->tables;
  a.ncells = h->C;
  for (int i = 0; i < 3; ++i) {
    a.grid[i] = h->grid[i];
    a.inv_dx[i] = 1.0 / h->dx[i];
  }
  a.picard = h->picard;
  for (int i = 0; i < 8; ++i) a.cst[i] = h->prm.pde_const[i];
  return a;
}

static int main_grid(aderdg_t h) {
  const int cpb = h->use_lin ? h->ks->LIN_CPB : h->ks->CPB;
  const long long nt = (h->C + cpb - 1) / cpb;
  return (int)std::min<long long>(nt, 0x7fffffffll);
}

// The cell sweep of the fused form: line-owner kernel for linear PDEs,
// node-owner kernel otherwise.
static cudaError_t fused_form_sweep(aderdg_t h, int stage, const SweepArgs &a, int grid, cudaStream_t s) {
  if (h->use_lin && (h->ncp || h->nsrc)) return h->ks->lin_sweep_ext(stage, a, grid, s);
  return h->use_lin ? h->ks->lin_sweep(stage, a, grid, s) : h->ks->sweep(stage, a, grid, s);
}

static aderdg_status launch_err(aderdg_t h, cudaError_t e, const char *what) {
  h->launches += 1;
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  return ADERDG_OK;
}

// The point-source coefficients of the coming sweep (after its control step).
static aderdg_status source_coefficients(aderdg_t h, cudaStream_t s) {
  if (!h->nsrc) return ADERDG_OK;
  src_coef_kernel<<<1, 64, 0, s>>>(h->ctl, h->d_srct, h->scp, h->d_srcco);
  return launch_err(h, cudaGetLastError(), "source coefficient kernel");
}

// Fused form: pre-control, optional rerun STP, one sweep of `stage`, post-control.
static aderdg_status fused_sweep(aderdg_t h, void *Q, int stage, cudaStream_t s) {
  ctl_pre_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp);
  aderdg_status st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  if ((st = source_coefficients(h, s))) return st;
  if (h->gate_needed && h->cp.fixed_dt <= 0.0) {
    SweepArgs g = sweep_args(h, Q);
    g.gate = 1;
    g.pred_dt_old = 1;
    g.hull_out = h->hull[h->cur];
    st = launch_err(h, timed(h, kTagStp, s, [&] { return fused_form_sweep(h, kPredict, g, h->grid_gate, s); }),
                    "rerun STP sweep");
    if (st) return st;
  }
  SweepArgs a = sweep_args(h, Q);
  st = launch_err(h, timed(h, stage == kFused ? kTagFused : kTagCorrect, s,
                           [&] { return fused_form_sweep(h, stage, a, main_grid(h), s); }),
                  "fused sweep");
  if (st) return st;
  if (stage == kFused) h->cur ^= 1;
  ctl_post_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp, 0);
  return launch_err(h, cudaGetLastError(), "control kernel");
}

// One whole Algorithm-1 step of the multi-pass forms.
static aderdg_status multipass_step(aderdg_t h, void *Q, cudaStream_t s) {
  aderdg_status st;
  if (h->form == ADERDG_FORM_HULL3) {
    SweepArgs a = sweep_args(h, Q);
    a.pred_dt_old = 1;
    a.hull_out = h->hull[0];
    st = launch_err(h, timed(h, kTagStp, s, [&] { return h->ks->sweep(kPredict, a, main_grid(h), s); }),
                    "STP sweep");
    if (st) return st;
    a.hull_in = h->hull[0];
    st = launch_err(h, timed(h, kTagRiemann, s, [&] { return h->ks->riemann(a, h->grid_riemann, s); }),
                    "Riemann sweep");
    if (st) return st;
    st = launch_err(h, timed(h, kTagCorrect, s, [&] { return h->ks->sweep(kCorrectFs, a, main_grid(h), s); }),
                    "corrector sweep");
    if (st) return st;
  } else {
    MultiArgs a = multi_args(h, Q);
    for (int ph = 0; ph < 4; ++ph) {
      st = launch_err(h, timed(h, kTagT1 + ph, s, [&] { return h->ks->table1(ph, a, s); }), "Table 1 phase");
      if (st) return st;
    }
  }
  ctl_post_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp, 1);
  return launch_err(h, cudaGetLastError(), "control kernel");
}

extern "C" aderdg_status aderdg_begin(aderdg_t h, void *dev_Q, double fixed_dt, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (!dev_Q) return fail(h, ADERDG_EINVAL, "dev_Q is NULL");
  if (((uintptr_t)dev_Q) % 16) return fail(h, ADERDG_EINVAL, "dev_Q must be 16-byte aligned");
  if (!(fixed_dt >= 0.0) || !std::isfinite(fixed_dt)) return fail(h, ADERDG_EINVAL, "fixed_dt must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->cp.fixed_dt = fixed_dt;
  h->cur = 0;
  ctl_reset_kernel<<<1, 1, 0, s>>>(h->ctl);
  aderdg_status st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  SweepArgs a = sweep_args(h, dev_Q);
  st = launch_err(h, h->ks->lambda(a, h->grid_lambda, s), "lambda reduction");
  if (st) return st;
  const int multipass = h->form != ADERDG_FORM_FUSED;
  ctl_begin_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp, multipass);
  st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  if ((st = source_coefficients(h, s))) return st;
  if (!multipass) {
    a.hull_out = h->hull[0];
    st = launch_err(h, timed(h, kTagStp, s, [&] { return fused_form_sweep(h, kPredict, a, main_grid(h), s); }),
                    "first STP sweep");
    if (st) return st;
  }
  h->begun = true;
  h->begun_Q = dev_Q;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_advance(aderdg_t h, void *dev_Q, int k, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (!h->begun || dev_Q != h->begun_Q) return fail(h, ADERDG_EINVAL, "aderdg_advance without a matching aderdg_begin");
  if (k < 0) return fail(h, ADERDG_EINVAL, "k must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  for (int i = 0; i < k; ++i) {
    aderdg_status st = h->form == ADERDG_FORM_FUSED ? fused_sweep(h, dev_Q, kFused, s)
                                                     : multipass_step(h, dev_Q, s);
    if (st) return st;
  }
  return ADERDG_OK;
}

static aderdg_status read_ctl(aderdg_t h, DevCtl *c, cudaStream_t s) {
  CK(h, cudaMemcpyAsync(c, h->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, s), "control read-back");
  CK(h, cudaStreamSynchronize(s), "stream synchronise");
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_end(aderdg_t h, void *dev_Q, double *t_inout, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (!h->begun || dev_Q != h->begun_Q) return fail(h, ADERDG_EINVAL, "aderdg_end without a matching aderdg_begin");
  cudaStream_t s = (cudaStream_t)stream;
  h->last_stream = s;
  h->begun = false;
  aderdg_status st = h->form == ADERDG_FORM_FUSED ? fused_sweep(h, dev_Q, kCorrect, s)
                                                   : multipass_step(h, dev_Q, s);
  if (st) return st;
  DevCtl c;
  st = read_ctl(h, &c, s);
  if (st) return st;
  if (t_inout) *t_inout += c.t;
  if (c.error == ADERDG_ENONFINITE) return fail(h, ADERDG_ENONFINITE, "non-finite wave speed in the state");
  if (c.error) return fail(h, (aderdg_status)c.error, "zero wave speed: no CFL step exists; pass fixed_dt");
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_step(aderdg_t h, void *dev_Q, int nsteps, double fixed_dt,
                                     double *t_inout, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, ADERDG_EINVAL, "nsteps must be >= 0");
  if (nsteps == 0) return ADERDG_OK;
  aderdg_status st = aderdg_begin(h, dev_Q, fixed_dt, stream);
  if (!st) st = aderdg_advance(h, dev_Q, nsteps - 1, stream);
  if (st) {
    h->begun = false;
    return st;
  }
  return aderdg_end(h, dev_Q, t_inout, stream);
}

// Host-resident state, fused form: the state moves in 32 chunks of tiles, in on
// one copy stream and out on another.  For linear PDEs the wave speed, hence
// Delta t, comes from the material alone, so the first STP sweep (which reads
// only its own cells) starts on each chunk as it lands; the last corrector
// (which reads its own cells' Q and D and the face hull, not the neighbours' Q)
// hands each chunk to the device-to-host copy as soon as it is done.  In a
// one-step call the corrector of a chunk runs as soon as the STP sweeps of the
// chunks holding its cells' neighbours are done, so the copies out overlap the
// copies in (linear PDEs) or the STP sweeps (nonlinear PDEs, whose wave speed
// needs the whole state first).  Other forms: copy, step, copy.

static aderdg_status host_copy_setup(aderdg_t h) {
  if (h->copy_stream) return ADERDG_OK;
  CK(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
  CK(h, cudaStreamCreateWithFlags(&h->copy_stream_out, cudaStreamNonBlocking), "copy stream");
  for (int i = 0; i < 2 * kHostChunks + 1; ++i)
    CK(h, cudaEventCreateWithFlags(&h->host_ev[i], cudaEventDisableTiming), "copy events");
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_step_host(aderdg_t h, void *host_Q, int nsteps, double fixed_dt,
                                          double *t_inout, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (!host_Q) return fail(h, ADERDG_EINVAL, "host_Q is NULL");
  if (nsteps < 0) return fail(h, ADERDG_EINVAL, "nsteps must be >= 0");
  if (!(fixed_dt >= 0.0) || !std::isfinite(fixed_dt)) return fail(h, ADERDG_EINVAL, "fixed_dt must be >= 0");
  if (nsteps == 0) return ADERDG_OK;
  // the compensated pair keeps a second plane (the low words) after the states
  const size_t cell_bytes = (size_t)h->m * h->ks->NS * h->ks->q_bytes;
  const size_t plane = (size_t)h->C * cell_bytes;
  const int planes = h->ks->pair ? 2 : 1;
  const size_t bytes = plane * planes;
  if (h->stage_bytes < bytes) {
    if (h->stage_Q) cudaFree(h->stage_Q);
    h->stage_Q = nullptr;
    h->stage_bytes = 0;
    CK(h, cudaMalloc(&h->stage_Q, bytes), "staging allocation");
    h->stage_bytes = bytes;
  }
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char *dQ = static_cast<unsigned char *>(h->stage_Q);
  unsigned char *hQ = static_cast<unsigned char *>(host_Q);
  // cells [c0, c1) of every plane
  auto copy_cells = [&](unsigned char *dst, const unsigned char *src, long long c0, long long c1,
                        cudaMemcpyKind kind, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < planes && e == cudaSuccess; ++p)
      e = cudaMemcpyAsync(dst + p * plane + c0 * cell_bytes, src + p * plane + c0 * cell_bytes,
                          (c1 - c0) * cell_bytes, kind, st);
    return e;
  };
  if (h->form != ADERDG_FORM_FUSED) {
    CK(h, cudaMemcpyAsync(dQ, hQ, bytes, cudaMemcpyHostToDevice, s), "host-to-device copy");
    aderdg_status st = aderdg_step(h, dQ, nsteps, fixed_dt, t_inout, stream);
    if (st && st != ADERDG_ENONFINITE) return st;
    CK(h, cudaMemcpyAsync(hQ, dQ, bytes, cudaMemcpyDeviceToHost, s), "device-to-host copy");
    CK(h, cudaStreamSynchronize(s), "stream synchronise");
    return st;
  }
  aderdg_status st = host_copy_setup(h);
  if (st) return st;
  cudaStream_t cs = h->copy_stream, co = h->copy_stream_out;
  cudaEvent_t *ev_in = h->host_ev, *ev_out = h->host_ev + kHostChunks, ev_start = h->host_ev[2 * kHostChunks];
  const int cpb = h->use_lin ? h->ks->LIN_CPB : h->ks->CPB;
  const long long ntiles = (h->C + cpb - 1) / cpb;
  const long long ct = (ntiles + kHostChunks - 1) / kHostChunks;  // tiles per chunk
  auto tiles_of = [&](int k, long long &t0, long long &t1) {
    t0 = std::min(ntiles, k * ct);
    t1 = std::min(ntiles, t0 + ct);
  };
  auto cells_of = [&](long long t0, long long t1, long long &c0, long long &c1) {
    c0 = std::min<long long>(h->C, t0 * cpb);
    c1 = std::min<long long>(h->C, t1 * cpb);
  };
  CK(h, cudaEventRecord(ev_start, s), "event");
  CK(h, cudaStreamWaitEvent(cs, ev_start, 0), "stream wait");
  CK(h, cudaStreamWaitEvent(co, ev_start, 0), "stream wait");

  // ---- begin: Delta t, then the first STP sweep chunk by chunk behind the copies
  h->last_stream = s;
  h->cp.fixed_dt = fixed_dt;
  h->cur = 0;
  ctl_reset_kernel<<<1, 1, 0, s>>>(h->ctl);
  st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  SweepArgs a = sweep_args(h, dQ);
  const bool overlap_in = h->ks->lambda_mat != nullptr;
  if (overlap_in) {
    const int g = h->mat ? h->grid_lambda : 1;
    st = launch_err(h, h->ks->lambda_mat(a, g, s), "lambda reduction");
    if (st) return st;
  } else {
    CK(h, cudaMemcpyAsync(dQ, hQ, bytes, cudaMemcpyHostToDevice, cs), "host-to-device copy");
    CK(h, cudaEventRecord(ev_in[0], cs), "event");
    CK(h, cudaStreamWaitEvent(s, ev_in[0], 0), "stream wait");
    st = launch_err(h, h->ks->lambda(a, h->grid_lambda, s), "lambda reduction");
    if (st) return st;
  }
  ctl_begin_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp, 0);
  st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  if ((st = source_coefficients(h, s))) return st;
  a.hull_out = h->hull[0];

  // One step: the control step before the correctors compares the dt_adm of
  // the initial state with the dt_new the first STP sweep used, so no STP
  // rerun can occur (unless the CFL factor exceeds 1), and it leaves dt_new as
  // it is: it may run between the STP chunks.  The corrector of chunk k needs
  // the hull of the cells up to S = G0 G1 (2D: G0) cells before and after its
  // own, across the periodic wrap: need[k] is the last STP chunk that covers
  // them.
  const bool interleave = nsteps == 1 && (fixed_dt > 0.0 || h->cp.cfl <= 1.0);
  const long long S = h->d == 3 ? (long long)h->grid[0] * h->grid[1] : (long long)h->grid[0];
  auto chunk_of = [&](long long cell) { return (int)((cell / cpb) / ct); };
  int need[kHostChunks];
  bool corrected[kHostChunks];
  for (int k = 0; k < kHostChunks; ++k) {
    long long t0, t1, c0, c1;
    tiles_of(k, t0, t1);
    cells_of(t0, t1, c0, c1);
    corrected[k] = t1 <= t0;
    int nd = k;
    if (t1 > t0) {
      nd = std::max(nd, chunk_of(std::min(h->C - 1, c1 - 1 + S)));
      if (c0 - S < 0) nd = std::max(nd, chunk_of(h->C - 1));
      if (c1 + S > h->C) nd = std::max(nd, chunk_of(std::min(h->C - 1, c1 + S - h->C - 1)));
    }
    need[k] = nd;
  }
  const SweepArgs c = sweep_args(h, dQ);
  bool pre_done = false;
  auto control_pre = [&]() -> aderdg_status {
    pre_done = true;
    ctl_pre_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp);
    aderdg_status e = launch_err(h, cudaGetLastError(), "control kernel");
    return e ? e : source_coefficients(h, s);
  };
  auto correct_chunk = [&](int k) -> aderdg_status {
    long long t0, t1, c0, c1;
    tiles_of(k, t0, t1);
    cells_of(t0, t1, c0, c1);
    corrected[k] = true;
    SweepArgs ck = c;
    ck.tile_lo = t0;
    ck.ntiles = t1;
    aderdg_status e = launch_err(
        h, timed(h, kTagCorrect, s, [&] { return fused_form_sweep(h, kCorrect, ck, (int)(t1 - t0), s); }),
        "corrector sweep");
    if (e) return e;
    CK(h, cudaEventRecord(ev_out[k], s), "event");
    CK(h, cudaStreamWaitEvent(co, ev_out[k], 0), "stream wait");
    CK(h, copy_cells(hQ, dQ, c0, c1, cudaMemcpyDeviceToHost, co), "device-to-host copy");
    return ADERDG_OK;
  };

  for (int k = 0; k < kHostChunks; ++k) {
    long long t0, t1, c0, c1;
    tiles_of(k, t0, t1);
    if (t1 <= t0) break;
    cells_of(t0, t1, c0, c1);
    if (overlap_in) {
      CK(h, copy_cells(dQ, hQ, c0, c1, cudaMemcpyHostToDevice, cs), "host-to-device copy");
      CK(h, cudaEventRecord(ev_in[k], cs), "event");
      CK(h, cudaStreamWaitEvent(s, ev_in[k], 0), "stream wait");
    }
    SweepArgs ak = a;
    ak.tile_lo = t0;
    ak.ntiles = t1;
    st = launch_err(h, timed(h, kTagStp, s, [&] { return fused_form_sweep(h, kPredict, ak, (int)(t1 - t0), s); }),
                    "first STP sweep");
    if (st) return st;
    if (interleave) {
      for (int kk = 0; kk < kHostChunks; ++kk) {
        if (corrected[kk] || need[kk] > k) continue;
        if (!pre_done && (st = control_pre())) return st;
        if ((st = correct_chunk(kk))) return st;
      }
    }
  }

  if (!interleave) {
    h->begun = true;
    h->begun_Q = dQ;
    // ---- the steps in between
    if (nsteps > 1) {
      st = aderdg_advance(h, dQ, nsteps - 1, stream);
      h->begun = false;
      if (st) return st;
    }
    h->begun = false;
    // ---- end: the last corrector chunk by chunk, each chunk copied back when done
    if ((st = control_pre())) return st;
    if (h->gate_needed && h->cp.fixed_dt <= 0.0) {
      SweepArgs g = sweep_args(h, dQ);
      g.gate = 1;
      g.pred_dt_old = 1;
      g.hull_out = h->hull[h->cur];
      st = launch_err(h, timed(h, kTagStp, s, [&] { return fused_form_sweep(h, kPredict, g, h->grid_gate, s); }),
                      "rerun STP sweep");
      if (st) return st;
    }
    const SweepArgs c2 = sweep_args(h, dQ);  // the hull of the last STP sweep
    for (int k = 0; k < kHostChunks; ++k) {
      long long t0, t1, c0, c1;
      tiles_of(k, t0, t1);
      if (t1 <= t0) break;
      cells_of(t0, t1, c0, c1);
      SweepArgs ck = c2;
      ck.tile_lo = t0;
      ck.ntiles = t1;
      st = launch_err(
          h, timed(h, kTagCorrect, s, [&] { return fused_form_sweep(h, kCorrect, ck, (int)(t1 - t0), s); }),
          "corrector sweep");
      if (st) return st;
      CK(h, cudaEventRecord(ev_out[k], s), "event");
      CK(h, cudaStreamWaitEvent(co, ev_out[k], 0), "stream wait");
      CK(h, copy_cells(hQ, dQ, c0, c1, cudaMemcpyDeviceToHost, co), "device-to-host copy");
    }
  }
  ctl_post_kernel<<<1, 1, 0, s>>>(h->ctl, h->cp, 0);
  st = launch_err(h, cudaGetLastError(), "control kernel");
  if (st) return st;
  DevCtl cb;
  st = read_ctl(h, &cb, s);
  if (st) return st;
  CK(h, cudaStreamSynchronize(cs), "copy stream synchronise");
  CK(h, cudaStreamSynchronize(co), "copy stream synchronise");
  if (t_inout) *t_inout += cb.t;
  if (cb.error == ADERDG_ENONFINITE) return fail(h, ADERDG_ENONFINITE, "non-finite wave speed in the state");
  if (cb.error) return fail(h, (aderdg_status)cb.error, "zero wave speed: no CFL step exists; pass fixed_dt");
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_set_material(aderdg_t h, const float *dev_mat, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (h->pde != ADERDG_ELASTICITY) return fail(h, ADERDG_EINVAL, "per-cell material needs ELASTICITY");
  cudaStream_t s = (cudaStream_t)stream;
  if (!dev_mat) {
    if (h->mat) {
      CK(h, cudaStreamSynchronize(s), "stream synchronise");
      cudaFree(h->mat);
    }
    h->mat = nullptr;
    // back to the uniform constants (entry 0)
    CK(h, h->ks->mat_pre(h->prm.pde_const, nullptr, 1, h->matp, s), "material constants");
    CK(h, cudaStreamSynchronize(s), "stream synchronise");
    return ADERDG_OK;
  }
  CK(h, cudaStreamSynchronize(s), "stream synchronise");  // no sweep in flight reads the old arrays
  if (!h->mat) CK(h, cudaMalloc((void **)&h->mat, sizeof(float) * 3 * h->C), "material allocation");
  if (h->matp_cap < h->C) {
    cudaFree(h->matp);
    h->matp = nullptr;
    h->matp_cap = 0;
    CK(h, cudaMalloc(&h->matp, (size_t)h->ks->mat_bytes * h->C), "material allocation");
    h->matp_cap = h->C;
  }
  CK(h, cudaMemcpyAsync(h->mat, dev_mat, sizeof(float) * 3 * h->C, cudaMemcpyDeviceToDevice, s), "material copy");
  CK(h, h->ks->mat_pre(h->prm.pde_const, h->mat, h->C, h->matp, s), "material constants");
  CK(h, cudaStreamSynchronize(s), "stream synchronise");
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_set_sources(aderdg_t h, int n, const aderdg_source *host_src, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (n < 0 || n > kMaxSources || (n > 0 && !host_src))
    return fail(h, ADERDG_EINVAL, "n must be in [0, 64] and host_src non-NULL");
  if (n > 0 && !h->use_lin)
    return fail(h, ADERDG_EUNSUPPORTED, "point sources need a linear PDE, the fused form and the time-modal predictor");
  if (n > 0 && !h->ks->lin_sweep_ext)
    return fail(h, ADERDG_EUNSUPPORTED, "point sources not compiled for this configuration");
  Basis1D B;
  if (!build_basis(h->N, B)) return fail(h, ADERDG_EINVAL, "basis construction failed");
  std::vector<SrcDev> dev(n);
  std::vector<SrcTime> tim(n);
  for (int k = 0; k < n; ++k) {
    const aderdg_source &S = host_src[k];
    bool ok = (S.kind == 0 || S.kind == 1) && std::isfinite(S.t0) && std::isfinite(S.f0);
    for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(S.pos[a]);
    for (int c = 0; c < 9; ++c) ok = ok && std::isfinite(S.amp[c]);
    for (int q = 0; q < 8; ++q) ok = ok && std::isfinite(S.coef[q]);
    if (!ok) return fail(h, ADERDG_EINVAL, "a source has kind outside 0/1 or a non-finite value");
    SrcDev &D = dev[k];
    std::memset(&D, 0, sizeof D);
    long long cell = 0, stride = 1;
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < kMaxn; ++i) D.e[a][i] = 1.0;
    for (int a = 0; a < h->d; ++a) {
      const double x = S.pos[a] / h->dx[a];
      long long ci = (long long)std::floor(x);
      ci = std::min<long long>(std::max<long long>(ci, 0), h->grid[a] - 1);
      double phi[kBasisMaxN + 1];
      lagrange_values(B, x - (double)ci, phi);   // outside the grid: extrapolated
      for (int i = 0; i <= h->N; ++i) D.e[a][i] = phi[i] / (B.w[i] * h->dx[a]);
      cell += ci * stride;
      stride *= h->grid[a];
    }
    D.cell = cell;
    for (int c = 0; c < 9; ++c) D.amp[c] = c < h->m ? S.amp[c] : 0.0;
    SrcTime &T = tim[k];
    std::memset(&T, 0, sizeof T);
    T.kind = S.kind;
    T.t0 = S.t0;
    T.f0 = S.f0;
    for (int q = 0; q < 8; ++q) T.coef[q] = S.coef[q];
  }
  cudaStream_t s = (cudaStream_t)stream;
  CK(h, cudaStreamSynchronize(s), "stream synchronise");
  if (n > 0 && !h->d_src) {
    CK(h, cudaMalloc((void **)&h->d_src, sizeof(SrcDev) * kMaxSources), "source allocation");
    CK(h, cudaMalloc((void **)&h->d_srct, sizeof(SrcTime) * kMaxSources), "source allocation");
    CK(h, cudaMalloc((void **)&h->d_srcco, sizeof(double) * kSrcCo * kMaxSources), "source allocation");
    CK(h, cudaMemset(h->d_srcco, 0, sizeof(double) * kSrcCo * kMaxSources), "source initialisation");
  }
  if (n > 0) {
    CK(h, cudaMemcpy(h->d_src, dev.data(), sizeof(SrcDev) * n, cudaMemcpyHostToDevice), "source copy");
    CK(h, cudaMemcpy(h->d_srct, tim.data(), sizeof(SrcTime) * n, cudaMemcpyHostToDevice), "source copy");
  }
  h->nsrc = n;
  h->scp.nsrc = n;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_get_dt_history(aderdg_t h, double *host_dt, int cap, int *n_out) {
  if (!h || !host_dt || !n_out || cap < 0) return fail(h, ADERDG_EINVAL, "bad argument");
  DevCtl c;
  aderdg_status st = read_ctl(h, &c, h->last_stream);
  if (st) return st;
  long long n = std::min<long long>(std::min<long long>(c.step, h->hist_cap), cap);
  if (n > 0) CK(h, cudaMemcpy(host_dt, h->hist, sizeof(double) * n, cudaMemcpyDeviceToHost), "history copy");
  *n_out = (int)n;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_get_stats(aderdg_t h, aderdg_stats *out) {
  if (!h || !out) return fail(h, ADERDG_EINVAL, "bad argument");
  DevCtl c;
  aderdg_status st = read_ctl(h, &c, h->last_stream);
  if (st) return st;
  out->t = c.t;
  out->dt_old = c.dt_old;
  out->dt_new = c.dt_new;
  out->lambda_max = c.lam_last;
  out->steps = c.step;
  out->reruns = c.reruns;
  out->launches = h->launches;
  out->device_error = c.error;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_nodes(int N, double *xi, double *w) {
  if (N < 0 || N > kBasisMaxN || !xi || !w) return fail(nullptr, ADERDG_EINVAL, "bad argument");
  return gauss_legendre01(N, xi, w) ? ADERDG_OK : fail(nullptr, ADERDG_EINVAL, "basis failed");
}

extern "C" aderdg_status aderdg_footprint(aderdg_t h, double *bytes_per_cell) {
  if (!h || !bytes_per_cell) return fail(h, ADERDG_EINVAL, "bad argument");
  *bytes_per_cell = (double)h->persistent_bytes;
  return ADERDG_OK;
}

// ---------------------------------------------------------------------------
// Adjoint of the receiver misfit (linear PDEs, fused form)

namespace {

struct DevBuf {
  void *p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
};

std::vector<int> receiver_comps(int pde, int d) {
  std::vector<int> c;
  if (pde == ADERDG_ADVECTION) c.push_back(0);
  else if (pde == ADERDG_ACOUSTICS)
    for (int a = 0; a < d; ++a) c.push_back(1 + a);
  else if (pde == ADERDG_ELASTICITY)
    for (int a = 0; a < d; ++a) c.push_back((d == 3 ? 6 : 3) + a);
  return c;
}

}  // namespace

extern "C" aderdg_status aderdg_step_adjoint(aderdg_t h, const void *dev_Q0, int nsteps, double fixed_dt,
                                             const float *dev_recv_pos, int R, const float *dev_obs,
                                             void *dev_gQ0, float *dev_gmat, int checkpoint_every,
                                             double *misfit_out, void *stream) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  if (!dev_Q0 || !dev_recv_pos || !dev_obs || !dev_gQ0 || nsteps < 1 || R < 1)
    return fail(h, ADERDG_EINVAL, "bad argument");
  if (!h->use_lin || !h->ks->adj_cell)
    return fail(h, ADERDG_EUNSUPPORTED, "adjoint not compiled for this configuration (linear PDEs, fused form)");
  if (h->ks->real_bytes != h->ks->q_bytes || h->ks->pair)
    return fail(h, ADERDG_EUNSUPPORTED, "adjoint needs FP32 or FP64");
  if (h->nsrc || h->ncp)
    return fail(h, ADERDG_EUNSUPPORTED, "the adjoint covers the per-cell flux without point sources");
  if (dev_gmat && (h->pde != ADERDG_ELASTICITY || !h->mat))
    return fail(h, ADERDG_EINVAL, "material gradient needs ELASTICITY with aderdg_set_material");
  if (!(fixed_dt >= 0.0)) return fail(h, ADERDG_EINVAL, "fixed_dt must be >= 0");
  const int ce = checkpoint_every > 0 ? checkpoint_every : 30;
  cudaStream_t s = (cudaStream_t)stream;
  const int d = h->d, m = h->m, NS = h->ks->NS, NF = h->ks->NF;
  const size_t qb = h->ks->q_bytes, rb = h->ks->real_bytes;
  const size_t state = (size_t)h->C * m * NS * qb;
  const std::vector<int> comps = receiver_comps(h->pde, d);
  const int nc = (int)comps.size();

  // receivers: cell and Lagrange weights of each position (host, FP64)
  std::vector<float> pos((size_t)R * d);
  CK(h, cudaMemcpy(pos.data(), dev_recv_pos, sizeof(float) * pos.size(), cudaMemcpyDeviceToHost), "receiver copy");
  Basis1D B;
  build_basis(h->N, B);
  const int n = h->N + 1;
  std::vector<long long> rcell(R);
  std::vector<double> rw((size_t)R * NS);
  for (int r = 0; r < R; ++r) {
    long long cell = 0, stride = 1;
    double phi[3][kBasisMaxN + 1];
    for (int a = 0; a < d; ++a) {
      const double x = pos[(size_t)r * d + a] / h->dx[a];
      long long ci = (long long)std::floor(x);
      ci = std::max(0ll, std::min<long long>(ci, h->grid[a] - 1));
      const double loc = x - ci;
      for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int b = 0; b < n; ++b)
          if (b != i) v *= (loc - B.xi[b]) / (B.xi[i] - B.xi[b]);
        phi[a][i] = v;
      }
      cell += ci * stride;
      stride *= h->grid[a];
    }
    rcell[r] = cell;
    for (int i = 0; i < NS; ++i) {
      double v = 1.0;
      int rem = i;
      for (int a = 0; a < d; ++a) {
        v *= phi[a][rem % n];
        rem /= n;
      }
      rw[(size_t)r * NS + i] = v;
    }
  }
  // the cell kernel's tables by value: the forward ones and the same built from
  // the transposed 1D operators Dm^T and Kvol^T (the transposed contractions)
  std::vector<unsigned char> htabT(h->htab.size());
  {
    Basis1D BT = B;
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) {
        BT.Dm[i * n + k] = B.Dm[k * n + i];
        BT.Kvol[i * n + k] = B.Kvol[k * n + i];
      }
    if (rb == 4) fill_tables(BT, *reinterpret_cast<Tables<float> *>(htabT.data()));
    else fill_tables(BT, *reinterpret_cast<Tables<double> *>(htabT.data()));
  }
  DevBuf d_rcell, d_rw, d_comps, d_traces, d_res, d_Qw, d_ck, d_seg, d_lam0, d_lam1, d_psi, d_gmat, d_zs;
  const int nseg = (nsteps + ce - 1) / ce;
  // The transposed step of a linear PDE does not depend on the state; the
  // forward states (checkpoints, segment recompute, their face hull) enter only
  // the material gradient.
  const bool need_fwd = dev_gmat != nullptr;
  if (d_rcell.alloc(sizeof(long long) * R) || d_rw.alloc(sizeof(double) * rw.size()) ||
      d_comps.alloc(sizeof(int) * nc) || d_traces.alloc(sizeof(double) * (size_t)nsteps * R * nc) ||
      d_res.alloc(sizeof(double) * (size_t)nsteps * R * nc) || d_Qw.alloc(state) ||
      (need_fwd && (d_ck.alloc(state * nseg) || d_seg.alloc(state * ce))) ||
      d_lam0.alloc((size_t)h->C * m * NS * rb) ||
      d_lam1.alloc((size_t)h->C * m * NS * rb) || d_psi.alloc((size_t)h->C * 2 * d * m * NF * rb) ||
      d_gmat.alloc(sizeof(double) * 3 * h->C))
    return fail(h, ADERDG_ENOMEM, "adjoint scratch allocation failed");
  // forward powers of the material gradient: one slot of picard - 1 levels per
  // block of the cell kernel (it loops over the tiles with at most that many blocks)
  long long zs_blocks = 0;
  if (need_fwd && h->picard > 1) {
    const long long tiles = (h->C + h->ks->adj_cpb - 1) / h->ks->adj_cpb;
    zs_blocks = std::min<long long>(tiles, (long long)h->nsm * 4);
    if (d_zs.alloc((size_t)zs_blocks * (h->picard - 1) * h->ks->adj_zlevel * rb))
      return fail(h, ADERDG_ENOMEM, "adjoint scratch allocation failed");
  }
  CK(h, cudaMemcpy(d_rcell.p, rcell.data(), sizeof(long long) * R, cudaMemcpyHostToDevice), "copy");
  CK(h, cudaMemcpy(d_rw.p, rw.data(), sizeof(double) * rw.size(), cudaMemcpyHostToDevice), "copy");
  CK(h, cudaMemcpy(d_comps.p, comps.data(), sizeof(int) * nc, cudaMemcpyHostToDevice), "copy");
  auto sample = [&](const void *Q, int k) {
    double *out = reinterpret_cast<double *>(d_traces.p) + (size_t)k * R * nc;
    if (qb == 4)
      rec_sample_kernel<float><<<R, 128, 0, s>>>(reinterpret_cast<const float *>(Q), (const long long *)d_rcell.p,
                                                 (const double *)d_rw.p, R, NS, m, (const int *)d_comps.p, nc, out);
    else
      rec_sample_kernel<double><<<R, 128, 0, s>>>(reinterpret_cast<const double *>(Q), (const long long *)d_rcell.p,
                                                  (const double *)d_rw.p, R, NS, m, (const int *)d_comps.p, nc, out);
    h->launches += 1;
    return cudaGetLastError();
  };
  aderdg_status st;
  // the step size, once, from the initial state (the CFL rule of the handle)
  double dt = fixed_dt;
  CK(h, cudaMemcpyAsync(d_Qw.p, dev_Q0, state, cudaMemcpyDeviceToDevice, s), "copy");
  if (!(dt > 0.0)) {
    st = aderdg_begin(h, d_Qw.p, 0.0, s);
    h->begun = false;
    if (st) return st;
    DevCtl c;
    st = read_ctl(h, &c, s);
    if (st) return st;
    if (c.error) return fail(h, (aderdg_status)c.error, "non-finite or zero wave speed in the initial state");
    dt = c.dt_new;
  }
  // forward pass: checkpoints every ce steps, receiver traces after every step
  if (need_fwd) CK(h, cudaMemcpyAsync(d_ck.p, dev_Q0, state, cudaMemcpyDeviceToDevice, s), "checkpoint");
  st = aderdg_begin(h, d_Qw.p, dt, s);
  if (st) return st;
  for (int k = 1; k <= nsteps; ++k) {
    st = k < nsteps ? aderdg_advance(h, d_Qw.p, 1, s) : aderdg_end(h, d_Qw.p, nullptr, s);
    if (st) return st;
    CK(h, sample(d_Qw.p, k - 1), "receiver sampling");
    if (need_fwd && k % ce == 0 && k < nsteps)
      CK(h, cudaMemcpyAsync((char *)d_ck.p + state * (k / ce), d_Qw.p, state, cudaMemcpyDeviceToDevice, s),
         "checkpoint");
  }
  // misfit J = 1/2 sum_k sum_r |u_r^k - d_r^k|^2 dt, residuals for the backward pass
  const size_t ntr = (size_t)nsteps * R * nc;
  std::vector<double> tr(ntr), res(ntr);
  std::vector<float> obs(ntr);
  CK(h, cudaMemcpyAsync(tr.data(), d_traces.p, sizeof(double) * ntr, cudaMemcpyDeviceToHost, s), "copy");
  CK(h, cudaMemcpyAsync(obs.data(), dev_obs, sizeof(float) * ntr, cudaMemcpyDeviceToHost, s), "copy");
  CK(h, cudaStreamSynchronize(s), "stream synchronise");
  double J = 0.0;
  for (size_t i = 0; i < ntr; ++i) {
    const double e = tr[i] - (double)obs[i];
    J += 0.5 * dt * e * e;
    res[i] = dt * e;
  }
  CK(h, cudaMemcpyAsync(d_res.p, res.data(), sizeof(double) * ntr, cudaMemcpyHostToDevice, s), "copy");
  CK(h, cudaMemsetAsync(d_lam0.p, 0, (size_t)h->C * m * NS * rb, s), "memset");
  CK(h, cudaMemsetAsync(d_gmat.p, 0, sizeof(double) * 3 * h->C, s), "memset");

  // backward pass, segment by segment from the last checkpoint
  void *lam_a = d_lam0.p, *lam_b = d_lam1.p;
  AdjArgs aa{};
  aa.mat = h->mat;
  aa.gmat = dev_gmat ? reinterpret_cast<double *>(d_gmat.p) : nullptr;
  aa.tables = h->tables;
  aa.ncells = h->C;
  for (int i = 0; i < 3; ++i) {
    aa.grid[i] = h->grid[i];
    aa.inv_dx[i] = 1.0 / h->dx[i];
  }
  for (int i = 0; i < 8; ++i) aa.cst[i] = h->prm.pde_const[i];
  aa.picard = h->picard;
  aa.hsl = h->ks->HSL;
  aa.fsz = h->ks->HSL / (2 * d);
  aa.dt = dt;
  aa.psi = d_psi.p;
  aa.hull = h->hull[0];
  aa.htab = h->htab.data();
  aa.htabT = htabT.data();
  aa.zs = d_zs.p;
  aa.zs_blocks = zs_blocks;
  aa.matp = h->matp;
  for (int i = 0; i < 3; ++i) aa.scf[i] = (float)(dt * aa.inv_dx[i]);
  // one transposed step: the receiver term of step k, then (material
  // gradient) the forward face hull of Q^{k-1} and the adjoint kernels
  auto adjoint_step = [&](int k, const void *Qprev) -> aderdg_status {
    const double *rk = reinterpret_cast<const double *>(d_res.p) + (size_t)(k - 1) * R * nc;
    const long long nt = (long long)R * NS;
    if (rb == 4)
      rec_adjoint_kernel<float><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(
          (float *)lam_a, (const long long *)d_rcell.p, (const double *)d_rw.p, R, NS, m, (const int *)d_comps.p, nc, rk);
    else
      rec_adjoint_kernel<double><<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(
          (double *)lam_a, (const long long *)d_rcell.p, (const double *)d_rw.p, R, NS, m, (const int *)d_comps.p, nc, rk);
    aderdg_status e = launch_err(h, cudaGetLastError(), "receiver adjoint");
    if (e) return e;
    if (Qprev) {
      SweepArgs sa = sweep_args(h, const_cast<void *>(Qprev));
      sa.Q_out = nullptr;
      sa.hull_out = h->hull[0];
      e = launch_err(h, fused_form_sweep(h, kPredict, sa, main_grid(h), s), "adjoint STP sweep");
      if (e) return e;
    }
    aa.lam_in = lam_a;
    aa.lam_out = lam_b;
    aa.Qk = Qprev;
    e = launch_err(h, h->ks->adj_faces(aa, s), "adjoint face kernel");
    if (e) return e;
    e = launch_err(h, h->ks->adj_cell(aa, s), "adjoint cell kernel");
    if (e) return e;
    std::swap(lam_a, lam_b);
    return ADERDG_OK;
  };
  if (!need_fwd) {
    for (int k = nsteps; k > 0; --k)
      if ((st = adjoint_step(k, nullptr))) return st;
  }
  for (int seg = need_fwd ? nseg - 1 : -1; seg >= 0; --seg) {
    const int k0 = seg * ce, k1 = std::min(nsteps, k0 + ce);
    char *segs = reinterpret_cast<char *>(d_seg.p);
    CK(h, cudaMemcpyAsync(segs, (char *)d_ck.p + state * seg, state, cudaMemcpyDeviceToDevice, s), "copy");
    if (k1 - k0 > 1) {
      CK(h, cudaMemcpyAsync(d_Qw.p, segs, state, cudaMemcpyDeviceToDevice, s), "copy");
      st = aderdg_begin(h, d_Qw.p, dt, s);
      if (st) return st;
      for (int k = k0 + 1; k < k1; ++k) {
        st = aderdg_advance(h, d_Qw.p, 1, s);
        if (st) return st;
        CK(h, cudaMemcpyAsync(segs + state * (k - k0), d_Qw.p, state, cudaMemcpyDeviceToDevice, s), "copy");
      }
      h->begun = false;
    }
    for (int k = k1; k > k0; --k)
      if ((st = adjoint_step(k, segs + state * (k - 1 - k0)))) return st;
  }
  CK(h, cudaMemcpyAsync(dev_gQ0, lam_a, state, cudaMemcpyDeviceToDevice, s), "gradient copy");
  if (dev_gmat) {
    const long long n3 = 3 * h->C;
    d2f_kernel<<<(unsigned)((n3 + 255) / 256), 256, 0, s>>>((const double *)d_gmat.p, dev_gmat, n3);
    st = launch_err(h, cudaGetLastError(), "conversion");
    if (st) return st;
  }
  CK(h, cudaStreamSynchronize(s), "stream synchronise");
  if (misfit_out) *misfit_out = J;
  h->last_stream = s;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_profile(aderdg_t h, int enable) {
  if (!h) return fail(nullptr, ADERDG_EINVAL, "handle is NULL");
  h->prof_on = enable != 0;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_profile_read(aderdg_t h, int kernel, double *ms_total, long long *count) {
  if (!h || !ms_total || !count) return fail(h, ADERDG_EINVAL, "bad argument");
  double ms = 0.0;
  long long n = 0;
  std::vector<aderdg_ctx::Prof> keep;
  for (auto &p : h->prof) {
    if (p.tag != kernel) {
      keep.push_back(p);
      continue;
    }
    CK(h, cudaEventSynchronize(p.b), "event synchronise");
    float e = 0.f;
    CK(h, cudaEventElapsedTime(&e, p.a, p.b), "event elapsed time");
    ms += e;
    ++n;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  h->prof.swap(keep);
  *ms_total = ms;
  *count = n;
  return ADERDG_OK;
}

extern "C" aderdg_status aderdg_destroy(aderdg_t h) {
  if (!h) return ADERDG_OK;
  cudaDeviceSynchronize();
  for (auto &p : h->prof) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  free_all(h);
  delete h;
  return ADERDG_OK;
}

extern "C" const char *aderdg_last_error(aderdg_t h) {
  if (h) return h->err.c_str();
  return g_create_error.c_str();
}
