// control.cuh -- the time-step control of Algorithms 1 and 2 on the device
// (one thread per controlled problem).
//   ctl_pre  (fused form, before each corrector sweep; Technique 5):
//            rerun = dt_adm < dt_new
//            dt_old = rerun ? C dt_adm : dt_new
//            dt_new = C dt_adm (strict) or (dt_old + C dt_adm)/2 (creeping)
//   ctl_post (after each corrector sweep): lambda_max -> dt_adm, simulated
//            time, dt history; the multi-pass forms set the next step's dt
//            here (Algorithm 1).
#pragma once
#include <cfloat>

#include "aderdg.h"
#include "common.cuh"

namespace aderdg {

__device__ __forceinline__ double ctl_lambda(const DevCtl *c) {
  return __longlong_as_double((long long)c->lam_bits);
}

__device__ __forceinline__ void ctl_pre(DevCtl *c, const CtlParams &p) {
  if (p.fixed_dt > 0.0) {
    c->rerun = 0;
    c->dt_old = c->dt_new = p.fixed_dt;
  } else {
    if (c->dt_adm < c->dt_new) {
      c->rerun = 1;
      c->reruns += 1;
      c->dt_old = p.cfl * c->dt_adm;
    } else {
      c->rerun = 0;
      c->dt_old = c->dt_new;
    }
    c->dt_new = p.policy == 1 ? 0.5 * (c->dt_old + p.cfl * c->dt_adm) : p.cfl * c->dt_adm;
  }
  c->lam_bits = 0ull;
}

__device__ __forceinline__ void ctl_post(DevCtl *c, const CtlParams &p, int multipass) {
  const double lam = ctl_lambda(c);
  c->lam_last = lam;
  c->lam_bits = 0ull;
  if (!(lam <= DBL_MAX) && !c->error) c->error = ADERDG_ENONFINITE;
  c->step += 1;
  c->t += c->dt_old;
  if (c->step <= c->hist_cap) c->hist[c->step - 1] = c->dt_old;
  if (p.fixed_dt > 0.0) return;
  if (lam > 0.0 && lam <= DBL_MAX) {
    c->dt_adm = p.dt_scale / lam;
    if (c->step == p.inject_step) c->dt_adm *= p.inject_factor;
  } else if (lam == 0.0 && !c->error) {
    c->error = ADERDG_EINVAL;
  }
  if (multipass) c->dt_old = p.cfl * c->dt_adm;  // Algorithm 1: dt of the next step
}

__device__ __forceinline__ void ctl_begin(DevCtl *c, const CtlParams &p, int multipass) {
  const double lam = ctl_lambda(c);
  c->lam_last = lam;
  c->lam_bits = 0ull;
  if (!(lam <= DBL_MAX)) c->error = ADERDG_ENONFINITE;
  if (p.fixed_dt > 0.0) {
    c->dt_adm = INFINITY;
    c->dt_old = c->dt_new = p.fixed_dt;
  } else if (lam > 0.0 && lam <= DBL_MAX) {
    c->dt_adm = p.dt_scale / lam;
    c->dt_new = p.cfl * c->dt_adm;
    c->dt_old = multipass ? c->dt_new : 0.0;  // first fused sweep: dt_old = 0 (Technique 3)
  } else {
    if (!c->error) c->error = ADERDG_EINVAL;  // zero wave speed: no CFL step exists
    c->dt_old = c->dt_new = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Point sources: the coefficients of one sweep (layout: kSrcCo in common.cuh).
// With M = K1^-1 diag(w) the Picard iteration of Eq. 3 with a source term is
// q <- 1 u - dt (M (x) L) q + dt (M svec) (x) sigma, whose time average after R
// iterations is sum_s (-dt L)^s [g_s u + dt h_s sigma], h_s = w . M^(s+1) svec
// (h_R = 0): the Horner form of the predictor gains dt h_s sigma at level s.
struct SrcCoefParams {
  int n, R, nsrc, pad_;
  double xi[kMaxn], w[kMaxn], M[kMaxn * kMaxn];
};

__device__ __forceinline__ double src_time(const SrcTime &S, double t) {
  const double tau = t - S.t0;
  if (S.kind == 1) {
    double a = 3.14159265358979323846 * S.f0 * tau;
    a *= a;
    return (1.0 - 2.0 * a) * exp(-a);
  }
  double v = 0.0;
  for (int q = 7; q >= 0; --q) v = v * tau + S.coef[q];
  return v;
}

__device__ __forceinline__ void src_horner(const SrcTime &S, const SrcCoefParams &p, double t0, double dt,
                                           double *dst) {
  double y[kMaxn], z[kMaxn];
  for (int l = 0; l < p.n; ++l) y[l] = src_time(S, t0 + p.xi[l] * dt);
  for (int s = 0; s < p.R; ++s) {
    double h = 0.0;
    for (int k = 0; k < p.n; ++k) {
      double acc = 0.0;
      for (int l = 0; l < p.n; ++l) acc += p.M[k * p.n + l] * y[l];
      z[k] = acc;
      h += p.w[k] * acc;
    }
    for (int k = 0; k < p.n; ++k) y[k] = z[k];
    dst[s] = dt * h;
  }
}

__device__ __forceinline__ void src_coef(const DevCtl *c, const SrcTime &S, const SrcCoefParams &p, double *co) {
  const double t = c->t, dto = c->dt_old, dtn = c->dt_new;
  double I = 0.0;
  for (int l = 0; l < p.n; ++l) I += p.w[l] * src_time(S, t + p.xi[l] * dto);
  co[0] = dto * I;
  src_horner(S, p, t + dto, dtn, co + 1);
  src_horner(S, p, t, dtn, co + 1 + kMaxPicard);
  src_horner(S, p, t, dto, co + 1 + 2 * kMaxPicard);
}

__device__ __forceinline__ void ctl_reset(DevCtl *c) {
  c->lam_bits = 0ull;
  c->t = 0.0;
  c->step = 0;
  c->reruns = 0;
  c->rerun = 0;
  c->error = 0;
  c->dt_old = c->dt_new = 0.0;
  c->dt_adm = INFINITY;
}

}  // namespace aderdg
