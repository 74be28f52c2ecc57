/*
 * aderdg.h -- C ABI of libaderdg, a GB300 (sm_103a) implementation of the
 * single-touch ADER-DG time step on a regular periodic Cartesian mesh
 * (Charrier & Weinzierl, arXiv:1801.08682).
 *
 * Scope.  The PDE is Eq. 1 with B = S = delta = 0 (Sec. 3):
 *   dQ/dt + div F(Q) = 0,  Q(x,t) in R^m,  x in [0, G_0 dx_0) x ... (periodic).
 * Each cell holds m (N+1)^d nodal values on Gauss-Legendre points (Sec. 3).
 * A time step applies Eq. 6: predict (Eq. 3), extrapolate, solveRiemann
 * (Eq. 4, Rusanov), integrateVolume + integrateFace + update (Eq. 2) and
 * calcTimeStep (Table 1), executed by default in the shifted, fused,
 * optimistic order of Algorithm 2 (Techniques 1-5, Sec. 5).
 *
 * Conventions for every entry point
 *   - Status codes, never exceptions or aborts.  A failing call leaves a
 *     message in aderdg_last_error().
 *   - "dev_" pointers are CUDA device pointers on the current device;
 *     "host_" pointers are host memory (pinned or pageable).  The caller
 *     owns every pointer it passes; the library never frees them.
 *   - The library owns its scratch (D, the face hull, time-step control
 *     block, multi-pass buffers); aderdg_destroy frees it.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Kernels are enqueued on it in order.
 *   - Layout of a state Q: Q[cell][comp][node], C-contiguous.
 *       cell = c0 + G0 (c1 + G1 c2)          (axis 0 fastest)
 *       node = i0 + n (i1 + n i2), n = N + 1 (axis 0 fastest)
 *     Element type: float (precision FP32) or double (FP64, FP32_ACC64);
 *     FP32_PAIR holds two float planes of this layout, the state and its
 *     low-order words (2 C m (N+1)^d floats).
 *     The node positions inside a cell are x = (c + xi_i) dx with xi from
 *     aderdg_nodes().
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef ADERDG_H
#define ADERDG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aderdg_ctx *aderdg_t;

typedef enum {
  ADERDG_OK = 0,
  ADERDG_EINVAL = 1,       /* bad argument; nothing was launched */
  ADERDG_ENOMEM = 2,       /* device or host allocation failed */
  ADERDG_ECUDA = 3,        /* a CUDA runtime call failed */
  ADERDG_ENONFINITE = 4,   /* a NaN/Inf wave speed was seen by the device */
  ADERDG_ETIMEOUT = 5,     /* a bounded device wait gave up */
  ADERDG_EUNSUPPORTED = 6  /* (pde, d, N, precision, form) not compiled in */
} aderdg_status;

/* PDE families (Eq. 1, conservative flux only).
 *   ADVECTION   m = 1        F_j = a_j u                      pde_const = a_0, a_1, a_2
 *   ACOUSTICS   m = d + 1    Q = (p, v), F_j = (K v_j, p/rho e_j), K = rho c^2
 *                                                              pde_const = rho, c
 *   EULER       m = d + 2    Q = (rho, j, E), Sec. 7 (p = (gamma-1)(E - |j|^2/(2 rho)))
 *                                                              pde_const = gamma
 *   ELASTICITY  m = 9 (3D: sxx syy szz sxy syz sxz vx vy vz) or 5 (2D: sxx syy sxy vx vy)
 *               velocity-stress, F_j = -A_j Q with lambda = rho(cp^2 - 2 cs^2),
 *               mu = rho cs^2; per-cell material via aderdg_set_material,
 *               otherwise pde_const = rho, cp, cs. */
typedef enum {
  ADERDG_ADVECTION = 0,
  ADERDG_ACOUSTICS = 1,
  ADERDG_EULER = 2,
  ADERDG_ELASTICITY = 3
} aderdg_pde;

typedef enum {
  ADERDG_FP32 = 0,        /* everything in float; Q is float */
  ADERDG_FP64 = 1,        /* everything in double; Q is double */
  ADERDG_FP32_ACC64 = 2,  /* float predictor/Riemann, Q is double and
                             accumulated Q += update in double */
  ADERDG_FP32_PAIR = 3    /* float predictor/Riemann; the state is a
                             compensated FP32 pair: Q is two float planes
                             [2][cell][comp][node], the FP32 state (hi) and
                             the low-order word of every DoF (lo), and the
                             corrector adds the update by TwoSum into (hi, lo),
                             renormalised so that hi = fl(hi + lo).  The
                             predictor and the wave speeds read hi.  Initialise
                             lo to zero, or to the rounding error of an FP64
                             state: lo = fl(Q64 - hi).  Fused and three-sweep
                             forms; no adjoint */
} aderdg_precision;

typedef enum {
  ADERDG_FORM_FUSED = 0,     /* Algorithm 2: one single-touch sweep per step */
  ADERDG_FORM_HULL3 = 1,     /* Algorithm 1 with the space-time hull only:
                                STP, Riemann and corrector as three sweeps */
  ADERDG_FORM_TABLE1 = 2     /* Algorithm 1 with the task outputs of Table 1
                                stored explicitly (space-time predictor and
                                space-time face data) */
} aderdg_form;

typedef enum {
  ADERDG_DT_STRICT = 0,    /* dt_new = C dt_adm (Alg. 2, first choice) */
  ADERDG_DT_CREEPING = 1   /* dt_new = (dt_old + C dt_adm)/2 (Alg. 2, second choice) */
} aderdg_dt_policy;

typedef enum {
  ADERDG_PREDICT_AUTO = 0,      /* linear PDEs: time-modal Picard; Euler: space-time */
  ADERDG_PREDICT_SPACETIME = 1, /* always the space-time Picard iteration */
  /* the space-time Picard iteration (Eq. 3) with the flux-divergence
   * contractions sum_j (1/dx_j) Dm_j F_j on the tensor cores: TF32 operands,
   * FP32 accumulation (mma.sync m16n8k8); FP32 configurations only.  Results
   * agree with the FP32 forms to about 1e-4 relative per step (TF32 keeps
   * 10 mantissa bits); everything else as ADERDG_PREDICT_SPACETIME. */
  ADERDG_PREDICT_SPACETIME_TF32 = 2
} aderdg_predictor;

/* How a per-cell material meets its neighbour at a face.
 *   PER_CELL_FLUX   each cell keeps the conservative flux F_j = -A_j(cell) Q
 *                   and each side of a face applies its own A_j in the
 *                   Rusanov flux; this converges to continuity of A_j Q
 *                   across a jump (default; the adjoint differentiates it)
 *   NONCONSERVATIVE the non-conservative products B_j(x) dQ/dx_j of Eq. 1
 *                   (Sec. 1: the B_i anticipate material changes): strong
 *                   volume term and path-conservative Rusanov fluctuations
 *                   along the straight path in (lambda, mu, 1/rho); velocity
 *                   and traction stay continuous across a jump, as the
 *                   physics requires.  With a uniform material both are the
 *                   same scheme. */
typedef enum {
  ADERDG_JUMPS_PER_CELL_FLUX = 0,
  ADERDG_JUMPS_NONCONSERVATIVE = 1
} aderdg_material_jumps;

/* Zero-initialised = defaults. */
typedef struct {
  double pde_const[8];  /* see aderdg_pde */
  double cfl;           /* C_dT of Alg. 1/2 in (0, 1]; 0 -> max(0.3, 0.9 - 0.1 N).
                           The admissible step is
                           dt_adm = min_j dx_j / (d (2N+1) lambda_max); the
                           default keeps 0.1 below the factor measured stable
                           for N = 2..6 in 2D/3D acoustics (0.8 .. 0.4) */
  int picard_iters;     /* Picard iterations of Eq. 3; 0 -> N + 1 */
  int precision;        /* aderdg_precision */
  int form;             /* aderdg_form */
  int dt_policy;        /* aderdg_dt_policy */
  int predictor;        /* aderdg_predictor */
  int inject_step;      /* >= 1: multiply dt_adm computed in that step (counted
                           from 1 since aderdg_begin) by inject_factor; a
                           host-side fault injection for the rerun path */
  double inject_factor;
  int material_jumps;   /* an aderdg_material_jumps value: ELASTICITY with a
                           per-cell material, fused form, time-modal predictor */
} aderdg_params;

typedef struct {
  double t;             /* simulated time */
  double dt_old;        /* step size of the last corrector */
  double dt_new;        /* step size of the pending predictor */
  double lambda_max;    /* last reduced spectral radius */
  long long steps;      /* corrector sweeps since aderdg_begin */
  long long reruns;     /* STP reruns (Technique 5) since aderdg_begin */
  long long launches;   /* kernels launched by this handle since creation */
  int device_error;     /* device error word (aderdg_status), 0 = none */
} aderdg_stats;

/* Create a solver for a d-dimensional (d = 2, 3) periodic grid of
 * grid[0] x grid[1] (x grid[2]) cells of size dx[0..d-1], polynomial order
 * N (0 <= N <= 6; N = 0 is the finite-volume case of Appendix A), m
 * variables (must equal the PDE's m for d).  params may be NULL.
 * Allocates D and the face hull on the current device.  The handle stays
 * bound to that device.  Errors: EINVAL (bad sizes, m mismatch, cfl out of
 * range), EUNSUPPORTED (combination not compiled), ENOMEM, ECUDA. */
aderdg_status aderdg_create(int d, int N, int m, aderdg_pde pde, const int grid[3],
                            const double dx[3], const aderdg_params *params, aderdg_t *out);

/* Per-cell material [C][3] = (rho, cp, cs) as float, device pointer, for
 * ELASTICITY; copied into library memory (the caller may free it after the
 * call returns).  NULL returns to the uniform pde_const material.
 * Defines the flux F_j = -A_j(cell) Q of Eq. 1 cell by cell; each side of a
 * face applies its own A_j in the Rusanov flux of Eq. 4, with the wave speed
 * s = max(cp_L, cp_R) (the paper leaves heterogeneous material to the
 * non-conservative B_i terms of Eq. 1, Sec. 1; this is their conservative
 * per-cell reading).  Errors: EINVAL (wrong PDE, non-positive values are not
 * checked). */
aderdg_status aderdg_set_material(aderdg_t h, const float *dev_mat, void *stream);

/* Point source a s(t) delta(x - pos): the delta terms of Eq. 1 (Sec. 1:
 * earthquake point sources).  The delta is projected onto the cell holding
 * pos (a position outside the grid is clamped to the boundary cell) as the
 * nodal values sigma_{c,i} = amp[c] prod_j phi_{i_j}(xi_j) / (w_{i_j} dx_j)
 * (lumped mass, Sec. 3 basis); it enters the predictor (Eq. 3) at every time
 * node and the update (Eq. 2) as dt sum_k w_k s(t + xi_k dt) sigma. */
typedef struct {
  double pos[3];        /* physical position (the first d entries) */
  double amp[9];        /* amplitude of every variable (the first m entries) */
  int kind;             /* 0: s(t) = sum_p coef[p] (t - t0)^p (p <= 7);
                           1: Ricker wavelet (1 - 2a) exp(-a), a = (pi f0 (t - t0))^2 */
  int pad_;
  double t0, f0;
  double coef[8];
} aderdg_source;

/* Replace the handle's point sources by n sources (0 <= n <= 64; n = 0
 * removes them); host_src is host memory owned by the caller (copied before
 * the call returns).  Linear PDEs, fused form, time-modal predictor.  Times
 * are simulated times since aderdg_begin.  Errors: EINVAL (NULL handle or
 * pointer, n out of range, kind not 0/1, a non-finite value), EUNSUPPORTED
 * (nonlinear PDE, multi-pass form or space-time predictor), ENOMEM, ECUDA. */
aderdg_status aderdg_set_sources(aderdg_t h, int n, const aderdg_source *host_src, void *stream);

/* Advance dev_Q (in place) by nsteps time steps (Eq. 6 per step) and
 * synchronise the stream.  dev_Q must be 16-byte aligned (the corrector
 * stages its rows with bulk copies), else EINVAL.  fixed_dt > 0 fixes every
 * step size; otherwise
 * the CFL control of Alg. 2 (or Alg. 1 for the multi-pass forms) is used.
 * *t_inout (may be NULL) is advanced by the simulated time.  Equivalent to
 * aderdg_begin + aderdg_advance(nsteps - 1) + aderdg_end.  nsteps = 0 is
 * a no-op.  Errors: EINVAL, ENONFINITE (NaN/Inf reached the wave-speed
 * reduction; Q then holds the non-finite state), ECUDA. */
aderdg_status aderdg_step(aderdg_t h, void *dev_Q, int nsteps, double fixed_dt,
                          double *t_inout, void *stream);

/* Same as aderdg_step on a host state: copies host_Q to a library-owned
 * device buffer, steps, copies the result back into host_Q.  This is the
 * entry point for callers that keep their state in host memory.  Fused form:
 * the copies run in 32 chunks, in and out on two streams of the library's
 * own; the first STP sweep of linear PDEs starts on each chunk as it arrives
 * (Delta t then comes from the material alone; a non-finite state is reported
 * after the step, by the corrector's check) and each chunk of the last
 * corrector is copied back as soon as it is done.  With nsteps = 1 the
 * corrector of a chunk runs as soon as the chunks holding its cells'
 * neighbours have had their STP sweep, so the copies back overlap the copies
 * in (linear PDEs) or the STP sweeps (nonlinear PDEs).  Results equal
 * aderdg_step's.  host_Q should be pinned (page-locked) memory for the copies
 * to overlap. */
aderdg_status aderdg_step_host(aderdg_t h, void *host_Q, int nsteps, double fixed_dt,
                               double *t_inout, void *stream);

/* The three phases of aderdg_step, asynchronous on `stream` (no host
 * synchronisation, no error read-back except launch errors):
 *   begin    computes dt_adm of dev_Q, and runs the first STP sweep
 *            (Technique 3: the first corrector has dt_old = 0);
 *   advance  runs k fused sweeps (corrector of step s, STP of step s+1);
 *   end      runs the last corrector and synchronises the stream, reads the
 *            device error word and the simulated time.
 * The same dev_Q must be passed to all three, unmodified in between.
 * For the multi-pass forms begin/advance/end run whole Alg. 1 steps. */
aderdg_status aderdg_begin(aderdg_t h, void *dev_Q, double fixed_dt, void *stream);
aderdg_status aderdg_advance(aderdg_t h, void *dev_Q, int k, void *stream);
aderdg_status aderdg_end(aderdg_t h, void *dev_Q, double *t_inout, void *stream);

/* Gradient of a receiver misfit by the discrete adjoint of the step (not in
 * the paper; built on Eqs. 2-4 transposed term by term).  Linear PDEs, fused
 * form, FP32 or FP64.
 *   Forward: Q^0 = dev_Q0 (not modified), nsteps steps with one fixed step
 *   size: fixed_dt if > 0, else C_dT dt_adm(Q^0).  After every step k the
 *   receivers record the velocity (acoustics, elasticity) or the scalar
 *   (advection) u_r^k at positions dev_recv_pos [R][d] (float, device).
 *   Misfit J = 1/2 sum_{k=1..nsteps} sum_r |u_r^k - d_r^k|^2 dt with
 *   observations dev_obs [nsteps][R][nc] (float, device; nc = d, or 1 for
 *   advection).
 *   Output: dev_gQ0 = dJ/dQ^0 (same type and layout as Q), dev_gmat =
 *   dJ/d(rho, cp, cs) [C][3] float for ELASTICITY with a per-cell material
 *   (NULL = not wanted), *misfit_out = J.
 * With dev_gmat, the forward states are kept every checkpoint_every steps
 * (0 -> 30) and recomputed segment by segment for the backward pass; scratch
 * (one state per checkpoint plus one state per step of a segment) is
 * allocated for the call and freed before it returns.  Without it no forward
 * state is kept: the transposed step of a linear PDE does not depend on the
 * state, and the receiver values of the forward run suffice.  Synchronises the
 * stream.
 * Errors: EINVAL, EUNSUPPORTED (nonlinear PDE, multi-pass form or not
 * compiled), ENOMEM, ECUDA. */
aderdg_status aderdg_step_adjoint(aderdg_t h, const void *dev_Q0, int nsteps, double fixed_dt,
                                  const float *dev_recv_pos, int R, const float *dev_obs,
                                  void *dev_gQ0, float *dev_gmat, int checkpoint_every,
                                  double *misfit_out, void *stream);

/* Step sizes used by the correctors since aderdg_begin (oldest first), at
 * most cap values; *n_out receives the number written.  These are the
 * dt_old of Algorithm 2's timeStep calls, chosen by the optimistic control of
 * Technique 5 (Sec. 5): dt_new = C dt_adm, an STP rerun when dt_adm < dt_new.
 * host_dt is host memory owned by the caller.  Synchronises.  Errors: EINVAL
 * (NULL handle or pointers, cap < 0), ECUDA. */
aderdg_status aderdg_get_dt_history(aderdg_t h, double *host_dt, int cap, int *n_out);

/* Counters of the handle: the time-step state of Algorithm 2 (t, dt_old,
 * dt_new, the last lambda_max of calcTimeStep, Table 1), the corrector sweeps
 * and the STP reruns of Technique 5 (Sec. 5), the kernels launched and the
 * device error word.  Synchronises the handle's last stream.  Errors: EINVAL
 * (NULL handle or out), ECUDA. */
aderdg_status aderdg_get_stats(aderdg_t h, aderdg_stats *out);

/* Gauss-Legendre nodes xi[0..N] in [0,1] and weights w[0..N] (sum 1) used
 * by the library (Sec. 3).  Host-only, no handle needed. */
aderdg_status aderdg_nodes(int N, double *xi, double *w);

/* Persistent device bytes per cell held by the handle (Q excluded): fused
 * form D and both face-hull buffers; three-sweep form D, one hull and F*;
 * Table 1 form F*, the space-time predictor and fluxes and their face data.
 * Compare with the footprints of Corollary "hull" (Sec. 6) and the task
 * volumes of Table 1.  Errors: EINVAL (NULL handle or out). */
aderdg_status aderdg_footprint(aderdg_t h, double *bytes_per_cell);

/* ---- Ensembles: many independent scenarios in one persistent launch ----
 * (not in the paper; every scenario runs Algorithm 2 with the fused sweep of
 * Sec. 5, and the persistent work list replaces the grid traversal that
 * issues the tasks of Sec. 5 cell by cell).  Scenarios: d = 2, N = 2..6, ACOUSTICS (m = 3) or
 * ELASTICITY (m = 5, uniform material pde_const), FP32, fused form; each
 * keeps its own CFL control and time step.  The states are packed in one
 * float buffer, scenario s at element offset aderdg_batch_offsets()[s], each
 * in the layout of a single state; offsets are multiples of 32 elements
 * (128 B, for the vector line loads), the gaps between scenarios are not
 * touched, and offsets[count] is the buffer length in elements (dev_Q must
 * be 16-byte aligned, else EINVAL).  aderdg_batch_step advances every
 * scenario by nsteps steps (one fused sweep of all scenarios per step):
 *   mode 0  persistent launches, the steady-state sweeps replayed from a
 *           CUDA graph captured on the first call (default)
 *   mode 1  persistent launches without the graph
 *   mode 2  one launch per scenario and sweep (the reference form)
 * and synchronises.  aderdg_batch_autotune times a few steps on a copy of
 * dev_Q (dev_Q is not modified) for every persistent-grid size (1..3 blocks
 * per SM, each with its own build of the persistent kernel: up to 255, 128
 * and 85 registers per thread) and work granularity (1, 2, 4, 8 tiles per
 * item) and keeps the fastest.  The batch owns a stream; calls order after `stream` and return
 * after the work is done.  Errors: EINVAL (also: a scenario with rho, c or cp
 * <= 0, cs < 0, or a CFL number outside (0, 1]; every scenario is checked
 * before any device call), EUNSUPPORTED, ENOMEM, ECUDA, ENONFINITE (any
 * scenario). */
typedef struct aderdg_batch_ctx *aderdg_batch_t;
typedef struct {
  int d, N, m;
  aderdg_pde pde;
  int grid[3];
  double dx[3];
  double pde_const[8];
  double cfl;           /* 0 -> max(0.3, 0.9 - 0.1 N) */
} aderdg_scenario;

aderdg_status aderdg_batch_create(int count, const aderdg_scenario *scen, aderdg_batch_t *out);
aderdg_status aderdg_batch_offsets(aderdg_batch_t b, long long *elem_offsets /* [count + 1] */);
aderdg_status aderdg_batch_step(aderdg_batch_t b, float *dev_Q, int nsteps, int mode, void *stream);
aderdg_status aderdg_batch_autotune(aderdg_batch_t b, float *dev_Q, int steps, void *stream);
aderdg_status aderdg_batch_get_tuning(aderdg_batch_t b, int *blocks_per_sm, int *tiles_per_item,
                                      long long *launches);
/* Events around every persistent fused sweep launched outside the graph
 * (mode 1) while enabled; profile_read synchronises, returns the summed
 * milliseconds and the number of timed sweeps since enabling or the last
 * read, and clears them. */
aderdg_status aderdg_batch_profile(aderdg_batch_t b, int enable);
aderdg_status aderdg_batch_profile_read(aderdg_batch_t b, double *ms_total, long long *count);
aderdg_status aderdg_batch_destroy(aderdg_batch_t b);

/* Kernel timing with CUDA events recorded on the launching stream around
 * every launch of the handle's main kernels while enabled (enable = 1); the
 * sweeps are the task groups of Algorithm 2 (fused), Algorithm 1 (three
 * sweeps) and Table 1 (one phase per task).  Not in the paper, whose
 * measurements are hardware counters (Sec. 7).  Errors: EINVAL (NULL handle
 * or pointers), ECUDA; a kernel number outside 0..7 reads as no launches.
 * kernel: 0 fused sweep, 1 STP sweep (first sweep, rerun, three-sweep
 * form), 2 corrector sweep, 3 Riemann sweep (three-sweep form),
 * 4..7 the Table 1 phases predict, extrapolate, solveRiemann, corrector.
 * profile_read synchronises, returns the summed milliseconds and the launch
 * count of that kernel since the last read, and clears them. */
aderdg_status aderdg_profile(aderdg_t h, int enable);
aderdg_status aderdg_profile_read(aderdg_t h, int kernel, double *ms_total, long long *count);

/* Free everything aderdg_create allocated (D, the face hull, the multi-pass
 * buffers of Table 1, the control block, the material copy) after waiting
 * for the device (cudaDeviceSynchronize); the caller's buffers are untouched.
 * NULL is a no-op returning ADERDG_OK. */
aderdg_status aderdg_destroy(aderdg_t h);

/* aderdg_step without a handle and without allocating: for callers that may
 * not call cudaMalloc or cudaFree while they run (a plugin whose host
 * application owns the device memory budget or forbids allocations after
 * start-up; a time-critical loop that must not add the device-wide
 * synchronisation of cudaFree).  The paper has no counterpart of this entry
 * point.
 *
 * Same arguments and results as aderdg_create + aderdg_step in the fused form
 * (params->form must be ADERDG_FORM_FUSED; the same PDE constants are
 * required), plus dev_mat (per-cell material [C][3] float on the device for
 * ELASTICITY, or NULL).  The step's scratch (D, two face-hull buffers, control
 * block, tables, a 1024-entry dt history) lives in one file-scope device array
 * of 16 MiB that every GPU loading the library holds until the process exits;
 * a problem whose scratch does not fit returns ADERDG_EINVAL with nothing
 * launched (roughly 1,500 cells of 3D acoustics at N = 5 in FP32, 4,000 at
 * N = 3).  Every argument is checked before any CUDA call.
 *   - The first call on a device fetches the array's device address with
 *     cudaGetSymbolAddress; make that first call before any stream capture.
 *   - The call is synchronous: it enqueues the step on `stream` and waits for
 *     that stream before returning, so it blocks the calling host thread.
 *   - All calls on a device share the array and leave their contents in it;
 *     calls that overlap on the GPU (other streams, other host threads) race.
 *   - Errors are returned as status codes only; aderdg_last_error is not set. */
aderdg_status aderdg_step_noalloc(int d, int N, int m, aderdg_pde pde, const int grid[3],
                                  const double dx[3], const aderdg_params *params,
                                  const float *dev_mat, void *dev_Q, int nsteps, double fixed_dt,
                                  double *t_inout, void *stream);

/* Measured FP32 fused multiply-add rate of the current device in TFLOP/s
 * (2 FLOP per FMA): the best of `repeats` timed launches (CUDA events on
 * `stream`) of a kernel of independent FMA chains on every SM.  The
 * denominator of a compute-roofline fraction; not part of the method.
 * Allocates and frees a small buffer; synchronises the stream.  Errors:
 * EINVAL (NULL tflops, repeats outside 1..1000), ENOMEM, ECUDA. */
aderdg_status aderdg_fp32_fma_peak(int repeats, double *tflops, void *stream);

/* Last error message of the handle, or of the calling thread's last failed
 * aderdg_create when h is NULL.  Never NULL. */
const char *aderdg_last_error(aderdg_t h);

#ifdef __cplusplus
}
#endif
#endif /* ADERDG_H */
