/*
 * rslb.h -- C ABI of the GB300 (sm_103a) R-SLB library.
 *
 * The library implements the time step of the quadrature-based relativistic
 * lattice Boltzmann method R-SLB(N_Omega; Q_xi) of Ambrus & Blaga, "High-order
 * quadrature-based lattice Boltzmann models for the flow of ultrarelativistic
 * rarefied gases":
 *   - momenta on a Gauss-Laguerre (|p|) x Gauss-Legendre (xi = cos theta) set
 *     (Sec. III B-E, Eqs. pjk, fjk);
 *   - Sod shock tube: WENO5 advection (Sec. III F, Eqs. flux_weno,
 *     weno5_omega), Landau matching (Sec. II E, Eqs. E_landau-pi_val),
 *     truncated Maxwell-Juttner f^eq (Sec. III D, Eq. feq_trunc),
 *     Anderson-Witting relaxation (Eq. L_Sod) and TVD-RK3 (Eq. rk3);
 *   - Bjorken flow: the same collision and RK3 with the momentum-space
 *     derivative matrices K^L and K^P (Eqs. K_lag_disc, K_leg_disc,
 *     L_Bjorken), batched over many independent runs.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: RSLB_OK (0) or an RSLB_ERR_* code.
 *     rslb_last_error() returns a static, thread-local description of the most
 *     recent failure in the calling thread.  Nothing aborts, exits or traps.
 *   - Velocity index v = k*Q_xi + j (k: radial node, j: polar node, ascending
 *     xi).  Populations are the weighted f_jk of Eq. fjk (T0 = 1).
 *   - Pointers passed in are owned by the caller and must stay valid until the
 *     call returns (host pointers) or until the next synchronising call on the
 *     handle (device pointers).  The library owns every allocation it makes
 *     and frees it in the matching *_destroy call.
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  rslb_step and rslb_bjorken_step only enqueue work on it;
 *     device-side errors (non-physical states) are reported by the next
 *     rslb_sync, rslb_moments, rslb_get_state or rslb_bjorken_read call.
 */
#ifndef RSLB_H
#define RSLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define RSLB_OK 0
#define RSLB_ERR_ARG 1          /* invalid argument or configuration */
#define RSLB_ERR_CFL 2          /* CFL = max|xi| dt / dz >= 1 (Eq. CFL) */
#define RSLB_ERR_STIFF 3        /* dt >= tau (explicit RK3 limit, Sec. III F) */
#define RSLB_ERR_ALLOC 4        /* device allocation failed */
#define RSLB_ERR_CUDA 5         /* a CUDA runtime call failed */
#define RSLB_ERR_NONPHYSICAL 6  /* a cell left the physical domain (n, E <= 0,
                                   |beta| >= 1, non-finite) */
#define RSLB_ERR_UNSUPPORTED 7  /* size beyond what the kernels support */
#define RSLB_ERR_TIMEOUT 8      /* a bounded wait inside a kernel ran out (the
                                   kernel left its work and freed what it held) */

/* ---- enumerations ---- */
#define RSLB_F32 0 /* populations, fluxes, relaxation in FP32; Landau in FP64 */
#define RSLB_F64 1 /* everything in FP64 */

/* Cells per CTA tile of the packed FP32x2 shock-tube stage kernel. */
#define RSLB_PACKED_TILE_CELLS 28

#define RSLB_BC_FIXED_EQ 0 /* ghost cells = left/right equilibria (Sec. IV A) */
#define RSLB_BC_OUTFLOW 1  /* ghost cells = first/last interior cell */
#define RSLB_BC_PERIODIC 2 /* periodic domain */

#define RSLB_TAU_CONST 0 /* constant relaxation time tau */
#define RSLB_TAU_ETAS 1  /* tau = tau_AW0/T [1 - ln(lambda_bar lambda_ref)/4]
                            (Eq. Sod:tau) */
#define RSLB_TAU_NONE 2  /* collisionless (free streaming, Sec. IV C) */

/* Fields of rslb_moments, in this order (each an array of Z doubles). */
#define RSLB_FIELD_N 0
#define RSLB_FIELD_E 1
#define RSLB_FIELD_P 2
#define RSLB_FIELD_T 3
#define RSLB_FIELD_BETA 4
#define RSLB_FIELD_GAMMA 5
#define RSLB_FIELD_LAMBDA 6 /* relative fugacity n/T^3 */
#define RSLB_FIELD_Q 7      /* heat flux, Eq. q_val */
#define RSLB_FIELD_PI 8     /* shear stress, Eq. pi_val */
#define RSLB_FIELD_NT 9
#define RSLB_FIELD_NZ 10
#define RSLB_FIELD_TTT 11
#define RSLB_FIELD_TTZ 12
#define RSLB_FIELD_TZZ 13
#define RSLB_NFIELDS 14

/*
 * Gauss-Legendre nodes/weights in xi (Sec. III C, Eq. quad_xi and the weight
 * formula after it) and Gauss-Laguerre nodes/weights for e^{-x} x^2 (Sec.
 * III B, Eqs. quadL, wL), in FP64 on the host.  No device work.
 *   xi, w_xi: caller-owned host arrays of length Q_xi (nodes ascending);
 *   xk, w_L:  caller-owned host arrays of length Q_L (nodes ascending).
 * Either pair may be NULL to skip it.  1 <= Q_xi <= 4096, 1 <= Q_L <= 12.
 * Errors: RSLB_ERR_ARG.
 */
int rslb_quadrature(int Q_xi, int Q_L, double* xi, double* w_xi, double* xk,
                    double* w_L);

/* Sod shock-tube configuration (Secs. II E, III, IV A). */
typedef struct rslb_config {
  int Z;               /* number of cells, >= 1 */
  double z_min, z_max; /* domain; dz = (z_max - z_min)/Z */
  int Q_xi;            /* polar nodes, 1..2048 */
  int Q_L;             /* radial nodes, 1..8 (paper: 2) */
  int N_Omega;         /* f^eq truncation order in P_m, 0 <= N_Omega < Q_xi, <= 12 */
  int precision;       /* RSLB_F32 or RSLB_F64 */
  int bc;              /* RSLB_BC_* */
  int tau_mode;        /* RSLB_TAU_* */
  double tau;          /* RSLB_TAU_CONST: relaxation time > 0 */
  double tau_AW0;      /* RSLB_TAU_ETAS: tau_AW0 > 0 */
  double lambda_ref;   /* RSLB_TAU_ETAS: lambda_ref > 0 */
  double dt;           /* time step > 0 */
  /* Left/right states (n, T, beta): the Riemann initial state (left for
   * cell centres z < 0) and the RSLB_BC_FIXED_EQ ghost equilibria. */
  double nL, TL, betaL, nR, TR, betaR;
  /* Optional per-cell initial fields (host arrays of Z doubles, read once by
   * rslb_init).  If all three are non-NULL they replace the Riemann state. */
  const double* n0;
  const double* T0;
  const double* beta0;
  /* Cells per CTA tile of the stage kernel: 0 = automatic; otherwise
   * RSLB_PACKED_TILE_CELLS (the packed FP32x2 kernel: V >= 128,
   * N_Omega <= 7), 128, 64, 32 or 16 (RSLB_F32), 16 or
   * 8 (RSLB_F64).  A tuning knob; results agree to rounding. */
  int tile_cells;
  /* Form of the packed FP32x2 kernel: RSLB_PACKED_AUTO or
   * RSLB_PACKED_PER_TILE (one CTA per tile, two CTAs per SM), or
   * RSLB_PACKED_PERSISTENT (one CTA per SM walking the tiles with two tile
   * buffers and warp-specialised cell and sweep groups; RSLB_ERR_ARG where it
   * does not fit: it needs V <= ~700, Z >= RSLB_PACKED_TILE_CELLS + 8).  Both
   * forms give bitwise identical results. */
  int packed_form;
} rslb_config;

#define RSLB_PACKED_AUTO 0
#define RSLB_PACKED_PER_TILE 1
#define RSLB_PACKED_PERSISTENT 2

typedef struct rslb_handle rslb_handle;

/*
 * Validate cfg, build the velocity tables, allocate the device state (three
 * population buffers of V x Z values of the chosen precision) and set the
 * populations to the truncated f^eq of the initial state (Sec. IV A), on
 * `stream`.  On success *h owns everything and must be released with
 * rslb_destroy.
 * Errors: RSLB_ERR_ARG (bad cfg), RSLB_ERR_CFL (max|xi| dt/dz >= 1),
 * RSLB_ERR_STIFF (RSLB_TAU_CONST and dt >= tau), RSLB_ERR_UNSUPPORTED
 * (V = Q_xi*Q_L too large for one tile of 16 (FP32) or 8 (FP64) cells, or
 * V * ldz >= 2^31 populations in one buffer, ldz = Z rounded up to a multiple
 * of 32; checked before any device work), RSLB_ERR_ALLOC, RSLB_ERR_CUDA,
 * RSLB_ERR_NONPHYSICAL (an initial state with n <= 0, T <= 0 or |beta| >= 1).
 */
int rslb_init(rslb_handle** h, const rslb_config* cfg, void* stream);

/*
 * Enqueue nsteps TVD-RK3 steps (Eq. rk3) of L_Sod (Eq. L_Sod) on the handle's
 * stream: three fused stage kernels per step, each doing moments, Landau
 * matching, f^eq, WENO5 flux difference, relaxation and the RK combination
 * for every (cell, velocity).  Asynchronous; nsteps >= 0.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA (launch failure).
 */
int rslb_step(rslb_handle* h, int nsteps);

/*
 * Wait for the handle's stream and report any device-side error raised since
 * the last check (RSLB_ERR_NONPHYSICAL, with the first offending cell in
 * rslb_last_error()).
 */
int rslb_sync(rslb_handle* h);

/*
 * Per-cell macroscopic fields of the current state, in FP64, layout
 * out[field*Z + s] with the RSLB_FIELD_* order (RSLB_NFIELDS fields): the
 * moments N^mu, T^{mu nu} of the populations (Eq. macro_jk) and the Landau
 * frame quantities n, E, P, T, beta, gamma, lambda_bar, q, Pi (Sec. II E,
 * Eqs. E_landau-pi_val).  For FP32 populations the sums are formed as exact
 * products summed in double-float arithmetic.
 * out: caller-owned, host memory if out_on_device == 0, else device memory
 * on the handle's device.  Synchronises the stream.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA, RSLB_ERR_NONPHYSICAL.
 */
int rslb_moments(rslb_handle* h, double* out, int out_on_device);

/*
 * Copy the populations out of / into the handle: f[v*Z + s], V*Z values of
 * the handle's precision (float for RSLB_F32, double for RSLB_F64).  Host
 * memory if on_device == 0 (pinned memory gives asynchronous copies), else
 * device memory.  rslb_get_state synchronises; rslb_set_state is
 * stream-ordered.  Used for checkpoint/resume and by the end-to-end path.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA.
 */
int rslb_get_state(rslb_handle* h, void* f, int on_device);
int rslb_set_state(rslb_handle* h, const void* f, int on_device);

/* Simulation time and step count of the handle (host-side bookkeeping). */
int rslb_time(const rslb_handle* h, double* t, long long* steps);

/* The stage kernel the handle launches: cells per CTA tile
 * (RSLB_PACKED_TILE_CELLS = packed FP32x2 kernel) and threads per CTA (the
 * persistent pipelined form of the packed kernel has more threads than
 * 8 * RSLB_PACKED_TILE_CELLS).  Errors: RSLB_ERR_ARG. */
int rslb_launch_info(const rslb_handle* h, int* tile_cells, int* threads);

/*
 * Allocation-free shock-tube step.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc or any allocating routine: code that runs
 * while another component owns all device memory (a framework's caching
 * allocator, a fixed memory budget), plugins loaded into a host that forbids
 * allocation in its compute callbacks, or real-time loops where an allocation's
 * implicit device synchronisation is not acceptable.  This entry point does
 * the same work as rslb_init + rslb_step without allocating anything: the RK
 * stage buffers, velocity tables and error word live in one static device
 * array of RSLB_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the
 * library holds until the process exits.
 *
 *   cfg:    the configuration, as for rslb_init (n0/T0/beta0, tile_cells and
 *           packed_form are ignored; the populations come from f);
 *   f:      caller-owned device array of V*Z values in the cfg precision
 *           (f[v*Z + s], v = k*Q_xi + j), advanced in place by nsteps steps,
 *           the same TVD-RK3 steps as rslb_step performs;
 *   stream: cudaStream_t as void* (NULL = legacy default stream).
 *
 * Limits: Q_xi*Q_L <= RSLB_NOALLOC_MAX_VELOCITIES, Q_L <= 8, and three stage
 * buffers of V x ceil32(Z) values plus O(V) tables must fit the static array;
 * larger problems are rejected with RSLB_ERR_UNSUPPORTED before any device
 * work.  The call synchronises the stream before returning and reports device
 * errors (RSLB_ERR_NONPHYSICAL) directly.
 * The first call on a device looks up the array's device address and opts
 * the stage kernels into large shared memory on that device (once per
 * device); make that first call before any stream capture.  Every call shares
 * the one array, which keeps the previous call's contents (each call clears
 * what it needs), so calls that overlap on the GPU -- from several threads or
 * streams -- race on it and must be serialised by the caller.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_CFL, RSLB_ERR_STIFF, RSLB_ERR_UNSUPPORTED,
 * RSLB_ERR_CUDA, RSLB_ERR_NONPHYSICAL.
 */
#define RSLB_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define RSLB_NOALLOC_MAX_VELOCITIES 1024
int rslb_sod_step_noalloc(const rslb_config* cfg, void* f, int nsteps, void* stream);

/* Release everything owned by h (synchronises its stream).  NULL is a no-op. */
void rslb_destroy(rslb_handle* h);

/* ------------------------------------------------------------------------ */
/* Batches of independent shock tubes (uneven Z, Q_xi, tau, states).         */
/* ------------------------------------------------------------------------ */

typedef struct rslb_sod_run {
  int Z;                  /* cells */
  int Q_xi;               /* polar nodes */
  double tau;             /* RSLB_TAU_CONST: constant relaxation time > 0 */
  double nL, TL, nR, TR;  /* chambers at rest (Sec. IV A) */
  double t_end;           /* final time > 0 */
  int tau_mode;           /* RSLB_TAU_CONST, RSLB_TAU_ETAS or RSLB_TAU_NONE */
  double tau_AW0;         /* RSLB_TAU_ETAS: tau_AW0 > 0 (Eq. Sod:tau) */
  double lambda_ref;      /* RSLB_TAU_ETAS: lambda_ref > 0 */
  int N_Omega;            /* f^eq truncation of this run; -1: the batch's rule */
  double dt;              /* > 0: this time step (t_end is rounded to whole steps;
                             required unless tau_mode is RSLB_TAU_CONST);
                             0: automatic (see rslb_sod_batch_init) */
} rslb_sod_run;

typedef struct rslb_sod_batch_opts {
  int Q_L;             /* radial nodes (shared) */
  int N_Omega;         /* -1: min(Q_xi - 1, 5) for each run */
  int precision;       /* RSLB_F32 or RSLB_F64 */
  int bc;              /* RSLB_BC_FIXED_EQ or RSLB_BC_OUTFLOW */
  double z_min, z_max; /* domain of every run */
  double cfl;          /* dt <= cfl dz / max|xi| (Eq. CFL) */
  double dt_over_tau;  /* dt <= dt_over_tau * tau (explicit RK3 limit) */
  int autotune;        /* 1: time the candidate tile kernels per velocity class */
} rslb_sod_batch_opts;

typedef struct rslb_sod_batch rslb_sod_batch;

/*
 * Set up nruns shock tubes.  A run with dt = 0 (constant tau only) gets
 * dt = t_end / ceil(t_end / dt_max) with dt_max = min(cfl dz / max|xi|,
 * dt_over_tau * tau), i.e. it reaches t_end exactly after its own number of
 * steps; a run with dt > 0 takes round(t_end / dt) steps of dt.  Runs are grouped by velocity
 * count; each group is advanced by one persistent launch per RK stage that
 * walks the tiles of its runs (runs with fewer steps drop out as they
 * finish).  With autotune, the tile kernel and CTAs per SM of each group are
 * chosen by timing the candidates on the actual state.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_UNSUPPORTED, RSLB_ERR_ALLOC, RSLB_ERR_CUDA.
 */
int rslb_sod_batch_init(rslb_sod_batch** b, const rslb_sod_run* runs, int nruns,
                        const rslb_sod_batch_opts* opts, void* stream);

/*
 * Enqueue nsteps batch steps (each active run advances one RK3 step, Eq. rk3;
 * runs stop at their own step count).  Steps are replayed from a captured
 * CUDA graph on non-default streams.  Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA.
 */
int rslb_sod_batch_step(rslb_sod_batch* b, int nsteps);

/* Batch bookkeeping: the largest per-run step count, steps enqueued so far,
 * and the cell-velocity updates all runs perform in total to their t_end. */
int rslb_sod_batch_info(const rslb_sod_batch* b, long long* max_steps, long long* steps_done,
                        double* total_cv_updates);

/* Per-run step count and time step. */
int rslb_sod_batch_run_info(const rslb_sod_batch* b, int run, long long* nsteps, double* dt);

/* The tuner's choice for velocity group g (groups in ascending V): tile
 * width (cells per CTA) and CTAs per SM; returns RSLB_ERR_ARG past the last. */
int rslb_sod_batch_tuning(const rslb_sod_batch* b, int g, int* V, int* tile_cells,
                          int* ctas_per_sm);

/* Moments of one run (as rslb_moments; out: host, RSLB_NFIELDS * Z). */
int rslb_sod_batch_moments(rslb_sod_batch* b, int run, double* out);

void rslb_sod_batch_destroy(rslb_sod_batch* b);

/* ------------------------------------------------------------------------ */
/* Boost-invariant (Bjorken) flow, batched over independent runs (Sec. V).  */
/* ------------------------------------------------------------------------ */

#define RSLB_GAS_PARTON 0 /* n_eq = P^{3/4}, T = P^{1/4} (Eqs. bjorken_mu0,
                             bjorken_tauAW0) */
#define RSLB_GAS_IDEAL 1  /* n_eq = n, T = P/n (Eq. bjorken_tauAW_mu) */

#define RSLB_KP_SIMT 0   /* K^P contraction on the CUDA cores in the working
                            precision (FP64 or FP32) */
#define RSLB_KP_TF32X3 2 /* K^P contraction on the tcgen05 tensor cores
                            (kind::tf32, accumulators in tensor memory):
                            both operands split x = hi + lo with
                            hi = tf32(x), products hi*hi + hi*lo + lo*hi,
                            FP32 accumulation.  RSLB_F32 only, Q_L <= 4. */

/* Number of per-run outputs of rslb_bjorken_read, in this order:
 * tau, n = N^tau, E = T^{tau tau}, P = E/3, T, Pi = P_L - P,
 * P_L = T^{eta eta}, P_T = (E - P_L)/2   (Eqs. bjorken_SET, bjorken_P) */
#define RSLB_BJ_NOUT 8

typedef struct rslb_bjorken_run {
  int Q_xi;       /* polar nodes of this run, 2 .. 512 */
  int gas;        /* RSLB_GAS_* */
  double tau_AW0; /* relaxation scale of Eq. bjorken_tauAW (units of tau0);
                     <= 0 or infinite: collisionless */
} rslb_bjorken_run;

typedef struct rslb_bjorken_opts {
  int Q_L;        /* radial nodes, 1..8 (shared by all runs) */
  int precision;  /* RSLB_F32 or RSLB_F64 */
  int kp_mode;    /* RSLB_KP_* */
  double tau0;    /* initial proper time, > 0 (the paper's nondimensional 1) */
  double dtau;    /* time step, > 0 */
} rslb_bjorken_opts;

typedef struct rslb_bjorken rslb_bjorken;

/*
 * Set up nruns independent Bjorken runs (Secs. II F, III, V A): each starts
 * from the isotropic equilibrium f = e^{-p}/(8 pi) at tau = tau0
 * (Eq. bjorken_f0), i.e. populations f_jk = w_j w_k / 4 (Eq. fjk).  Builds
 * the K^P matrix (Eq. K_leg_disc) of every distinct Q_xi and K^L
 * (Eq. K_lag_disc) on the device in FP64.  runs: caller-owned host array of
 * nruns entries, read during the call.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_STIFF (dtau >= the initial tau_AW of a run),
 * RSLB_ERR_UNSUPPORTED, RSLB_ERR_ALLOC, RSLB_ERR_CUDA.
 */
int rslb_bjorken_init(rslb_bjorken** b, const rslb_bjorken_run* runs, int nruns,
                      const rslb_bjorken_opts* opts, void* stream);

/*
 * Enqueue nsteps TVD-RK3 steps (Eq. rk3) of L_Bjorken (Eq. L_Bjorken) for
 * every run, with stage times tau_n, tau_n + dtau, tau_n + dtau/2.  Per
 * stage: moments, equilibrium (gas law), f^eq at u = 0 (Eq. Bjorken_MB via
 * Eqs. feq_trunc, fjk), the K^L term, the K^P contraction, relaxation and
 * the RK combination.  Asynchronous.  Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA.
 */
int rslb_bjorken_step(rslb_bjorken* b, int nsteps);

/*
 * Per-run observables of the current state: out[r*RSLB_BJ_NOUT + i] in the
 * callers' run order (see RSLB_BJ_NOUT).  out: caller-owned host memory, or
 * device memory if out_on_device.  Synchronises.  Errors: RSLB_ERR_ARG,
 * RSLB_ERR_CUDA, RSLB_ERR_NONPHYSICAL (a run with P <= 0 or non-finite).
 */
int rslb_bjorken_read(rslb_bjorken* b, double* out, int out_on_device);

/*
 * Populations of all runs, concatenated in the callers' run order, each run
 * f[k*Q_xi + j] (Q_L*Q_xi values), in the handle's precision; host memory.
 * rslb_bjorken_get_state synchronises.  Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA.
 */
int rslb_bjorken_get_state(rslb_bjorken* b, void* f);
int rslb_bjorken_set_state(rslb_bjorken* b, const void* f);

/*
 * The xi-derivative contraction alone: y_r = K^P f_r (Eq. K_leg_disc applied
 * to the radial columns of every run, y[k*Q_xi + j] = sum_j' K^P_{j j'}
 * f[k*Q_xi + j']) on the current state, computed by the handle's tensor-core
 * path, written like rslb_bjorken_get_state (FP32, callers' run order, host
 * memory).  Synchronises.  Errors: RSLB_ERR_ARG, RSLB_ERR_UNSUPPORTED
 * (kp_mode other than RSLB_KP_TF32X3), RSLB_ERR_CUDA.
 */
int rslb_bjorken_kp_apply(rslb_bjorken* b, void* y);

/*
 * Self-test of the tensor-core kernel's failure handling (not part of the
 * method): one contraction-only launch in which the worker warps never signal
 * that their operand tiles are ready, so the issuing thread's bounded wait
 * (~0.3 s) runs out.  Each CTA then records the time-out, waits (bounded) for
 * the copies it issued, frees its tensor memory and returns; the state is
 * untouched and the handle stays usable.  Expected result: RSLB_ERR_TIMEOUT.
 * Synchronises.  Errors: RSLB_ERR_ARG, RSLB_ERR_UNSUPPORTED (kp_mode other than
 * RSLB_KP_TF32X3), RSLB_ERR_CUDA, RSLB_ERR_TIMEOUT.
 */
int rslb_bjorken_selftest_timeout(rslb_bjorken* b);

/* Release everything owned by b (synchronises).  NULL is a no-op. */
void rslb_bjorken_destroy(rslb_bjorken* b);

/* ------------------------------------------------------------------------ */
/* Learned closure of a low-order velocity set (an addition to the paper's  */
/* method).  A per-cell MLP, trained on data generated by the method with a */
/* high-order velocity set, corrects the low-order populations after every  */
/* RK3 step; the correction leaves each cell's N^t, T^tt, T^tz unchanged.   */
/* ------------------------------------------------------------------------ */

typedef struct rslb_mlp rslb_mlp;

/*
 * Network n_in -> n_hidden -> n_hidden -> n_out, SiLU after both hidden
 * layers, BF16 weights (an FP32 master copy is kept for training), FP32
 * biases and accumulation.  Parameters (flat FP32 vector, this order):
 * W1 [n_hidden][n_in], b1 [n_hidden], W2 [n_hidden][n_hidden], b2 [n_hidden],
 * W3 [n_out][n_hidden], b3 [n_out]; initialised from `seed` (weights normal
 * with variance 1/fan_in, the output layer scaled by 0.1, biases zero).
 * Limits: n_in <= 128, n_hidden in {16, 32, 64}, n_out <= 32.
 * Errors: RSLB_ERR_ARG, RSLB_ERR_UNSUPPORTED, RSLB_ERR_ALLOC, RSLB_ERR_CUDA.
 */
int rslb_mlp_create(rslb_mlp** m, int n_in, int n_hidden, int n_out, unsigned long long seed,
                    void* stream);
int rslb_mlp_num_params(const rslb_mlp* m);
/* Master parameters to / from caller-owned host memory (set resets Adam). */
int rslb_mlp_get_params(rslb_mlp* m, float* theta);
int rslb_mlp_set_params(rslb_mlp* m, const float* theta);

/*
 * Fixed (not trained) normalisation: the network sees (x - mu) * inv_sd and
 * its output is multiplied by out_sd (identity after rslb_mlp_create).
 * set/get: caller-owned host arrays of n_in, n_in and n_out floats.
 * fit: from training data on the device (X [n][n_in], T [n][n_out]): mu and
 * 1/sd = the column means and inverse standard deviations of X, out_sd = the
 * column root-mean-squares of T (1 for constant or zero columns);
 * synchronises.
 */
int rslb_mlp_set_normalization(rslb_mlp* m, const float* mu, const float* inv_sd,
                               const float* out_sd);
int rslb_mlp_get_normalization(rslb_mlp* m, float* mu, float* inv_sd, float* out_sd);
int rslb_mlp_fit_normalization(rslb_mlp* m, const float* X, const float* T, int n);

/* Y [n][n_out] = out_sd * net((X [n][n_in] - mu) * inv_sd); device pointers;
 * asynchronous. */
int rslb_mlp_forward(rslb_mlp* m, const float* X, int n, float* Y);

/*
 * Mean-squared loss L = sum (y - t / out_sd)^2 / (n n_out) over the n
 * samples, y = net((x - mu) * inv_sd) the network in normalised units
 * (X [n][n_in], T [n][n_out], device), and its gradient with respect to the
 * parameters, by the library's backward kernels (weights as used in the
 * forward pass, i.e. BF16-rounded).  loss: host; grad: host, or NULL.
 * Synchronises.
 */
int rslb_mlp_loss_grad(rslb_mlp* m, const float* X, const float* T, int n, double* loss,
                       float* grad);

/*
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8) on minibatches of `batch` samples,
 * reshuffled each epoch from `seed`; epoch_loss (host, `epochs` entries, or
 * NULL) receives each epoch's mean loss.  Synchronises.
 */
int rslb_mlp_train(rslb_mlp* m, const float* X, const float* T, int n, int epochs, int batch,
                   double lr, unsigned long long seed, double* epoch_loss);
void rslb_mlp_destroy(rslb_mlp* m);

/*
 * State of `lo` := R(state of `hi`): per radial node, the Legendre moments
 * m < Q_xi(lo) of the high-order populations re-expanded at the low-order
 * nodes, f^lo_{ik} = w_i sum_m (2m+1)/2 P_m(xi_i) sum_j P_m(xi_j) f^hi_{jk}
 * (Gauss-Legendre exactness keeps the moments of Eq. macro_jk).  Both
 * handles RSLB_F32 with equal Z and Q_L.  Synchronises.
 */
int rslb_restrict(rslb_handle* hi, rslb_handle* lo);

/*
 * One training sample per cell: lo := R(hi); X [Z][3V+1] (device) = features
 * of lo (over n_s: the populations of cell s, f_{s+1} - f_s, f_s - f_{s-1};
 * then log10 tau; outflow copies at the ends); then both handles advance one
 * RK3 step and
 * T [Z][V] (device) = P(R(hi) - lo) / n_s with P the projection that removes
 * the components along the collision invariants (1, p, p xi) weighted by
 * w_j w_k.  V = Q_L Q_xi(lo) <= 32.  Synchronises.
 */
int rslb_closure_sample(rslb_handle* hi, rslb_handle* lo, double tau, float* X, float* T);

/*
 * nsteps RK3 steps of `lo`, each followed in every cell by f += alpha
 * P(n_s net(features)), alpha <= 1 the largest factor that leaves every
 * positive population at least half of itself.  The network must be
 * (3V+1) -> V.  Asynchronous.
 */
int rslb_closure_step(rslb_handle* lo, rslb_mlp* m, double tau, int nsteps);

/* ------------------------------------------------------------------------ */
/* Measurement support (not part of the method).                            */
/* ------------------------------------------------------------------------ */

/*
 * FP64 fused multiply-add rate of the current device: reps launches of
 * 8 x (SM count) blocks of 256 threads, each thread running 8 independent
 * DFMA chains of 4096 steps, timed with CUDA events on `stream` (after one
 * untimed launch).  *fma_per_s receives DFMA operations (lanes) per second.
 * Changes no device setting.  Errors: RSLB_ERR_ARG, RSLB_ERR_CUDA.
 */
int rslb_measure_fp64_fma(int reps, double* fma_per_s, void* stream);

/* Description of the last failure in the calling thread ("" if none). */
const char* rslb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSLB_H */
