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

/* ---- enumerations ---- */
#define RSLB_F32 0 /* populations, fluxes, relaxation in FP32; Landau in FP64 */
#define RSLB_F64 1 /* everything in FP64 */

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
  /* Cells per CTA tile of the stage kernel: 0 = automatic (largest tile that
   * keeps two CTAs per SM); otherwise 32 or 16 (RSLB_F32), 16 or 8
   * (RSLB_F64).  A tuning knob; results do not depend on it. */
  int tile_cells;
} rslb_config;

typedef struct rslb_handle rslb_handle;

/*
 * Validate cfg, build the velocity tables, allocate the device state (three
 * population buffers of V x Z values of the chosen precision) and set the
 * populations to the truncated f^eq of the initial state (Sec. IV A), on
 * `stream`.  On success *h owns everything and must be released with
 * rslb_destroy.
 * Errors: RSLB_ERR_ARG (bad cfg), RSLB_ERR_CFL (max|xi| dt/dz >= 1),
 * RSLB_ERR_STIFF (RSLB_TAU_CONST and dt >= tau), RSLB_ERR_UNSUPPORTED
 * (V = Q_xi*Q_L too large for one tile), RSLB_ERR_ALLOC, RSLB_ERR_CUDA,
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
 * out[field*Z + s] with the RSLB_FIELD_* order (RSLB_NFIELDS fields).
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

/*
 * Allocation-free shock-tube step (no counterpart in the paper; a service for
 * callers that cannot allocate device memory).
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
 *   cfg:    the configuration, as for rslb_init (n0/T0/beta0 and tile_cells
 *           are ignored; the populations come from f);
 *   f:      caller-owned device array of V*Z values in the cfg precision
 *           (f[v*Z + s], v = k*Q_xi + j), advanced in place by nsteps TVD-RK3
 *           steps (Eq. rk3 of L_Sod, Eq. L_Sod);
 *   stream: cudaStream_t as void* (NULL = legacy default stream).
 *
 * Limits: Q_xi*Q_L <= RSLB_NOALLOC_MAX_VELOCITIES, Q_L <= 8, and three stage
 * buffers of V x ceil32(Z) values plus O(V) tables must fit the static array;
 * larger problems are rejected with RSLB_ERR_UNSUPPORTED before any device
 * work.  The call synchronises the stream before returning and reports device
 * errors (RSLB_ERR_NONPHYSICAL) directly.
 * The first call on a device looks up the array's device address (once per
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

/* Description of the last failure in the calling thread ("" if none). */
const char* rslb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RSLB_H */
