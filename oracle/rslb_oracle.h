/*
 * rslb_oracle.h -- FP64 CPU oracle of the R-SLB method (Ambrus & Blaga,
 * "High-order quadrature-based lattice Boltzmann models for the flow of
 * ultrarelativistic rarefied gases").
 *
 * TEST INFRASTRUCTURE ONLY.  This header and rslb_oracle.c are the slow,
 * plain reference that the GPU library is checked against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the GPU library neither includes this header nor links this code, and
 * this code includes nothing from the GPU library.
 *
 * Conventions (all FP64):
 *   velocity index  v = k*Q_xi + j   (k: radial node, j: polar node; both 0-based)
 *   Sod populations f[s*V + v], s = 0..Z-1 (interior cells only)
 *   Bjorken populations f[v]
 * Every function returns 0 on success, a positive ORC_ERR_* code otherwise.
 */
#ifndef RSLB_ORACLE_H
#define RSLB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_ARG = 1,
  ORC_ERR_NONPHYSICAL = 2,
  ORC_ERR_NOCONV = 3
};

enum { ORC_BC_FIXED_EQ = 0, ORC_BC_OUTFLOW = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_TAU_CONST = 0, ORC_TAU_ETAS = 1, ORC_TAU_NONE = 2 };
enum { ORC_GAS_PARTON = 0, ORC_GAS_IDEAL = 1 };

/* Number of per-cell output fields of orc_sod_moments, in this order:
 * n, E, P, T, beta, gamma, lambda_bar, q, Pi, Nt, Nz, Ttt, Ttz, Tzz */
#define ORC_SOD_NFIELDS 14
/* Per-step output of orc_bjorken_run, in this order:
 * tau, n, E, P, T, Pi, P_L, P_T */
#define ORC_BJ_NOUT 8

double orc_legendre(int m, double x);
double orc_laguerre2(int l, double x);

int orc_gauss_legendre(int Q, double* x, double* w);
int orc_gauss_laguerre2(int Q, double* x, double* w);

/* a[l*(N_Omega+1)+m] = a^{(eq)}_{l,m}, l = 0,1 (Sec. III D, Eq. aeq_aux). */
int orc_aeq(double n, double theta, double u, int N_Omega, double* a);

/* f^eq_{jk} of Eqs. feq_trunc and fjk for a cell in state (n, T, beta). */
int orc_feq(int Q_xi, int Q_L, int N_Omega, double n, double T, double beta,
            double* feq);

/* Moments of Eq. macro_jk: M[0..4] = Nt, Nz, Ttt, Ttz, Tzz. */
int orc_moments(int Q_xi, int Q_L, const double* f, double* M);

/* Landau matching of Eqs. E_landau, u_landau, q_val, pi_val.
 * out[0..8] = n, E, P, T, beta, gamma, lambda_bar, q, Pi. */
int orc_landau(const double* M, double* out);

/* One WENO5 face flux from five upwind-ordered J values (Eqs. flux_weno,
 * weno5_omega and the limiting rules (i)-(iii)). */
double orc_weno5_face(double a, double b, double c, double d, double e);

/* K^L (Q_L x Q_L, Eq. K_lag_disc) and K^P (Q_xi x Q_xi, Eq. K_leg_disc),
 * row-major. */
int orc_kl_matrix(int Q_L, double* K);
int orc_kp_matrix(int Q_xi, double* K);

typedef struct {
  int Z;
  double z_min, z_max;
  int Q_xi, Q_L, N_Omega;
  int bc;        /* ORC_BC_* */
  int tau_mode;  /* ORC_TAU_* */
  double tau;    /* ORC_TAU_CONST */
  double tau_AW0, lambda_ref; /* ORC_TAU_ETAS */
  double dt;
  /* left/right states: used for the piecewise initial state and the
   * FIXED_EQ ghost cells */
  double nL, TL, betaL, nR, TR, betaR;
} orc_sod_params;

/* f[Z][V] <- f^eq of the per-cell fields (n, T, beta) (each length Z). */
int orc_sod_init_fields(const orc_sod_params* p, const double* n,
                        const double* T, const double* beta, double* f);
/* f[Z][V] <- left state for z_s < 0, right state otherwise (Sec. IV A). */
int orc_sod_init_riemann(const orc_sod_params* p, double* f);
/* nsteps TVD-RK3 steps (Eq. rk3) of L_Sod (Eq. L_Sod), in place. */
int orc_sod_steps(const orc_sod_params* p, double* f, int nsteps);
/* out[field*Z + s], ORC_SOD_NFIELDS fields. */
int orc_sod_moments(const orc_sod_params* p, const double* f, double* out);
/* L_Sod[f] for the interior cells (out[Z][V]); exposed for unit pins. */
int orc_sod_rhs(const orc_sod_params* p, const double* f, double* Lf);

typedef struct {
  int Q_xi, Q_L, N_Omega;
  int gas;        /* ORC_GAS_* */
  double tau_AW0; /* <= 0 or inf: collisionless */
  double tau0, dtau;
} orc_bjorken_params;

/* Runs nsteps RK3 steps of L_Bjorken (Eq. L_Bjorken) from f (in/out, V
 * values; if init != 0, f is first set to the isotropic state of
 * Eq. bjorken_f0).  out (may be NULL) gets ORC_BJ_NOUT values for each of
 * the nsteps+1 times tau0 + i*dtau. */
int orc_bjorken_run(const orc_bjorken_params* p, double* f, int init,
                    int nsteps, double* out);
int orc_bjorken_rhs(const orc_bjorken_params* p, const double* f, double tau,
                    double* Lf);

#ifdef __cplusplus
}
#endif
#endif
