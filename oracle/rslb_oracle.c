/*
 * rslb_oracle.c -- plain, slow FP64 CPU oracle of the R-SLB method of
 * Ambrus & Blaga ("High-order quadrature-based lattice Boltzmann models for
 * the flow of ultrarelativistic rarefied gases").
 *
 * TEST INFRASTRUCTURE ONLY: the GPU library is checked against this file.
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or constant with the GPU path.
 *
 * Every routine follows the paper's definitions in the paper's order, with
 * no blocking or fusion.  Summation order is fixed: radial node k outer,
 * polar node j inner, both ascending.  Readings of points where the paper is
 * silent or ambiguous are marked "Reading:".
 */
#include "rslb_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* Orthogonal polynomials                                              */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_m(x) (Sec. III C), Bonnet's recurrence
 * (m+1) P_{m+1} = (2m+1) x P_m - m P_{m-1}. */
double orc_legendre(int m, double x) {
  if (m < 0) return 0.0;
  if (m == 0) return 1.0;
  double p0 = 1.0, p1 = x;
  for (int i = 1; i < m; ++i) {
    double p2 = ((2.0 * i + 1.0) * x * p1 - i * p0) / (i + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

static double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

/* Generalised Laguerre polynomial L_l^{(2)}(x) (Sec. III B; explicit sum in
 * Eq. lag_expl).  Evaluated by the equivalent three-term recurrence
 * (n+1) L_{n+1} = (2n+3-x) L_n - (n+2) L_{n-1}, L_0 = 1, L_1 = 3 - x, which
 * avoids the cancellation of the alternating explicit sum at large x. */
double orc_laguerre2(int l, double x) {
  if (l < 0) return 0.0;
  if (l == 0) return 1.0;
  double p0 = 1.0, p1 = 3.0 - x;
  for (int n = 1; n < l; ++n) {
    double p2 = ((2.0 * n + 3.0 - x) * p1 - (n + 2.0) * p0) / (n + 1.0);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* ------------------------------------------------------------------ */
/* Quadratures                                                         */
/* ------------------------------------------------------------------ */

/* Gauss-Legendre nodes = roots of P_Q, weights
 * w = 2(1-x^2)/[(Q+1) P_{Q+1}(x)]^2 (Sec. III C, after Eq. quad_xi), in the
 * equivalent derivative form explained below.
 * Reading: the tabulated nodes of the supplemental material are not
 * available, so the roots are found by Newton's method in FP64 from the
 * asymptotic guess cos(pi(4i-1)/(4Q+2)), iterated two more times after the
 * step falls below a few ulps of 1; pairs are made exactly symmetric.
 * Ascending. */
int orc_gauss_legendre(int Q, double* x, double* w) {
  if (Q < 1 || Q > 4096 || !x || !w) return ORC_ERR_ARG;
  for (int i = 0; i < Q / 2; ++i) {
    double z = cos(M_PI * (4.0 * (i + 1) - 1.0) / (4.0 * Q + 2.0));
    int extra = 0, it;
    for (it = 0; it < 200; ++it) {
      double p0 = 1.0, p1 = z;
      for (int r = 1; r < Q; ++r) {
        double p2 = ((2.0 * r + 1.0) * z * p1 - r * p0) / (r + 1.0);
        p0 = p1;
        p1 = p2;
      }
      /* p1 = P_Q(z), p0 = P_{Q-1}(z) */
      double dp = Q * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) <= 4.0 * DBL_EPSILON) {
        if (++extra > 2) break;
      }
    }
    if (it == 200) return ORC_ERR_NOCONV;
    x[Q - 1 - i] = z;
    x[i] = -z;
  }
  if (Q % 2) x[Q / 2] = 0.0;
  for (int i = 0; i < (Q + 1) / 2; ++i) {
    double z = x[Q - 1 - i];
    /* At a root of P_Q, (Q+1) P_{Q+1} = -Q P_{Q-1} = (1 - z^2) P'_Q, so the
     * printed weight equals 2/((1 - z^2) P'_Q(z)^2).  That form is used
     * because, with P'_Q = Q (z P_Q - P_{Q-1})/(z^2 - 1) evaluated at the
     * rounded root, it is insensitive to the last bit of z; the printed
     * form loses up to 8 digits at the edge nodes when Q ~ 1000. */
    double pq = orc_legendre(Q, z), pqm1 = orc_legendre(Q - 1, z);
    double dp = Q * (z * pq - pqm1) / ((z - 1.0) * (z + 1.0));
    double wi = 2.0 / ((1.0 - z) * (1.0 + z) * dp * dp);
    w[Q - 1 - i] = wi;
    w[i] = wi;
  }
  return ORC_OK;
}

/* Gauss-Laguerre nodes for the weight e^{-x} x^2: roots of L^{(2)}_Q and
 * w = x (Q+2)/((Q+1)[L^{(2)}_{Q+1}(x)]^2) (Sec. III B, Eqs. quadL, wL).
 * Roots are bracketed on a fine grid, bisected, then polished by Newton
 * with x L'_Q = Q L_Q - (Q+2) L_{Q-1}.  At a root (Q+1) L_{Q+1} = x L'_Q, so
 * the printed weight equals (Q+1)(Q+2)/(x L'_Q(x)^2), the form used here
 * (insensitive to the last bit of x, like the Legendre case). */
int orc_gauss_laguerre2(int Q, double* x, double* w) {
  if (Q < 1 || Q > 12 || !x || !w) return ORC_ERR_ARG;
  const double xmax = 4.0 * Q + 6.0;
  const int ngrid = 100000;
  int found = 0;
  double a = 0.0, fa = orc_laguerre2(Q, a);
  for (int g = 1; g <= ngrid && found < Q; ++g) {
    double b = xmax * g / ngrid, fb = orc_laguerre2(Q, b);
    if ((fa < 0.0) != (fb < 0.0)) {
      double lo = a, hi = b, flo = fa;
      for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double fm = orc_laguerre2(Q, mid);
        if (fm == 0.0) { lo = hi = mid; break; }
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      double z = 0.5 * (lo + hi);
      for (int it = 0; it < 3; ++it) {
        double lq = orc_laguerre2(Q, z), lq1 = orc_laguerre2(Q - 1, z);
        double d = (Q * lq - (Q + 2.0) * lq1) / z;
        if (d != 0.0) z -= lq / d;
      }
      x[found++] = z;
    }
    a = b;
    fa = fb;
  }
  if (found != Q) return ORC_ERR_NOCONV;
  for (int k = 0; k < Q; ++k) {
    double z = x[k];
    double d = (Q * orc_laguerre2(Q, z) - (Q + 2.0) * orc_laguerre2(Q - 1, z)) / z;
    w[k] = (Q + 1.0) * (Q + 2.0) / (z * d * d);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Equilibrium distribution                                            */
/* ------------------------------------------------------------------ */

#define ORC_AEQ_NODES 96

/* a^{(eq)}_{l,m} for l = 0,1 and 0 <= m <= N_Omega: the Legendre
 * coefficients of F^{(eq)}_l in cos(gamma_u), defined by the integral of
 * Eq. aeq_aux (Sec. III D):
 *   a_{l,m} = n(l+1)(l+2)/(8 pi) int_{-1}^{1} dc (u0 - u c)^{-3}
 *             (1 - theta/(u0 - u c))^l P_m(c).
 * Reading: the closed forms of App. A lose all accuracy in FP64 for
 * moderate u (they cancel), so the defining integral itself is evaluated.
 * With u0 = cosh A, u = sinh A and the exact change of variables
 * u0 - u c = e^{-s}, s = A t, the integral becomes
 *   (A/u) int_{-1}^{1} dt e^{2s} (1 - theta e^{s})^l P_m(c(s)),
 *   c(s) = (2 sinh^2(A/2) - expm1(-s)) / u,
 * whose integrand is a short sum of exponentials in s; a 96-node
 * Gauss-Legendre rule in t integrates it to round-off for A < 5. */
int orc_aeq(double n, double theta, double u, int N_Omega, double* a) {
  static double gx[ORC_AEQ_NODES], gw[ORC_AEQ_NODES];
  static int ready = 0;
  if (N_Omega < 0 || N_Omega > 64 || !a || !(u >= 0.0) || !(u < 70.0))
    return ORC_ERR_ARG;
  if (!ready) {
    if (orc_gauss_legendre(ORC_AEQ_NODES, gx, gw)) return ORC_ERR_NOCONV;
    ready = 1;
  }
  const int NM = N_Omega + 1;
  const double A = asinh(u);
  const double ratio = (u > 0.0) ? A / u : 1.0;
  const double sh2 = 2.0 * sinh(0.5 * A) * sinh(0.5 * A);
  for (int l = 0; l <= 1; ++l)
    for (int m = 0; m < NM; ++m) a[l * NM + m] = 0.0;
  for (int i = 0; i < ORC_AEQ_NODES; ++i) {
    double t = gx[i];
    double s = A * t;
    double c = (u > 0.0) ? (sh2 - expm1(-s)) / u : t;
    for (int l = 0; l <= 1; ++l) {
      double g = exp(2.0 * s) * pow(1.0 - theta * exp(s), l);
      for (int m = 0; m < NM; ++m) a[l * NM + m] += gw[i] * g * orc_legendre(m, c);
    }
  }
  for (int l = 0; l <= 1; ++l)
    for (int m = 0; m < NM; ++m)
      a[l * NM + m] *= n * (l + 1.0) * (l + 2.0) / (8.0 * M_PI) * ratio;
  return ORC_OK;
}

typedef struct {
  int Q_xi, Q_L, N_Omega, V;
  double *xi, *wxi, *xk, *wk;
} orc_model;

static void model_free(orc_model* md) {
  free(md->xi);
  free(md->wxi);
  free(md->xk);
  free(md->wk);
  memset(md, 0, sizeof(*md));
}

static int model_build(orc_model* md, int Q_xi, int Q_L, int N_Omega) {
  memset(md, 0, sizeof(*md));
  if (Q_xi < 1 || Q_xi > 4096 || Q_L < 1 || Q_L > 12 || N_Omega < 0 ||
      N_Omega > 64)
    return ORC_ERR_ARG;
  md->Q_xi = Q_xi;
  md->Q_L = Q_L;
  md->N_Omega = N_Omega;
  md->V = Q_xi * Q_L;
  md->xi = (double*)malloc(sizeof(double) * Q_xi);
  md->wxi = (double*)malloc(sizeof(double) * Q_xi);
  md->xk = (double*)malloc(sizeof(double) * Q_L);
  md->wk = (double*)malloc(sizeof(double) * Q_L);
  if (!md->xi || !md->wxi || !md->xk || !md->wk) {
    model_free(md);
    return ORC_ERR_ARG;
  }
  int rc = orc_gauss_legendre(Q_xi, md->xi, md->wxi);
  if (!rc) rc = orc_gauss_laguerre2(Q_L, md->xk, md->wk);
  if (rc) model_free(md);
  return rc;
}

/* f^{eq}_{jk} = 2 pi T0^3 e^{x_k} w_j w_k f^{eq}_{N_L=1,N_Omega}(p_k, xi_j)
 * (Eq. fjk applied to Eq. feq_trunc, T0 = 1), with
 * cos(gamma_u) = sgn(u^3) xi_j for flow along z (end of Sec. III D).
 * Reading: at beta = 0 every a_{l,m>=1} vanishes, so the sign is moot. */
static int model_feq(const orc_model* md, double n, double T, double beta,
                     double* feq) {
  if (!(n > 0.0) || !(T > 0.0) || !(fabs(beta) < 1.0)) return ORC_ERR_NONPHYSICAL;
  const int NM = md->N_Omega + 1;
  double a[2 * 65];
  double gamma = 1.0 / sqrt(1.0 - beta * beta);
  double u = gamma * fabs(beta);
  int rc = orc_aeq(n, T, u, md->N_Omega, a);
  if (rc) return rc;
  double sgn = (beta < 0.0) ? -1.0 : 1.0;
  for (int k = 0; k < md->Q_L; ++k) {
    for (int j = 0; j < md->Q_xi; ++j) {
      double sum = 0.0;
      for (int l = 0; l <= 1; ++l) {
        double inner = 0.0;
        for (int m = 0; m < NM; ++m)
          inner += 0.5 * (2.0 * m + 1.0) * a[l * NM + m] *
                   orc_legendre(m, sgn * md->xi[j]);
        sum += orc_laguerre2(l, md->xk[k]) / ((l + 1.0) * (l + 2.0)) * inner;
      }
      feq[k * md->Q_xi + j] = 2.0 * M_PI * md->wxi[j] * md->wk[k] * sum;
    }
  }
  return ORC_OK;
}

int orc_feq(int Q_xi, int Q_L, int N_Omega, double n, double T, double beta,
            double* feq) {
  orc_model md;
  int rc = model_build(&md, Q_xi, Q_L, N_Omega);
  if (rc) return rc;
  rc = model_feq(&md, n, T, beta, feq);
  model_free(&md);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Moments and Landau matching                                         */
/* ------------------------------------------------------------------ */

/* N^t = sum f, N^z = sum f xi, T^tt = sum f p, T^tz = sum f p xi,
 * T^zz = sum f p xi^2 (Eq. macro_jk), p_k = T0 x_k with T0 = 1. */
static void model_moments(const orc_model* md, const double* f, double* M) {
  for (int i = 0; i < 5; ++i) M[i] = 0.0;
  for (int k = 0; k < md->Q_L; ++k) {
    double p = md->xk[k];
    for (int j = 0; j < md->Q_xi; ++j) {
      double fv = f[k * md->Q_xi + j], xi = md->xi[j];
      M[0] += fv;
      M[1] += fv * xi;
      M[2] += fv * p;
      M[3] += fv * p * xi;
      M[4] += fv * p * xi * xi;
    }
  }
}

int orc_moments(int Q_xi, int Q_L, const double* f, double* M) {
  orc_model md;
  int rc = model_build(&md, Q_xi, Q_L, 0);
  if (rc) return rc;
  model_moments(&md, f, M);
  model_free(&md);
  return ORC_OK;
}

/* Landau frame for the 1-D stress tensor: E (Eq. E_landau), beta and gamma
 * (Eq. u_landau), n = -u.N, P = E/3, T = P/n (Eq. T_def),
 * lambda_bar = n/T^3, q (Eq. q_val), Pi (Eq. pi_val). */
int orc_landau(const double* M, double* out) {
  double Nt = M[0], Nz = M[1], Ttt = M[2], Ttz = M[3], Tzz = M[4];
  double disc = (Ttt + Tzz) * (Ttt + Tzz) - 4.0 * Ttz * Ttz;
  if (!(disc >= 0.0)) return ORC_ERR_NONPHYSICAL;
  double E = 0.5 * (Ttt - Tzz + sqrt(disc));
  if (!(E > 0.0)) return ORC_ERR_NONPHYSICAL;
  double beta = Ttz / (E + Tzz);
  if (!(fabs(beta) < 1.0)) return ORC_ERR_NONPHYSICAL;
  double gamma = 1.0 / sqrt(1.0 - beta * beta);
  double n = gamma * (Nt - beta * Nz);
  if (!(n > 0.0)) return ORC_ERR_NONPHYSICAL;
  double P = E / 3.0;
  double T = P / n;
  out[0] = n;
  out[1] = E;
  out[2] = P;
  out[3] = T;
  out[4] = beta;
  out[5] = gamma;
  out[6] = n / (T * T * T);
  out[7] = -4.0 * T * (Nz - n * beta * gamma);
  out[8] = 2.0 * E / 3.0 - Ttt + Tzz;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* WENO5 (Sec. III F)                                                  */
/* ------------------------------------------------------------------ */

/* Face flux F_{s+1/2} from the upwind-ordered values
 * (a, b, c, d, e) = (J_{s-2}, J_{s-1}, J_s, J_{s+1}, J_{s+2}) (Eq. flux_weno
 * with the three interpolants, the smoothness functions sigma_q and
 * Eq. weno5_omega with delta = (0.1, 0.6, 0.3)).  No epsilon is added; the
 * limiting rules (i)-(iii) are applied instead, in that order.
 * Reading: "sigma_q = 0" is taken literally (exactly zero); in addition, a
 * nonzero sigma_q whose square underflows (so that delta_q/sigma_q^2 would
 * be infinite) is treated as zero, which is the limit the rules describe. */
double orc_weno5_face(double a, double b, double c, double d, double e) {
  const double delta[3] = {0.1, 0.6, 0.3};
  double F[3], sig[3], om[3];
  F[0] = a / 3.0 - 7.0 * b / 6.0 + 11.0 * c / 6.0;
  F[1] = -b / 6.0 + 5.0 * c / 6.0 + d / 3.0;
  F[2] = c / 3.0 + 5.0 * d / 6.0 - e / 6.0;
  sig[0] = 13.0 / 12.0 * (a - 2.0 * b + c) * (a - 2.0 * b + c) +
           0.25 * (a - 4.0 * b + 3.0 * c) * (a - 4.0 * b + 3.0 * c);
  sig[1] = 13.0 / 12.0 * (b - 2.0 * c + d) * (b - 2.0 * c + d) +
           0.25 * (b - d) * (b - d);
  sig[2] = 13.0 / 12.0 * (c - 2.0 * d + e) * (c - 2.0 * d + e) +
           0.25 * (3.0 * c - 4.0 * d + e) * (3.0 * c - 4.0 * d + e);
  if (sig[0] == sig[1] && sig[1] == sig[2]) {
    /* rule (i) */
    om[0] = delta[0];
    om[1] = delta[1];
    om[2] = delta[2];
  } else {
    int zero[3], nz = 0;
    for (int q = 0; q < 3; ++q) {
      zero[q] = (sig[q] == 0.0) || (sig[q] * sig[q] == 0.0);
      nz += zero[q];
    }
    if (nz == 2) {
      /* rule (ii): sigma vanishes for all q but one (p) */
      double dsum = 0.0;
      for (int q = 0; q < 3; ++q)
        if (zero[q]) dsum += delta[q];
      for (int q = 0; q < 3; ++q) om[q] = zero[q] ? delta[q] / dsum : 0.0;
    } else if (nz == 1) {
      /* rule (iii): sigma vanishes only for q = p */
      for (int q = 0; q < 3; ++q) om[q] = zero[q] ? 1.0 : 0.0;
    } else {
      double wt[3], sum = 0.0;
      for (int q = 0; q < 3; ++q) {
        wt[q] = delta[q] / (sig[q] * sig[q]);
        sum += wt[q];
      }
      for (int q = 0; q < 3; ++q) om[q] = wt[q] / sum;
    }
  }
  return om[0] * F[0] + om[1] * F[1] + om[2] * F[2];
}

/* ------------------------------------------------------------------ */
/* Sod shock tube (Secs. II E, III F, IV A)                            */
/* ------------------------------------------------------------------ */

typedef struct {
  orc_model md;
  double *fL, *fR; /* FIXED_EQ ghost populations */
  double *g;       /* extended state [(Z+6)][V] */
  double *feq, *coll, *J, *F;
} sod_ws;

static void sod_ws_free(sod_ws* w) {
  model_free(&w->md);
  free(w->fL);
  free(w->fR);
  free(w->g);
  free(w->feq);
  free(w->coll);
  free(w->J);
  free(w->F);
  memset(w, 0, sizeof(*w));
}

static int sod_check(const orc_sod_params* p) {
  if (!p || p->Z < 1 || !(p->z_max > p->z_min) || p->N_Omega < 0 ||
      p->bc < 0 || p->bc > 2 || p->tau_mode < 0 || p->tau_mode > 2 ||
      !(p->dt > 0.0))
    return ORC_ERR_ARG;
  if (p->tau_mode == ORC_TAU_CONST && !(p->tau > 0.0)) return ORC_ERR_ARG;
  if (p->tau_mode == ORC_TAU_ETAS && !(p->tau_AW0 > 0.0 && p->lambda_ref > 0.0))
    return ORC_ERR_ARG;
  return ORC_OK;
}

static int sod_ws_build(sod_ws* w, const orc_sod_params* p) {
  memset(w, 0, sizeof(*w));
  int rc = sod_check(p);
  if (rc) return rc;
  rc = model_build(&w->md, p->Q_xi, p->Q_L, p->N_Omega);
  if (rc) return rc;
  const int V = w->md.V, Z = p->Z;
  w->fL = (double*)malloc(sizeof(double) * V);
  w->fR = (double*)malloc(sizeof(double) * V);
  w->g = (double*)malloc(sizeof(double) * (size_t)(Z + 6) * V);
  w->feq = (double*)malloc(sizeof(double) * (size_t)Z * V);
  w->coll = (double*)malloc(sizeof(double) * (size_t)Z * V);
  w->J = (double*)malloc(sizeof(double) * (size_t)(Z + 6));
  w->F = (double*)malloc(sizeof(double) * (size_t)(Z + 1));
  if (!w->fL || !w->fR || !w->g || !w->feq || !w->coll || !w->J || !w->F) {
    sod_ws_free(w);
    return ORC_ERR_ARG;
  }
  if (p->bc == ORC_BC_FIXED_EQ) {
    rc = model_feq(&w->md, p->nL, p->TL, p->betaL, w->fL);
    if (!rc) rc = model_feq(&w->md, p->nR, p->TR, p->betaR, w->fR);
    if (rc) {
      sod_ws_free(w);
      return rc;
    }
  }
  return ORC_OK;
}

/* Ghost cells, three on each side (Sec. IV A).  FIXED_EQ: the left/right
 * equilibria (the paper's choice).  Reading: OUTFLOW copies the first/last
 * interior cell into its three ghosts (zero gradient); PERIODIC wraps. */
static void sod_extend(const orc_sod_params* p, sod_ws* w, const double* f) {
  const int V = w->md.V, Z = p->Z;
  for (int s = -3; s < Z + 3; ++s) {
    const double* src;
    if (s >= 0 && s < Z) {
      src = f + (size_t)s * V;
    } else if (p->bc == ORC_BC_FIXED_EQ) {
      src = (s < 0) ? w->fL : w->fR;
    } else if (p->bc == ORC_BC_OUTFLOW) {
      src = f + (size_t)((s < 0) ? 0 : Z - 1) * V;
    } else {
      int sp = ((s % Z) + Z) % Z;
      src = f + (size_t)sp * V;
    }
    memcpy(w->g + (size_t)(s + 3) * V, src, sizeof(double) * V);
  }
}

/* L_Sod[f] of Eq. L_Sod: - (xi dz f) - (u^0 - u^z xi_j)/tau_AW (f - f^eq). */
static int sod_rhs_ws(const orc_sod_params* p, sod_ws* w, const double* f,
                      double* Lf) {
  const int V = w->md.V, Z = p->Z, Qx = w->md.Q_xi;
  const double dz = (p->z_max - p->z_min) / Z;
  sod_extend(p, w, f);
  /* collision term per (cell, velocity) */
  for (int s = 0; s < Z; ++s) {
    const double* fs = f + (size_t)s * V;
    double* cs = w->coll + (size_t)s * V;
    if (p->tau_mode == ORC_TAU_NONE) {
      for (int v = 0; v < V; ++v) cs[v] = 0.0;
      continue;
    }
    double M[5], L[9];
    model_moments(&w->md, fs, M);
    int rc = orc_landau(M, L);
    if (rc) return rc;
    double n = L[0], T = L[3], beta = L[4], gamma = L[5];
    double tau;
    if (p->tau_mode == ORC_TAU_CONST) {
      tau = p->tau;
    } else {
      /* Eq. Sod:tau: tau_AW = tau_AW0/T [1 - ln(lambda_bar lambda_ref)/4] */
      tau = p->tau_AW0 / T * (1.0 - 0.25 * log(n / (T * T * T) * p->lambda_ref));
    }
    double* fe = w->feq + (size_t)s * V;
    rc = model_feq(&w->md, n, T, beta, fe);
    if (rc) return rc;
    for (int k = 0; k < w->md.Q_L; ++k)
      for (int j = 0; j < Qx; ++j) {
        int v = k * Qx + j;
        double u0 = gamma, uz = gamma * beta;
        cs[v] = (u0 - uz * w->md.xi[j]) / tau * (fs[v] - fe[v]);
      }
  }
  /* advection, velocity by velocity */
  for (int v = 0; v < V; ++v) {
    double xi = w->md.xi[v % Qx];
    for (int e = 0; e < Z + 6; ++e) w->J[e] = xi * w->g[(size_t)e * V + v];
    /* J[e] holds J_{e-3}; F[i] holds F_{i-1/2}, i = 0..Z */
#define JJ(s) (w->J[(s) + 3])
    for (int i = 0; i <= Z; ++i) {
      int s = i - 1; /* face s+1/2 */
      if (xi > 0.0)
        w->F[i] = orc_weno5_face(JJ(s - 2), JJ(s - 1), JJ(s), JJ(s + 1), JJ(s + 2));
      else if (xi < 0.0)
        w->F[i] = orc_weno5_face(JJ(s + 3), JJ(s + 2), JJ(s + 1), JJ(s), JJ(s - 1));
      else
        w->F[i] = 0.0;
    }
#undef JJ
    for (int s = 0; s < Z; ++s)
      Lf[(size_t)s * V + v] =
          -(w->F[s + 1] - w->F[s]) / dz - w->coll[(size_t)s * V + v];
  }
  return ORC_OK;
}

int orc_sod_rhs(const orc_sod_params* p, const double* f, double* Lf) {
  sod_ws w;
  int rc = sod_ws_build(&w, p);
  if (rc) return rc;
  rc = sod_rhs_ws(p, &w, f, Lf);
  sod_ws_free(&w);
  return rc;
}

int orc_sod_init_fields(const orc_sod_params* p, const double* n,
                        const double* T, const double* beta, double* f) {
  orc_model md;
  if (!p || p->Z < 1) return ORC_ERR_ARG;
  int rc = model_build(&md, p->Q_xi, p->Q_L, p->N_Omega);
  if (rc) return rc;
  for (int s = 0; s < p->Z && !rc; ++s)
    rc = model_feq(&md, n[s], T[s], beta[s], f + (size_t)s * md.V);
  model_free(&md);
  return rc;
}

/* Cell centres z_s = z_min + (s + 1/2) dz; left state for z_s < 0. */
int orc_sod_init_riemann(const orc_sod_params* p, double* f) {
  orc_model md;
  if (!p || p->Z < 1 || !(p->z_max > p->z_min)) return ORC_ERR_ARG;
  int rc = model_build(&md, p->Q_xi, p->Q_L, p->N_Omega);
  if (rc) return rc;
  const double dz = (p->z_max - p->z_min) / p->Z;
  for (int s = 0; s < p->Z && !rc; ++s) {
    double z = p->z_min + (s + 0.5) * dz;
    if (z < 0.0)
      rc = model_feq(&md, p->nL, p->TL, p->betaL, f + (size_t)s * md.V);
    else
      rc = model_feq(&md, p->nR, p->TR, p->betaR, f + (size_t)s * md.V);
  }
  model_free(&md);
  return rc;
}

/* Shu-Osher TVD-RK3 (Eq. rk3, Tab. II). */
int orc_sod_steps(const orc_sod_params* p, double* f, int nsteps) {
  sod_ws w;
  int rc = sod_ws_build(&w, p);
  if (rc) return rc;
  const size_t N = (size_t)p->Z * w.md.V;
  double* L = (double*)malloc(sizeof(double) * N);
  double* f1 = (double*)malloc(sizeof(double) * N);
  double* f2 = (double*)malloc(sizeof(double) * N);
  if (!L || !f1 || !f2) rc = ORC_ERR_ARG;
  const double dt = p->dt;
  for (int n = 0; n < nsteps && !rc; ++n) {
    rc = sod_rhs_ws(p, &w, f, L);
    if (rc) break;
    for (size_t i = 0; i < N; ++i) f1[i] = f[i] + dt * L[i];
    rc = sod_rhs_ws(p, &w, f1, L);
    if (rc) break;
    for (size_t i = 0; i < N; ++i)
      f2[i] = 0.75 * f[i] + 0.25 * f1[i] + 0.25 * dt * L[i];
    rc = sod_rhs_ws(p, &w, f2, L);
    if (rc) break;
    for (size_t i = 0; i < N; ++i)
      f[i] = f[i] / 3.0 + 2.0 / 3.0 * f2[i] + 2.0 / 3.0 * dt * L[i];
  }
  free(L);
  free(f1);
  free(f2);
  sod_ws_free(&w);
  return rc;
}

int orc_sod_moments(const orc_sod_params* p, const double* f, double* out) {
  orc_model md;
  if (!p || p->Z < 1) return ORC_ERR_ARG;
  int rc = model_build(&md, p->Q_xi, p->Q_L, 0);
  if (rc) return rc;
  const int Z = p->Z;
  for (int s = 0; s < Z && !rc; ++s) {
    double M[5], L[9];
    model_moments(&md, f + (size_t)s * md.V, M);
    rc = orc_landau(M, L);
    if (rc) break;
    for (int i = 0; i < 9; ++i) out[(size_t)i * Z + s] = L[i];
    for (int i = 0; i < 5; ++i) out[(size_t)(9 + i) * Z + s] = M[i];
  }
  model_free(&md);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Momentum-space derivative matrices (Sec. III E)                     */
/* ------------------------------------------------------------------ */

/* K^L_{k,k'} = w_k sum_{l=1}^{Q_L-1} L_l(x_k) [(l+2) L_{l-1}(x_k') -
 * l L_l(x_k')] / ((l+1)(l+2))   (Eq. K_lag_disc). */
static void kl_fill(const orc_model* md, double* K) {
  const int Q = md->Q_L;
  for (int k = 0; k < Q; ++k)
    for (int kp = 0; kp < Q; ++kp) {
      double s = 0.0;
      for (int l = 1; l <= Q - 1; ++l)
        s += orc_laguerre2(l, md->xk[k]) *
             ((l + 2.0) * orc_laguerre2(l - 1, md->xk[kp]) -
              l * orc_laguerre2(l, md->xk[kp])) /
             ((l + 1.0) * (l + 2.0));
      K[k * Q + kp] = md->wk[k] * s;
    }
}

/* K^P_{j,j'} of Eq. K_leg_disc, sums read with the printed limits:
 *   w_j sum_{m=1}^{Q-3} m(m+1)(m+2)/(2(2m+3)) P_m(xi_j) P_{m+2}(xi_j')
 * - w_j sum_{m=1}^{Q-1} m(m+1)/2 P_m(xi_j) [ (2m+1) P_m(xi_j')/((2m-1)(2m+3))
 *                                          + (m-1)/(2m-1) P_{m-2}(xi_j') ]. */
static void kp_fill(const orc_model* md, double* K) {
  const int Q = md->Q_xi;
  /* table P[m][j] = P_m(xi_j), m = 0 .. Q+1 (values of Sec. III C) */
  double* P = (double*)malloc(sizeof(double) * (size_t)(Q + 2) * Q);
  for (int m = 0; m < Q + 2; ++m)
    for (int j = 0; j < Q; ++j) P[(size_t)m * Q + j] = orc_legendre(m, md->xi[j]);
#define PM(m, j) ((m) < 0 ? 0.0 : P[(size_t)(m) * Q + (j)])
  for (int j = 0; j < Q; ++j)
    for (int jp = 0; jp < Q; ++jp) {
      double s1 = 0.0, s2 = 0.0;
      for (int m = 1; m <= Q - 3; ++m)
        s1 += m * (m + 1.0) * (m + 2.0) / (2.0 * (2.0 * m + 3.0)) * PM(m, j) * PM(m + 2, jp);
      for (int m = 1; m <= Q - 1; ++m)
        s2 += m * (m + 1.0) / 2.0 * PM(m, j) *
              ((2.0 * m + 1.0) * PM(m, jp) / ((2.0 * m - 1.0) * (2.0 * m + 3.0)) +
               (m - 1.0) / (2.0 * m - 1.0) * PM(m - 2, jp));
      K[j * Q + jp] = md->wxi[j] * (s1 - s2);
    }
#undef PM
  free(P);
}

int orc_kl_matrix(int Q_L, double* K) {
  orc_model md;
  int rc = model_build(&md, 1, Q_L, 0);
  if (rc) return rc;
  kl_fill(&md, K);
  model_free(&md);
  return ORC_OK;
}

int orc_kp_matrix(int Q_xi, double* K) {
  orc_model md;
  int rc = model_build(&md, Q_xi, 1, 0);
  if (rc) return rc;
  kp_fill(&md, K);
  model_free(&md);
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Bjorken flow (Secs. II F, III F, V)                                 */
/* ------------------------------------------------------------------ */

typedef struct {
  orc_model md;
  double *KL, *KP, *feq;
} bj_ws;

static void bj_ws_free(bj_ws* w) {
  model_free(&w->md);
  free(w->KL);
  free(w->KP);
  free(w->feq);
  memset(w, 0, sizeof(*w));
}

static int bj_ws_build(bj_ws* w, const orc_bjorken_params* p) {
  memset(w, 0, sizeof(*w));
  if (!p || !(p->tau0 > 0.0) || !(p->dtau > 0.0) || p->gas < 0 || p->gas > 1)
    return ORC_ERR_ARG;
  int rc = model_build(&w->md, p->Q_xi, p->Q_L, p->N_Omega);
  if (rc) return rc;
  w->KL = (double*)malloc(sizeof(double) * p->Q_L * p->Q_L);
  w->KP = (double*)malloc(sizeof(double) * (size_t)p->Q_xi * p->Q_xi);
  w->feq = (double*)malloc(sizeof(double) * w->md.V);
  if (!w->KL || !w->KP || !w->feq) {
    bj_ws_free(w);
    return ORC_ERR_ARG;
  }
  kl_fill(&w->md, w->KL);
  kp_fill(&w->md, w->KP);
  return ORC_OK;
}

static int bj_collisionless(const orc_bjorken_params* p) {
  return !(p->tau_AW0 > 0.0) || isinf(p->tau_AW0);
}

/* Equilibrium state of a homogeneous Bjorken cell at rest (u = (1,0,0,0),
 * Eq. bjorken_u): E = T^{tau tau}, P = E/3.
 *  parton gas (Eqs. bjorken_mu0, bjorken_tauAW0): T = P^{1/4},
 *    n_eq = P^{3/4}, tau_AW = tau_AW0/T;
 *  ideal gas (Eq. bjorken_tauAW_mu): n = N^tau, T = P/n, n_eq = n,
 *    tau_AW = tau_AW0/T [1 - ln(n/T^3)/4]  (Eq. bjorken_tauAW with
 *    lambda_ref = 1). */
static int bj_equilibrium(const orc_bjorken_params* p, const orc_model* md,
                          const double* f, double* n_eq, double* T,
                          double* tau_aw) {
  double M[5];
  model_moments(md, f, M);
  double P = M[2] / 3.0;
  if (!(P > 0.0)) return ORC_ERR_NONPHYSICAL;
  if (p->gas == ORC_GAS_PARTON) {
    *T = pow(P, 0.25);
    *n_eq = pow(P, 0.75);
    *tau_aw = p->tau_AW0 / *T;
  } else {
    double n = M[0];
    if (!(n > 0.0)) return ORC_ERR_NONPHYSICAL;
    *T = P / n;
    *n_eq = n;
    *tau_aw = p->tau_AW0 / *T * (1.0 - 0.25 * log(n / (*T * *T * *T)));
  }
  return ORC_OK;
}

/* L_Bjorken[f] of Eq. L_Bjorken at proper time tau. */
static int bj_rhs_ws(const orc_bjorken_params* p, bj_ws* w, const double* f,
                     double tau, double* Lf) {
  const orc_model* md = &w->md;
  const int Qx = md->Q_xi, QL = md->Q_L;
  int coll = !bj_collisionless(p);
  double tau_aw = 1.0;
  if (coll) {
    double n_eq, T;
    int rc = bj_equilibrium(p, md, f, &n_eq, &T, &tau_aw);
    if (rc) return rc;
    rc = model_feq(md, n_eq, T, 0.0, w->feq);
    if (rc) return rc;
  }
  for (int k = 0; k < QL; ++k)
    for (int j = 0; j < Qx; ++j) {
      int v = k * Qx + j;
      double kl = 0.0, kp = 0.0;
      for (int kq = 0; kq < QL; ++kq) kl += w->KL[k * QL + kq] * f[kq * Qx + j];
      for (int jq = 0; jq < Qx; ++jq) kp += w->KP[j * Qx + jq] * f[k * Qx + jq];
      double xi = md->xi[j];
      double r = -f[v] / tau + xi * xi / tau * kl + kp / tau;
      if (coll) r -= (f[v] - w->feq[v]) / tau_aw;
      Lf[v] = r;
    }
  return ORC_OK;
}

int orc_bjorken_rhs(const orc_bjorken_params* p, const double* f, double tau,
                    double* Lf) {
  bj_ws w;
  int rc = bj_ws_build(&w, p);
  if (rc) return rc;
  rc = bj_rhs_ws(p, &w, f, tau, Lf);
  bj_ws_free(&w);
  return rc;
}

static int bj_output(const orc_bjorken_params* p, const orc_model* md,
                     const double* f, double tau, double* o) {
  double M[5];
  model_moments(md, f, M);
  double E = M[2], P = E / 3.0, PL = M[4];
  double T;
  if (p->gas == ORC_GAS_PARTON) {
    T = (P > 0.0) ? pow(P, 0.25) : NAN;
  } else {
    T = P / M[0];
  }
  o[0] = tau;
  o[1] = M[0];
  o[2] = E;
  o[3] = P;
  o[4] = T;
  o[5] = PL - P; /* Eq. bjorken_P: P_L = P + Pi */
  o[6] = PL;
  o[7] = 0.5 * (E - PL); /* T^{xx} = (T^{tt} - T^{zz})/2 (Eq. TxxTyy) */
  return ORC_OK;
}

/* RK3 with stage times tau_n, tau_n + dtau, tau_n + dtau/2 (the Butcher
 * nodes c = (0, 1, 1/2) of Tab. II).  Reading: L is evaluated at each
 * stage's own time, with tau_AW from the stage state. */
int orc_bjorken_run(const orc_bjorken_params* p, double* f, int init,
                    int nsteps, double* out) {
  bj_ws w;
  int rc = bj_ws_build(&w, p);
  if (rc) return rc;
  const int V = w.md.V;
  double* L = (double*)malloc(sizeof(double) * V);
  double* f1 = (double*)malloc(sizeof(double) * V);
  double* f2 = (double*)malloc(sizeof(double) * V);
  if (!L || !f1 || !f2) rc = ORC_ERR_ARG;
  /* isotropic initial state f = e^{-p}/(8 pi) at tau = 1 (Eq. bjorken_f0):
   * the equilibrium with n = 1, T = 1 */
  if (!rc && init) rc = model_feq(&w.md, 1.0, 1.0, 0.0, f);
  const double dtau = p->dtau;
  if (!rc && out) bj_output(p, &w.md, f, p->tau0, out);
  for (int n = 0; n < nsteps && !rc; ++n) {
    double tn = p->tau0 + n * dtau;
    rc = bj_rhs_ws(p, &w, f, tn, L);
    if (rc) break;
    for (int v = 0; v < V; ++v) f1[v] = f[v] + dtau * L[v];
    rc = bj_rhs_ws(p, &w, f1, tn + dtau, L);
    if (rc) break;
    for (int v = 0; v < V; ++v) f2[v] = 0.75 * f[v] + 0.25 * f1[v] + 0.25 * dtau * L[v];
    rc = bj_rhs_ws(p, &w, f2, tn + 0.5 * dtau, L);
    if (rc) break;
    for (int v = 0; v < V; ++v)
      f[v] = f[v] / 3.0 + 2.0 / 3.0 * f2[v] + 2.0 / 3.0 * dtau * L[v];
    if (out) bj_output(p, &w.md, f, p->tau0 + (n + 1) * dtau, out + (size_t)(n + 1) * ORC_BJ_NOUT);
  }
  free(L);
  free(f1);
  free(f2);
  bj_ws_free(&w);
  return rc;
}
