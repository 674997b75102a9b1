"""Closed-form results printed in the paper, used to pin the FP64 oracle.

Each function restates one analytic result of Ambrus & Blaga (the paper's
section and equation are named in its docstring).  None of them shares code or
arithmetic with ``oracle/``: they are independent routes to the same numbers.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp
from scipy.optimize import brentq

CS = 1.0 / math.sqrt(3.0)  # ultrarelativistic sound speed, Sec. IV B 1


# ---------------------------------------------------------------------------
# App. A: closed forms of the f^eq expansion coefficients
# ---------------------------------------------------------------------------
def a_tilde_closed(l, s, u, theta):
    """tilde a^{(eq)}_{l,s} of App. A (valid for u > 0; unstable for small u)."""
    u0 = math.sqrt(1.0 + u * u)
    ash = math.asinh(u)
    t0 = [
        1.0,
        u / u0,
        3.0 / (2 * u**3 * u0) * ash + 1.0 - 3.0 / (2 * u**2),
        15.0 / (2 * u**4) * ash - (15 + 5 * u**2 - 2 * u**4) / (2 * u**3 * u0),
        15.0 / (4 * u**5 * u0) * (7 + 6 * u**2) * ash - (105 + 20 * u**2 - 4 * u**4) / (4 * u**4),
        105.0 / (4 * u**6) * (3 + 2 * u**2) * ash
        - (315 + 315 * u**2 + 28 * u**4 - 4 * u**6) / (4 * u**5 * u0),
        105.0 / (16 * u**7 * u0) * (33 + 48 * u**2 + 16 * u**4) * ash
        - (3465 + 2730 * u**2 + 168 * u**4 - 16 * u**6) / (16 * u**6),
    ]
    if l == 0:
        return t0[s]
    th = theta
    d1 = [
        -th / (3 * u0) * (3 + 4 * u**2),
        -4 * u * th / 3,
        -4 * th * u**2 / (3 * u0),
        5 * th / (2 * u**4 * u0) * ash - th / (6 * u**3) * (15 - 10 * u**2 + 8 * u**4),
        35 * th / (2 * u**5) * ash - th / (6 * u**4 * u0) * (105 + 35 * u**2 - 14 * u**4 + 8 * u**6),
        35 * th / (4 * u**6 * u0) * (9 + 8 * u**2) * ash
        - th / (12 * u**5) * (945 + 210 * u**2 - 56 * u**4 + 16 * u**6),
        105 * th / (4 * u**7) * (11 + 8 * u**2) * ash
        - th / (12 * u**6 * u0) * (3465 + 3675 * u**2 + 378 * u**4 - 72 * u**6 + 16 * u**8),
    ]
    return t0[s] + d1[s]


def a_tilde_series(l, s, u, theta):
    """Maclaurin series of App. A (through u^11), for small u.

    Reading: the printed l=1, s=3 series has a doubled minus sign before the
    u^7 term; the alternating-sign reading is used.
    """
    u0 = math.sqrt(1.0 + u * u)
    s0 = {
        0: 1.0,
        1: u / u0,
        2: 4 * u**2 / 5 - 24 * u**4 / 35 + 64 * u**6 / 105 - 128 * u**8 / 231 + 512 * u**10 / 1001,
        3: 4 * u**3 / 7 - 2 * u**5 / 3 + 15 * u**7 / 22 - 35 * u**9 / 52 + 21 * u**11 / 32,
        4: 8 * u**4 / 21 - 128 * u**6 / 231 + 640 * u**8 / 1001 - 2048 * u**10 / 3003,
        5: 8 * u**5 / 33 - 60 * u**7 / 143 + 7 * u**9 / 13 - 21 * u**11 / 34,
        6: 64 * u**6 / 429 - 128 * u**8 / 429 + 1024 * u**10 / 2431,
    }
    if l == 0:
        return s0[s]
    th = theta
    s1 = {
        0: -th / (3 * u0) * (3 + 4 * u**2),
        1: -4 * u * th / 3,
        2: -4 * th / 3 * u**2 + 2 * th / 3 * u**4 - th / 2 * u**6 + 5 * th / 12 * u**8
        - 35 * th / 96 * u**10,
        3: -8 * th / 7 * u**3 + 64 * th / 63 * u**5 - 640 * th / 693 * u**7
        + 2560 * th / 3003 * u**9 - 1024 * th / 1287 * u**11,
        4: -8 * th / 9 * u**4 + 12 * th / 11 * u**6 - 15 * th / 13 * u**8 + 7 * th / 6 * u**10,
        5: -64 * th / 99 * u**5 + 1280 * th / 1287 * u**7 - 512 * th / 429 * u**9
        + 28672 * th / 21879 * u**11,
        6: -64 * th / 143 * u**6 + 32 * th / 39 * u**8 - 56 * th / 51 * u**10,
    }
    return s0[s] + s1[s]


def a_from_tilde(n, l, u, at):
    """a_{l,s} = n (l+1)(l+2)/(4 pi) u^0 tilde a_{l,s} (App. A)."""
    return n * (l + 1) * (l + 2) / (4 * math.pi) * math.sqrt(1 + u * u) * at


# ---------------------------------------------------------------------------
# Sec. IV B 1: exact inviscid Riemann problem for massless particles
# ---------------------------------------------------------------------------
class Riemann:
    """Exact ultrarelativistic Sod solution for left/right states at rest."""

    def __init__(self, nL, PL, nR, PR):
        self.nL, self.PL, self.nR, self.PR = nL, PL, nR, PR
        r3 = math.sqrt(3.0)

        def plateau_eq(PC):  # Eq. Sod:PC
            a = (PL / PC) ** (r3 / 2)
            return (a - 1) / (a + 1) - math.sqrt(3 * (PC - PR) ** 2 / ((PC + 3 * PR) * (3 * PC + PR)))

        self.PC = brentq(plateau_eq, PR * (1 + 1e-14), PL, xtol=1e-16, rtol=1e-15, maxiter=500)
        PC = self.PC
        self.beta_shock = math.sqrt((PR + 3 * PC) / (3 * (PC + 3 * PR)))  # Eq. Sod:uplateau
        self.beta_C = math.sqrt(3 * (PC - PR) ** 2 / ((PC + 3 * PR) * (3 * PC + PR)))
        q = (PC / PL) ** (r3 / 2)
        self.zeta_T = (r3 - 1 - (r3 + 1) * q) / (r3 - 1 + (r3 + 1) * q)  # Eq. Sod:xiT
        self.nI = nL * (PC / PL) ** 0.75  # Eq. Sod:nI
        self.nII = nR * math.sqrt(PC * (PR + 3 * PC) / (PR * (PC + 3 * PR)))  # Eq. Sod:nII

    def profile(self, z, t):
        """(n, P, beta) at positions z, time t (full solution of Sec. IV B 1)."""
        z = np.asarray(z, dtype=float)
        zeta = z / t
        n = np.empty_like(z)
        P = np.empty_like(z)
        b = np.empty_like(z)
        zH, zT, zC, zS = -CS, self.zeta_T, self.beta_C, self.beta_shock
        for i, x in enumerate(zeta):
            if x < zH:
                n[i], P[i], b[i] = self.nL, self.PL, 0.0
            elif x < zT:
                r = (1 - CS) * (1 - x) / ((1 + CS) * (1 + x))
                b[i] = (CS + x) / (1 + CS * x)  # Eq. betastar
                P[i] = self.PL * r ** (2 / math.sqrt(3))  # Eq. Pstar
                n[i] = self.nL * r ** (math.sqrt(3) / 2)  # Eq. nstar
            elif x < zC:
                n[i], P[i], b[i] = self.nI, self.PC, self.beta_C
            elif x < zS:
                n[i], P[i], b[i] = self.nII, self.PC, self.beta_C
            else:
                n[i], P[i], b[i] = self.nR, self.PR, 0.0
        return n, P, b


# ---------------------------------------------------------------------------
# Sec. IV C 1: ballistic (collisionless) Sod, continuum momentum space
# ---------------------------------------------------------------------------
def ballistic_sod(zeta, nL, PL, nR, PR):
    """(N^t, N^z, T^tt, T^tz, T^zz) of Eqs. Sod:bal:Nmu and Sod:bal:Tmunu."""
    zeta = np.clip(np.asarray(zeta, dtype=float), -1.0, 1.0)
    Nt = (nL + nR) / 2 - (nL - nR) / 2 * zeta
    Nz = (nL - nR) / 4 * (1 - zeta**2)
    Ttt = 1.5 * (PL + PR) - 1.5 * (PL - PR) * zeta
    Ttz = 0.75 * (PL - PR) * (1 - zeta**2)
    Tzz = 0.5 * (PL + PR) - 0.5 * (PL - PR) * zeta**3
    return Nt, Nz, Ttt, Ttz, Tzz


# ---------------------------------------------------------------------------
# Sec. V: Bjorken flow
# ---------------------------------------------------------------------------
def bjorken_ballistic(tau):
    """(P, P_L) of the free-streaming solution, Eq. bjorken_bal."""
    tau = np.asarray(tau, dtype=float)
    r = np.sqrt(tau**2 - 1.0)
    rs = np.where(r > 1e-3, r, 1.0)
    at = np.where(r > 1e-3, np.arctan(rs) / rs, 1.0 - r**2 / 3.0)
    P = 0.5 * (at + 1.0 / tau**2)
    # near tau = 1 the bracket cancels; its Taylor expansion is 1 - 6 r^2/5
    PL = np.where(r > 1e-3, 1.5 / (rs * rs) * (at - 1.0 / tau**2), 1.0 - 1.2 * r**2)
    return P, PL


def bjorken_hydro1_parton(tau, tau_AW0):
    """(P, Pi) of first-order hydrodynamics for the parton gas, Eq. bjorken_mu0_hydro1."""
    tau = np.asarray(tau, dtype=float)
    br = 1.0 + 2.0 * tau_AW0 / 15.0 * (1.0 - tau ** (-2.0 / 3.0))
    return tau ** (-4.0 / 3.0) * br**4, -16.0 * tau_AW0 / (15.0 * tau**2) * br**3


def bjorken_hydro2_parton(tau, tau_AW0):
    """(P, Pi) of second-order hydrodynamics for the parton gas (Eq. bjorken_mu0_hydro2),
    integrated from P(1) = 1, Pi(1) = 0."""
    tau = np.asarray(tau, dtype=float)

    def rhs(t, y):
        P, Pi = y
        return [-4.0 * P / (3.0 * t) - Pi / (3.0 * t),
                -P**0.25 / tau_AW0 * Pi - 38.0 / 21.0 * Pi / t - 16.0 / 15.0 * P / t]

    sol = solve_ivp(rhs, (1.0, float(tau.max())), [1.0, 0.0], t_eval=tau, rtol=1e-11, atol=1e-13,
                    method="LSODA")
    return sol.y[0], sol.y[1]


HBARC_GEV_FM = 0.1973269804  # hbar c in GeV fm


def tau_aw0_bjorken(eta_s, T0_GeV, tau0_fm):
    """tau_AW0 = 5 hbar (eta/s) / (tau0 k_B T0) in units of tau0 (Eq. bjorken_tauAW)."""
    return 5.0 * HBARC_GEV_FM * eta_s / (tau0_fm * T0_GeV)


# ---------------------------------------------------------------------------
# Sec. IV B 2: integrated heat flux and shear stress near the inviscid limit
# ---------------------------------------------------------------------------
def dissipation_integrals(nL, TL, nR, TR, tau_coef_etas, lambda_ref=1.0, method="ce"):
    """Eqs. intq and intpi: the integrals of q over the contact and the shock
    and of Pi over the shock, from the inviscid plateau states (Eqs. Sod:PC -
    Sod:nII), T = P/n, the relative fugacity lambda_bar = P/T^4 = n/T^3,
    tau_AW = tau_AW0/T [1 - ln(lambda_bar lambda_ref)/4] (Eq. Sod:tau) and the
    Chapman-Enskog (eta = 4/5 P tau_AW, lambda_heat = 4/3 P tau_AW/T, Eq.
    tcoeff_ce) or Grad (2/3 and 4/5, Eq. tcoeff_grad) transport coefficients."""
    R = Riemann(nL, nL * TL, nR, nR * TR)
    PC, vC, vS = R.PC, R.beta_C, R.beta_shock
    gC2 = 1.0 / (1.0 - vC * vC)
    ce, cl = (4.0 / 5.0, 4.0 / 3.0) if method == "ce" else (2.0 / 3.0, 4.0 / 5.0)

    def state(n, P):
        T = P / n
        lam = n / T**3
        tau = tau_coef_etas / T * (1.0 - 0.25 * math.log(lam * lambda_ref))
        return T, lam, ce * P * tau, cl * P * tau / T

    T1, l1, e1, k1 = state(R.nI, PC)
    T2, l2, e2, k2 = state(R.nII, PC)
    TR_, lR, eR, kR = state(nR, nR * TR)
    q_c = (k1 * T1 + k2 * T2) * math.log(l2 / l1) / 8.0
    q_s = (kR * TR_ + k2 * T2 * gC2 * (1.0 - vC * vS)) * math.log(lR / l2) / 8.0
    pi_s = 2.0 * vC * math.sqrt(gC2) / 3.0 * (eR + e2 * (1.0 - vC * vS))
    return {"q_contact": q_c, "q_shock": q_s, "Pi_shock": pi_s, "zeta_C": vC, "zeta_S": vS}


# ---------------------------------------------------------------------------
# Sec. V C: semi-analytic solution of the relaxation-time Bjorken flow of a
# parton gas (Eqs. flork_sol, flork_sol_aux)
# ---------------------------------------------------------------------------
def _H(y):
    """H(y) = y^2 + arctan(sqrt(y^-2 - 1))/sqrt(y^-2 - 1) for 0 < y <= 1."""
    y = np.asarray(y, dtype=float)
    s = np.sqrt(np.maximum(1.0 / (y * y) - 1.0, 0.0))
    ss = np.where(s > 1e-4, s, 1.0)
    at = np.where(s > 1e-4, np.arctan(ss) / ss, 1.0 - s * s / 3.0 + s**4 / 5.0)
    return y * y + at


def _HL(y):
    """H_L(y) = y^2 d/dy [H(y)/y] = y H'(y) - H(y), with H' from its closed form:
    d/dy [arctan(s)/s] = (ds/dy)(1/(s (1 + s^2)) - arctan(s)/s^2), s = sqrt(y^-2 - 1),
    ds/dy = -1/(y^3 s)."""
    y = np.asarray(y, dtype=float)
    s = np.sqrt(np.maximum(1.0 / (y * y) - 1.0, 0.0))
    big = s > 1e-3
    ss = np.where(big, s, 1.0)
    dterm = np.where(big, (-1.0 / (y**3 * ss)) * (1.0 / (ss * (1.0 + ss * ss)) - np.arctan(ss) / ss**2),
                     # series of arctan(s)/s = 1 - s^2/3 + s^4/5 with s^2 = y^-2 - 1
                     (2.0 / (3.0 * y**3)) - (4.0 / 5.0) * (1.0 / y**2 - 1.0) / y**3)
    Hp = 2.0 * y + dterm
    return y * Hp - _H(y)


def florkowski_parton(tau_AW0, tau_f=40.0, dtau=0.04, tol=1e-7, max_iter=500):
    """(tau, T, n, P_L) of Eqs. flork_sol by the iteration the paper describes:
    T_(0) = tau^(-1/3), trapezoidal quadrature on an equidistant grid, stop
    when the L2 norm (over [1, tau_f]) of T_(n) - T_(n-1) is below tol.
    Parton gas: tau_AW = tau_AW0 / T, P = T^4."""
    tau = np.arange(1.0, tau_f + 0.5 * dtau, dtau)
    N = len(tau)
    T = tau ** (-1.0 / 3.0)

    def cumtrap(f):
        out = np.zeros(N)
        out[1:] = np.cumsum(0.5 * (f[1:] + f[:-1]) * dtau)
        return out

    H1 = _H(1.0)
    for _ in range(max_iter):
        I = cumtrap(T)  # int_1^tau T
        T4 = np.empty(N)
        src = T**4 * T / (2.0 * tau_AW0)  # T^4 / (2 tau_AW), tau_AW = tau_AW0 / T
        for i in range(N):
            D = np.exp(-(I[i] - I[: i + 1]) / tau_AW0)  # D(tau_i, tau')
            g = src[: i + 1] * D * _H(tau[: i + 1] / tau[i])
            integral = 0.5 * dtau * (g[1:] + g[:-1]).sum() if i > 0 else 0.0
            T4[i] = D[0] * _H(1.0 / tau[i]) / H1 + integral
        Tn = T4**0.25
        L2 = math.sqrt(_trap((Tn - T) ** 2, dtau) / (tau_f - 1.0))
        T = Tn
        if L2 <= tol:
            break
    I = cumtrap(T)
    n = np.empty(N)
    PL = np.empty(N)
    for i in range(N):
        D = np.exp(-(I[i] - I[: i + 1]) / tau_AW0)
        gn = T[: i + 1] ** 3 * tau[: i + 1] * T[: i + 1] / tau_AW0 * D
        gp = T[: i + 1] ** 5 / (2.0 * tau_AW0) * D * _HL(tau[: i + 1] / tau[i])
        In = 0.5 * dtau * (gn[1:] + gn[:-1]).sum() if i > 0 else 0.0
        Ip = 0.5 * dtau * (gp[1:] + gp[:-1]).sum() if i > 0 else 0.0
        n[i] = (D[0] + In) / tau[i]
        PL[i] = 3.0 * (D[0] * _HL(1.0 / tau[i]) / H1 + Ip)
    return tau, T, n, PL


def _trap(f, h):
    return float(0.5 * h * (f[1:] + f[:-1]).sum())
