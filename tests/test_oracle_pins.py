"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against an independent route: numbers printed in
the paper (tests/golden), closed forms (tests/exact.py), library routines
(scipy), invariants, or brute-force integration.  None of these tests needs a
GPU.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

import oracle
from tests import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- quadrature
def test_table1_laguerre_nodes_and_weights():
    g = _golden("table1_laguerre_QL2.json")
    x, w = oracle.gauss_laguerre2(g["Q_L"])
    np.testing.assert_allclose(x, g["nodes"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(w, g["weights"], rtol=0, atol=1e-14)


def test_laguerre_polynomial_explicit_sum():
    """L_l^{(2)} against the explicit sum of Eq. lag_expl, in exact rationals."""
    from fractions import Fraction
    for l in range(0, 7):
        for x in (Fraction(0), Fraction(1, 3), Fraction(5, 2), Fraction(7)):
            ref = sum((-x) ** s * math.factorial(l + 2) /
                      Fraction(math.factorial(s) * math.factorial(s + 2) * math.factorial(l - s))
                      for s in range(l + 1))
            assert abs(oracle.laguerre2(l, float(x)) - float(ref)) < 1e-13 * max(1, abs(float(ref)))


@pytest.mark.parametrize("Q", [2, 3, 4, 6, 8])
def test_laguerre_matches_scipy_and_moments(Q):
    x, w = oracle.gauss_laguerre2(Q)
    xs, ws = sp.roots_genlaguerre(Q, 2)
    np.testing.assert_allclose(x, xs, rtol=1e-13)
    # the paper's weights integrate e^{-x} x^2 (scipy's convention too)
    np.testing.assert_allclose(w, ws, rtol=1e-12)
    # exact for polynomial degree < 2Q: int e^{-x} x^{2+s} = (s+2)!
    for s in range(2 * Q):
        assert abs(np.sum(w * x**s) / math.factorial(s + 2) - 1) < 1e-12


@pytest.mark.parametrize("Q", [1, 2, 3, 8, 20, 50, 200, 512])
def test_legendre_matches_scipy_and_moments(Q):
    x, w = oracle.gauss_legendre(Q)
    xs, ws = sp.roots_legendre(Q)
    np.testing.assert_allclose(x, xs, rtol=0, atol=2e-15)
    # scipy's own weights are good to ~1e-12 (1e-8 at high Q); the tight pin is
    # the 40-digit check below
    np.testing.assert_allclose(w, ws, rtol=1e-8 if Q > 100 else 1e-11, atol=0)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_array_equal(x, -x[::-1])
    np.testing.assert_array_equal(w, w[::-1])
    for r in range(0, min(2 * Q, 40), 2):
        assert abs(np.sum(w * x**r) - 2.0 / (r + 1)) < 1e-13


@pytest.mark.parametrize("Q", [50, 200, 1000])
def test_legendre_against_40_digit_newton(Q):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, w = oracle.gauss_legendre(Q)
    for i in [0, 1, Q // 3, Q // 2]:
        z = mp.mpf(x[i])
        for _ in range(6):
            p = mp.legendre(Q, z)
            z -= p / (Q * (z * p - mp.legendre(Q - 1, z)) / (z * z - 1))
        wm = 2 * (1 - z * z) / ((Q + 1) * mp.legendre(Q + 1, z)) ** 2
        assert abs(float(z) - x[i]) <= 2.3e-16
        # conditioning of 1 - x^2 at the edge node limits the weight to ~1e-11
        assert abs(float(wm / w[i]) - 1) < 5e-11


# ------------------------------------------------------- f^eq coefficients
@pytest.mark.parametrize("u", [1.0, 2.0, 5.0])
@pytest.mark.parametrize("theta", [0.4, 1.0, 1.7])
def test_aeq_against_appendix_a_closed_forms(u, theta):
    n = 0.83
    a = oracle.aeq(n, theta, u, 6)
    for l in (0, 1):
        for s in range(7):
            ref = exact.a_from_tilde(n, l, u, exact.a_tilde_closed(l, s, u, theta))
            assert abs(a[l, s] - ref) <= 1e-12 * abs(a[0, 0]), (l, s)


@pytest.mark.parametrize("u", [1e-3, 3e-3, 1e-2])
def test_aeq_against_appendix_a_series(u):
    n, theta = 1.3, 0.7
    a = oracle.aeq(n, theta, u, 6)
    for l in (0, 1):
        for s in range(7):
            ref = exact.a_from_tilde(n, l, u, exact.a_tilde_series(l, s, u, theta))
            # series truncation O(u^12); round-off relative to a_00
            assert abs(a[l, s] - ref) <= 2e-15 * abs(a[0, 0]) + 1e-13 * abs(ref), (l, s)


@pytest.mark.parametrize("u", [1e-4, 1e-2, 0.3, 1.0, 2.0, 5.0, 20.0, 50.0])
def test_sixteen_node_rule_reproduces_aeq(u):
    """The FP32 stage kernels evaluate a_{l,m} (N_Omega <= 7) with a 16-node
    Gauss-Legendre rule in s = A t after the substitution u0 - u cos(gamma) =
    e^{-s} (Eq. aeq_aux): J3_m = int e^{2s} P_m(c), J4_m = int e^{3s} P_m(c),
    a_{0,m} = n (A/u) J3_m / (4 pi), a_{1,m} = 3 n (A/u) (J3_m - theta J4_m) / (4 pi).
    Written out here in numpy, that rule matches the oracle to 2e-14 of a_{l,0}
    for u <= 20 and to 5e-13 at u = 50 (beta = 0.9998), far inside FP32."""
    from numpy.polynomial.legendre import leggauss
    n, theta, nomega = 1.3, 0.8, 7
    t, w = leggauss(16)
    A = math.asinh(u)
    s = A * t
    c = (2.0 * math.sinh(A / 2) ** 2 - np.expm1(-s)) / u
    e1 = np.exp(s)
    w3 = w * e1 * e1
    w4 = w3 * e1
    P = np.zeros((nomega + 1, t.size))
    P[0] = 1.0
    P[1] = c
    for m in range(1, nomega):
        P[m + 1] = ((2 * m + 1) * c * P[m] - m * P[m - 1]) / (m + 1)
    J3, J4 = P @ w3, P @ w4
    got = np.vstack([n * (A / u) * J3, 3.0 * n * (A / u) * (J3 - theta * J4)]) / (4.0 * math.pi)
    ref = oracle.aeq(n, theta, u, nomega)
    tol = 3e-14 if u <= 20.0 else 1e-12
    assert np.abs(got - ref).max() <= tol * np.abs(ref[:, 0]).max()


def test_aeq_at_rest_and_leading_order():
    a = oracle.aeq(2.0, 0.6, 0.0, 6)
    assert abs(a[0, 0] - 2.0 / (2 * math.pi)) < 1e-15
    assert abs(a[1, 0] - 6 * 2.0 * 2 * (1 - 0.6) / (8 * math.pi)) < 1e-15
    assert np.abs(a[:, 1:]).max() < 1e-15 * a[0, 0]
    # leading term of a_{l,m} is O((u/u0)^m) (Sec. III D)
    r = [oracle.aeq(1.0, 1.0, u, 6)[0, 4] for u in (1e-2, 2e-2)]
    assert abs(r[1] / r[0] - 16.0) < 1e-2


def test_aeq_brute_force_integral():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for (u, theta) in [(0.3, 0.8), (0.9, 1.2), (2.5, 0.5)]:
        a = oracle.aeq(1.0, theta, u, 12)
        u0 = math.sqrt(1 + u * u)
        for l in (0, 1):
            # up to the largest truncation order the kernels accept (N_Omega = 12)
            for m in (0, 2, 5, 7, 9, 12):
                f = lambda c: (u0 - u * c) ** -3 * (1 - theta / (u0 - u * c)) ** l * mp.legendre(m, c)
                ref = (l + 1) * (l + 2) / (8 * mp.pi) * mp.quad(f, [-1, 0, 1])
                assert abs(a[l, m] - float(ref)) < 1e-13 * abs(a[0, 0])


# ------------------------------------------------------------ MJ moments
def _mj_moments(n, T, beta):
    g = 1 / math.sqrt(1 - beta * beta)
    P = n * T
    E = 3 * P
    return np.array([n * g, n * g * beta, (E + P) * g * g - P, (E + P) * g * g * beta,
                     (E + P) * g * g * beta * beta + P])


@pytest.mark.parametrize("QL", [2, 3])
@pytest.mark.parametrize("NO", [2, 5, 12])
@pytest.mark.parametrize("state", [(1.0, 1.0, 0.0), (0.125, 0.8, 0.6), (0.4, 0.5, -0.9),
                                   (2.0, 1.6, 0.95)])
def test_truncated_feq_reproduces_mj_moments(QL, NO, state):
    """N^mu = n u^mu and T^{mu nu} = (E+P) u u + P eta with E = 3P = 3nT, exactly
    from the truncated f^eq on the discrete set (Sec. III B-E)."""
    n, T, beta = state
    Qx = max(NO + 1, 6)
    f = oracle.feq(Qx, QL, NO, n, T, beta)
    M = oracle.moments(Qx, QL, f)
    ref = _mj_moments(n, T, beta)
    np.testing.assert_allclose(M, ref, rtol=2e-14, atol=2e-14 * abs(ref).max())
    L = oracle.landau(M)
    # the printed Landau formula cancels as |beta| -> 1 (Eq. E_landau)
    tol = 1e-13 / (1 - abs(beta))
    assert abs(L["n"] / n - 1) < tol
    assert abs(L["T"] / T - 1) < tol
    assert abs(L["beta"] - beta) < tol
    assert abs(L["E"] - 3 * L["P"]) < 1e-14 * L["E"]
    assert abs(L["Pi"]) < 1e-12 * L["E"] and abs(L["q"]) < 1e-12 * L["E"]


def test_feq_rest_frame_special_case():
    """At beta = 0: f^eq_jk = (n w_j w_k /4)[1 + (3 - x_k)(1 - T)], the u = 0 case
    of Eqs. feq_trunc and fjk with L_1^{(2)}(x) = 3 - x."""
    Qx, QL = 7, 3
    xj, wj = sp.roots_legendre(Qx)
    xk, wk = sp.roots_genlaguerre(QL, 2)
    n, T = 0.7, 1.4
    f = oracle.feq(Qx, QL, 5, n, T, 0.0).reshape(QL, Qx)
    ref = n * np.outer(wk * (1 + (3 - xk) * (1 - T)), wj) / 4
    np.testing.assert_allclose(f, ref, rtol=1e-13)


def test_brute_force_moments_on_tiny_velocity_set():
    """Quadrature sums of the populations equal the continuum integrals of
    Eq. momsr for f = truncated f^eq, by adaptive integration (Q_xi=3, Q_L=2)."""
    n, T, beta, NO = 0.9, 0.7, 0.45, 2
    Qx, QL = 3, 2
    g = 1 / math.sqrt(1 - beta**2)
    u = g * abs(beta)
    a = oracle.aeq(n, T, u, NO)

    def f(p, xi):  # truncated f^eq of Eq. feq_trunc, T0 = 1
        L = [1.0, 3.0 - p]
        s = 0.0
        for l in (0, 1):
            s += L[l] / ((l + 1) * (l + 2)) * sum(
                (2 * m + 1) / 2 * a[l, m] * sp.eval_legendre(m, xi) for m in range(NO + 1))
        return math.exp(-p) * s

    fpop = oracle.feq(Qx, QL, NO, n, T, beta)
    xj, _ = oracle.gauss_legendre(Qx)
    xk, _ = oracle.gauss_laguerre2(QL)
    for (s, r) in [(0, 0), (0, 1), (1, 0), (1, 1), (1, 2)]:
        cont, _ = integrate.dblquad(lambda p, xi: 2 * math.pi * p ** (s + 2) * xi**r * f(p, xi),
                                    -1, 1, 0, 60, epsabs=1e-13, epsrel=1e-12)
        disc = sum(fpop[k * Qx + j] * xj[j] ** r * xk[k] ** s for k in range(QL) for j in range(Qx))
        assert abs(disc - cont) < 1e-10 * abs(cont) + 1e-12


# -------------------------------------------------------------- Landau
def test_landau_factored_vs_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    f = oracle.feq(20, 3, 5, 0.3, 0.9, 0.8)
    M = oracle.moments(20, 3, f)
    L = oracle.landau(M)
    Nt, Nz, Ttt, Ttz, Tzz = [mp.mpf(v) for v in M]
    E = (Ttt - Tzz + mp.sqrt((Ttt + Tzz) ** 2 - 4 * Ttz**2)) / 2
    b = Ttz / (E + Tzz)
    nn = (Nt - b * Nz) / mp.sqrt(1 - b * b)
    assert abs(L["E"] / float(E) - 1) < 1e-14
    assert abs(L["beta"] - float(b)) < 1e-14
    assert abs(L["n"] / float(nn) - 1) < 1e-14


def test_landau_rejects_nonphysical():
    with pytest.raises(oracle.OracleError):
        oracle.landau(np.array([1.0, 0.0, -1.0, 0.0, 0.5]))
    with pytest.raises(oracle.OracleError):
        oracle.landau(np.array([-1.0, 0.0, 3.0, 0.0, 1.0]))


def _rest_populations(Qx, QL, shape):
    """Populations w_j w_k/4 [1 + shape(x_k, xi_j)] on scipy's nodes: the rest-frame
    equilibrium n = T = 1 (Eq. fjk) times a chosen perturbation."""
    xj, wj = sp.roots_legendre(Qx)
    xk, wk = sp.roots_genlaguerre(QL, 2)
    X, XI = np.meshgrid(xk, xj, indexing="ij")  # [k][j], v = k*Qx + j
    return (np.outer(wk, wj) / 4.0 * (1.0 + shape(X, XI))).ravel()


@pytest.mark.parametrize("a", [0.3, -0.45])
def test_landau_shear_stress_at_rest_closed_form(a):
    """f = f^eq_rest (1 + a P_2(xi)): by hand, N^t = 1, N^z = T^tz = 0, T^tt = 3,
    T^zz = (3/2)(2/3 + 4a/15) = 1 + 2a/5 (int xi^2 P_2 = 4/15), so the Landau
    frame is at rest with n = 1, E = 3, P = T = 1, and Pi = T^zz - P = 2a/5
    (Eq. pi_val with T^tt = E), q = 0 (Eq. q_val with N^z = 0)."""
    Qx, QL = 6, 3
    f = _rest_populations(Qx, QL, lambda x, xi: a * 0.5 * (3 * xi**2 - 1))
    L = oracle.landau(oracle.moments(Qx, QL, f))
    assert abs(L["Pi"] - 0.4 * a) < 1e-14
    assert abs(L["q"]) < 1e-14
    assert abs(L["beta"]) < 1e-15
    for k, v in (("n", 1.0), ("E", 3.0), ("P", 1.0), ("T", 1.0), ("gamma", 1.0)):
        assert abs(L[k] - v) < 1e-14, (k, L[k])


@pytest.mark.parametrize("b", [0.2, -0.35])
def test_landau_heat_flux_at_rest_closed_form(b):
    """f = f^eq_rest (1 + b (x - 4) xi): the radial factor makes T^tz vanish
    (int e^-x x^3 (x - 4) = 24 - 24 = 0), so beta = 0, while
    N^z = (b/4)(int e^-x x^2 (x - 4))(2/3) = (b/4)(-2)(2/3) = -b/3.  With n = T = 1,
    q = -4T(N^z - n beta gamma) = 4b/3 and Pi = 0 (T^tt = 3, T^zz = 1)."""
    Qx, QL = 6, 3
    f = _rest_populations(Qx, QL, lambda x, xi: b * (x - 4.0) * xi)
    M = oracle.moments(Qx, QL, f)
    assert abs(M[3]) < 1e-14 and abs(M[1] + b / 3.0) < 1e-14
    L = oracle.landau(M)
    assert abs(L["q"] - 4.0 * b / 3.0) < 1e-14
    assert abs(L["Pi"]) < 1e-14
    assert abs(L["beta"]) < 1e-15
    assert abs(L["n"] - 1.0) < 1e-14 and abs(L["T"] - 1.0) < 1e-14


def _boost(M, v):
    """Moments (N^t, N^z, T^tt, T^tz, T^zz) seen from a frame moving with velocity v
    along z: N' = Lambda N, T' = Lambda T Lambda^T."""
    g = 1.0 / math.sqrt(1.0 - v * v)
    Lm = np.array([[g, -g * v], [-g * v, g]])
    N = Lm @ np.array([M[0], M[1]])
    T = Lm @ np.array([[M[2], M[3]], [M[3], M[4]]]) @ Lm.T
    return np.array([N[0], N[1], T[0, 0], T[0, 1], T[1, 1]])


@pytest.mark.parametrize("v", [0.3, -0.7, 0.9])
def test_landau_lorentz_covariance_off_equilibrium(v):
    """An anisotropic, heat-conducting state with q and Pi far from zero, seen from a
    boosted frame.  n, E, P, T and Pi are Lorentz scalars (Pi^{ab} = Pi (z^a z^b -
    transverse/2) with the unit vector z = gamma(beta, 0, 0, 1)); q^a = q (beta, 0, 0, 1)
    = (q/gamma) z^a, so q/gamma is the invariant; beta adds relativistically.  The
    printed heat flux must also satisfy q^a = -4T (N^a - n u^a) in its time component
    (Eq. qL with E + P = 4nT), which Eq. q_val does not use, and n = u_a N^a."""
    Qx, QL = 10, 3
    f = _rest_populations(Qx, QL, lambda x, xi: 0.3 * 0.5 * (3 * xi**2 - 1) +
                          0.2 * (x - 4.0) * xi + 0.1 * xi)
    M = oracle.moments(Qx, QL, f)
    L0 = oracle.landau(M)
    assert abs(L0["Pi"]) > 0.05 and abs(L0["q"]) > 0.05 and abs(L0["beta"]) > 1e-3
    for ref in (L0, oracle.landau(_boost(M, v))):
        Mr = M if ref is L0 else _boost(M, v)
        g, b, n, T = ref["gamma"], ref["beta"], ref["n"], ref["T"]
        assert abs(ref["q"] * b + 4.0 * T * (Mr[0] - n * g)) < 1e-13
        assert abs(n - g * (Mr[0] - b * Mr[1])) < 1e-13
    L1 = oracle.landau(_boost(M, v))
    for k in ("n", "E", "P", "T"):
        assert abs(L1[k] / L0[k] - 1.0) < 1e-13, (k, L0[k], L1[k])
    assert abs(L1["Pi"] - L0["Pi"]) < 1e-13 * L0["E"]
    assert abs(L1["q"] / L1["gamma"] - L0["q"] / L0["gamma"]) < 1e-13 * L0["E"]
    b0 = L0["beta"]
    assert abs(L1["beta"] - (b0 - v) / (1.0 - b0 * v)) < 1e-14


# -------------------------------------------------------------- WENO5
def test_weno_constant_and_quadratic_exactness():
    assert oracle.weno5_face(0.3, 0.3, 0.3, 0.3, 0.3) == pytest.approx(0.3, abs=1e-16)
    # cell averages of a quadratic: every candidate reconstructs the face value
    # exactly, so the flux is exact whatever the weights (Sec. III F)
    h = 0.1
    P = lambda z: 1.3 - 0.7 * z + 2.1 * z * z
    prim = lambda z: 1.3 * z - 0.35 * z * z + 0.7 * z**3
    avg = [(prim((s + 0.5) * h) - prim((s - 0.5) * h)) / h for s in (-2, -1, 0, 1, 2)]
    assert oracle.weno5_face(*avg) == pytest.approx(P(0.5 * h), rel=1e-13)


def test_weno_limit_rules():
    # rule (iii): sigma_1 = 0 only (J_{s-2} = J_{s-1} = J_s): all weight on F^1,
    # which reproduces the constant exactly however steep the data downwind
    assert oracle.weno5_face(2.0, 2.0, 2.0, 10.0, -4.0) == pytest.approx(2.0, rel=1e-15)
    # rule (ii): sigma_1 = sigma_2 = 0, sigma_3 != 0: F^3 gets weight 0
    assert oracle.weno5_face(1.5, 1.5, 1.5, 1.5, 50.0) == pytest.approx(1.5, rel=1e-15)
    # rule (i): all sigma equal (linear data: sigma_q = 1) -> ideal weights; every
    # candidate is exact on linear data, so the face value is 2.5
    assert oracle.weno5_face(0.0, 1.0, 2.0, 3.0, 4.0) == pytest.approx(2.5, rel=1e-15)
    # general case: sigma_q > 0 with a jump downwind -> the weight of the stencil
    # across the jump is tiny, so the flux stays near the smooth upwind values
    v = oracle.weno5_face(1.0, 1.1, 1.2, 5.0, 5.0)
    assert 1.2 < v < 1.3


def _advect_error(Z, order_check=False):
    """Linear advection on a periodic domain with collisions off: populations are
    translated exactly by xi_j t; WENO5 + RK3 must converge at high order."""
    Qx, QL = 2, 2
    p = oracle.sod_params(Z, Qx, QL, N_Omega=1, z_min=0.0, z_max=1.0, bc="periodic",
                          tau_mode="none", dt=0.2 / Z)
    xi, _ = oracle.gauss_legendre(Qx)
    zc = (np.arange(Z) + 0.5) / Z
    h = 1.0 / Z
    # cell averages of 1 + 0.3 sin(2 pi z) per population
    avg = lambda c: 1 + 0.3 * (np.cos(2 * np.pi * (c - h / 2)) - np.cos(2 * np.pi * (c + h / 2))) / (2 * np.pi * h)
    f0 = np.stack([avg(zc)] * (Qx * QL), axis=1)
    nsteps = Z // 2
    t = nsteps * p.dt
    f = oracle.sod_steps(p, f0, nsteps)
    err = 0.0
    for v in range(Qx * QL):
        ref = avg(zc - xi[v % Qx] * t)
        err = max(err, np.abs(f[:, v] - ref).max())
    return err


def test_weno_rk3_advection_convergence():
    e1, e2 = _advect_error(40), _advect_error(80)
    # fifth order in space at fixed CFL (RK3 error is smaller at this CFL)
    assert e2 < e1 / 2**4.2, (e1, e2)


# ------------------------------------------------------- K^L and K^P
@pytest.mark.parametrize("Q", [8, 20, 64])
def test_kp_exact_on_polynomials(Q):
    """K^P applied to populations w_j g(xi_j) gives w_j d/dxi[xi(1-xi^2) g] at the
    nodes, exactly for g = xi^d with d <= Q-4 (Eqs. f_leg_force_K, K_leg_disc)."""
    K = oracle.kp_matrix(Q)
    x, w = oracle.gauss_legendre(Q)
    for d in range(0, Q - 3):
        out = K @ (w * x**d)
        ref = w * ((d + 1) * x**d - (d + 3) * x ** (d + 2))
        assert np.abs(out - ref).max() < 1e-10 * max(1.0, np.abs(ref).max()) * Q, d


def test_kl_qL2_closed_form():
    """Eq. K_lag_disc1: K^L_{kk'} = w_k (3 - x_k) x_k' / 6 for Q_L = 2."""
    K = oracle.kl_matrix(2)
    x, w = oracle.gauss_laguerre2(2)
    np.testing.assert_allclose(K, np.outer(w * (3 - x), x) / 6, rtol=1e-14)


@pytest.mark.parametrize("QL", [2, 3, 4])
def test_kl_exact_on_polynomials(QL):
    """K^L applied to populations 2 pi w_k q(x_k) (f = e^{-p} q(p)) reproduces
    (1/p^2) d(f p^3)/dp = e^{-p}[3q + p q' - p q] for deg q <= Q_L - 2."""
    K = oracle.kl_matrix(QL)
    x, w = oracle.gauss_laguerre2(QL)
    for d in range(0, QL - 1):
        q = x**d
        dq = d * x ** max(d - 1, 0) if d > 0 else 0 * x
        ref = w * (3 * q + x * dq - x * q)
        np.testing.assert_allclose(K @ (w * q), ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------- Sod: invariants, limits
def _smooth_periodic_state(Z):
    zc = (np.arange(Z) + 0.5) / Z
    n = 1 + 0.3 * np.sin(2 * np.pi * zc)
    T = 1 + 0.2 * np.cos(2 * np.pi * zc)
    b = 0.4 * np.sin(4 * np.pi * zc)
    return n, T, b


@pytest.mark.parametrize("NO", [2, 5])
def test_sod_conservation_periodic(NO):
    """sum_s N^t, T^tt, T^tz are conserved to round-off on a periodic domain
    (Eqs. cons, collinv; requires N_Omega >= 2)."""
    Z = 48
    p = oracle.sod_params(Z, 8, 3, N_Omega=NO, z_min=0.0, z_max=1.0, bc="periodic",
                          tau_mode="const", tau=2e-3, dt=1e-3)
    f = oracle.sod_init_fields(p, *_smooth_periodic_state(Z))
    m0 = oracle.sod_moments(p, f)
    f = oracle.sod_steps(p, f, 60)
    m1 = oracle.sod_moments(p, f)
    for k in ("Nt", "Ttt", "Ttz"):
        assert abs(m1[k].sum() - m0[k].sum()) < 1e-13 * np.abs(m0[k]).sum(), k
    # and the state really evolved
    assert np.abs(m1["beta"] - m0["beta"]).max() > 1e-3


def test_sod_uniform_state_is_stationary():
    p = oracle.sod_params(16, 6, 2, bc="outflow", tau=1e-2, dt=1e-3,
                          left=(0.5, 0.9, 0.3), right=(0.5, 0.9, 0.3))
    f = oracle.sod_init_riemann(p)
    L = oracle.sod_rhs(p, f)
    assert np.abs(L).max() < 1e-12 * np.abs(f).max() / p.dt


def test_sod_mirror_symmetry():
    """z -> -z with xi_j -> -xi_j maps solutions to solutions."""
    Z, Qx = 32, 6
    p = oracle.sod_params(Z, Qx, 2, bc="outflow", tau=5e-3, dt=1e-3, left=(1, 1, 0),
                          right=(0.125, 0.8, 0))
    q = oracle.sod_params(Z, Qx, 2, bc="outflow", tau=5e-3, dt=1e-3, left=(0.125, 0.8, 0),
                          right=(1, 1, 0))
    f = oracle.sod_steps(p, oracle.sod_init_riemann(p), 40)
    g = oracle.sod_steps(q, oracle.sod_init_riemann(q), 40)
    fm = f.reshape(Z, 2, Qx)[::-1, :, ::-1].reshape(Z, -1)
    np.testing.assert_allclose(g, fm, rtol=0, atol=1e-14 * np.abs(f).max())


@pytest.mark.slow
def test_sod_inviscid_limit_plateau():
    """Small tau: the plateau values approach the exact inviscid Riemann
    solution of Sec. IV B 1 (state of the shock-tube workload)."""
    Z = 400
    p = oracle.sod_params(Z, 8, 2, N_Omega=5, bc="fixed_eq", tau_mode="const", tau=1e-3,
                          dt=5e-4, left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0))
    f = oracle.sod_steps(p, oracle.sod_init_riemann(p), 800)
    t = 800 * p.dt
    m = oracle.sod_moments(p, f)
    R = exact.Riemann(1.0, 1.0, 0.125, 0.1)
    zc = -1 + (np.arange(Z) + 0.5) * 2 / Z
    for zeta, key, ref in [(0.5 * (R.zeta_T + R.beta_C), "n", R.nI),
                           (0.5 * (R.beta_C + R.beta_shock), "n", R.nII),
                           (0.5 * (R.zeta_T + R.beta_shock), "P", R.PC),
                           (0.5 * (R.zeta_T + R.beta_shock), "beta", R.beta_C)]:
        s = np.argmin(abs(zc - zeta * t))
        assert abs(m[key][s] / ref - 1) < 0.02, (key, m[key][s], ref)
    # L1 distance of the density profile to the exact one is a few percent
    n_ex, _, _ = R.profile(zc, t)
    assert np.mean(np.abs(m["n"] - n_ex)) < 0.01


def test_exact_riemann_matches_printed_values():
    g = _golden("sod_inviscid_plateau_paper_state.json")
    R = exact.Riemann(g["left"]["n"], g["left"]["P"], g["right"]["n"], g["right"]["P"])
    tol = 0.5 * 10 ** -g["printed_digits"]
    for k, v in [("beta_shock", R.beta_shock), ("beta_C", R.beta_C), ("P_C", R.PC),
                 ("n_I", R.nI), ("n_II", R.nII), ("zeta_T", R.zeta_T), ("zeta_H", -exact.CS)]:
        assert abs(v - g[k]) <= tol + 1e-12, (k, v, g[k])


def _free_stream_exact(p, f0_left, f0_right, t):
    """Discrete-velocity free streaming: every population is its initial step
    translated by xi_j t, averaged over each cell."""
    Z = p.Z
    dz = (p.z_max - p.z_min) / Z
    xi, _ = oracle.gauss_legendre(p.Q_xi)
    lo = p.z_min + np.arange(Z) * dz
    out = np.zeros((Z, p.Q_xi * p.Q_L))
    for v in range(p.Q_xi * p.Q_L):
        front = xi[v % p.Q_xi] * t  # the step sits at z = xi_j t
        frac_left = np.clip((front - lo) / dz, 0.0, 1.0)
        out[:, v] = frac_left * f0_left[v] + (1 - frac_left) * f0_right[v]
    return out


def test_sod_ballistic_discrete_exact_and_continuum():
    """Collisionless limit (Sec. IV C): WENO5-RK3 converges to the exact
    discrete free-streaming solution as Z grows, and its moments approach the
    continuum solution of Eqs. Sod:bal:Nmu, Sod:bal:Tmunu as Q_xi grows."""
    errs = []
    for Z in (100, 200):
        p = oracle.sod_params(Z, 16, 2, bc="fixed_eq", tau_mode="none", dt=0.25 / Z,
                              z_min=-0.5, z_max=0.5, left=(1, 1, 0), right=(0.125, 0.5, 0))
        f0 = oracle.sod_init_riemann(p)
        nst = Z // 2
        f = oracle.sod_steps(p, f0, nst)
        ex = _free_stream_exact(p, f0[0], f0[-1], nst * p.dt)
        errs.append(np.abs(f - ex).sum() / Z)
    assert errs[1] < 0.7 * errs[0], errs

    Z, Qx = 200, 100
    p = oracle.sod_params(Z, Qx, 2, bc="fixed_eq", tau_mode="none", dt=0.25 / Z,
                          z_min=-0.5, z_max=0.5, left=(1, 1, 0), right=(0.125, 0.5, 0))
    nst = 120
    f = oracle.sod_steps(p, oracle.sod_init_riemann(p), nst)
    t = nst * p.dt
    zc = -0.5 + (np.arange(Z) + 0.5) / Z
    m = oracle.sod_moments(p, f)
    ref = exact.ballistic_sod(zc / t, 1.0, 1.0, 0.125, 0.0625)
    for key, r in zip(("Nt", "Nz", "Ttt", "Ttz", "Tzz"), ref):
        assert np.mean(np.abs(m[key] - r)) < 0.01 * np.abs(r).max(), key


# ---------------------------------------------------------------- Bjorken
def test_bjorken_ballistic_and_density():
    """Free streaming (Eq. bjorken_bal) and n tau = 1 (Eq. bjorken_n)."""
    p = oracle.bjorken_params(40, 2, N_Omega=5, gas="ideal", tau_AW0=math.inf, dtau=1e-2)
    _, h = oracle.bjorken_run(p, 400)
    assert np.abs(h["n"] * h["tau"] - 1).max() < 1e-12
    P, PL = exact.bjorken_ballistic(h["tau"])
    sel = h["tau"] >= 1.5
    assert np.abs(h["P"][sel] / P[sel] - 1).max() < 2e-3
    assert np.abs(h["PL"][sel] / PL[sel] - 1).max() < 2e-2
    # P_L = P + Pi (Eq. bjorken_P)
    np.testing.assert_allclose(h["PL"], h["P"] + h["Pi"], rtol=1e-13)


def test_bjorken_ideal_gas_density_exact_in_collisions():
    p = oracle.bjorken_params(6, 2, N_Omega=5, gas="ideal", tau_AW0=0.3, dtau=1e-2)
    _, h = oracle.bjorken_run(p, 300)
    assert np.abs(h["n"] * h["tau"] - 1).max() < 1e-12


def test_bjorken_ideal_cooling_hydro_limit():
    """Inviscid limit (Eq. bjorken_inv): T tau^{1/3} -> 1."""
    p = oracle.bjorken_params(20, 3, gas="parton", tau_AW0=2e-3, dtau=5e-4)
    _, h = oracle.bjorken_run(p, 4000)
    Ttau = h["T"] * h["tau"] ** (1 / 3)
    assert abs(Ttau[-1] - 1) < 5e-3
    # first-order hydro (Eq. bjorken_mu0_hydro1) is closer still
    P1, _ = exact.bjorken_hydro1_parton(h["tau"][-1], 2e-3)
    assert abs(h["P"][-1] / P1 - 1) < 2e-3


def test_bjorken_second_order_hydro():
    """4 pi eta/s = 0.3, T0 = 0.6 GeV: second-order hydrodynamics
    (Eq. bjorken_mu0_hydro2) tracks the kinetic P within a few per mille."""
    t0 = exact.tau_aw0_bjorken(0.3 / (4 * math.pi), 0.6, 0.25)
    p = oracle.bjorken_params(40, 2, gas="parton", tau_AW0=t0, dtau=1e-3)
    _, h = oracle.bjorken_run(p, 4000)
    P2, Pi2 = exact.bjorken_hydro2_parton(h["tau"], t0)
    sel = h["tau"] > 2.0
    assert np.abs(h["P"][sel] / P2[sel] - 1).max() < 1e-2
    assert np.abs(h["Pi"][sel] - Pi2[sel]).max() < 0.1 * np.abs(Pi2[sel]).max()


def test_bjorken_rk3_third_order():
    p = lambda dt: oracle.bjorken_params(12, 2, gas="parton", tau_AW0=0.5, dtau=dt)
    _, href = oracle.bjorken_run(p(1.25e-3), 1600)
    errs = []
    for dt, ns in [(4e-2, 50), (2e-2, 100)]:
        _, h = oracle.bjorken_run(p(dt), ns)
        errs.append(abs(h["P"][-1] - href["P"][-1]))
    assert 6.0 < errs[0] / errs[1] < 10.0, errs


# ------------------------------------------- Florkowski semi-analytic Bjorken
def test_florkowski_solution_free_streaming_limit():
    """Eqs. flork_sol with tau_AW0 -> infinity reduce to the ballistic solution
    (Eq. bjorken_bal): T^4 = P, P_L as printed, n tau = 1."""
    tau, T, n, PL = exact.florkowski_parton(1e8, tau_f=5.0, dtau=0.01)
    P, PLb = exact.bjorken_ballistic(tau)
    assert np.abs(T**4 - P).max() < 1e-7
    assert np.abs(PL - PLb).max() < 1e-6
    assert np.abs(n * tau - 1.0).max() < 1e-6


@pytest.mark.parametrize("eta_s_4pi", [1.0, 3.0, 10.0])
def test_bjorken_parton_matches_florkowski_semianalytic(eta_s_4pi):
    """Transition regime (Sec. V C, Fig. bjorken_flork): the FP64 oracle with
    Q_xi = 40, Q_L = 3, dtau = 1e-3 against the iterative solution of Eqs.
    flork_sol (T0 = 0.3 GeV, tau0 = 0.5 fm/c, tau to 10): T, n and P_L/P_T."""
    t0 = exact.tau_aw0_bjorken(eta_s_4pi / (4 * math.pi), 0.3, 0.5)
    tau, T, n, PL = exact.florkowski_parton(t0, tau_f=10.0, dtau=0.01)
    p = oracle.bjorken_params(40, 3, gas="parton", tau_AW0=t0, dtau=1e-3)
    _, h = oracle.bjorken_run(p, 9000)
    idx = np.round((tau - 1.0) / 1e-3).astype(int)
    PT = (3 * T**4 - PL) / 2
    assert np.abs(h["T"][idx] / T - 1).max() < 1e-4
    assert np.abs(h["n"][idx] / n - 1).max() < 2e-4
    assert np.abs(h["PL"][idx] / h["PT"][idx] - PL / PT).max() < 1e-4
