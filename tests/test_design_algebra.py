"""CPU checks of formulas the GPU kernels use in place of the paper's printed
ones, each against the oracle on the same populations: the five direct sums
of the output-moment kernel and the identities that give N^mu, T^{mu nu}
from them (Eq. macro_jk), and the factored Landau matching with a single
FP64 reciprocal (Sec. II E, Eqs. E_landau-pi_val)."""
import math

import numpy as np
import pytest

import oracle

Q_XI, Q_L = 20, 3


def _velocities():
    xi, _ = oracle.gauss_legendre(Q_XI)
    xk, _ = oracle.gauss_laguerre2(Q_L)
    return np.tile(xi, Q_L), np.repeat(xk, Q_XI)  # v = k Q_xi + j, p_k = x_k (T0 = 1)


def _state(n, T, beta, seed):
    f = oracle.feq(Q_XI, Q_L, 5, n, T, beta)
    rng = np.random.default_rng(seed)
    return f * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, f.size))  # off equilibrium


def _direct_sums(f):
    """N+-, A+-, D summed directly with non-negative weights."""
    x, p = _velocities()
    return ((f * (1 + x)).sum(), (f * (1 - x)).sum(), (f * p * (1 + x) ** 2).sum(),
            (f * p * (1 - x) ** 2).sum(), (f * p * (1 - x) * (1 + x)).sum())


def _landau_one_division(Np, Nm, Ap, Am, D):
    """The GPU's Landau matching: one reciprocal r = 1/(sqrt(ab) (a+b) X)."""
    a, b = math.sqrt(Ap), math.sqrt(Am)
    ab, apb = a * b, a + b
    sab = math.sqrt(ab)
    X = b * Np + a * Nm
    r = 1.0 / (sab * apb * X)
    h = 0.5 * apb * X * r
    E = 0.5 * (D + ab)
    beta = (a - b) * sab * X * r
    return dict(n=X * h, E=E, T=(2.0 / 3.0) * E * ab * apb * r, beta=beta, gamma=apb * h)


CASES = [(1.0, 1.0, 0.0, 1), (1.2, 0.9, 0.5, 2), (0.125, 0.8, -0.6, 3), (2.0, 0.3, 0.7, 4)]


@pytest.mark.parametrize("n,T,beta,seed", CASES)
def test_moment_identities(n, T, beta, seed):
    f = _state(n, T, beta, seed)
    Np, Nm, Ap, Am, D = _direct_sums(f)
    Nt, Nz, Ttt, Ttz, Tzz = oracle.moments(Q_XI, Q_L, f)
    tr = 0.25 * (Ap + Am)
    got = np.array([0.5 * (Np + Nm), 0.5 * (Np - Nm), tr + 0.5 * D, 0.25 * (Ap - Am), tr - 0.5 * D])
    ref = np.array([Nt, Nz, Ttt, Ttz, Tzz])
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("n,T,beta,seed", CASES)
def test_landau_with_one_division(n, T, beta, seed):
    f = _state(n, T, beta, seed)
    got = _landau_one_division(*_direct_sums(f))
    ref = oracle.landau(oracle.moments(Q_XI, Q_L, f))
    for k in ("n", "E", "T", "gamma"):
        assert abs(got[k] - ref[k]) <= 1e-13 * abs(ref[k]), k
    assert abs(got["beta"] - ref["beta"]) <= 1e-13


def test_weno_scale_from_exponent_bits():
    """2^(127-e) from an AND and a subtract on the FP32 bits (and the FP64
    analogue) brings a normal maximum into [1, 2) exactly; zero and subnormal
    maxima get the largest such power (the kernels' WENO scale)."""
    rng = np.random.default_rng(5)
    m32 = np.float32(10.0) ** rng.uniform(-37, 37, 1000).astype(np.float32)
    inv32 = (np.uint32(0x7F000000) - (m32.view(np.uint32) & np.uint32(0x7F800000))).view(np.float32)
    r = m32 * inv32
    assert np.all((r >= 1.0) & (r < 2.0))
    assert np.all(inv32 == np.float32(2.0) ** (-np.floor(np.log2(m32.astype(np.float64)))).astype(np.float32))
    z = np.array([0.0, 1e-40], dtype=np.float32)
    zinv = (np.uint32(0x7F000000) - (z.view(np.uint32) & np.uint32(0x7F800000))).view(np.float32)
    assert np.all(zinv == np.float32(2.0) ** 127)
    m64 = 10.0 ** rng.uniform(-300, 300, 1000)
    inv64 = (np.uint64(0x7FE0000000000000) -
             (m64.view(np.uint64) & np.uint64(0x7FF0000000000000))).view(np.float64)
    r64 = m64 * inv64
    assert np.all((r64 >= 1.0) & (r64 < 2.0))


def test_double_float_moment_sums():
    """The FP32 output-moment kernel's accumulation: the FP64 weight split as
    w_hi + w_lo (FP32), f w_hi formed exactly as product + fma remainder, hi
    parts added with TwoSum, remainders and errors in a plain FP32 low sum.
    Emulated step by step in FP32 (the remainder is exact, so evaluating it in
    FP64 is exact too); the result agrees with the exact sum to ~1e-14 (the
    low sum's own FP32 rounding over V terms bounds it by about V 2^-48)."""
    from fractions import Fraction
    rng = np.random.default_rng(9)
    V = 600
    f = rng.uniform(0.0, 1.0, V).astype(np.float32) * np.float32(1e-2)
    x, p = np.linspace(-0.99, 0.99, V), np.repeat([0.4, 2.2, 6.1], V // 3)
    w = p * (1 + x) ** 2
    wh = w.astype(np.float32)
    wl = (w - wh.astype(np.float64)).astype(np.float32)
    H = np.float32(0.0)
    L = np.float32(0.0)
    for fv, a, b in zip(f, wh, wl):
        ph = np.float32(fv * a)
        pl = np.float32(np.float64(fv) * np.float64(a) - np.float64(ph))  # exact remainder
        pl = np.float32(np.float64(fv) * np.float64(b) + np.float64(pl))   # fma(f, wl, pl)
        s = np.float32(H + ph)
        bp = np.float32(s - H)
        e = np.float32(np.float32(H - np.float32(s - bp)) + np.float32(ph - bp))
        H = s
        L = np.float32(L + np.float32(e + pl))
    got = float(H) + float(L)
    exact = sum(Fraction(float(fv)) * Fraction(float(wv)) for fv, wv in zip(f, w))
    assert abs(Fraction(got) - exact) <= Fraction(5, 10 ** 14) * abs(exact)


def _kp_entry_from_table(Q, xi, w, j, jp):
    """One K^P entry the way the GPU set-up builds it (Eq. K_leg_disc): the
    m-dependent factors of both sums and of both Legendre recurrences come
    from a per-m table, P_m(xi_j) advances by Bonnet's recurrence and the
    xi_j' values are carried as a window P_{m-2} .. P_{m+2}."""
    c = np.zeros((Q, 7))
    for m in range(Q):
        d = float(m)
        c[m] = [d * (d + 1) * (d + 2) / (2 * (2 * d + 3)),
                0.5 * d * (d + 1) * (2 * d + 1) / ((2 * d - 1) * (2 * d + 3)) if m else 0.0,
                0.5 * d * (d + 1) * (d - 1) / (2 * d - 1) if m else 0.0,
                (2 * d + 1) / (d + 1), d / (d + 1), (2 * d + 5) / (d + 3), (d + 2) / (d + 3)]
    x, y = xi[j], xi[jp]
    px, pxm1 = x, 1.0
    ym2, ym1, y0 = 0.0, 1.0, y
    yp1 = 0.5 * (3 * y * y - 1)
    yp2 = (5 * y * yp1 - 2 * y0) / 3
    s1 = s2 = 0.0
    for m in range(1, Q):
        if m <= Q - 3:
            s1 += c[m, 0] * px * yp2
        s2 += px * (c[m, 1] * y0 + c[m, 2] * ym2)
        px, pxm1 = c[m, 3] * x * px - c[m, 4] * pxm1, px
        yn = c[m, 5] * y * yp2 - c[m, 6] * yp1
        ym2, ym1, y0, yp1, yp2 = ym1, y0, yp1, yp2, yn
    return w[j] * (s1 - s2)


@pytest.mark.parametrize("Q", [8, 20, 41])
def test_kp_from_the_coefficient_table(Q):
    xi, w = oracle.gauss_legendre(Q)
    K = oracle.kp_matrix(Q)
    got = np.array([[_kp_entry_from_table(Q, xi, w, j, jp) for jp in range(Q)] for j in range(Q)])
    assert np.abs(got - K).max() <= 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("Q", [8, 9, 20, 33, 64, 129, 200])
def test_kp_even_odd_split_reproduces_kp(Q):
    """The tensor-core contraction uses K^P's centrosymmetry (K_{Q-1-j, Q-1-j'} =
    K_{j j'}, Eq. K_leg_disc on symmetric nodes): with h = floor(Q/2) mirror pairs
    and qh = ceil(Q/2), E_{ij} = K_{ij} + K_{i,Q-1-j} (qh x qh) acting on the even
    parts s_j = f_j + f_{Q-1-j} (s_h = f_h for odd Q) and O_{ij} = K_{ij} - K_{i,Q-1-j}
    (h x h) acting on the odd parts d_j = f_j - f_{Q-1-j} give
    (K f)_i = (E s + O d)_i / 2 and (K f)_{Q-1-i} = (E s - O d)_i / 2 (i < h), and
    (K f)_h = (E s)_h / 2 for the middle row.  Restated here in numpy on the
    oracle's K^P."""
    K = oracle.kp_matrix(Q)
    J = K[::-1, ::-1]
    assert np.array_equal(K, J), "K^P is exactly centrosymmetric in FP64"
    h, qh = Q // 2, Q - Q // 2
    E = K[:qh, :qh] + K[:qh, ::-1][:, :qh]
    O = K[:h, :h] - K[:h, ::-1][:, :h]
    rng = np.random.default_rng(Q)
    f = rng.normal(size=(Q, 3))
    s = f[:qh].copy()
    s[:h] += f[::-1][:h]
    d = f[:h] - f[::-1][:h]
    ye, yo = E @ s, O @ d
    y = np.empty_like(f)
    y[:h] = 0.5 * (ye[:h] + yo)
    y[Q - 1 - np.arange(h)] = 0.5 * (ye[:h] - yo)
    if Q % 2:
        y[h] = 0.5 * ye[h]
    ref = K @ f
    assert np.abs(y - ref).max() <= 1e-13 * np.abs(K).sum(1).max() * np.abs(f).max()
