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
