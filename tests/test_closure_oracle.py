"""Pins of the FP64 learned-closure reference (oracle/closure.py) against
facts that do not come from it: finite differences, exact moment
preservation of the restriction, exactness on equilibria whose Legendre
content fits the low-order set, and the conservation property."""

import numpy as np
import pytest

import oracle
from oracle import closure as C


def small_net(D=7, H=5, O=4, seed=3):
    rng = np.random.default_rng(seed)
    n = sum(C.param_sizes(D, H, O))
    theta = rng.normal(0, 0.5, size=n)
    X = rng.normal(0, 1, size=(11, D))
    T = rng.normal(0, 1, size=(11, O))
    return theta, X, T, D, H, O


def test_silu_derivative_closed_form():
    a = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (C.silu(a + h) - C.silu(a - h)) / (2 * h)
    assert np.abs(fd - C.dsilu(a)).max() < 1e-9


def test_backprop_matches_central_differences():
    theta, X, T, D, H, O = small_net()
    L, g = C.loss_grad(theta, X, T, D, H, O)
    idx = np.arange(len(theta))
    fd = C.fd_grad(theta, X, T, D, H, O, idx, h=1e-5)
    rel = np.abs(fd - g).max() / np.abs(g).max()
    assert rel < 1e-8, rel


def test_backprop_full_size_random_subset():
    """The closure's own shape (73 -> 64 -> 64 -> 24) on 1000 random parameters."""
    D, H, O = 73, 64, 24
    rng = np.random.default_rng(11)
    n = sum(C.param_sizes(D, H, O))
    theta = rng.normal(0, 1, size=n) / np.sqrt(np.repeat([D, 1, H, 1, H, 1], C.param_sizes(D, H, O)))
    X = rng.normal(0, 1, size=(16, D))
    T = rng.normal(0, 1, size=(16, O))
    _, g = C.loss_grad(theta, X, T, D, H, O)
    idx = rng.choice(n, size=1000, replace=False)
    fd = C.fd_grad(theta, X, T, D, H, O, idx, h=1e-5)
    rel = np.abs(fd - g[idx]).max() / np.abs(g[idx]).max()
    assert rel < 1e-8, rel


def test_forward_by_hand_two_two_two_one():
    """A 2 -> 2 -> 2 -> 1 network written out scalar by scalar: the flat layout
    (W1 [H][D] row-major, b1, W2 [H][H], b2, W3 [O][H], b3), W x (not x W) in every
    layer, SiLU a / (1 + e^-a) after both hidden layers and none after the last."""
    import math
    W1 = [[0.5, -1.0], [2.0, 0.25]]
    b1 = [0.1, -0.3]
    W2 = [[1.5, -0.5], [0.0, 1.0]]
    b2 = [-0.2, 0.4]
    W3 = [[-1.0, 2.0]]
    b3 = [0.05]
    theta = np.array([W1[0][0], W1[0][1], W1[1][0], W1[1][1], b1[0], b1[1],
                      W2[0][0], W2[0][1], W2[1][0], W2[1][1], b2[0], b2[1],
                      W3[0][0], W3[0][1], b3[0]])

    def silu(a):
        return a / (1.0 + math.exp(-a))

    for x in ([1.0, 2.0], [-0.7, 0.3]):
        h1 = [silu(W1[i][0] * x[0] + W1[i][1] * x[1] + b1[i]) for i in range(2)]
        h2 = [silu(W2[i][0] * h1[0] + W2[i][1] * h1[1] + b2[i]) for i in range(2)]
        y = W3[0][0] * h2[0] + W3[0][1] * h2[1] + b3[0]
        got, _ = C.forward(theta, np.array([x]), 2, 2, 1)
        assert abs(got[0, 0] - y) < 1e-15, (x, got, y)
    # x = (1, 2) worked on paper: a1 = (-1.4, 2.2), h1 = (-0.276943, 1.980549),
    # a2 = (-1.605688, 2.380549), h2 = (-0.268452, 2.178993), y = 4.676437
    y12, _ = C.forward(theta, np.array([[1.0, 2.0]]), 2, 2, 1)
    assert abs(y12[0, 0] - 4.676437) < 2e-6


def test_loss_is_mean_square():
    theta, X, T, D, H, O = small_net()
    y, _ = C.forward(theta, X, D, H, O)
    L, _ = C.loss_grad(theta, X, T, D, H, O)
    assert L == pytest.approx(float(np.mean((y - T) ** 2)), rel=1e-14)


@pytest.mark.parametrize("Q_lo", [8, 4])
def test_restriction_preserves_moments(Q_lo):
    """N^t, N^z, T^tt, T^tz, T^zz of the restricted populations equal the
    high-order ones (Eq. macro_jk; modes m <= 2 < Q_lo are kept exactly)."""
    QL, Q_hi = 3, 200
    rng = np.random.default_rng(5)
    f_hi = np.stack([oracle.feq(Q_hi, QL, 5, n, T, b) for n, T, b in
                     zip(rng.uniform(0.2, 1, 6), rng.uniform(0.5, 1.5, 6), rng.uniform(-0.8, 0.8, 6))])
    f_hi += rng.uniform(0, 1e-3, size=f_hi.shape)  # non-equilibrium part with all modes
    f_lo = C.restrict(f_hi, Q_hi, Q_lo, QL)
    for s in range(f_hi.shape[0]):
        Mh = oracle.moments(Q_hi, QL, f_hi[s])
        Ml = oracle.moments(Q_lo, QL, f_lo[s])
        assert np.abs(Mh - Ml).max() < 1e-13 * np.abs(Mh).max()


def test_restriction_is_exact_on_low_order_equilibria():
    """f^eq truncated at N_Omega = 5 has Legendre modes m <= 5 only, so its
    restriction to 8 nodes is the 8-node f^eq itself (Eqs. feq_trunc, fjk)."""
    QL = 3
    for n, T, b in [(1.0, 1.0, 0.0), (0.3, 0.8, 0.6), (0.7, 1.3, -0.9)]:
        f_hi = oracle.feq(200, QL, 5, n, T, b)[None, :]
        f_lo = C.restrict(f_hi, 200, 8, QL)[0]
        ref = oracle.feq(8, QL, 5, n, T, b)
        assert np.abs(f_lo - ref).max() < 1e-13 * np.abs(ref).max()


def test_projection_conserves_and_is_idempotent():
    Q, QL = 8, 3
    rng = np.random.default_rng(9)
    d = rng.normal(size=(5, Q * QL))
    p = C.project(d, Q, QL)
    Phi, W = C.invariants(Q, QL)
    assert np.abs(p @ Phi).max() < 1e-14 * np.abs(d).max() * 100
    assert np.abs(C.project(p, Q, QL) - p).max() < 1e-14 * 100
    # anything along W Phi is removed entirely
    inv = (rng.normal(size=(5, 3)) @ Phi.T) * W
    assert np.abs(C.project(inv, Q, QL)).max() < 1e-14 * 100


def test_correction_keeps_cell_invariants():
    Q, QL, H = 8, 3, 16
    V = Q * QL
    rng = np.random.default_rng(2)
    theta = rng.normal(0, 0.3, size=sum(C.param_sizes(3 * V + 1, H, V)))
    f = np.stack([oracle.feq(Q, QL, 5, 0.5 + 0.1 * s, 1.0, 0.1 * s) for s in range(6)])
    d = C.correction(theta, f, 0.01, Q, QL, H)
    Phi, _ = C.invariants(Q, QL)
    assert np.abs(d @ Phi).max() < 1e-13


def test_features_layout():
    f = np.arange(12.0).reshape(4, 3) + 1.0
    X = C.features(f, 0.1)
    n = f.sum(1)
    assert np.allclose(X[1, :3], f[1] / n[1])
    assert np.allclose(X[1, 3:6], (f[2] - f[1]) / n[1])
    assert np.allclose(X[1, 6:9], (f[1] - f[0]) / n[1])
    assert np.allclose(X[0, 6:9], 0.0)      # outflow copy at the left end
    assert np.allclose(X[3, 3:6], 0.0)      # outflow copy at the right end
    assert np.allclose(X[:, 9], -1.0)


def test_normalization_fit_and_use():
    rng = np.random.default_rng(8)
    X = rng.normal(3.0, 2.0, size=(5000, 4))
    X[:, 2] = 7.0  # constant column
    T = rng.normal(0.0, 0.5, size=(5000, 2))
    mu, isd, osd = C.fit_normalization(X, T)
    Xn = (X - mu) * isd
    assert np.abs(Xn[:, [0, 1, 3]].mean(0)).max() < 1e-12
    assert np.abs(Xn[:, [0, 1, 3]].std(0) - 1).max() < 1e-12
    assert isd[2] == 1.0 and np.all(Xn[:, 2] == 0.0)
    assert np.allclose(np.sqrt((T / osd) ** 2).mean(0) > 0, True)
    assert np.abs(np.sqrt(((T / osd) ** 2).mean(0)) - 1).max() < 1e-12
    theta = rng.normal(0, 0.3, size=sum(C.param_sizes(4, 16, 2)))
    y0, _ = C.forward(theta, Xn, 4, 16, 2)
    assert np.allclose(C.net(theta, X, 4, 16, 2, (mu, isd, osd)), y0 * osd, rtol=1e-14)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.14159265], dtype=np.float32)
    r = C.bf16_round(x)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == -2.5
    assert abs(r[4] - 3.140625) < 1e-12


def test_limiter_keeps_positive_populations_and_invariants():
    Q, QL, H = 8, 3, 16
    V = Q * QL
    rng = np.random.default_rng(4)
    theta = rng.normal(0, 3.0, size=sum(C.param_sizes(3 * V + 1, H, V)))  # large corrections
    f = np.stack([oracle.feq(Q, QL, 5, 0.5 + 0.1 * s, 1.0, 0.05 * s) for s in range(6)])
    d = C.correction(theta, f, 0.01, Q, QL, H)
    g = f + d
    pos = f > 0
    assert np.all(g[pos] >= (1 - C.LIMIT_THETA) * f[pos] - 1e-15)
    Phi, _ = C.invariants(Q, QL)
    assert np.abs(d @ Phi).max() < 1e-12
    # the limiter never amplifies: |delta'| <= |projected delta|
    X = C.features(f, 0.01)
    y, _ = C.forward(theta, X, 3 * V + 1, H, V)
    raw = C.project(f.sum(1)[:, None] * y, Q, QL)
    assert np.all(np.abs(d) <= np.abs(raw) + 1e-15)
