"""FP64 reference of the learned closure -- TEST INFRASTRUCTURE ONLY.

The paper has no learned closure; this module defines the one built here,
in plain numpy, so that the GPU kernels (restriction, features, MLP forward,
backward and the conserving correction) can be checked against it.  Only
``tests/`` may import it.

Definitions (velocity index v = k * Q + j, radial node k, polar node j):

* Restriction R from Q_hi to Q_lo polar nodes, radial index kept: the
  Legendre moments F_{m,k} = sum_j f_{jk} P_m(xi_j) (m < Q_lo) of the
  high-order populations, re-expanded at the low-order nodes,
      f^lo_{ik} = w_i sum_{m < Q_lo} (2m + 1)/2 F_{m,k} P_m(xi_i).
  Gauss-Legendre exactness (degree <= 2 Q_lo - 1) makes the low-order
  populations reproduce F_{m,k} for every m < Q_lo, in particular the
  moments N^mu and T^{mu nu} (m <= 2, Eq. macro_jk).
* Features of cell s (outflow copies at the ends), all divided by
  n_s = sum_v f_{v,s}: the populations of cell s, the forward differences
  f_{s+1} - f_s and the backward differences f_s - f_{s-1}, then log10(tau):
  3 V + 1 numbers.
* MLP: h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3 with
  silu(a) = a / (1 + e^{-a}).
* Normalisation (fixed, not trained): the network sees (x - mu) * inv_sd and
  its output is multiplied by out_sd; fit_normalization takes mu, sd as the
  column means and standard deviations of the training inputs and out_sd as
  the column root-mean-squares of the targets (1 where a column is constant).
* Correction of cell s: delta = n_s out_sd * y, made conserving by removing its
  component along the collision invariants phi = (1, p_k, p_k xi_j) in the
  quadrature-weighted sense,
      delta' = delta - W Phi (Phi^T W Phi)^{-1} Phi^T delta,  W = diag(w_j w_k),
  so that sum_v delta'_v phi_v = 0 (N^t, T^tt, T^tz unchanged).
* Positivity limiter: the conserving correction of a cell is scaled by
  alpha = min(1, min over v with f_v > 0 and delta'_v < 0 of
  LIMIT_THETA f_v / (-delta'_v)), so no positive population loses more than
  half of itself in one step; the scaling keeps sum_v delta'_v phi_v = 0.
* Loss: L = sum over samples and outputs of (y - t)^2 / (n_samples * n_out).

Flat parameter layout: W1 [H][D] row-major, b1 [H], W2 [H][H], b2 [H],
W3 [O][H], b3 [O].
"""
import numpy as np

from . import gauss_laguerre2, gauss_legendre, legendre


def param_sizes(D, H, O):
    return [H * D, H, H * H, H, O * H, O]


def unpack(theta, D, H, O):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = [], 0
    for n in param_sizes(D, H, O):
        out.append(theta[o:o + n])
        o += n
    W1, b1, W2, b2, W3, b3 = out
    return W1.reshape(H, D), b1, W2.reshape(H, H), b2, W3.reshape(O, H), b3


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def forward(theta, X, D, H, O):
    """X: [N][D] -> (y [N][O], cache)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, D, H, O)
    a1 = X @ W1.T + b1
    h1 = silu(a1)
    a2 = h1 @ W2.T + b2
    h2 = silu(a2)
    y = h2 @ W3.T + b3
    return y, (X, a1, h1, a2, h2)


def loss_grad(theta, X, T, D, H, O):
    """Mean-squared loss and its gradient with respect to theta (backprop)."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, D, H, O)
    y, (X, a1, h1, a2, h2) = forward(theta, X, D, H, O)
    N = X.shape[0]
    r = y - T
    L = float((r * r).sum() / (N * O))
    gy = 2.0 * r / (N * O)
    gW3 = gy.T @ h2
    gb3 = gy.sum(0)
    gh2 = gy @ W3
    ga2 = gh2 * dsilu(a2)
    gW2 = ga2.T @ h1
    gb2 = ga2.sum(0)
    gh1 = ga2 @ W2
    ga1 = gh1 * dsilu(a1)
    gW1 = ga1.T @ X
    gb1 = ga1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def fd_grad(theta, X, T, D, H, O, idx, h=1e-6):
    """Central finite differences of the loss at the parameters idx."""
    theta = np.array(theta, dtype=np.float64)
    g = np.zeros(len(idx))
    for n, i in enumerate(idx):
        t0 = theta[i]
        theta[i] = t0 + h
        lp = loss_grad(theta, X, T, D, H, O)[0]
        theta[i] = t0 - h
        lm = loss_grad(theta, X, T, D, H, O)[0]
        theta[i] = t0
        g[n] = (lp - lm) / (2.0 * h)
    return g


def restrict(f_hi, Q_hi, Q_lo, QL):
    """f_hi: [Z][QL*Q_hi] -> [Z][QL*Q_lo]."""
    xh, _ = gauss_legendre(Q_hi)
    xl, wl = gauss_legendre(Q_lo)
    Ph = np.array([[legendre(m, x) for x in xh] for m in range(Q_lo)])  # [m][j]
    Pl = np.array([[legendre(m, x) for x in xl] for m in range(Q_lo)])  # [m][i]
    c = (2.0 * np.arange(Q_lo) + 1.0) / 2.0
    Z = f_hi.shape[0]
    out = np.zeros((Z, QL * Q_lo))
    for k in range(QL):
        F = f_hi[:, k * Q_hi:(k + 1) * Q_hi] @ Ph.T  # [Z][m]
        out[:, k * Q_lo:(k + 1) * Q_lo] = wl * ((F * c) @ Pl)
    return out


def features(f_lo, tau):
    """f_lo: [Z][V] -> X [Z][3V + 1] (outflow copies at both ends)."""
    Z, V = f_lo.shape
    n = f_lo.sum(1)
    left = np.vstack([f_lo[:1], f_lo[:-1]])
    right = np.vstack([f_lo[1:], f_lo[-1:]])
    X = np.hstack([f_lo, right - f_lo, f_lo - left]) / n[:, None]
    return np.hstack([X, np.full((Z, 1), np.log10(tau))])


def identity_norm(D, O):
    return np.zeros(D), np.ones(D), np.ones(O)


def fit_normalization(X, T):
    """(mu, inv_sd, out_sd) from training inputs X [N][D] and targets T [N][O]."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    mu = X.mean(0)
    sd = np.sqrt(((X - mu) ** 2).mean(0))
    inv_sd = np.where(sd > 0, 1.0 / np.where(sd > 0, sd, 1.0), 1.0)
    rms = np.sqrt((T * T).mean(0))
    out_sd = np.where(rms > 0, rms, 1.0)
    return mu, inv_sd, out_sd


def net(theta, X, D, H, O, norm=None):
    """The normalised network: out_sd * MLP((X - mu) * inv_sd)."""
    mu, inv_sd, out_sd = norm if norm is not None else identity_norm(D, O)
    y, _ = forward(theta, (np.asarray(X) - mu) * inv_sd, D, H, O)
    return y * out_sd


def invariants(Q, QL, T0=1.0):
    """Phi [V][3] = (1, p, p xi) and the weights w_j w_k [V]."""
    xi, w = gauss_legendre(Q)
    xk, wk = gauss_laguerre2(QL)
    V = Q * QL
    Phi = np.zeros((V, 3))
    W = np.zeros(V)
    for k in range(QL):
        for j in range(Q):
            v = k * Q + j
            p = T0 * xk[k]
            Phi[v] = (1.0, p, p * xi[j])
            W[v] = w[j] * wk[k]
    return Phi, W


def project(delta, Q, QL):
    """Remove the invariant components: delta [Z][V] -> delta'."""
    Phi, W = invariants(Q, QL)
    G = Phi.T @ (W[:, None] * Phi)
    c = np.linalg.solve(G, (delta @ Phi).T).T  # [Z][3]
    return delta - (c @ Phi.T) * W


LIMIT_THETA = 0.5


def limit(delta, f):
    """Scale each cell's correction so positive populations stay positive."""
    alpha = np.ones(delta.shape[0])
    for s in range(delta.shape[0]):
        m = (f[s] > 0) & (delta[s] < 0)
        if m.any():
            alpha[s] = min(1.0, float(np.min(LIMIT_THETA * f[s][m] / -delta[s][m])))
    return delta * alpha[:, None]


def correction(theta, f_lo, tau, Q, QL, H, norm=None):
    """The conserving, limited correction delta' [Z][V] of every cell."""
    V = Q * QL
    X = features(f_lo, tau)
    y = net(theta, X, 3 * V + 1, H, V, norm)
    n = f_lo.sum(1)
    return limit(project(n[:, None] * y, Q, QL), f_lo)


def bf16_round(x):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP64."""
    a = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (a >> 16) & 1
    a = (a + 0x7FFF + lsb) & 0xFFFF0000
    return a.astype(np.uint32).view(np.float32).astype(np.float64)
