"""Seeded synthetic workloads (problem set-ups only -- no method arithmetic).

Both the GPU tests/benchmark and the oracle take their inputs from here.  The
shapes follow the paper's shock-tube and Bjorken set-ups (Secs. IV A, V A) at
the sizes of the benchmark configurations.
"""
import math

import numpy as np

SEED = 20161201

# Sod left/right states (n, P) at rest; T = P/n.
SOD_LEFT = (1.0, 1.0)
SOD_RIGHT = (0.125, 0.1)


def sod_states(left=SOD_LEFT, right=SOD_RIGHT):
    """(n, T, beta) tuples for the left and right chambers."""
    return (left[0], left[1] / left[0], 0.0), (right[0], right[1] / right[0], 0.0)


def sod_small():
    """Shock tube on [-1, 1]: 256 cells, 3 x 20 velocities, tau = 1e-3, outflow.

    The nominal step 2e-3 exceeds tau (explicit RK3 is unstable there), so it
    is taken in 4 substeps of 5e-4 (1600 steps to t = 0.8)."""
    L, R = sod_states()
    return dict(Z=256, Q_xi=20, Q_L=3, N_Omega=5, z_min=-1.0, z_max=1.0, bc="outflow",
                tau_mode="const", tau=1e-3, dt=5e-4, left=L, right=R, t_end=0.8)


def sod_large(tau=1e-2):
    """Shock tube at scale: 65536 cells, 3 x 200 velocities, CFL 0.5, to t = 0.8."""
    L, R = sod_states()
    Z = 65536
    dz = 2.0 / Z
    return dict(Z=Z, Q_xi=200, Q_L=3, N_Omega=5, z_min=-1.0, z_max=1.0, bc="outflow",
                tau_mode="const", tau=tau, dt=None, cfl=0.5, dz=dz, left=L, right=R, t_end=0.8)


SOD_LARGE_TAUS = (1e-4, 1e-2, 1.0, 10.0)


def bjorken_batch(nruns=16384, seed=SEED, qxi_lo=8, qxi_hi=512):
    """Batched Bjorken runs: Q_xi integer-uniform, eta/s log-uniform [0.01, 10],
    T0 uniform [0.3, 0.6] GeV; returned as arrays (Q_xi, eta_s, T0_GeV)."""
    rng = np.random.default_rng(seed)
    qxi = rng.integers(qxi_lo, qxi_hi + 1, size=nruns)
    eta_s = np.exp(rng.uniform(math.log(0.01), math.log(10.0), size=nruns))
    T0 = rng.uniform(0.3, 0.6, size=nruns)
    return qxi, eta_s, T0


def random_smooth_fields(Z, seed=SEED, beta_max=0.6):
    """Smooth seeded (n, T, beta) profiles for periodic tests."""
    rng = np.random.default_rng(seed)
    z = (np.arange(Z) + 0.5) / Z
    a = rng.uniform(0.1, 0.3, size=3)
    ph = rng.uniform(0, 2 * np.pi, size=3)
    n = 1.0 + a[0] * np.sin(2 * np.pi * z + ph[0])
    T = 1.0 + a[1] * np.sin(2 * np.pi * z + ph[1])
    beta = beta_max * np.sin(2 * np.pi * z + ph[2])
    return n, T, beta


def sod_sweep(nruns=4096, seed=SEED, z_lo=256, z_hi=8192, qxi=(8, 20, 50, 100, 200),
              tau_lo=1e-4, tau_hi=10.0, t_end=0.8):
    """Uneven batch of shock tubes: Z log-uniform in [z_lo, z_hi] (integer), Q_xi
    drawn from ``qxi``, tau log-uniform, left chamber (n, P) = (1, 1), right
    chamber density 1/8 and pressure 1/r with r uniform in [2, 20].  Returned as
    a list of run dicts (keys of ``rslb_sod_run``)."""
    rng = np.random.default_rng(seed + 4)
    Z = np.exp(rng.uniform(math.log(z_lo), math.log(z_hi + 1), size=nruns)).astype(np.int64)
    Z = np.clip(Z, z_lo, z_hi)
    Q = rng.choice(np.asarray(qxi), size=nruns)
    tau = np.exp(rng.uniform(math.log(tau_lo), math.log(tau_hi), size=nruns))
    ratio = rng.uniform(2.0, 20.0, size=nruns)
    nR = 0.125
    return [dict(Z=int(Z[r]), Q_xi=int(Q[r]), tau=float(tau[r]), nL=1.0, TL=1.0, nR=nR,
                 TR=float(1.0 / ratio[r] / nR), t_end=float(t_end)) for r in range(nruns)]
