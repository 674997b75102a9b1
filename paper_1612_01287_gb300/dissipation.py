"""Dissipative quantities across the shock and the contact discontinuity
(Sec. IV B 2, Eqs. intq and intpi).

Close to the inviscid limit the heat flux q (Eq. q_val) and the shear stress
Pi (Eq. pi_val) of the shock tube are peaked at the contact discontinuity
(z_C = beta_C t) and at the shock front (z_S = beta_shock t); the paper
compares their integrals over small vicinities of these points with the
Chapman-Enskog predictions.  This driver runs the tubes (one per eta/s) as a
batch on the GPU engine and integrates q and Pi over the given windows.
"""
import numpy as np


def window_integral(z, f, lo, hi):
    """int_lo^hi f dz of cell-averaged values f on cell centres z (midpoint
    rule: the cells whose centres lie in [lo, hi], each times its width)."""
    z = np.asarray(z, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    dz = z[1] - z[0]
    m = (z >= lo) & (z <= hi)
    return float(f[m].sum() * dz)


def sod_dissipation_integrals(etas, windows, Z=10000, Q_xi=6, Q_L=2, N_Omega=5, dt=5e-6,
                              t_end=0.5, left=(1.0, 1.0), right=(0.125, 0.5), tau_coef=0.3854,
                              lambda_ref=1.0, z_min=-0.5, z_max=0.5, precision="f64",
                              stream=None):
    """Integrals of q and Pi over windows (name -> (z_lo, z_hi)) at t_end for
    each eta/s, the paper's set-up of Sec. IV B (fixed-equilibrium ghosts,
    the eta/s law with tau_AW0 = tau_coef eta/s, Eq. Sod:tau1).
    Returns {"etas": [...], name: {"q": [...], "Pi": [...]}, "profiles": [...]}."""
    from . import SodBatch
    runs = [dict(Z=Z, Q_xi=int(Q_xi), t_end=t_end, dt=dt, tau_mode="etas",
                 tau_AW0=tau_coef * es, lambda_ref=lambda_ref, N_Omega=N_Omega,
                 nL=left[0], TL=left[1], nR=right[0], TR=right[1]) for es in etas]
    with SodBatch(runs, Q_L=Q_L, precision=precision, bc="fixed_eq", z_min=z_min, z_max=z_max,
                  autotune=False, stream=stream) as b:
        b.step(b.max_steps)
        prof = [b.moments(r) for r in range(len(runs))]
    z = z_min + (np.arange(Z) + 0.5) * (z_max - z_min) / Z
    out = {"etas": list(etas), "z": z, "profiles": prof}
    for name, (lo, hi) in windows.items():
        out[name] = {"q": [window_integral(z, p["q"], lo, hi) for p in prof],
                     "Pi": [window_integral(z, p["Pi"], lo, hi) for p in prof]}
    return out
