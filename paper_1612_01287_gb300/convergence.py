"""Convergence tests of the quadrature order (Secs. IV E and V E).

Sod shock tube (Sec. IV E): the error of Eq. eps_def,
    eps = max_j eps_j,  eps_j = max_z |d_j(z) - d_j,ref(z)| / (max_z d_j - min_z d_j),
over the profiles d_j in {n, T, gamma} at the final time, against a reference
model with many more nodes; a model has converged when eps < eps_th (Eq. eps_th).
Reading: the printed max_z[d_j - d_j,ref] is taken as the largest absolute
deviation (the text: "the largest error in a single point").

Bjorken flow (Sec. V E): the time-averaged L2 norm of Eq. bjork_L2,
    L2(A) = sqrt( int_1^tau_f dtau/(tau_f - 1) [A(tau) - A_ref(tau)]^2 ),
    L2 = max over A in {n, P, T, Pi},
integrated here by the trapezoidal rule on the sampled times; convergence when
L2 <= L2_th.

The sweeps run every (eta/s, Q_xi) model, and the references, as one batch on
the GPU engines (rslb_sod_batch_*, rslb_bjorken_*) and return the error of each
model and the smallest converged Q_xi per threshold.
"""
import math

import numpy as np

HBARC_GEV_FM = 0.1973269804
_trapezoid = getattr(np, "trapezoid", None) or np.trapz
SOD_FIELDS = ("n", "T", "gamma")
BJ_FIELDS = ("n", "P", "T", "Pi")


def eps_sod(prof, ref, fields=SOD_FIELDS):
    """Eq. eps_def for dicts of per-cell arrays (same grid)."""
    out = 0.0
    for k in fields:
        d = np.asarray(prof[k], dtype=np.float64)
        r = np.asarray(ref[k], dtype=np.float64)
        span = d.max() - d.min()
        dev = np.abs(d - r).max()
        out = max(out, dev / span if span > 0.0 else dev)
    return out


def l2_bjorken(tau, hist, ref, tau_f=None, fields=BJ_FIELDS):
    """Eq. bjork_L2 for histories sampled at the times `tau` (both dicts of
    arrays on the same samples); returns (L2, {field: L2(A)})."""
    t = np.asarray(tau, dtype=np.float64)
    t0 = t[0]
    tf = t[-1] if tau_f is None else tau_f
    per = {}
    for k in fields:
        e2 = (np.asarray(hist[k], dtype=np.float64) - np.asarray(ref[k], dtype=np.float64)) ** 2
        per[k] = math.sqrt(float(_trapezoid(e2, t)) / (tf - t0))
    return max(per.values()), per


def first_converged(qxis, errs, threshold, strict=True):
    """Smallest Q_xi whose error is below the threshold (strictly, as Eq.
    eps_th; or at most equal, as Eq. bjork_L2) and stays so for every larger
    Q_xi in the sweep (None if there is none)."""
    order = np.argsort(qxis)
    q = np.asarray(qxis)[order]
    e = np.asarray(errs)[order]
    ok = e < threshold if strict else e <= threshold
    for i in range(len(q)):
        if ok[i:].all():
            return int(q[i])
    return None


def sod_qxi_sweep(etas, qxis, Z=1000, t_end=0.5, dt=5e-4, Q_L=2, q_ref=500, n_omega_ref=5,
                  left=(1.0, 1.0), right=(0.125, 0.5), tau_coef=0.3854, lambda_ref=1.0,
                  z_min=-0.5, z_max=0.5, precision="f64", thresholds=(0.01, 0.02, 0.05),
                  stream=None):
    """Q_xi convergence of the shock tube (Sec. IV E, Table III).

    Every (eta/s, Q_xi) model with N_Omega = min(Q_xi - 1, 5), and for every
    eta/s the reference R-SLB(n_omega_ref; q_ref), run to t_end with the eta/s
    law tau_AW = tau_AW0/T [1 - ln(lambda_bar lambda_ref)/4],
    tau_AW0 = tau_coef eta/s (Eq. Sod:tau1), left/right chambers (n, T) at rest.
    Returns {"eps": [[eps(etas_i, q_j)]], "q_conv": {th: [q or None per etas]}}."""
    from . import SodBatch
    runs = []
    for es in etas:
        # explicit RK3 needs dt below ~2.5 tau; the smallest tau of the tube is
        # tau_AW0 / max T (the log factor is 1 in both chambers), so tubes
        # with a smaller tau than 2 dt take an even division of t_end instead
        tau_min = tau_coef * es / max(left[1], right[1])
        dt_r = dt if dt <= 0.5 * tau_min else t_end / math.ceil(t_end / (0.5 * tau_min))
        for j, q in enumerate(list(qxis) + [q_ref]):
            nom = n_omega_ref if j == len(qxis) else min(q - 1, 5)
            runs.append(dict(Z=Z, Q_xi=int(q), t_end=t_end, dt=dt_r, tau_mode="etas",
                             tau_AW0=tau_coef * es, lambda_ref=lambda_ref, N_Omega=nom,
                             nL=left[0], TL=left[1], nR=right[0], TR=right[1]))
    with SodBatch(runs, Q_L=Q_L, precision=precision, bc="fixed_eq", z_min=z_min, z_max=z_max,
                  autotune=False, stream=stream) as b:
        b.step(b.max_steps)
        prof = [b.moments(r) for r in range(len(runs))]
    nq = len(qxis) + 1  # per eta/s: the tested models, then the reference
    eps = np.zeros((len(etas), len(qxis)))
    for i in range(len(etas)):
        ref = prof[i * nq + len(qxis)]
        for j in range(len(qxis)):
            eps[i, j] = eps_sod(prof[i * nq + j], ref)
    conv = {th: [first_converged(qxis, eps[i], th) for i in range(len(etas))]
            for th in thresholds}
    return {"etas": list(etas), "qxis": list(qxis), "eps": eps.tolist(), "q_conv": conv}


def bjorken_tau_aw0(eta_s_4pi, T0_GeV, tau0_fm=0.5):
    """tau_AW0 = 5 hbar c (eta/s) / (tilde tau_0 T_0) with eta/s = (4 pi eta/s)/(4 pi)
    (Eq. bjorken_tauAW0; nondimensional tau from 1)."""
    return 5.0 * HBARC_GEV_FM * (eta_s_4pi / (4.0 * math.pi)) / (tau0_fm * T0_GeV)


def bjorken_qxi_sweep(eta_s_4pi, qxis, T0_GeV=0.3, gas="parton", tau_f=40.0, dtau=1e-3,
                      sample_every=50, Q_L=2, q_ref=100, precision="f64", kp_mode="simt",
                      thresholds=(1e-5, 1e-6), stream=None):
    """Q_xi convergence of the Bjorken flow (Sec. V E, Table IV): the L2 norm
    (Eq. bjork_L2) of n, P, T, Pi over tau in [1, tau_f] against R-SLB(5; q_ref)."""
    from . import Bjorken
    qs, taus = [], []
    for e4 in eta_s_4pi:
        t0 = bjorken_tau_aw0(e4, T0_GeV)
        for q in list(qxis) + [q_ref]:
            qs.append(int(q))
            taus.append(t0)
    nsteps = int(round((tau_f - 1.0) / dtau))
    hist = {k: [] for k in ("tau",) + BJ_FIELDS}
    with Bjorken(qs, gas, taus, Q_L=Q_L, precision=precision, kp_mode=kp_mode, dtau=dtau,
                 stream=stream) as b:
        done = 0
        while True:
            o = b.read()
            for k in hist:
                hist[k].append(np.asarray(o[k], dtype=np.float64).copy())
            if done >= nsteps:
                break
            n = min(sample_every, nsteps - done)
            b.step(n)
            done += n
    H = {k: np.array(v) for k, v in hist.items()}  # [sample][run]
    nq = len(qxis) + 1
    l2 = np.zeros((len(eta_s_4pi), len(qxis)))
    for i in range(len(eta_s_4pi)):
        r = i * nq + len(qxis)
        ref = {k: H[k][:, r] for k in BJ_FIELDS}
        for j in range(len(qxis)):
            c = i * nq + j
            l2[i, j], _ = l2_bjorken(H["tau"][:, c], {k: H[k][:, c] for k in BJ_FIELDS}, ref,
                                     tau_f=tau_f)
    conv = {th: [first_converged(qxis, l2[i], th, strict=False) for i in range(len(eta_s_4pi))]
            for th in thresholds}
    return {"eta_s_4pi": list(eta_s_4pi), "qxis": list(qxis), "l2": l2.tolist(), "q_conv": conv}


def main(argv=None):
    """The paper's two convergence sweeps on the current GPU, printed as JSON:
    the shock tube at Z = 1000, dt = 5e-4, t = 0.5 against R-SLB(5;500) with
    Q_L = 2 (Table III), and the Bjorken flow of a parton gas at T0 = 0.3 GeV
    over tau in [1, 40] against R-SLB(5;100) (Table IV)."""
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--which", default="sod,bjorken")
    ap.add_argument("--quick", action="store_true", help="fewer models, shorter runs")
    a = ap.parse_args(argv)
    out = {}
    if "sod" in a.which:
        etas = [1e-4, 1e-3, 1e-2, 0.083, 0.3, 1.0, 3.0, 18.0, 100.0]
        qxis = [4, 5, 6, 8, 10, 12, 16, 20, 30, 50, 70, 100, 150, 200, 300]
        if a.quick:
            etas, qxis = etas[::3], qxis[::3]
        out["sod"] = sod_qxi_sweep(etas, qxis)
    if "bjorken" in a.which:
        e4 = [1e-2, 5e-2, 0.3, 1.0, 10.0, 100.0, 1e3, 1e4]
        qxis = [3, 4, 5, 6, 8, 10, 12, 16, 20, 25, 33, 40, 50]
        if a.quick:
            e4, qxis = e4[::3], qxis[::3]
        out["bjorken"] = bjorken_qxi_sweep(e4, qxis, tau_f=40.0 if not a.quick else 5.0)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
