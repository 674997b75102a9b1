"""The convergence-test drivers of Secs. IV E and V E: the error measures
(Eqs. eps_def, bjork_L2) pinned on closed forms, and the GPU sweeps against
the same models run by the FP64 oracle."""
import math

import numpy as np
import pytest

import oracle
from paper_1612_01287_gb300 import convergence as C


def test_eps_is_the_largest_pointwise_deviation_over_the_range():
    z = np.linspace(-0.5, 0.5, 101)
    ref = {"n": 1.0 + 0.5 * np.tanh(z / 0.1), "T": 2.0 + z, "gamma": 1.0 + 0.1 * z * z}
    prof = {k: v.copy() for k, v in ref.items()}
    assert C.eps_sod(prof, ref) == 0.0
    prof["T"][40] += 3e-3          # T spans 1.5 .. 2.5 (after the bump, still 1.0)
    prof["n"][70] -= 1e-3          # n spans ~0.50 .. ~1.50
    span_n = prof["n"].max() - prof["n"].min()
    want = max(3e-3 / (prof["T"].max() - prof["T"].min()), 1e-3 / span_n)
    assert C.eps_sod(prof, ref) == pytest.approx(want, rel=1e-12)


def test_l2_closed_forms():
    """A constant offset c gives L2 = c; a linear drift a (tau - 1) over
    [1, tau_f] gives a (tau_f - 1)/sqrt(3)."""
    t = np.linspace(1.0, 40.0, 39001)
    ref = {k: np.cos(t) for k in C.BJ_FIELDS}
    h = {k: v + 2.5e-6 for k, v in ref.items()}
    L2, per = C.l2_bjorken(t, h, ref, tau_f=40.0)
    assert L2 == pytest.approx(2.5e-6, rel=1e-9)
    h = {k: v.copy() for k, v in ref.items()}
    h["Pi"] = ref["Pi"] + 1e-7 * (t - 1.0)
    L2, per = C.l2_bjorken(t, h, ref, tau_f=40.0)
    assert per["Pi"] == pytest.approx(1e-7 * 39.0 / math.sqrt(3.0), rel=1e-8)
    assert L2 == per["Pi"]


def test_first_converged_needs_all_larger_models_converged():
    q = [4, 6, 8, 12, 16]
    assert C.first_converged(q, [0.5, 0.005, 0.02, 0.004, 0.001], 0.01) == 12
    assert C.first_converged(q, [0.5, 0.1, 0.05, 0.02, 0.011], 0.01) is None
    assert C.first_converged(q, [1e-6, 1e-6, 1e-7, 1e-7, 0.0], 1e-6, strict=False) == 4


def test_bjorken_tau_aw0():
    """Eq. bjorken_tauAW0 with tau0 = 0.5 fm/c, T0 = 0.3 GeV: 5 hbar c (eta/s)/(tau0 T0)."""
    assert C.bjorken_tau_aw0(4 * math.pi, 0.3) == pytest.approx(5 * 0.1973269804 / 0.15)


@pytest.mark.gpu
def test_sod_sweep_matches_oracle_models():
    """A small sweep (Z = 64, two eta/s, Q_xi = 4, 8 against 16) on the batched
    engine in FP64; the same models run by the oracle give the same eps."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    etas, qxis, kw = [0.01, 1.0], [4, 8], dict(Z=64, t_end=0.04, dt=1e-3, q_ref=16, Q_L=2)
    res = C.sod_qxi_sweep(etas, qxis, **kw)
    for i, es in enumerate(etas):
        prof = {}
        for q in qxis + [16]:
            p = oracle.sod_params(64, q, 2, 5 if q == 16 else min(q - 1, 5), z_min=-0.5,
                                  z_max=0.5, bc="fixed_eq", tau_mode="etas",
                                  tau_AW0=0.3854 * es, lambda_ref=1.0, dt=1e-3,
                                  left=(1.0, 1.0, 0.0), right=(0.125, 0.5, 0.0))
            prof[q] = oracle.sod_moments(p, oracle.sod_steps(p, oracle.sod_init_riemann(p), 40))
        for j, q in enumerate(qxis):
            want = C.eps_sod(prof[q], prof[16])
            assert res["eps"][i][j] == pytest.approx(want, rel=1e-9, abs=1e-12), (es, q)
            assert want > 1e-4  # the models differ visibly


@pytest.mark.gpu
def test_bjorken_sweep_matches_oracle_models():
    """Bjorken L2 (Eq. bjork_L2) of Q_xi = 3, 6 against 12 over tau in [1, 1.5],
    FP64 SIMT engine against the oracle's histories on the same samples."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    e4, qxis = [0.3, 30.0], [3, 6]
    res = C.bjorken_qxi_sweep(e4, qxis, tau_f=1.5, sample_every=50, q_ref=12)
    for i, e in enumerate(e4):
        t0 = C.bjorken_tau_aw0(e, 0.3)
        hist = {}
        for q in qxis + [12]:
            _, h = oracle.bjorken_run(oracle.bjorken_params(q, 2, gas="parton", tau_AW0=t0,
                                                            dtau=1e-3), 500)
            hist[q] = {k: np.asarray(v)[::50] for k, v in h.items()}
        for j, q in enumerate(qxis):
            want, _ = C.l2_bjorken(hist[q]["tau"], hist[q], hist[12], tau_f=1.5)
            assert res["l2"][i][j] == pytest.approx(want, rel=1e-6, abs=1e-14), (e, q)
            assert want > 1e-8
