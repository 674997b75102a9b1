"""GPU parity of the batched Bjorken path against the FP64 oracle.

Each run of a mixed batch (different Q_xi, gas laws, relaxation scales,
collisionless) is compared with the oracle run of the same parameters:
max-normalised relative error on n, E and P_L, and Pi normalised by P.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1612_01287_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import build, load
    build.build()
    load()


def run_batch(Qs, gases, taus, precision, nsteps, dtau=1e-2, Q_L=3):
    from paper_1612_01287_gb300 import Bjorken
    with Bjorken(Qs, gases, taus, Q_L=Q_L, precision=precision, dtau=dtau) as b:
        b.step(nsteps)
        got = b.read()
        state = b.get_state()
    return got, state


def oracle_batch(Qs, gases, taus, nsteps, dtau=1e-2, Q_L=3):
    outs, states = [], []
    for Q, g, t in zip(Qs, gases, taus):
        p = oracle.bjorken_params(int(Q), Q_L, gas=g, tau_AW0=t, dtau=dtau)
        f, h = oracle.bjorken_run(p, nsteps)
        outs.append({k: v[-1] for k, v in h.items()})
        states.append(f)
    return outs, states


def errors(got, ref):
    e = {}
    for k in ("n", "E", "PL", "P"):
        r = np.array([o[k] for o in ref])
        e[k] = np.abs(got[k] - r).max() / np.abs(r).max()
    r = np.array([o["Pi"] for o in ref])
    P = np.array([o["P"] for o in ref])
    e["Pi"] = np.abs(got["Pi"] - r).max() / np.abs(P).max()
    return e


MIXED = ([8, 20, 37, 64, 100, 8, 20],
         ["parton", "ideal", "parton", "ideal", "parton", "parton", "ideal"],
         [0.05, 0.3, math.inf, 1.0, 0.1, 2.0, 0.02])


@pytest.mark.parametrize("precision,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_mixed_batch_parity(precision, tol):
    Qs, gases, taus = MIXED
    got, state = run_batch(Qs, gases, taus, precision, 60)
    ref, rstates = oracle_batch(Qs, gases, taus, 60)
    e = errors(got, ref)
    print(precision, e)
    for k, v in e.items():
        assert v <= tol, (k, e)
    if precision == "f64":
        flat = np.concatenate(rstates)
        assert np.abs(state - flat).max() <= 1e-12 * np.abs(flat).max()


def test_large_q_and_many_runs_fp64():
    """Q_xi = 512 (the largest of the batched workload) and a block of many runs
    sharing a small Q_xi."""
    Qs = [512, 300] + [10] * 70
    gases = ["parton"] * len(Qs)
    taus = [0.2, math.inf] + list(np.linspace(0.05, 1.0, 70))
    got, _ = run_batch(Qs, gases, taus, "f64", 8, dtau=2e-3)
    ref, _ = oracle_batch(Qs, gases, taus, 8, dtau=2e-3)
    e = errors(got, ref)
    for k, v in e.items():
        assert v <= 1e-12, (k, e)


def test_seeded_workload_sample_fp32():
    """A sample of the seeded batched workload (Q_xi in [8, 512], eta/s log-uniform,
    T0 uniform): FP32 path against the oracle."""
    qxi, eta_s, T0 = workloads.bjorken_batch(nruns=24)
    taus = [5 * 0.1973269804 * e / (0.5 * t) for e, t in zip(eta_s, T0)]
    got, _ = run_batch(qxi, ["parton"] * 24, taus, "f32", 20, dtau=1e-3)
    ref, _ = oracle_batch(qxi, ["parton"] * 24, taus, 20, dtau=1e-3)
    e = errors(got, ref)
    for k, v in e.items():
        assert v <= 1e-5, (k, e)


def test_density_conservation_ideal_gas():
    """n tau = 1 for the ideal gas (Eq. bjorken_n)."""
    from paper_1612_01287_gb300 import Bjorken
    with Bjorken([16, 64], "ideal", [0.3, 0.05], precision="f64", dtau=1e-2) as b:
        b.step(100)
        o = b.read()
    assert np.abs(o["n"] * o["tau"] - 1).max() < 1e-12


@pytest.mark.parametrize("precision,kp_mode,tol", [("f64", "simt", 1e-4), ("f32", "tf32x3", 1e-4)])
def test_transition_regime_against_florkowski(precision, kp_mode, tol):
    """4 pi eta/s = 1, 3, 10 at T0 = 0.3 GeV (Sec. V C): T and P_L/P_T of the GPU
    runs (Q_xi = 40, Q_L = 3, dtau = 1e-3, tau to 10) against the semi-analytic
    solution of Eqs. flork_sol."""
    import math
    from paper_1612_01287_gb300 import Bjorken
    from tests import exact
    e4 = [1.0, 3.0, 10.0]
    taus = [exact.tau_aw0_bjorken(e / (4 * math.pi), 0.3, 0.5) for e in e4]
    ref = [exact.florkowski_parton(t, tau_f=10.0, dtau=0.01) for t in taus]
    marks = [1.0 + 0.5 * k for k in range(1, 19)]
    got = []
    with Bjorken([40] * 3, "parton", taus, Q_L=3, precision=precision, kp_mode=kp_mode,
                 dtau=1e-3) as b:
        done = 0
        for m in marks:
            n = int(round((m - 1.0) / 1e-3)) - done
            b.step(n)
            done += n
            got.append(b.read())
    for r in range(3):
        tau, T, _, PL = ref[r]
        for m, o in zip(marks, got):
            i = int(round((m - 1.0) / 0.01))
            PT = (3 * T[i] ** 4 - PL[i]) / 2
            assert abs(o["T"][r] / T[i] - 1) < tol, (e4[r], m)
            assert abs(o["PL"][r] / o["PT"][r] - PL[i] / PT) < tol, (e4[r], m)
