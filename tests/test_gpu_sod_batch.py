"""Batched shock tubes (``rslb_sod_batch``): every run of an uneven batch must
follow the same trajectory as the single-run path with its own dt, stop at its
own step count, and agree with the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_1612_01287_gb300 import workloads
from tests.sodcase import PARITY_FIELDS, field_errors, run_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import build, load
    build.build()
    load()


RUNS = [dict(Z=97, Q_xi=8, tau=0.05, t_end=0.1),
        dict(Z=256, Q_xi=20, tau=1e-2, t_end=0.08),
        dict(Z=130, Q_xi=20, tau=0.3, t_end=0.12, TR=0.4),
        dict(Z=64, Q_xi=50, tau=2.0, t_end=0.05),
        dict(Z=200, Q_xi=8, tau=1e-3, t_end=0.02),
        dict(Z=33, Q_xi=201, tau=0.02, t_end=0.03, nR=0.2, TR=2.0)]


def single(R, nsteps, dt, precision):
    from paper_1612_01287_gb300 import Sod
    left = (R.get("nL", 1.0), R.get("TL", 1.0), 0.0)
    right = (R.get("nR", 0.125), R.get("TR", 0.8), 0.0)
    with Sod(R["Z"], R["Q_xi"], precision=precision, bc="outflow", tau=R["tau"], dt=dt,
             left=left, right=right) as s:
        s.step(nsteps)
        return s.moments()


def case_of(R, dt):
    return dict(Z=R["Z"], Q_xi=R["Q_xi"], tau=R["tau"], dt=dt, bc="outflow",
                left=(R.get("nL", 1.0), R.get("TL", 1.0), 0.0),
                right=(R.get("nR", 0.125), R.get("TR", 0.8), 0.0))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_matches_single_runs(precision):
    from paper_1612_01287_gb300 import SodBatch
    with SodBatch(RUNS, precision=precision, autotune=False) as b:
        b.run_to_end()
        assert b.steps_done == b.max_steps
        for r, R in enumerate(RUNS):
            n, dt = b.run_info(r)
            assert n == math.ceil(R["t_end"] / dt - 1e-9)
            assert abs(n * dt - R["t_end"]) < 1e-12
            got = b.moments(r)
            ref = single(R, n, dt, precision)
            # the batched and single-run kernels are separate compilations of
            # the same tile code, so they may round differently (FMA
            # contraction); a wrong step count or mixed-up tables shows up
            # orders of magnitude above these bounds
            tol = 1e-13 if precision == "f64" else 1e-6
            e = field_errors(got, ref)
            for k in PARITY_FIELDS:
                assert e[k] <= tol, (r, k, e)


def test_batch_oracle_parity_fp64_autotuned():
    from paper_1612_01287_gb300 import SodBatch
    with SodBatch(RUNS, precision="f64", autotune=True) as b:
        for V, B, K in b.tuning():
            assert B in (8, 16) and K in (1, 2), (V, B, K)
        b.run_to_end()
        for r, R in enumerate(RUNS):
            n, dt = b.run_info(r)
            _, mo = run_oracle(case_of(R, dt), n)
            e = field_errors(b.moments(r), mo)
            for k in PARITY_FIELDS:
                assert e[k] <= 1e-12, (r, k, e)


def test_finished_runs_stay_put():
    """Steps past a run's own count leave it unchanged (runs drop out)."""
    from paper_1612_01287_gb300 import SodBatch
    with SodBatch(RUNS[:3], precision="f32", autotune=False) as b:
        counts = [b.run_info(r)[0] for r in range(3)]
        short = int(np.argmin(counts))
        b.step(min(counts))
        before = b.moments(short)
        b.step(b.max_steps - b.steps_done + 9)
        after = b.moments(short)
        for k in ("n", "E", "Ttz"):
            assert np.array_equal(before[k], after[k])


def test_sweep_sample_fp32():
    """A sample of the seeded uneven sweep (Z log-uniform, Q_xi in {8..200},
    tau log-uniform, pressure ratio in [2, 20]) with short end times: batched
    FP32 against the oracle on the smaller runs, against single runs on all."""
    from paper_1612_01287_gb300 import SodBatch, quadrature
    runs = workloads.sod_sweep(nruns=10, z_hi=2048)
    for R in runs:
        xi = quadrature(R["Q_xi"], 3)[0]
        dtmax = min(0.5 * (2.0 / R["Z"]) / abs(xi[-1]), 0.5 * R["tau"])
        R["t_end"] = 12 * dtmax
    with SodBatch(runs, precision="f32", autotune=True) as b:
        b.run_to_end()
        for r, R in enumerate(runs):
            n, dt = b.run_info(r)
            assert n == 12
            got = b.moments(r)
            if R["Z"] * R["Q_xi"] <= 40000:
                _, mo = run_oracle(case_of(R, dt), n)
                e = field_errors(got, mo)
                for k in PARITY_FIELDS:
                    assert e[k] <= 1e-5, (r, k, e)
            ref = single(R, n, dt, "f32")
            for k in ("n", "E"):
                assert np.abs(got[k] - ref[k]).max() <= 1e-6 * np.abs(ref[k]).max()


def test_batch_rejects_bad_runs():
    from paper_1612_01287_gb300 import RslbError, SodBatch
    with pytest.raises(RslbError):
        SodBatch([dict(Z=0, Q_xi=8, tau=0.1, t_end=0.1)])
    with pytest.raises(RslbError):
        SodBatch([dict(Z=10, Q_xi=8, tau=-1.0, t_end=0.1)])


def test_tuning_is_cached_per_velocity_set():
    """A second batch with the same velocity sets reuses the first one's
    choice (tile kernel, CTAs per SM) without timing again."""
    import time
    from paper_1612_01287_gb300 import SodBatch
    runs = [dict(Z=600, Q_xi=50, tau=0.1, t_end=0.01), dict(Z=300, Q_xi=8, tau=0.1, t_end=0.01)]
    with SodBatch(runs, precision="f32", autotune=True) as b:
        first = b.tuning()
    t0 = time.perf_counter()
    with SodBatch(runs[::-1], precision="f32", autotune=True) as b:
        second = b.tuning()
    assert first == second
    assert time.perf_counter() - t0 < 30
