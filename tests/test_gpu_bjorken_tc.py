"""The tensor-core (tcgen05, 3xTF32) K^P contraction of the batched Bjorken
path: the contraction alone against an FP64 product with the oracle's K^P,
and whole runs against the FP64 oracle at the FP32 tolerance."""
import math

import numpy as np
import pytest

import oracle
from paper_1612_01287_gb300 import workloads
from tests.test_gpu_bjorken import MIXED, errors, oracle_batch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import build, load
    build.build()
    load()


def split_runs(flat, Qs, QL):
    out, o = [], 0
    for Q in Qs:
        out.append(flat[o:o + QL * Q].reshape(QL, Q))
        o += QL * Q
    return out


@pytest.mark.parametrize("QL", [2, 3])
def test_contraction_against_fp64(QL):
    """y = K^P f for Q spanning one to four M-tiles, ragged K-blocks and
    several column blocks per Q; errors relative to sum_j' |K||f|."""
    from paper_1612_01287_gb300 import Bjorken
    Qs = [8, 20, 33, 64, 100, 128, 129, 200, 257, 384, 511, 512] + [40] * 60
    rng = np.random.default_rng(workloads.SEED)
    with Bjorken(Qs, "parton", math.inf, Q_L=QL, precision="f32", kp_mode="tf32x3") as b:
        f = rng.uniform(0.0, 1.0, size=int(QL * sum(Qs))).astype(np.float32)
        f[::7] *= -0.5  # signed entries too
        b.set_state(f)
        y = b.kp_apply()
    worst = 0.0
    for Q, fr, yr in zip(Qs, split_runs(f.astype(np.float64), Qs, QL), split_runs(y, Qs, QL)):
        K = oracle.kp_matrix(Q)
        ref = fr @ K.T                    # [k][j] = sum_j' K[j][j'] f[k][j']
        scale = np.abs(fr) @ np.abs(K).T
        err = np.abs(yr - ref) / np.maximum(scale, 1e-300)
        worst = max(worst, float(err.max()))
    print("max |y - K f| / (|K| |f|):", worst)
    assert worst < 2e-5


@pytest.mark.parametrize("QL", [2, 3, 4])
def test_mixed_batch_parity_tf32x3(QL):
    """Q_L = 2 is the paper's radial set; 3 the workload's; 4 the largest the
    tensor-core epilogue takes."""
    from paper_1612_01287_gb300 import Bjorken
    Qs, gases, taus = MIXED
    with Bjorken(Qs, gases, taus, Q_L=QL, precision="f32", kp_mode="tf32x3", dtau=1e-2) as b:
        b.step(60)
        got = b.read()
    ref, _ = oracle_batch(Qs, gases, taus, 60, Q_L=QL)
    e = errors(got, ref)
    print("tf32x3", e)
    for k, v in e.items():
        assert v <= 1e-5, (k, e)


def test_seeded_workload_sample_tf32x3():
    from paper_1612_01287_gb300 import Bjorken
    qxi, eta_s, T0 = workloads.bjorken_batch(nruns=24)
    taus = [5 * 0.1973269804 * e / (0.5 * t) for e, t in zip(eta_s, T0)]
    with Bjorken(qxi, "parton", taus, Q_L=3, precision="f32", kp_mode="tf32x3", dtau=1e-3) as b:
        b.step(20)
        got = b.read()
    ref, _ = oracle_batch(qxi, ["parton"] * 24, taus, 20, dtau=1e-3)
    e = errors(got, ref)
    print("tf32x3 workload", e)
    for k, v in e.items():
        assert v <= 1e-5, (k, e)


def test_graph_replayed_steps_match_plain_launches():
    """On a non-default stream the tensor-core steps run as graphs of two
    steps (one per parity of the moment buffers), the odd remainder as plain
    launches, the stage times read from a device step counter: uneven step
    counts give bitwise the states of plain launches on the default stream."""
    import torch
    from paper_1612_01287_gb300 import Bjorken
    Qs, gases, taus = MIXED
    st = torch.cuda.Stream()
    kw = dict(Q_L=3, precision="f32", kp_mode="tf32x3", dtau=1e-2)
    with Bjorken(Qs, gases, taus, **kw) as a, Bjorken(Qs, gases, taus, stream=st, **kw) as b:
        a.step(18)
        for n in (7, 6, 1, 4):
            b.step(n)
        st.synchronize()
        fa, fb = a.get_state(), b.get_state()
        ra, rb = a.read(), b.read()
    assert np.array_equal(fa, fb)
    for k in ra:
        assert np.array_equal(ra[k], rb[k]), k


def test_tf32x3_tracks_simt_fp32():
    """The two FP32 contraction paths agree on a long ideal-gas run."""
    from paper_1612_01287_gb300 import Bjorken
    Qs = [16, 64, 200]
    res = []
    for mode in ("simt", "tf32x3"):
        with Bjorken(Qs, "ideal", [0.3, 0.05, 1.0], precision="f32", kp_mode=mode,
                     dtau=1e-2) as b:
            b.step(200)
            res.append(b.read())
    for k in ("E", "PL"):
        a, c = res[0][k], res[1][k]
        assert np.abs(a - c).max() <= 1e-5 * np.abs(a).max(), k
    assert np.abs(res[1]["n"] * res[1]["tau"] - 1).max() < 1e-5


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    """Failure handling of the tensor-core kernel: in a self-test launch the
    worker warps never signal their operand tiles (a flag that nothing sets).
    The issuing thread's bounded mbarrier wait runs out; every CTA records the
    time-out, waits for the copies it issued, frees its tensor memory and
    returns.  The host reads RSLB_ERR_TIMEOUT; the same handle then steps and
    matches the oracle as if nothing had happened."""
    import time
    from paper_1612_01287_gb300 import Bjorken
    Qs, taus = [8, 33, 130], [0.05, 0.5, math.inf]
    with Bjorken(Qs, "parton", taus, Q_L=3, precision="f32", kp_mode="tf32x3", dtau=1e-2) as b:
        t0 = time.perf_counter()
        rc, msg = b.selftest_timeout()
        waited = time.perf_counter() - t0
        assert rc == 8, (rc, msg)
        assert "bounded wait" in msg
        assert waited < 30.0
        b.step(20)
        got = b.read()
    ref, _ = oracle_batch(Qs, ["parton"] * 3, taus, 20)
    e = errors(got, ref)
    for k, v in e.items():
        assert v <= 1e-5, (k, e)
