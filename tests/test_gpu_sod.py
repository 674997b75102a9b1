"""GPU parity of the Sod shock-tube path against the FP64 oracle.

Tolerances: the FP64 path must match to 1e-12 and the FP32 path to 1e-5 in
the max-normalised error max_s|a-b|/max_s|b| on n, E, beta and Pi (the shear
stress of Eq. pi_val); FP64 populations are also compared element by element.
"""

import numpy as np
import pytest

import oracle
from paper_1612_01287_gb300 import workloads
from paper_1612_01287_gb300._lib import PACKED_TILE_CELLS as PACKED
from tests import sodcase

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import build, load
    build.build()
    load()


def small_case():
    w = workloads.sod_small()
    w.pop("t_end")
    return w


def test_small_workload_fp64_parity():
    """The 256-cell, 60-velocity shock tube, 100 steps: FP64 parity."""
    errs = sodcase.compare(small_case(), 100, "f64", TOL64, TOL64)
    print("fp64 100-step errors", errs)


def test_small_workload_full_run_fp64_within_rounding_envelope():
    """Full run to t = 0.8 (1600 steps).  The WENO5 weights make the scheme
    amplify rounding: the oracle nudged by one ulp every 16 steps drifts from
    itself by ~1e-8 over this run.  The GPU must stay within that envelope."""
    case = small_case()
    errs = sodcase.compare(case, 1600, "f64", 1.0, None)
    env = sodcase.oracle_rounding_envelope(case, 1600)
    print("fp64 full-run errors", errs, "oracle envelope", env)
    for k in sodcase.PARITY_FIELDS:
        assert errs[k] <= 100.0 * env[k] + TOL64, (k, errs, env)


def test_small_workload_fp32_parity():
    errs = sodcase.compare(small_case(), 100, "f32", TOL32)
    print("fp32 100-step errors", errs)


def test_small_workload_full_run_fp32_within_rounding_envelope():
    """Full run to t = 0.8 in FP32.  FP32 storage and arithmetic perturb every
    stage by about one FP32 ulp, and the WENO5 weights amplify such
    perturbations: the oracle, with its stage values rounded to FP32 and nudged
    by one FP32 ulp at every stage, drifts from itself by ~1e-5 over this run.
    The GPU must stay within 10 times that envelope."""
    case = small_case()
    errs = sodcase.compare(case, 1600, "f32", 1.0, None)
    env = sodcase.oracle_fp32_envelope(case, 1600)
    print("fp32 full-run errors", errs, "oracle fp32 envelope", env)
    for k in sodcase.PARITY_FIELDS:
        assert errs[k] <= 10.0 * env[k] + TOL32, (k, errs, env)


@pytest.mark.parametrize("precision,tol", [("f64", TOL64), ("f32", TOL32)])
def test_ragged_fixed_eq_odd_qxi(precision, tol):
    """Z not a multiple of the tile, fixed-equilibrium ghosts, odd Q_xi (a xi = 0
    node), Q_L = 2 as in the paper, N_Omega = 3."""
    case = dict(Z=100, Q_xi=7, Q_L=2, N_Omega=3, bc="fixed_eq", tau=2e-3, dt=1e-3,
                z_min=-0.5, z_max=0.5, left=(1.0, 1.0, 0.0), right=(0.125, 0.5, 0.0))
    sodcase.compare(case, 60, precision, tol, tol if precision == "f64" else None)


@pytest.mark.parametrize("precision,tol", [("f64", TOL64), ("f32", TOL32)])
def test_periodic_etas_smooth_flow(precision, tol):
    """Periodic domain, smooth moving state, the eta/s relaxation-time law."""
    Z = 64
    case = dict(Z=Z, Q_xi=12, Q_L=3, N_Omega=5, bc="periodic", tau_mode="etas", tau_AW0=4e-3,
                lambda_ref=1.0, dt=2e-3, z_min=0.0, z_max=1.0,
                fields=workloads.random_smooth_fields(Z))
    sodcase.compare(case, 40, precision, tol, tol if precision == "f64" else None)


@pytest.mark.parametrize("precision,tol", [("f64", TOL64), ("f32", TOL32)])
def test_collisionless(precision, tol):
    case = dict(Z=80, Q_xi=10, Q_L=2, bc="fixed_eq", tau_mode="none", dt=5e-3, z_min=-0.5,
                z_max=0.5, left=(1.0, 1.0, 0.0), right=(0.125, 0.5, 0.0))
    sodcase.compare(case, 40, precision, tol, tol if precision == "f64" else None)


@pytest.mark.parametrize("Q_xi,Q_L", [(4, 2), (20, 3), (50, 3)])
def test_small_velocity_sets_segmented_rows(Q_xi, Q_L):
    """V = 8, 60, 150: rows split into segments across threads."""
    case = dict(Z=96, Q_xi=Q_xi, Q_L=Q_L, N_Omega=min(Q_xi - 1, 5), bc="outflow", tau=1e-3,
                dt=5e-4, left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0))
    sodcase.compare(case, 30, "f64", TOL64, TOL64)


@pytest.mark.parametrize("Z", [1, 2, 3, 33])
def test_tiny_domains(Z):
    case = dict(Z=Z, Q_xi=6, Q_L=2, bc="outflow", tau=1e-2, dt=2e-3, z_min=-1.0, z_max=1.0,
                left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0))
    sodcase.compare(case, 10, "f64", TOL64, TOL64)


@pytest.mark.parametrize("precision,tol,Q_xi", [("f64", TOL64, 200), ("f32", TOL32, 200),
                                                ("f64", TOL64, 300), ("f32", TOL32, 300)])
def test_large_velocity_sets(precision, tol, Q_xi):
    """V = 600 (the large workload) and V = 900 (narrower tiles)."""
    case = dict(Z=48, Q_xi=Q_xi, Q_L=3, N_Omega=5, bc="outflow", tau=1e-2, dt=1e-3,
                left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0))
    sodcase.compare(case, 6, precision, tol, tol if precision == "f64" else None)


@pytest.mark.parametrize("precision,tiles,tol,Q_xi", [("f32", (PACKED, 64, 32, 16), 1e-6, 100),
                                                      ("f32", (128, 64, 32, 16), 1e-6, 8),
                                                      ("f64", (16, 8), 1e-13, 100),
                                                      ("f64", (16, 8), 1e-13, 8)])
def test_tile_width_does_not_change_results(precision, tiles, tol, Q_xi):
    """V = 300 and V = 24 (moments summed per lane below 128 velocities)."""
    from paper_1612_01287_gb300 import Sod
    case = sodcase.gpu_kwargs(small_case())
    case.update(Z=200, Q_xi=Q_xi)
    out = []
    for B in tiles:
        with Sod(precision=precision, tile_cells=B, **case) as s:
            s.step(20)
            out.append(s.moments())
    for other in out[1:]:
        errs = sodcase.field_errors(other, out[0])
        assert max(errs.values()) <= tol, errs


@pytest.mark.parametrize("precision,tol,Q_xi,N_Omega", [
    ("f64", TOL64, 16, 7), ("f64", TOL64, 16, 10), ("f64", TOL64, 16, 12),
    ("f32", TOL32, 16, 7), ("f32", TOL32, 16, 10), ("f32", TOL32, 16, 12),
    ("f32", TOL32, 50, 7), ("f32", TOL32, 50, 12)])
def test_truncation_orders_above_six(precision, tol, Q_xi, N_Omega):
    """f^eq truncated above the paper's largest order (App. A stops at m = 6): the
    a_{l,m} integrals by the 16-node rule (FP32, N_Omega = 7), the 32-node rule
    (FP64; FP32 above 7) and, at 150 velocities, the packed FP32x2 kernel
    (N_Omega = 7) or the scalar kernel (N_Omega = 12).  Boosted chambers, so that
    the high Legendre orders carry weight (Eq. feq_trunc)."""
    case = dict(Z=72, Q_xi=Q_xi, Q_L=3, N_Omega=N_Omega, bc="fixed_eq", tau=5e-3, dt=1e-3,
                left=(0.8, 1.2, 0.6), right=(0.3, 0.7, -0.5))
    if precision == "f32" and Q_xi == 50:
        from paper_1612_01287_gb300 import Sod
        with Sod(precision="f32", **sodcase.gpu_kwargs(case)) as s:
            assert (s.launch_info()[0] == PACKED) == (N_Omega <= 7)
    errs = sodcase.compare(case, 30, precision, tol, tol if precision == "f64" else None)
    print(precision, Q_xi, N_Omega, errs)


def test_moving_states_negative_beta_fp64():
    """Boosted initial states (sgn(beta) enters f^eq through P_m(sgn(beta) xi))."""
    case = dict(Z=64, Q_xi=16, Q_L=3, N_Omega=6, bc="fixed_eq", tau=5e-3, dt=1e-3,
                left=(0.8, 1.2, 0.5), right=(0.3, 0.7, -0.6))
    sodcase.compare(case, 40, "f64", TOL64, TOL64)


@pytest.mark.parametrize("precision,tol,tau", [("f64", TOL64, 1e-2), ("f32", TOL32, 1e-4),
                                               ("f32", TOL32, 1e-2), ("f32", TOL32, 1.0),
                                               ("f32", TOL32, 10.0)])
def test_full_size_sampled_cells(precision, tol, tau):
    """65536 cells x 600 velocities (the benchmark launch, every relaxation time of
    the benchmark in FP32: dt/tau = 0.15 down to 1.5e-6): two steps on the GPU;
    sampled cells are recomputed by the oracle on a window wide enough that its
    own boundaries cannot reach the sample (each RK stage reaches 3 cells)."""
    from paper_1612_01287_gb300 import Sod
    w = workloads.sod_large(tau=tau)
    Z, dz = w["Z"], w["dz"]
    xi, _, _, _ = __import__("paper_1612_01287_gb300").quadrature(w["Q_xi"], w["Q_L"])
    dt = w["cfl"] * dz / np.abs(xi).max()
    steps = 2
    with Sod(Z=Z, Q_xi=w["Q_xi"], Q_L=w["Q_L"], N_Omega=w["N_Omega"], bc=w["bc"], tau=w["tau"],
             dt=dt, left=w["left"], right=w["right"], precision=precision) as s:
        if precision == "f32":
            assert s.launch_info()[0] == PACKED
        s.step(steps)
        mg = s.moments()
    R = 9 * steps + 6
    rng = np.random.default_rng(7)
    samples = sorted(set([0, 1, Z // 2 - 2, Z // 2 - 1, Z // 2, Z // 2 + 1, Z - 1]
                         + list(rng.integers(0, Z, size=3))))
    keys = sodcase.PARITY_FIELDS + ("P",)
    got = {k: [] for k in keys}
    ref = {k: [] for k in keys}
    nL, TL, bL = w["left"]
    nR, TR, bR = w["right"]
    for s0 in samples:
        lo, hi = max(0, s0 - R), min(Z, s0 + R + 1)
        zc = -1.0 + (np.arange(lo, hi) + 0.5) * dz
        fields = (np.where(zc < 0, nL, nR), np.where(zc < 0, TL, TR), np.where(zc < 0, bL, bR))
        case = dict(Z=hi - lo, Q_xi=w["Q_xi"], Q_L=w["Q_L"], N_Omega=w["N_Omega"], bc="outflow",
                    tau=w["tau"], dt=dt, z_min=-1.0 + lo * dz, z_max=-1.0 + hi * dz,
                    fields=fields)
        _, mo = sodcase.run_oracle(case, steps)
        for k in keys:
            got[k].append(mg[k][s0])
            ref[k].append(mo[k][s0 - lo])
    errs = sodcase.field_errors(got, ref)
    for k in sodcase.PARITY_FIELDS:
        assert errs[k] <= tol, (k, errs, samples)


def test_checkpoint_resume_is_bitwise():
    from paper_1612_01287_gb300 import Sod
    case = sodcase.gpu_kwargs(small_case())
    with Sod(precision="f32", **case) as a:
        a.step(30)
        ref = a.get_state()
    with Sod(precision="f32", **case) as b:
        b.step(12)
        snap = b.get_state()
    with Sod(precision="f32", **case) as c:
        c.set_state(snap)
        c.step(18)
        got = c.get_state()
    np.testing.assert_array_equal(got, ref)


def test_deterministic_repeat():
    from paper_1612_01287_gb300 import Sod
    case = sodcase.gpu_kwargs(small_case())
    out = []
    for _ in range(2):
        with Sod(precision="f32", **case) as s:
            s.step(20)
            out.append(s.get_state())
    np.testing.assert_array_equal(out[0], out[1])


def test_nonphysical_state_reported():
    """A negative density is caught on the device and reported on the host."""
    from paper_1612_01287_gb300 import RslbError, Sod
    Z = 32
    n = np.ones(Z)
    n[5] = -1.0
    with pytest.raises(RslbError) as ei:
        Sod(Z=Z, Q_xi=6, Q_L=2, bc="outflow", tau=1e-2, dt=1e-3,
            fields=(n, np.ones(Z), np.zeros(Z)))
    assert ei.value.code == 6
    # a NaN planted in the populations is reported by the next sync
    with Sod(Z=Z, Q_xi=6, Q_L=2, bc="outflow", tau=1e-2, dt=1e-3, precision="f64") as s:
        f = s.get_state()
        f[:, 7] = np.nan
        s.set_state(f)
        s.step(1)
        with pytest.raises(RslbError) as ei:
            s.sync()
        assert ei.value.code == 6 and "cell" in str(ei.value)


def test_graph_captured_steps_match_plain_launches():
    """On a non-default stream rslb_step replays a captured graph of 8 steps;
    the result is bitwise the one of plain launches."""
    import torch
    from paper_1612_01287_gb300 import Sod
    case = sodcase.gpu_kwargs(small_case())
    with Sod(precision="f32", **case) as a:
        a.step(20)
        ref = a.get_state()
    s = torch.cuda.Stream()
    with Sod(precision="f32", stream=s, **case) as b:
        b.step(20)
        b.step(3)
        b.step(16)
        got = b.get_state()
    with Sod(precision="f32", **case) as c:
        c.step(39)
        ref39 = c.get_state()
    np.testing.assert_array_equal(got, ref39)
    assert not np.array_equal(ref, ref39)


@pytest.mark.parametrize("bc", ["fixed_eq", "periodic", "outflow"])
@pytest.mark.parametrize("precision,tol", [("f32", TOL32), ("f64", TOL64)])
def test_boundary_tiles_at_many_velocities(bc, precision, tol):
    """150 velocities (the packed FP32 kernel, bulk-tensor staging of the
    interior tiles) on 130 cells: interior tiles, both boundary tiles with each
    boundary rule, and a ragged last tile."""
    from paper_1612_01287_gb300 import Sod
    n, T, b = workloads.random_smooth_fields(130, beta_max=0.4)
    case = dict(Z=130, Q_xi=50, Q_L=3, N_Omega=5, bc=bc, tau=5e-3, dt=1e-3, fields=(n, T, b))
    if precision == "f32":
        with Sod(precision="f32", **sodcase.gpu_kwargs(case)) as s:
            assert s.launch_info()[0] == PACKED
    errs = sodcase.compare(case, 20, precision, tol)
    print(bc, precision, errs)


@pytest.mark.parametrize("Z,Q_xi,bc,tau_mode", [
    (36, 200, "outflow", "const"),      # two tiles, the second ragged
    (100, 200, "fixed_eq", "const"),    # ragged last tile, fixed ghosts
    (300, 200, "periodic", "etas"),     # periodic ghosts, eta/s law
    (130, 200, "outflow", "none"),      # collisionless
    (1000, 200, "outflow", "const"),    # several tiles per CTA at this grid
    (140, 50, "fixed_eq", "const"),     # 150 velocities: one sweep round
    (200, 180, "outflow", "etas"),      # 540 velocities, uneven rounds
])
def test_persistent_packed_kernel_is_bitwise_the_per_tile_kernel(Z, Q_xi, bc, tau_mode):
    """The persistent pipelined form of the packed FP32x2 kernel (one CTA per SM,
    two tile buffers, bulk-tensor staging of every tile including the boundary
    ones, ghost cells filled afterwards) runs the same phase code as the
    one-CTA-per-tile form: the populations agree bitwise after 13 steps."""
    from paper_1612_01287_gb300 import Sod
    n, T, b = workloads.random_smooth_fields(Z, beta_max=0.5)
    case = dict(Z=Z, Q_xi=Q_xi, Q_L=3, N_Omega=5, bc=bc, tau_mode=tau_mode, tau=5e-3,
                tau_AW0=4e-3, lambda_ref=1.0, dt=1e-3, fields=(n, T, b))
    out = {}
    for form in ("per_tile", "persistent"):
        with Sod(precision="f32", packed_form=form, **case) as s:
            tc, nt = s.launch_info()
            assert tc == PACKED
            s.step(13)
            out[form] = (nt, s.get_state())
    assert out["persistent"][0] != out["per_tile"][0]
    np.testing.assert_array_equal(out["persistent"][1], out["per_tile"][1])


def test_packed_kernel_forms_are_selected_as_asked():
    from paper_1612_01287_gb300 import RslbError, Sod
    case = dict(Q_xi=200, Q_L=3, N_Omega=5, bc="outflow", tau=1e-2, dt=1e-4)
    with Sod(Z=64, precision="f32", **case) as s:
        assert s.launch_info() == (PACKED, 8 * PACKED)
    with Sod(Z=64, precision="f32", packed_form="persistent", **case) as s:
        assert s.launch_info() == (PACKED, 512)
    with pytest.raises(RslbError):  # too short for its bulk copies
        Sod(Z=30, precision="f32", packed_form="persistent", **case)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("f32", 1e-12)])
@pytest.mark.parametrize("Z,Q_xi", [(1000, 50), (77, 7)])
def test_output_moments_of_a_given_state(precision, tol, Z, Q_xi):
    """rslb_moments on a state loaded with rslb_set_state equals the oracle's
    moments and Landau matching (Eq. macro_jk, Eqs. E_landau-pi_val) of the
    same stored values.  The FP32 path sums exact products as double-floats,
    so it is held to FP64-level agreement too.  Z is not a multiple of the
    block width and the velocity chunks are uneven."""
    from paper_1612_01287_gb300 import Sod
    rng = np.random.default_rng(20261203 + Z)
    zc = np.linspace(-1.0, 1.0, Z)
    n = 1.0 + 0.5 * np.sin(3.0 * zc)
    T = 0.8 + 0.3 * np.cos(2.0 * zc)
    beta = 0.7 * np.sin(5.0 * zc)  # at |beta| = 0.9 the truncated f^eq is too negative
    # for the noisy state below to stay physical
    case = dict(Z=Z, Q_xi=Q_xi, Q_L=3, bc="outflow", tau=1e-2, dt=1e-4)
    p = sodcase.oracle_params(case)
    f = oracle.sod_init_fields(p, n, T, beta)  # oracle layout [Z][V]
    f = f * (1.0 + 0.05 * rng.uniform(-1.0, 1.0, f.shape))  # off equilibrium: Pi, q != 0
    with Sod(precision=precision, fields=(n, T, beta), **case) as s:
        s.set_state(f.T)  # library layout [V][Z]
        stored = s.get_state().astype(np.float64)
        mg = s.moments()
    mo = oracle.sod_moments(p, np.ascontiguousarray(stored.T))
    # q = -4T(N^z - n beta gamma) and Pi = 2E/3 - D are differences of nearly
    # equal terms: their rounding is measured against the size of those terms
    scale = {k: np.abs(mo[k]).max() for k in oracle.SOD_FIELDS}
    scale["q"] = np.abs(4.0 * mo["T"] * mo["Nz"]).max()
    scale["Pi"] = np.abs(mo["E"]).max()
    for k in oracle.SOD_FIELDS:
        err = np.abs(mg[k] - mo[k]).max() / scale[k]
        assert err <= tol, (k, err)
