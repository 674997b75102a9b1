"""The allocation-free shock-tube entry point (rslb_sod_step_noalloc).

It serves callers that may not allocate device memory; its stage buffers live in
a static device array.  These tests check it against the regular handle-based
entry points (rslb_init + rslb_step) on two calls in a row, and that oversized
problems are refused.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

CASES = [
    ("f64", dict(Z=200, Q_xi=20, Q_L=3, N_Omega=5, bc="outflow", tau=1e-3, dt=5e-4), 1e-12),
    ("f32", dict(Z=200, Q_xi=20, Q_L=3, N_Omega=5, bc="outflow", tau=1e-3, dt=5e-4), 1e-6),
    ("f64", dict(Z=150, Q_xi=7, Q_L=2, N_Omega=3, bc="fixed_eq", tau=2e-3, dt=1e-3,
                 z_min=-0.5, z_max=0.5, right=(0.125, 0.5, 0.0)), 1e-12),
    # 150 velocities: the packed FP32x2 stage kernel, whose bulk-tensor maps then
    # point into the static array
    ("f32", dict(Z=130, Q_xi=50, Q_L=3, N_Omega=5, bc="outflow", tau=5e-3, dt=1e-3), 1e-6),
    # periodic domain with the eta/s relaxation-time law, packed kernel
    ("f32", dict(Z=96, Q_xi=50, Q_L=3, N_Omega=5, bc="periodic", tau_mode="etas", tau_AW0=4e-3,
                 lambda_ref=1.0, dt=1e-3), 1e-6),
]


@pytest.mark.gpu
@pytest.mark.parametrize("precision,case,tol", CASES)
def test_noalloc_matches_handle_path_on_two_calls(precision, case, tol):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1612_01287_gb300 import Sod, build
    from paper_1612_01287_gb300._lib import sod_step_noalloc
    build.build()
    dtype = torch.float64 if precision == "f64" else torch.float32
    with Sod(precision=precision, **case) as ref:
        f0 = ref.get_state()
        # the caller owns the populations; the entry point allocates nothing
        f = torch.from_numpy(f0.copy()).to("cuda", dtype=dtype).contiguous()
        stream = torch.cuda.current_stream()
        for nsteps in (7, 5):
            sod_step_noalloc(f.data_ptr(), nsteps, precision=precision, stream=stream, **case)
            ref.step(nsteps)
            want = ref.get_state()
            got = f.cpu().numpy()
            err = np.abs(got.astype(np.float64) - want).max() / np.abs(want).max()
            assert err <= tol, (nsteps, err)


def test_noalloc_rejects_oversized_problem():
    """Too large for the static scratch array: refused before any device work."""
    from paper_1612_01287_gb300 import RslbError, build
    from paper_1612_01287_gb300._lib import sod_step_noalloc
    build.build()
    with pytest.raises(RslbError) as ei:
        sod_step_noalloc(1, 1, Z=1_000_000, Q_xi=200, Q_L=3, tau=1e-2, dt=1e-7)
    assert ei.value.code == 7 and "scratch" in str(ei.value)
    with pytest.raises(RslbError) as ei:
        sod_step_noalloc(1, 1, Z=64, Q_xi=600, Q_L=3, tau=1e-2, dt=1e-4)
    assert ei.value.code == 7
