"""Helpers that run one shock-tube case on the GPU library and on the oracle
from the same parameters and compare them field by field."""
import numpy as np

import oracle

PARITY_FIELDS = ("n", "E", "beta", "Pi")


def oracle_params(case):
    return oracle.sod_params(case["Z"], case["Q_xi"], case.get("Q_L", 3), case.get("N_Omega"),
                             z_min=case.get("z_min", -1.0), z_max=case.get("z_max", 1.0),
                             bc=case.get("bc", "outflow"), tau_mode=case.get("tau_mode", "const"),
                             tau=case.get("tau", 1e-3), tau_AW0=case.get("tau_AW0", 0.0),
                             lambda_ref=case.get("lambda_ref", 1.0), dt=case["dt"],
                             left=case.get("left", (1.0, 1.0, 0.0)),
                             right=case.get("right", (0.125, 0.8, 0.0)))


def gpu_kwargs(case):
    keys = ("Z", "Q_xi", "Q_L", "N_Omega", "z_min", "z_max", "bc", "tau_mode", "tau", "tau_AW0",
            "lambda_ref", "dt", "left", "right", "fields")
    return {k: case[k] for k in keys if k in case}


def run_oracle(case, steps):
    p = oracle_params(case)
    if "fields" in case:
        f = oracle.sod_init_fields(p, *case["fields"])
    else:
        f = oracle.sod_init_riemann(p)
    f = oracle.sod_steps(p, f, steps)
    return f, oracle.sod_moments(p, f)


def run_gpu(case, steps, precision):
    from paper_1612_01287_gb300 import Sod
    with Sod(precision=precision, **gpu_kwargs(case)) as s:
        s.step(steps)
        m = s.moments()
        f = s.get_state()
    return f, m


def rel_err(a, b):
    """max_s |a - b| / max_s |b| (normalised by the field's maximum)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    if scale == 0.0:
        return np.abs(a).max()
    return np.abs(a - b).max() / scale


def compare(case, steps, precision, tol_fields, tol_pop=None):
    """Run both sides; return dict of errors; assert against the tolerances."""
    fg, mg = run_gpu(case, steps, precision)
    fo, mo = run_oracle(case, steps)
    errs = {k: rel_err(mg[k], mo[k]) for k in PARITY_FIELDS}
    errs["populations"] = rel_err(fg, fo.T)
    for k in PARITY_FIELDS:
        assert errs[k] <= tol_fields, (k, errs)
    if tol_pop is not None:
        assert errs["populations"] <= tol_pop, errs
    return errs
