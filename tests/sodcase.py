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
    """max_s |a - b| / max_s |b| (normalised by the reference field's maximum)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    if scale == 0.0:
        return np.abs(a).max()
    return np.abs(a - b).max() / scale


def field_errors(mg, mo):
    """Parity metric on n, E, beta, Pi.

    n and E: max-normalised relative error.  beta: absolute error (beta is a
    velocity in units of c, and vanishes in the unperturbed chambers).  Pi: error
    normalised by the pressure scale max_s P (Pi is a small difference of O(P)
    stresses, Eq. pi_val, so its own maximum is not a meaningful scale)."""
    e = {"n": rel_err(mg["n"], mo["n"]), "E": rel_err(mg["E"], mo["E"]),
         "beta": float(np.abs(np.asarray(mg["beta"]) - np.asarray(mo["beta"])).max())}
    e["Pi"] = float(np.abs(np.asarray(mg["Pi"]) - np.asarray(mo["Pi"])).max() / np.abs(mo["P"]).max())
    return e


def compare(case, steps, precision, tol_fields, tol_pop=None):
    """Run both sides; return dict of errors; assert against the tolerances."""
    fg, mg = run_gpu(case, steps, precision)
    fo, mo = run_oracle(case, steps)
    errs = field_errors(mg, mo)
    errs["populations"] = rel_err(fg, fo.T)
    for k in PARITY_FIELDS:
        assert errs[k] <= tol_fields, (k, errs)
    if tol_pop is not None:
        assert errs["populations"] <= tol_pop, errs
    return errs


def oracle_rounding_envelope(case, steps, every=16, seed=3):
    """How far the oracle itself moves when its state is nudged by one ulp (random
    sign, every `every` steps): the size of differences that rounding alone
    produces in this nonlinear scheme over `steps` steps."""
    p = oracle_params(case)
    f = oracle.sod_init_fields(p, *case["fields"]) if "fields" in case else oracle.sod_init_riemann(p)
    rng = np.random.default_rng(seed)
    g = f.copy()
    done = 0
    while done < steps:
        n = min(every, steps - done)
        f = oracle.sod_steps(p, f, n)
        g = np.nextafter(g, np.where(rng.random(g.shape) < 0.5, -np.inf, np.inf))
        g = oracle.sod_steps(p, g, n)
        done += n
    mf, mg = oracle.sod_moments(p, f), oracle.sod_moments(p, g)
    e = field_errors(mg, mf)
    e["populations"] = rel_err(g, f)
    return e


def oracle_fp32_envelope(case, steps, seed=3):
    """How far the oracle moves when each of its RK stage values (Eq. rk3) is
    rounded to FP32 and then nudged by one FP32 ulp (random sign): the size of
    differences that FP32 storage and arithmetic, about one ulp per stage,
    produce in this nonlinear scheme over `steps` steps.  The stages are
    composed here from the oracle's right-hand side L(f) (Eq. L_Sod)."""
    p = oracle_params(case)
    f = oracle.sod_init_fields(p, *case["fields"]) if "fields" in case else oracle.sod_init_riemann(p)
    rng = np.random.default_rng(seed)

    def r32(x):
        y = x.astype(np.float32)
        away = np.where(rng.random(y.shape) < 0.5, -np.inf, np.inf).astype(np.float32)
        return np.nextafter(y, away).astype(np.float64)

    dt = p.dt
    g = r32(f)
    for _ in range(steps):
        g1 = r32(g + dt * oracle.sod_rhs(p, g))
        g2 = r32(0.75 * g + 0.25 * (g1 + dt * oracle.sod_rhs(p, g1)))
        g = r32(g / 3.0 + 2.0 / 3.0 * (g2 + dt * oracle.sod_rhs(p, g2)))
    f = oracle.sod_steps(p, f, steps)
    return field_errors(oracle.sod_moments(p, g), oracle.sod_moments(p, f))
