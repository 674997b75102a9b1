"""FP64 CPU oracle of the R-SLB method -- TEST INFRASTRUCTURE ONLY.

ctypes binding of ``rslb_oracle.c``: the plain, slow reference against which the
GPU library is checked.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the GPU library and its binding) never does.

Velocity index convention: ``v = k * Q_xi + j`` (radial node k, polar node j).
Sod populations are returned cell-major, shape ``(Z, V)``.
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

SOD_FIELDS = ("n", "E", "P", "T", "beta", "gamma", "lambda_bar", "q", "Pi",
              "Nt", "Nz", "Ttt", "Ttz", "Tzz")
BJ_FIELDS = ("tau", "n", "E", "P", "T", "Pi", "PL", "PT")

BC = {"fixed_eq": 0, "outflow": 1, "periodic": 2}
TAU = {"const": 0, "etas": 1, "none": 2}
GAS = {"parton": 0, "ideal": 1}

_ERR = {1: "bad argument", 2: "nonphysical state", 3: "no convergence"}


class OracleError(RuntimeError):
    pass


class _SodParams(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_int), ("z_min", ctypes.c_double), ("z_max", ctypes.c_double),
                ("Q_xi", ctypes.c_int), ("Q_L", ctypes.c_int), ("N_Omega", ctypes.c_int),
                ("bc", ctypes.c_int), ("tau_mode", ctypes.c_int), ("tau", ctypes.c_double),
                ("tau_AW0", ctypes.c_double), ("lambda_ref", ctypes.c_double),
                ("dt", ctypes.c_double),
                ("nL", ctypes.c_double), ("TL", ctypes.c_double), ("betaL", ctypes.c_double),
                ("nR", ctypes.c_double), ("TR", ctypes.c_double), ("betaR", ctypes.c_double)]


class _BjParams(ctypes.Structure):
    _fields_ = [("Q_xi", ctypes.c_int), ("Q_L", ctypes.c_int), ("N_Omega", ctypes.c_int),
                ("gas", ctypes.c_int), ("tau_AW0", ctypes.c_double),
                ("tau0", ctypes.c_double), ("dtau", ctypes.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_legendre.restype = d
        _lib.orc_legendre.argtypes = [i, d]
        _lib.orc_laguerre2.restype = d
        _lib.orc_laguerre2.argtypes = [i, d]
        _lib.orc_weno5_face.restype = d
        _lib.orc_weno5_face.argtypes = [d, d, d, d, d]
        for name, args in (("orc_gauss_legendre", [i, p, p]),
                           ("orc_gauss_laguerre2", [i, p, p]),
                           ("orc_aeq", [d, d, d, i, p]),
                           ("orc_feq", [i, i, i, d, d, d, p]),
                           ("orc_moments", [i, i, p, p]),
                           ("orc_landau", [p, p]),
                           ("orc_kl_matrix", [i, p]),
                           ("orc_kp_matrix", [i, p]),
                           ("orc_sod_init_fields", [p, p, p, p, p]),
                           ("orc_sod_init_riemann", [p, p]),
                           ("orc_sod_steps", [p, p, i]),
                           ("orc_sod_moments", [p, p, p]),
                           ("orc_sod_rhs", [p, p, p]),
                           ("orc_bjorken_run", [p, p, i, i, p]),
                           ("orc_bjorken_rhs", [p, p, d, p])):
            fn = getattr(_lib, name)
            fn.restype = i
            fn.argtypes = args
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise OracleError("%s: %s (code %d)" % (what, _ERR.get(rc, "error"), rc))


def legendre(m, x):
    return lib().orc_legendre(int(m), float(x))


def laguerre2(l, x):
    return lib().orc_laguerre2(int(l), float(x))


def gauss_legendre(Q):
    x = np.zeros(Q)
    w = np.zeros(Q)
    _check(lib().orc_gauss_legendre(int(Q), _ptr(x), _ptr(w)), "gauss_legendre")
    return x, w


def gauss_laguerre2(Q):
    x = np.zeros(Q)
    w = np.zeros(Q)
    _check(lib().orc_gauss_laguerre2(int(Q), _ptr(x), _ptr(w)), "gauss_laguerre2")
    return x, w


def aeq(n, theta, u, N_Omega):
    """a^{(eq)}_{l,m}, shape (2, N_Omega+1)."""
    a = np.zeros(2 * (N_Omega + 1))
    _check(lib().orc_aeq(float(n), float(theta), float(u), int(N_Omega), _ptr(a)), "aeq")
    return a.reshape(2, N_Omega + 1)


def feq(Q_xi, Q_L, N_Omega, n, T, beta):
    """f^eq_{jk} populations, flat length Q_L*Q_xi with v = k*Q_xi + j."""
    f = np.zeros(Q_xi * Q_L)
    _check(lib().orc_feq(int(Q_xi), int(Q_L), int(N_Omega), float(n), float(T), float(beta),
                         _ptr(f)), "feq")
    return f


def moments(Q_xi, Q_L, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    M = np.zeros(5)
    _check(lib().orc_moments(int(Q_xi), int(Q_L), _ptr(f), _ptr(M)), "moments")
    return M


def landau(M):
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = np.zeros(9)
    _check(lib().orc_landau(_ptr(M), _ptr(out)), "landau")
    return dict(zip(SOD_FIELDS[:9], out))


def weno5_face(a, b, c, d, e):
    return lib().orc_weno5_face(float(a), float(b), float(c), float(d), float(e))


def kl_matrix(Q_L):
    K = np.zeros(Q_L * Q_L)
    _check(lib().orc_kl_matrix(int(Q_L), _ptr(K)), "kl_matrix")
    return K.reshape(Q_L, Q_L)


def kp_matrix(Q_xi):
    K = np.zeros(Q_xi * Q_xi)
    _check(lib().orc_kp_matrix(int(Q_xi), _ptr(K)), "kp_matrix")
    return K.reshape(Q_xi, Q_xi)


def sod_params(Z, Q_xi, Q_L=3, N_Omega=None, z_min=-1.0, z_max=1.0, bc="outflow",
               tau_mode="const", tau=1e-3, tau_AW0=0.0, lambda_ref=1.0, dt=5e-4,
               left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0)):
    """Sod parameters; ``left``/``right`` are (n, T, beta)."""
    if N_Omega is None:
        N_Omega = min(Q_xi - 1, 5)
    return _SodParams(int(Z), float(z_min), float(z_max), int(Q_xi), int(Q_L), int(N_Omega),
                      BC[bc] if isinstance(bc, str) else int(bc),
                      TAU[tau_mode] if isinstance(tau_mode, str) else int(tau_mode),
                      float(tau), float(tau_AW0), float(lambda_ref), float(dt),
                      float(left[0]), float(left[1]), float(left[2]),
                      float(right[0]), float(right[1]), float(right[2]))


def _V(p):
    return p.Q_xi * p.Q_L


def sod_init_riemann(p):
    f = np.zeros((p.Z, _V(p)))
    _check(lib().orc_sod_init_riemann(ctypes.byref(p), _ptr(f)), "sod_init_riemann")
    return f


def sod_init_fields(p, n, T, beta):
    n = np.ascontiguousarray(n, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    f = np.zeros((p.Z, _V(p)))
    _check(lib().orc_sod_init_fields(ctypes.byref(p), _ptr(n), _ptr(T), _ptr(beta), _ptr(f)),
           "sod_init_fields")
    return f


def sod_steps(p, f, nsteps):
    """Advance f (Z, V) by nsteps RK3 steps; returns a new array."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    _check(lib().orc_sod_steps(ctypes.byref(p), _ptr(f), int(nsteps)), "sod_steps")
    return f


def sod_rhs(p, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    L = np.zeros_like(f)
    _check(lib().orc_sod_rhs(ctypes.byref(p), _ptr(f), _ptr(L)), "sod_rhs")
    return L


def sod_moments(p, f):
    """Dict of per-cell fields (each length Z)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(len(SOD_FIELDS) * p.Z)
    _check(lib().orc_sod_moments(ctypes.byref(p), _ptr(f), _ptr(out)), "sod_moments")
    out = out.reshape(len(SOD_FIELDS), p.Z)
    return {k: out[i] for i, k in enumerate(SOD_FIELDS)}


def bjorken_params(Q_xi, Q_L=3, N_Omega=None, gas="parton", tau_AW0=math.inf, tau0=1.0,
                   dtau=1e-3):
    if N_Omega is None:
        N_Omega = min(Q_xi - 1, 5)
    return _BjParams(int(Q_xi), int(Q_L), int(N_Omega),
                     GAS[gas] if isinstance(gas, str) else int(gas),
                     float(tau_AW0), float(tau0), float(dtau))


def bjorken_run(p, nsteps, f=None):
    """Run nsteps; returns (f_final, history dict of arrays of length nsteps+1)."""
    V = p.Q_xi * p.Q_L
    init = f is None
    f = np.zeros(V) if f is None else np.array(f, dtype=np.float64, copy=True)
    out = np.zeros((nsteps + 1) * len(BJ_FIELDS))
    _check(lib().orc_bjorken_run(ctypes.byref(p), _ptr(f), int(init), int(nsteps), _ptr(out)),
           "bjorken_run")
    out = out.reshape(nsteps + 1, len(BJ_FIELDS))
    return f, {k: out[:, i] for i, k in enumerate(BJ_FIELDS)}


def bjorken_rhs(p, f, tau):
    f = np.ascontiguousarray(f, dtype=np.float64)
    L = np.zeros_like(f)
    _check(lib().orc_bjorken_rhs(ctypes.byref(p), _ptr(f), float(tau), _ptr(L)), "bjorken_rhs")
    return L
