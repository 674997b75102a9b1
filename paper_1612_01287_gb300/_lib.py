"""ctypes binding of the R-SLB C ABI (include/rslb.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``_build/librslb.so``.  The library must have been built (``build.build()``);
importing the binding without it raises immediately -- there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import build as _build

FIELDS = ("n", "E", "P", "T", "beta", "gamma", "lambda_bar", "q", "Pi",
          "Nt", "Nz", "Ttt", "Ttz", "Tzz")

OK = 0
ERR = {1: "RSLB_ERR_ARG", 2: "RSLB_ERR_CFL", 3: "RSLB_ERR_STIFF", 4: "RSLB_ERR_ALLOC",
       5: "RSLB_ERR_CUDA", 6: "RSLB_ERR_NONPHYSICAL", 7: "RSLB_ERR_UNSUPPORTED"}
F32, F64 = 0, 1
PACKED_TILE_CELLS = 28  # RSLB_PACKED_TILE_CELLS
BC = {"fixed_eq": 0, "outflow": 1, "periodic": 2}
TAU = {"const": 0, "etas": 1, "none": 2}


class RslbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERR.get(code, "error %d" % code), msg))
        self.code = code


class Config(ctypes.Structure):
    """Mirror of ``rslb_config``."""
    _fields_ = [("Z", ctypes.c_int), ("z_min", ctypes.c_double), ("z_max", ctypes.c_double),
                ("Q_xi", ctypes.c_int), ("Q_L", ctypes.c_int), ("N_Omega", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc", ctypes.c_int), ("tau_mode", ctypes.c_int),
                ("tau", ctypes.c_double), ("tau_AW0", ctypes.c_double),
                ("lambda_ref", ctypes.c_double), ("dt", ctypes.c_double),
                ("nL", ctypes.c_double), ("TL", ctypes.c_double), ("betaL", ctypes.c_double),
                ("nR", ctypes.c_double), ("TR", ctypes.c_double), ("betaR", ctypes.c_double),
                ("n0", ctypes.c_void_p), ("T0", ctypes.c_void_p), ("beta0", ctypes.c_void_p),
                ("tile_cells", ctypes.c_int), ("packed_form", ctypes.c_int)]


PACKED_FORMS = {"auto": 0, "per_tile": 1, "persistent": 2}


_lib = None


def lib_path():
    return _build.LIB_PATH


def load():
    """Load the built library (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("R-SLB CUDA library not built (%s missing); run "
                           "paper_1612_01287_gb300.build.build() first" % path)
    L = ctypes.CDLL(path)
    i, p, d = ctypes.c_int, ctypes.c_void_p, ctypes.c_double
    sig = {
        "rslb_quadrature": (i, [i, i, p, p, p, p]),
        "rslb_init": (i, [ctypes.POINTER(p), ctypes.POINTER(Config), p]),
        "rslb_step": (i, [p, i]),
        "rslb_sync": (i, [p]),
        "rslb_moments": (i, [p, p, i]),
        "rslb_get_state": (i, [p, p, i]),
        "rslb_set_state": (i, [p, p, i]),
        "rslb_time": (i, [p, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]),
        "rslb_launch_info": (i, [p, ctypes.POINTER(i), ctypes.POINTER(i)]),
        "rslb_destroy": (None, [p]),
        "rslb_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != OK:
        msg = load().rslb_last_error()
        raise RslbError(rc, msg.decode() if msg else "")


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def quadrature(Q_xi, Q_L):
    """(xi, w_xi, x_k, w_L) from ``rslb_quadrature``."""
    xi, wx = np.zeros(Q_xi), np.zeros(Q_xi)
    xk, wk = np.zeros(Q_L), np.zeros(Q_L)
    _check(load().rslb_quadrature(int(Q_xi), int(Q_L), _ptr(xi), _ptr(wx), _ptr(xk), _ptr(wk)))
    return xi, wx, xk, wk


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


class Sod:
    """One Sod shock-tube simulation on the current CUDA device (``rslb_handle``)."""

    def __init__(self, Z, Q_xi, Q_L=3, N_Omega=None, z_min=-1.0, z_max=1.0, precision="f32",
                 bc="outflow", tau_mode="const", tau=1e-3, tau_AW0=0.0, lambda_ref=1.0, dt=5e-4,
                 left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0), fields=None, stream=None,
                 tile_cells=0, packed_form="auto"):
        """left/right: (n, T, beta); fields: optional (n0, T0, beta0) arrays of length Z."""
        if N_Omega is None:
            N_Omega = min(Q_xi - 1, 5)
        self.Z, self.Q_xi, self.Q_L = int(Z), int(Q_xi), int(Q_L)
        self.V = self.Q_xi * self.Q_L
        if precision not in ("f32", "fp32", "f64", "fp64", F32, F64):
            raise ValueError("precision must be 'f32' or 'f64'")
        self.fp64 = precision in ("f64", "fp64", F64)
        self.dtype = np.float64 if self.fp64 else np.float32
        self._keep = None
        cfg = Config(self.Z, z_min, z_max, self.Q_xi, self.Q_L, int(N_Omega),
                     F64 if self.fp64 else F32, BC[bc] if isinstance(bc, str) else int(bc),
                     TAU[tau_mode] if isinstance(tau_mode, str) else int(tau_mode),
                     tau, tau_AW0, lambda_ref, dt, left[0], left[1], left[2],
                     right[0], right[1], right[2], None, None, None, int(tile_cells),
                     PACKED_FORMS[packed_form])
        if fields is not None:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in fields]
            self._keep = arrs
            cfg.n0, cfg.T0, cfg.beta0 = (a.ctypes.data for a in arrs)
        self._h = ctypes.c_void_p()
        self._stream = _stream_ptr(stream)
        _check(load().rslb_init(ctypes.byref(self._h), ctypes.byref(cfg), self._stream))
        self._keep = None

    def step(self, nsteps=1):
        _check(load().rslb_step(self._h, int(nsteps)))

    def sync(self):
        _check(load().rslb_sync(self._h))

    def moments(self, out=None):
        """Dict of FP64 numpy arrays (host) -- or fill a device buffer if ``out`` is a
        CUDA torch tensor of shape (14, Z)."""
        if out is not None:
            _check(load().rslb_moments(self._h, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        buf = np.zeros((len(FIELDS), self.Z))
        _check(load().rslb_moments(self._h, _ptr(buf), 0))
        return {k: buf[i] for i, k in enumerate(FIELDS)}

    def moments_into(self, host_buf):
        """Fill a caller-owned host array (14*Z doubles, e.g. pinned memory)."""
        _check(load().rslb_moments(self._h, ctypes.c_void_p(host_buf), 0))

    def get_state(self):
        """Populations as a (V, Z) array of the handle's precision."""
        f = np.zeros((self.V, self.Z), dtype=self.dtype)
        _check(load().rslb_get_state(self._h, _ptr(f), 0))
        return f

    def set_state(self, f):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        assert f.shape == (self.V, self.Z)
        _check(load().rslb_set_state(self._h, _ptr(f), 0))
        self.sync()

    def set_state_ptr(self, ptr, on_device):
        """Stream-ordered copy from a raw pointer (host pinned or device)."""
        _check(load().rslb_set_state(self._h, ctypes.c_void_p(ptr), int(on_device)))

    def time(self):
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(load().rslb_time(self._h, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def launch_info(self):
        """(cells per CTA tile, threads per CTA) of the stage kernel."""
        B, T = ctypes.c_int(), ctypes.c_int()
        _check(load().rslb_launch_info(self._h, ctypes.byref(B), ctypes.byref(T)))
        return B.value, T.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().rslb_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def sod_step_noalloc(f_ptr, nsteps, Z, Q_xi, Q_L=3, N_Omega=None, z_min=-1.0, z_max=1.0,
                     precision="f32", bc="outflow", tau_mode="const", tau=1e-3, tau_AW0=0.0,
                     lambda_ref=1.0, dt=5e-4, left=(1.0, 1.0, 0.0), right=(0.125, 0.8, 0.0),
                     stream=None):
    """Advance caller-owned device populations (pointer ``f_ptr``, V*Z values of the
    given precision) by ``nsteps`` steps with ``rslb_sod_step_noalloc``, which
    allocates no device memory (for callers that may not allocate)."""
    L = load()
    fn = L.rslb_sod_step_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    if N_Omega is None:
        N_Omega = min(Q_xi - 1, 5)
    if precision not in ("f32", "fp32", "f64", "fp64", F32, F64):
        raise ValueError("precision must be 'f32' or 'f64'")
    fp64 = precision in ("f64", "fp64", F64)
    cfg = Config(int(Z), z_min, z_max, int(Q_xi), int(Q_L), int(N_Omega), F64 if fp64 else F32,
                 BC[bc] if isinstance(bc, str) else int(bc),
                 TAU[tau_mode] if isinstance(tau_mode, str) else int(tau_mode),
                 tau, tau_AW0, lambda_ref, dt, left[0], left[1], left[2],
                 right[0], right[1], right[2], None, None, None, 0, 0)
    _check(fn(ctypes.byref(cfg), ctypes.c_void_p(f_ptr), int(nsteps), _stream_ptr(stream)))


def measure_fp64_fma(reps=20, stream=None):
    """DFMA lane operations per second of the current device
    (``rslb_measure_fp64_fma``)."""
    L = load()
    fn = L.rslb_measure_fp64_fma
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    out = ctypes.c_double()
    _check(fn(int(reps), ctypes.byref(out), _stream_ptr(stream)))
    return out.value


BJ_FIELDS = ("tau", "n", "E", "P", "T", "Pi", "PL", "PT")
GAS = {"parton": 0, "ideal": 1}
KP = {"simt": 0, "tf32x3": 2}


class BjorkenRun(ctypes.Structure):
    """Mirror of ``rslb_bjorken_run``."""
    _fields_ = [("Q_xi", ctypes.c_int), ("gas", ctypes.c_int), ("tau_AW0", ctypes.c_double)]


class BjorkenOpts(ctypes.Structure):
    """Mirror of ``rslb_bjorken_opts``."""
    _fields_ = [("Q_L", ctypes.c_int), ("precision", ctypes.c_int), ("kp_mode", ctypes.c_int),
                ("tau0", ctypes.c_double), ("dtau", ctypes.c_double)]


def _bj_sigs(L):
    if getattr(L, "_bj_ready", False):
        return
    i, p = ctypes.c_int, ctypes.c_void_p
    for name, (res, args) in {
        "rslb_bjorken_init": (i, [ctypes.POINTER(p), ctypes.POINTER(BjorkenRun), i,
                                  ctypes.POINTER(BjorkenOpts), p]),
        "rslb_bjorken_step": (i, [p, i]),
        "rslb_bjorken_read": (i, [p, p, i]),
        "rslb_bjorken_get_state": (i, [p, p]),
        "rslb_bjorken_set_state": (i, [p, p]),
        "rslb_bjorken_kp_apply": (i, [p, p]),
        "rslb_bjorken_destroy": (None, [p]),
    }.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._bj_ready = True


class Bjorken:
    """A batch of independent boost-invariant runs (``rslb_bjorken``)."""

    def __init__(self, Q_xi, gas="parton", tau_AW0=float("inf"), Q_L=3, precision="f32",
                 kp_mode="simt", tau0=1.0, dtau=1e-3, stream=None):
        """Q_xi, gas, tau_AW0: per-run sequences (scalars are broadcast)."""
        L = load()
        _bj_sigs(L)
        Q_xi = np.atleast_1d(np.asarray(Q_xi, dtype=np.int64))
        n = len(Q_xi)
        gas = np.broadcast_to(np.asarray([GAS[g] if isinstance(g, str) else int(g)
                                          for g in np.atleast_1d(gas)]), (n,))
        t0 = np.broadcast_to(np.atleast_1d(np.asarray(tau_AW0, dtype=np.float64)), (n,))
        runs = (BjorkenRun * n)()
        for r in range(n):
            runs[r].Q_xi = int(Q_xi[r])
            runs[r].gas = int(gas[r])
            runs[r].tau_AW0 = float(t0[r])
        if precision not in ("f32", "fp32", "f64", "fp64", F32, F64):
            raise ValueError("precision must be 'f32' or 'f64'")
        self.fp64 = precision in ("f64", "fp64", F64)
        self.dtype = np.float64 if self.fp64 else np.float32
        opts = BjorkenOpts(int(Q_L), F64 if self.fp64 else F32,
                           KP[kp_mode] if isinstance(kp_mode, str) else int(kp_mode),
                           float(tau0), float(dtau))
        self.nruns, self.Q_xi, self.Q_L = n, Q_xi.copy(), int(Q_L)
        self._h = ctypes.c_void_p()
        _check(L.rslb_bjorken_init(ctypes.byref(self._h), runs, n, ctypes.byref(opts),
                                   _stream_ptr(stream)))

    def step(self, nsteps=1):
        _check(load().rslb_bjorken_step(self._h, int(nsteps)))

    def read(self):
        out = np.zeros((self.nruns, len(BJ_FIELDS)))
        _check(load().rslb_bjorken_read(self._h, _ptr(out), 0))
        return {k: out[:, i] for i, k in enumerate(BJ_FIELDS)}

    def read_into(self, ptr, on_device):
        _check(load().rslb_bjorken_read(self._h, ctypes.c_void_p(ptr), int(on_device)))

    def get_state(self):
        f = np.zeros(int(self.Q_L * self.Q_xi.sum()), dtype=self.dtype)
        _check(load().rslb_bjorken_get_state(self._h, _ptr(f)))
        return f

    def set_state(self, f):
        f = np.ascontiguousarray(f, dtype=self.dtype)
        _check(load().rslb_bjorken_set_state(self._h, _ptr(f)))

    def selftest_timeout(self):
        """Run the tensor-core kernel's failure-handling self-test
        (``rslb_bjorken_selftest_timeout``); returns its status code
        (RSLB_ERR_TIMEOUT = 8 expected) and message without raising."""
        L = load()
        rc = L.rslb_bjorken_selftest_timeout(self._h)
        msg = L.rslb_last_error()
        return rc, msg.decode() if msg else ""

    def kp_apply(self):
        """K^P f of every run's current state (tensor-core path), like get_state."""
        y = np.zeros(int(self.Q_L * self.Q_xi.sum()), dtype=np.float32)
        _check(load().rslb_bjorken_kp_apply(self._h, _ptr(y)))
        return y

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().rslb_bjorken_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class SodRun(ctypes.Structure):
    """Mirror of ``rslb_sod_run``."""
    _fields_ = [("Z", ctypes.c_int), ("Q_xi", ctypes.c_int), ("tau", ctypes.c_double),
                ("nL", ctypes.c_double), ("TL", ctypes.c_double), ("nR", ctypes.c_double),
                ("TR", ctypes.c_double), ("t_end", ctypes.c_double), ("tau_mode", ctypes.c_int),
                ("tau_AW0", ctypes.c_double), ("lambda_ref", ctypes.c_double),
                ("N_Omega", ctypes.c_int), ("dt", ctypes.c_double)]


class SodBatchOpts(ctypes.Structure):
    """Mirror of ``rslb_sod_batch_opts``."""
    _fields_ = [("Q_L", ctypes.c_int), ("N_Omega", ctypes.c_int), ("precision", ctypes.c_int),
                ("bc", ctypes.c_int), ("z_min", ctypes.c_double), ("z_max", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt_over_tau", ctypes.c_double),
                ("autotune", ctypes.c_int)]


def _batch_sigs(L):
    if getattr(L, "_batch_ready", False):
        return
    i, p, ll, d = ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double
    P = ctypes.POINTER
    for name, (res, args) in {
        "rslb_sod_batch_init": (i, [P(p), P(SodRun), i, P(SodBatchOpts), p]),
        "rslb_sod_batch_step": (i, [p, i]),
        "rslb_sod_batch_info": (i, [p, P(ll), P(ll), P(d)]),
        "rslb_sod_batch_run_info": (i, [p, i, P(ll), P(d)]),
        "rslb_sod_batch_tuning": (i, [p, i, P(i), P(i), P(i)]),
        "rslb_sod_batch_moments": (i, [p, i, p]),
        "rslb_sod_batch_destroy": (None, [p]),
    }.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._batch_ready = True


class SodBatch:
    """Many independent shock tubes advanced together (``rslb_sod_batch``).

    ``runs``: sequence of dicts with keys Z, Q_xi, t_end and tau (constant
    relaxation time) or tau_mode "etas" with tau_AW0, lambda_ref and dt, and
    optionally nL, TL, nR, TR (default: the chambers of Sec. IV A), N_Omega,
    dt."""

    def __init__(self, runs, Q_L=3, N_Omega=-1, precision="f32", bc="outflow", z_min=-1.0,
                 z_max=1.0, cfl=0.5, dt_over_tau=0.5, autotune=True, stream=None):
        L = load()
        _batch_sigs(L)
        n = len(runs)
        arr = (SodRun * n)()
        for r, R in enumerate(runs):
            tm = R.get("tau_mode", "const")
            arr[r] = SodRun(int(R["Z"]), int(R["Q_xi"]), float(R.get("tau", 0.0)),
                            float(R.get("nL", 1.0)), float(R.get("TL", 1.0)),
                            float(R.get("nR", 0.125)), float(R.get("TR", 0.8)),
                            float(R["t_end"]), TAU[tm] if isinstance(tm, str) else int(tm),
                            float(R.get("tau_AW0", 0.0)), float(R.get("lambda_ref", 1.0)),
                            int(R.get("N_Omega", -1)), float(R.get("dt", 0.0)))
        if precision not in ("f32", "fp32", "f64", "fp64", F32, F64):
            raise ValueError("precision must be 'f32' or 'f64'")
        self.fp64 = precision in ("f64", "fp64", F64)
        opts = SodBatchOpts(int(Q_L), int(N_Omega), F64 if self.fp64 else F32,
                            BC[bc] if isinstance(bc, str) else int(bc), float(z_min),
                            float(z_max), float(cfl), float(dt_over_tau), int(bool(autotune)))
        self.nruns = n
        self.Z = [int(R["Z"]) for R in runs]
        self._h = ctypes.c_void_p()
        _check(L.rslb_sod_batch_init(ctypes.byref(self._h), arr, n, ctypes.byref(opts),
                                     _stream_ptr(stream)))

    def step(self, nsteps=1):
        _check(load().rslb_sod_batch_step(self._h, int(nsteps)))

    def run_to_end(self):
        self.step(self.max_steps - self.steps_done)

    def _info(self):
        a, b, c = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_double()
        _check(load().rslb_sod_batch_info(self._h, ctypes.byref(a), ctypes.byref(b),
                                          ctypes.byref(c)))
        return a.value, b.value, c.value

    @property
    def max_steps(self):
        return self._info()[0]

    @property
    def steps_done(self):
        return self._info()[1]

    @property
    def total_cv_updates(self):
        return self._info()[2]

    def run_info(self, r):
        n, dt = ctypes.c_longlong(), ctypes.c_double()
        _check(load().rslb_sod_batch_run_info(self._h, int(r), ctypes.byref(n), ctypes.byref(dt)))
        return n.value, dt.value

    def tuning(self):
        """[(V, tile_cells, ctas_per_sm)] per velocity group."""
        out, g = [], 0
        L = load()
        while True:
            V, B, K = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
            if L.rslb_sod_batch_tuning(self._h, g, ctypes.byref(V), ctypes.byref(B),
                                       ctypes.byref(K)) != OK:
                return out
            out.append((V.value, B.value, K.value))
            g += 1

    def moments(self, r):
        out = np.zeros((len(FIELDS), self.Z[r]))
        _check(load().rslb_sod_batch_moments(self._h, int(r), _ptr(out)))
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().rslb_sod_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _mlp_sigs(L):
    if getattr(L, "_mlp_ready", False):
        return
    i, p, d, u64 = ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_ulonglong
    for name, (res, args) in {
        "rslb_mlp_create": (i, [ctypes.POINTER(p), i, i, i, u64, p]),
        "rslb_mlp_num_params": (i, [p]),
        "rslb_mlp_get_params": (i, [p, p]),
        "rslb_mlp_set_params": (i, [p, p]),
        "rslb_mlp_forward": (i, [p, p, i, p]),
        "rslb_mlp_set_normalization": (i, [p, p, p, p]),
        "rslb_mlp_get_normalization": (i, [p, p, p, p]),
        "rslb_mlp_fit_normalization": (i, [p, p, p, i]),
        "rslb_mlp_loss_grad": (i, [p, p, p, i, ctypes.POINTER(d), p]),
        "rslb_mlp_train": (i, [p, p, p, i, i, i, d, u64, p]),
        "rslb_mlp_destroy": (None, [p]),
        "rslb_restrict": (i, [p, p]),
        "rslb_closure_sample": (i, [p, p, d, p, p]),
        "rslb_closure_step": (i, [p, p, d, i]),
    }.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    L._mlp_ready = True


class MLP:
    """The closure network (``rslb_mlp``); arrays passed as device pointers
    (ints, e.g. ``tensor.data_ptr()``) unless noted."""

    def __init__(self, n_in, n_hidden, n_out, seed=0, stream=None):
        L = load()
        _mlp_sigs(L)
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        self._h = ctypes.c_void_p()
        _check(L.rslb_mlp_create(ctypes.byref(self._h), self.n_in, self.n_hidden, self.n_out,
                                 int(seed), _stream_ptr(stream)))
        self.num_params = L.rslb_mlp_num_params(self._h)

    def get_params(self):
        t = np.zeros(self.num_params, dtype=np.float32)
        _check(load().rslb_mlp_get_params(self._h, _ptr(t)))
        return t

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.size == self.num_params
        _check(load().rslb_mlp_set_params(self._h, _ptr(t)))

    def set_normalization(self, mu, inv_sd, out_sd):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (mu, inv_sd, out_sd)]
        _check(load().rslb_mlp_set_normalization(self._h, *(_ptr(x) for x in a)))

    def get_normalization(self):
        a = [np.zeros(self.n_in, np.float32), np.zeros(self.n_in, np.float32),
             np.zeros(self.n_out, np.float32)]
        _check(load().rslb_mlp_get_normalization(self._h, *(_ptr(x) for x in a)))
        return tuple(a)

    def fit_normalization(self, X_ptr, T_ptr, n):
        _check(load().rslb_mlp_fit_normalization(self._h, ctypes.c_void_p(X_ptr),
                                                 ctypes.c_void_p(T_ptr), int(n)))

    def forward(self, X_ptr, n, Y_ptr):
        _check(load().rslb_mlp_forward(self._h, ctypes.c_void_p(X_ptr), int(n),
                                       ctypes.c_void_p(Y_ptr)))

    def loss_grad(self, X_ptr, T_ptr, n):
        loss = ctypes.c_double()
        g = np.zeros(self.num_params, dtype=np.float32)
        _check(load().rslb_mlp_loss_grad(self._h, ctypes.c_void_p(X_ptr), ctypes.c_void_p(T_ptr),
                                         int(n), ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, X_ptr, T_ptr, n, epochs, batch=4096, lr=1e-3, seed=0):
        losses = np.zeros(max(int(epochs), 1))
        _check(load().rslb_mlp_train(self._h, ctypes.c_void_p(X_ptr), ctypes.c_void_p(T_ptr),
                                     int(n), int(epochs), int(batch), float(lr), int(seed),
                                     _ptr(losses)))
        return losses[:int(epochs)]

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().rslb_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def restrict(hi, lo):
    """State of Sod handle ``lo`` := restriction of ``hi``'s state."""
    L = load()
    _mlp_sigs(L)
    _check(L.rslb_restrict(hi._h, lo._h))


def closure_sample(hi, lo, tau, X_ptr, T_ptr):
    L = load()
    _mlp_sigs(L)
    _check(L.rslb_closure_sample(hi._h, lo._h, float(tau), ctypes.c_void_p(X_ptr),
                                 ctypes.c_void_p(T_ptr)))


def closure_step(lo, mlp, tau, nsteps=1):
    L = load()
    _mlp_sigs(L)
    _check(L.rslb_closure_step(lo._h, mlp._h, float(tau), int(nsteps)))
