"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports every
function that include/rslb.h declares, and the host-side parts (quadrature,
argument validation) behave as documented.  No GPU compute is launched."""
import os
import re

import numpy as np
import pytest
import scipy.special as sp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_01287_gb300 import build, load
    build.build()
    return load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rslb_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "rslb_init" in names and "rslb_step" in names and "rslb_quadrature" in names
    for name in sorted(names):
        assert hasattr(lib, name), name


def test_library_targets_sm_103a():
    from paper_1612_01287_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


@pytest.mark.parametrize("Q_xi,Q_L", [(1, 1), (2, 2), (7, 3), (20, 3), (200, 3), (512, 8)])
def test_quadrature_abi(lib, Q_xi, Q_L):
    from paper_1612_01287_gb300 import quadrature
    xi, wx, xk, wk = quadrature(Q_xi, Q_L)
    xs, ws = sp.roots_legendre(Q_xi)
    np.testing.assert_allclose(xi, xs, atol=2e-15, rtol=0)
    np.testing.assert_allclose(wx, ws, rtol=1e-8 if Q_xi > 100 else 1e-11)
    # independent implementations (library vs oracle) agree to round-off
    xo, wo = oracle.gauss_legendre(Q_xi)
    np.testing.assert_allclose(xi, xo, atol=4e-16, rtol=0)
    np.testing.assert_allclose(wx, wo, rtol=2e-13 if Q_xi < 300 else 5e-11)
    lo, lw = oracle.gauss_laguerre2(Q_L)
    np.testing.assert_allclose(xk, lo, rtol=4e-15)
    np.testing.assert_allclose(wk, lw, rtol=4e-14)


def test_quadrature_rejects_bad_orders(lib):
    from paper_1612_01287_gb300 import RslbError, quadrature
    with pytest.raises(RslbError):
        quadrature(0, 2)
    with pytest.raises(RslbError):
        quadrature(4, 13)


@pytest.mark.parametrize("kw,code", [
    (dict(Z=0), 1),
    (dict(N_Omega=6, Q_xi=6), 1),
    (dict(Q_L=9), 1),
    (dict(tau=-1.0), 1),
    (dict(dt=0.1), 2),            # CFL >= 1
    (dict(dt=2e-3, tau=1e-3), 3),  # dt >= tau: stiff
    (dict(bc="periodic", Z=4), 1),
    (dict(Z=4_000_000, Q_xi=200, Q_L=3, dt=1e-7), 7),  # V x ldz >= 2^31 populations
])
def test_host_side_validation(lib, kw, code):
    """Argument errors are rejected on the host before any device work."""
    from paper_1612_01287_gb300 import RslbError, Sod
    base = dict(Z=64, Q_xi=6, Q_L=2, tau=1e-2, dt=1e-3)
    base.update(kw)
    with pytest.raises(RslbError) as ei:
        Sod(**base)
    assert ei.value.code == code


def test_last_error_is_reset(lib):
    from paper_1612_01287_gb300 import quadrature
    quadrature(3, 2)
    assert lib.rslb_last_error() == b""


def test_destroy_null_is_noop(lib):
    lib.rslb_destroy(None)
