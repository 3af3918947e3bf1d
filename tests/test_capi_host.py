"""The C-ABI library without a GPU: it loads, exports every function that
include/lcmg.h declares, and its host-only calls (L-curve corner, lambda
window, defaults, argument errors) agree with the oracle."""
import numpy as np
import pytest

import problemgen as pg
from oracle import lcurve

L = pytest.importorskip("paper_2306_11067_gb300.lcmg")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2306_11067_gb300 import build
    build.build()


def test_library_exports_every_header_function():
    lib = L.lib()
    names = L.header_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(L._SIGS), set(names) ^ set(L._SIGS)


def test_default_params():
    p = L.lcmg_default_params()
    assert (p.nu, p.coarse_max, p.maxit, p.check_every, p.graphs) == (2, 16, 10000, 16, 1)
    assert (p.tol, p.q, p.d_min) == (1e-6, 2.0, 1e-3)
    # execution-path options: the measured-fastest combination on GB300
    assert (p.fused, p.tail_points, p.pdl, p.fold, p.staged, p.vfuse) == (0, 0, 0, 0, 0, 1)
    assert L.lcmg_version().startswith("lcmg")


def test_cull_matches_oracle_exhaustive():
    for m in range(10, 65):
        assert L.lcmg_cull_lambdas(m, 0) == (1, m)
        for i in range(1, m + 1):
            assert L.lcmg_cull_lambdas(m, i) == lcurve.lambda_window(m, i)
    with pytest.raises(L.LcmgError):
        L.lcmg_cull_lambdas(10, 11)


def test_corner_matches_oracle_random_curves():
    g = pg.rng(5)
    for trial in range(300):
        k = int(g.integers(3, 40))
        rho = np.sort(10.0 ** g.uniform(-2, 3, k))
        eta = np.sort(10.0 ** g.uniform(-2, 3, k))[::-1].copy()
        assert L.lcmg_lcurve_corner(rho, eta) == lcurve.corner(rho, eta), trial


def test_corner_argument_errors():
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_lcurve_corner([1.0, 2.0], [2.0, 1.0])
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    with pytest.raises(L.LcmgError):
        L.lcmg_lcurve_corner([1.0, -2.0, 3.0], [3.0, 2.0, 1.0])


def test_server_rejects_bad_arguments_without_a_device():
    """Argument checks of the serving entry points run before any CUDA call."""
    import ctypes as C
    h = C.c_void_p()
    p = L.lcmg_default_params()
    assert L.lib().lcmg_server_create(C.byref(h), 0, 1 << 30, 0, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert L.lib().lcmg_server_create(C.byref(h), 0, 0, 2, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert L.lib().lcmg_server_create(None, 0, 1 << 30, 2, C.byref(p)) == L.LCMG_ERR_INVALID_ARG
    assert b"bad arguments" in L.lib().lcmg_server_last_error()
    assert L.lib().lcmg_server_destroy(None) == L.LCMG_OK
