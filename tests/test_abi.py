"""The C ABI library loads and exports every function include/rpca.h declares (CPU only:
no compute call is made without a GPU)."""
import ctypes

import pytest

P = pytest.importorskip("paper_1711_05519_gb300")


@pytest.fixture(scope="module")
def lib():
    from paper_1711_05519_gb300 import build

    build.build()
    return P.lib()


def test_exports_every_declared_function(lib):
    names = P.header_functions()
    assert len(names) >= 10
    missing = [f for f in names if not hasattr(lib, f)]
    assert not missing, missing


def test_host_only_calls(lib):
    p = P.rpca.Params()
    assert lib.rpca_params_default(ctypes.byref(p)) == P.OK
    assert (p.max_iter, p.trim, p.precision, p.zeta_mode) == (100, 1, 1, 0)
    assert P.status_string(P.CAPACITY) == "RPCA_ERR_CAPACITY"
    assert P.status_string(99) == "RPCA_UNKNOWN_STATUS"
    assert lib.rpca_create(None, None, None) == P.INVALID_ARG
    assert lib.rpca_params_default(None) == P.INVALID_ARG
    ctx = ctypes.c_void_p()
    bad = P.rpca.Params()
    lib.rpca_params_default(ctypes.byref(bad))
    bad.beta, bad.gamma, bad.tol = 0.1, 1.5, 1e-5  # gamma must be < 1
    assert lib.rpca_create(ctypes.byref(ctx), ctypes.byref(bad), None) == P.INVALID_ARG
    assert lib.rpca_solve_host(None, 10, 10, 1, 0.1, 0.5, 1e-5, None, None, None, None, None, 0, None, None,
                               None) == P.INVALID_ARG
