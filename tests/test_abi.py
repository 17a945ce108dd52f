"""CPU checks of the C ABI: the library builds, loads and exports every entry
point that include/gpfagp.h declares; argument validation happens on the
host before any device work; without a GPU the product fails loudly instead
of falling back to the CPU."""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2403_12797_gb300 import _lib

HAS_GPU = False
try:
    import torch
    HAS_GPU = torch.cuda.is_available()
except Exception:  # pragma: no cover
    pass


def test_header_declares_the_boundary():
    names = set(_lib.declared_symbols())
    for need in ("gp_fit", "gp_predict", "gp_free", "gp_fit_ex", "gp_predict_ex", "gp_gram_ex",
                 "gp_fit_batch", "gp_predict_batch", "gp_last_error", "gp_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    for name in _lib.declared_symbols():
        assert hasattr(L, name), name


def test_strerror_and_version_are_host_only():
    assert _lib.strerror(_lib.GP_ENOTPD) == "matrix A is not positive definite"
    assert "sm_103a" in _lib.version()


def _fit_rc(N=10, p=1, n=3, eps=1.0, alpha=1.0, sigma2=0.1, prec=3):
    L = _lib.lib()
    X = np.zeros((max(N, 1), max(p, 1)))
    y = np.zeros(max(N, 1))
    out = C.c_void_p()
    rc = L.gp_fit_ex(X.ctypes.data, y.ctypes.data, N, p, n, eps, alpha, sigma2, prec, None, 0,
                     C.byref(out))
    return rc, out.value


@pytest.mark.parametrize("kw", [dict(N=0), dict(p=0), dict(p=33), dict(n=0), dict(eps=0.0),
                                dict(alpha=-1.0), dict(sigma2=math.nan), dict(sigma2=math.inf),
                                dict(p=4, n=14), dict(prec=7)])
def test_invalid_arguments_rejected_on_host(kw):
    rc, h = _fit_rc(**kw)
    assert rc == _lib.GP_EINVAL and not h
    assert _lib.lib().gp_last_error() == _lib.GP_EINVAL


def test_null_pointers_rejected():
    L = _lib.lib()
    out = C.c_void_p()
    assert L.gp_fit_ex(None, None, 10, 1, 3, 1.0, 1.0, 0.1, 3, None, 0, C.byref(out)) == _lib.GP_EINVAL
    assert L.gp_predict_ex(None, None, 5, None, None, None, 0) == _lib.GP_EINVAL
    L.gp_free(None)  # no-op


@pytest.mark.skipif(HAS_GPU, reason="checks the no-GPU path")
def test_no_gpu_fails_loudly():
    rc, h = _fit_rc()
    assert rc == _lib.GP_ENODEV and not h
    with pytest.raises(_lib.GPError):
        _lib.fit(np.zeros((4, 1)), np.zeros(4), 3, 1.0, 1.0, 0.1)
