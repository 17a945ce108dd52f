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
    with pytest.raises(_lib.GPError) as e:
        _lib.fit_predict(np.zeros((4, 1)), np.zeros(4), 3, 1.0, 1.0, 0.1, np.zeros((2, 1)))
    assert e.value.status == _lib.GP_ENODEV


def _fit_predict_rc(N=10, p=1, n=3, Ns=4, xs=True, mean=True, out=True, **kw):
    L = _lib.lib()
    X, y = np.zeros((max(N, 1), p)), np.zeros(max(N, 1))
    Xs, m, v = np.zeros((max(Ns, 1), p)), np.zeros(max(Ns, 1)), np.zeros(max(Ns, 1))
    h = C.c_void_p()
    rc = L.gp_fit_predict_ex(X.ctypes.data, y.ctypes.data, N, p, n, kw.get("eps", 1.0), 1.0, 0.1,
                             kw.get("prec", 3), Xs.ctypes.data if xs else None, Ns,
                             m.ctypes.data if mean else None, v.ctypes.data, None, 0,
                             C.byref(h) if out else None)
    return rc, h.value


@pytest.mark.parametrize("kw", [dict(Ns=-1), dict(xs=False), dict(mean=False), dict(out=False),
                                dict(N=0), dict(eps=0.0), dict(prec=7)])
def test_fit_predict_arguments_rejected_on_host(kw):
    rc, h = _fit_predict_rc(**kw)
    assert rc == _lib.GP_EINVAL and not h


def test_fit_predict_python_rejects_mismatched_inputs():
    with pytest.raises(ValueError):  # Xs with another column count
        _lib.fit_predict(np.zeros((4, 2)), np.zeros(4), 3, 1.0, 1.0, 0.1, np.zeros((2, 3)))


@pytest.mark.parametrize("kw", [dict(N=0), dict(p=0), dict(n=0), dict(eps=0.0), dict(alpha=-1.0),
                                dict(null="X"), dict(null="ebx"), dict(null="ebx4"), dict(null="colexp")])
def test_column_exponents_arguments_rejected_on_host(kw):
    # argument checks come before any device work, so these run without a GPU
    a = dict(N=16, p=2, n=3, eps=1.0, alpha=1.0)
    a.update({k: v for k, v in kw.items() if k != "null"})
    X = np.zeros((16, 2))
    ebx = np.zeros(64, dtype=np.int8)
    ebx4 = np.zeros(64, dtype=np.int8)
    ce = np.zeros(16, dtype=np.int32)
    ptr = {"X": X.ctypes.data, "ebx": ebx.ctypes.data, "ebx4": ebx4.ctypes.data, "colexp": ce.ctypes.data}
    if "null" in kw:
        ptr[kw["null"]] = None
    rc = _lib.lib().gp_debug_column_exponents(ptr["X"], a["N"], a["p"], a["n"], a["eps"], a["alpha"],
                                              ptr["ebx"], ptr["ebx4"], ptr["colexp"])
    assert rc == _lib.GP_EINVAL


# ---- the mixed Gram's row-split plan (host logic, no GPU)

_W = (1.0, 1.24, 1.17)  # per-block costs of the pair classes the planner uses
_BLOCK = 1024            # rows per split block of the one-CTA mixed Gram (GP_TAB_BLOCK)


def _plan_cost(T, n, rows):
    npc = (T, T - 1, (T - 1) * (T - 2) // 2)
    return max((rows[c] // _BLOCK + 1) * _W[c] for c in range(3) if npc[c] > 0)


@pytest.mark.parametrize("T,Npad,target", [(1, 50_048, 152), (2, 100_096, 152), (3, 300_032, 152),
                                           (4, 200_064, 152), (4, 20_096, 152), (4, 2_048, 152),
                                           (5, 1_000_064, 64), (8, 131_072, 40), (17, 400_000, 152)])
def test_gram_split_plan_invariants(T, Npad, target):
    n, rows, ctas = _lib.debug_gram_splits(T, Npad, target)
    npairs = T * (T + 1) // 2
    npc = (T, T - 1, (T - 1) * (T - 2) // 2)
    for c in range(3):
        assert rows[c] % _BLOCK == 0 and rows[c] >= _BLOCK
        # every split has rows, and the splits cover every row
        assert (n[c] - 1) * rows[c] < Npad <= n[c] * rows[c]
    assert ctas == sum(npc[c] * n[c] for c in range(3))
    if npairs <= target:
        assert ctas <= target  # one wave
        # never worse than the best uniform split that fits the same wave
        ns = target // npairs
        r = -(-((Npad + _BLOCK - 1) // _BLOCK) // ns) * _BLOCK
        assert _plan_cost(T, n, rows) <= _plan_cost(T, [ns] * 3, [r] * 3) + 1e-9
    else:  # more pairs than CTAs: one split size for every class
        assert n[0] == n[1] == n[2] and rows[0] == rows[1] == rows[2]


def test_gram_split_plan_of_the_benchmark_workload():
    # M = 400 (four 128-column tile rows), N = 200,000 (Npad 200,064), 152 SMs:
    # 13 / 17 / 16 splits of 16 / 12 / 13 blocks, 151 CTAs (one uniform split
    # would need 14 blocks per split for every pair)
    n, rows, ctas = _lib.debug_gram_splits(4, 200_064, 152)
    assert n == [13, 17, 16] and rows == [16 * _BLOCK, 12 * _BLOCK, 13 * _BLOCK] and ctas == 151


def test_gram_split_plan_rejects_bad_arguments():
    with pytest.raises(_lib.GPError):
        _lib.debug_gram_splits(0, 1000, 152)
    with pytest.raises(_lib.GPError):
        _lib.debug_gram_splits(4, 1000, 0)
