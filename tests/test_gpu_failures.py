"""Failure detection on the GPU, with no fault, trap or hang.

Two failures the library must report instead of hanging or returning
garbage:
  * a bounded device wait that runs out: the cooperative Cholesky's grid
    barrier is given a 50 ms limit and one CTA is made to leave before it
    arrives (a test hook; nothing is left in flight), so the other CTAs give
    up and the call returns GP_ETIMEOUT -- and the device stays usable;
  * a matrix A that is genuinely not positive definite in floating point:
    a Gram of rank 3 (three distinct training points, repeated) with a noise
    variance of 1e-300, so sigma^2 Lambda^{-1} (Eq. 10-11) is far below the
    rounding level of G. Past the first three pivots the Schur complement is
    zero up to rounding, so a pivot comes out non-positive and the call
    returns GP_ENOTPD with that column (>= 3) as the detail.
"""
import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_barrier_wait_that_runs_out_returns_timeout(prec):
    pr = W.workload2(N=20_000, Ns=200)  # M = 400: a cooperative Cholesky of many CTAs
    _lib.debug_barrier_timeout(0.05, 1)
    try:
        with pytest.raises(_lib.GPError) as e:
            _lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    finally:
        _lib.debug_barrier_timeout(0.0, -1)
    assert e.value.status == _lib.GP_ETIMEOUT
    assert e.value.detail == 100  # the grid barrier's site
    # the context is still usable: the same fit now succeeds and is right
    m = _lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    try:
        mean, var = m.predict(pr.Xs)
        mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
        mo, vo = O.predict(mdl, pr.Xs)
        tol = 1e-10 if prec == "fp64" else 1e-4
        assert O.relerr(mean, mo) < tol
    finally:
        m.free()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rank_deficient_gram_with_vanishing_noise_is_not_positive_definite(prec):
    r = np.random.default_rng(3)
    base = r.uniform(-1.0, 1.0, size=(3, 2))
    X = np.ascontiguousarray(np.repeat(base, 10, axis=0))  # 30 rows, 3 distinct points
    y = r.standard_normal(30)
    n = 10                                                 # M = 100 columns
    with pytest.raises(_lib.GPError) as e:
        _lib.fit(X, y, n, 1.0, 1.0, 1e-300, prec=prec)
    assert e.value.status == _lib.GP_ENOTPD
    assert 3 <= e.value.detail < n * n
    # the same library fits the same data with a noise variance that keeps A
    # positive definite
    m = _lib.fit(X, y, n, 1.0, 1.0, 1e-2, prec=prec)
    m.free()
