"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself (a textbook table, a closed form, an independent route to
the same posterior, or a limit the mathematics fixes), so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line)
    return rows


def _ev(expr):
    return float(eval(expr, {"__builtins__": {}}, {k: getattr(math, k) for k in dir(math)}))


# ---------------------------------------------------------------- Hermite / quadrature

def test_hermite_recurrence_matches_textbook_table():
    t = np.linspace(-3.0, 3.0, 13)
    H = O.hermite_phys(8, t)
    for row in _read_golden("hermite_phys_coeffs.txt"):
        k, coeffs = row.split(":")
        c = [float(v) for v in coeffs.split()]
        ref = np.polynomial.polynomial.polyval(t, c)
        np.testing.assert_allclose(H[:, int(k)], ref, rtol=1e-14, atol=1e-12)


def test_gauss_hermite_closed_form_small():
    rows = [r.split(";") for r in _read_golden("gauss_hermite_small.txt")]
    for K in (1, 2, 3):
        ref = sorted((_ev(a), _ev(b)) for k, a, b in rows if int(k) == K)
        t, w = O.gauss_hermite(K)
        order = np.argsort(t)
        np.testing.assert_allclose(t[order], [r[0] for r in ref], atol=1e-14)
        np.testing.assert_allclose(w[order], [r[1] for r in ref], rtol=1e-13)


@pytest.mark.parametrize("K", [5, 17, 40])
def test_gauss_hermite_matches_numpy(K):
    t, w = O.gauss_hermite(K)
    tr, wr = np.polynomial.hermite.hermgauss(K)
    o = np.argsort(t)
    np.testing.assert_allclose(t[o], tr, atol=1e-12)
    np.testing.assert_allclose(w[o], wr, rtol=1e-9, atol=1e-14)


# ---------------------------------------------------------------- eigenpairs

def test_eigenvalue_worked_example():
    vals = {k.strip(): _ev(v) for k, v in (r.split(";") for r in _read_golden("eigenvalues_eps1_rho1.txt"))}
    beta, delta2 = O.se_constants(1.0, 1.0)
    assert beta == pytest.approx(vals["beta"], rel=1e-15)
    assert delta2 == pytest.approx(vals["delta2"], rel=1e-14)
    lam = O.eigenvalues_1d(5, 1.0, 1.0)
    assert lam[0] == pytest.approx(vals["lambda_1"], rel=1e-14)
    assert lam[1] == pytest.approx(vals["lambda_2"], rel=1e-14)
    assert lam[4] == pytest.approx(vals["lambda_5"], rel=1e-13)


def _orthonormality_error(n, eps, rho, K=None):
    """max |int phi_m phi_k (rho/sqrt(pi)) exp(-rho^2 x^2) dx - delta_mk| by Gauss-Hermite.

    With x = t / (rho beta) the integrand becomes a polynomial times exp(-t^2)
    exactly when delta^2 = rho^2 (beta^2 - 1) / 2, so K >= n nodes are exact.
    """
    K = K or n + 2
    beta, _ = O.se_constants(eps, rho)
    t, w = O.gauss_hermite(K)
    x = t / (rho * beta)
    Phi = O.eigenfunctions_1d(x, n, eps, rho)                 # (K, n)
    weight = (rho / math.sqrt(math.pi)) * np.exp(-rho ** 2 * x ** 2)
    g = weight * np.exp(t ** 2) / (rho * beta)                # change of variables
    Gm = (Phi * (w * g)[:, None]).T @ Phi
    return float(np.max(np.abs(Gm - np.eye(n))))


@pytest.mark.parametrize("eps,rho", [(1.0, 1.0), (1.0, 0.8), (1.2, 1.0), (0.5, 2.0), (2.0, 0.5)])
def test_eigenfunctions_orthonormal(eps, rho):
    assert _orthonormality_error(30, eps, rho) < 1e-11


def test_eigenfunctions_orthonormal_large_n_normalised_branch():
    n = O.LITERAL_MAX_N + 30
    assert _orthonormality_error(n, 1.0, 1.0, K=n + 4) < 1e-9


def test_normalised_recurrence_equals_literal(monkeypatch):
    x = np.linspace(-2.5, 2.5, 41)
    a = O.eigenfunctions_1d(x, 60, 1.1, 0.9)
    monkeypatch.setattr(O, "LITERAL_MAX_N", 0)
    b = O.eigenfunctions_1d(x, 60, 1.1, 0.9)
    np.testing.assert_allclose(b, a, rtol=1e-11, atol=1e-14)


def _mercer_error_1d(n, eps, rho):
    x = np.linspace(-1.0, 1.0, 33)
    K = O.kernel_approx(x[:, None], x[:, None], n, eps, rho)
    return float(np.max(np.abs(K - O.kernel_se(x[:, None], x[:, None], eps))))


@pytest.mark.parametrize("eps,rho", [(1.0, 1.0), (1.0, 0.8), (1.2, 1.0), (0.5, 2.0)])
def test_mercer_sum_converges_to_se_kernel(eps, rho):
    errs = [_mercer_error_1d(n, eps, rho) for n in (4, 8, 16, 32, 60)]
    assert errs[-1] < 1e-12
    assert all(b < a or b < 1e-14 for a, b in zip(errs[:-1], errs[1:]))


def test_mercer_workload_truncation_errors():
    # Truncation error of the workloads' own n: small, and far below 1.
    assert _mercer_error_1d(10, 1.0, 1.0) < 1e-3
    assert _mercer_error_1d(20, 1.0, 0.8) < 1e-6
    assert _mercer_error_1d(16, 1.2, 1.0) < 1e-4


@pytest.mark.parametrize("p,n", [(2, 30), (3, 22)])
def test_mercer_tensor_product_pd(p, n):
    r = np.random.Generator(np.random.PCG64(7))
    X1 = r.uniform(-1, 1, size=(9, p))
    X2 = r.uniform(-1, 1, size=(7, p))
    K = O.kernel_approx(X1, X2, n, 1.0, 1.0)
    np.testing.assert_allclose(K, O.kernel_se(X1, X2, 1.0), atol=1e-11)


def test_multi_index_order_last_dimension_fastest():
    idx = O.multi_index(3, 2)
    assert idx.tolist()[:4] == [[0, 0], [0, 1], [0, 2], [1, 0]]
    m = np.arange(27)
    idx3 = O.multi_index(3, 3)
    np.testing.assert_array_equal(idx3 @ np.array([9, 3, 1]), m)


# ---------------------------------------------------------------- planted mistakes fail

def test_wrong_delta_reading_is_rejected(monkeypatch):
    def wrong(eps, rho):
        beta = (1.0 + (2.0 * eps / rho) ** 2) ** 0.25
        return beta, rho / 2.0 * (beta ** 2 - 1.0)     # Eq. 14 as printed
    assert _mercer_error_1d(40, 1.0, 0.8) < 1e-12
    monkeypatch.setattr(O, "se_constants", wrong)
    assert _mercer_error_1d(40, 1.0, 0.8) > 1e-3
    assert _orthonormality_error(20, 1.0, 0.8) > 1e-3


def test_probabilists_hermite_is_rejected(monkeypatch):
    def he(n, t):
        t = np.asarray(t, dtype=np.float64)
        H = np.empty(t.shape + (n,))
        H[..., 0] = 1.0
        if n > 1:
            H[..., 1] = t
        for k in range(1, n - 1):
            H[..., k + 1] = t * H[..., k] - k * H[..., k - 1]
        return H
    monkeypatch.setattr(O, "hermite_phys", he)
    assert _orthonormality_error(12, 1.0, 1.0) > 1e-2
    assert _mercer_error_1d(30, 1.0, 1.0) > 1e-2


def test_dropped_noise_term_is_caught(monkeypatch):
    pr = W.random_problem(11, 40, 9, 1, 6)
    ref_m, ref_v = O.posterior_nxn(pr.X, pr.y, pr.Xs, pr.n, pr.eps, pr.alpha, pr.sigma2)
    monkeypatch.setattr(O, "noise_diagonal", lambda n, p, e, r, s: np.zeros(n ** p))
    mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    assert O.relerr(m, ref_m) > 1e-6 or O.relerr(v, ref_v) > 1e-6


# ---------------------------------------------------------------- closed form, brute force

def test_closed_form_p1_n1():
    pr = W.random_problem(3, 25, 6, 1, 1, eps=0.9, alpha=1.3, sigma2=0.04)
    eps, rho, s2 = pr.eps, pr.alpha, pr.sigma2
    beta = (1 + (2 * eps / rho) ** 2) ** 0.25
    d2 = rho ** 2 * (beta ** 2 - 1) / 2
    lam1 = math.sqrt(rho ** 2 / (rho ** 2 + d2 + eps ** 2))
    phi1 = lambda x: math.sqrt(beta) * math.exp(-d2 * x * x)   # gamma_1 H_0 = sqrt(beta)
    S = sum(phi1(x) ** 2 for x in pr.X[:, 0])
    B = sum(phi1(x) * yy for x, yy in zip(pr.X[:, 0], pr.y))
    den = S + s2 / lam1
    mdl = O.fit(pr.X, pr.y, 1, eps, rho, s2)
    m, v = O.predict(mdl, pr.Xs)
    for i, xs in enumerate(pr.Xs[:, 0]):
        assert m[i] == pytest.approx(phi1(xs) * B / den, rel=1e-13)
        assert v[i] == pytest.approx(s2 * phi1(xs) ** 2 / den, rel=1e-13)


@pytest.mark.parametrize("N,p,n", [(5, 1, 8), (50, 1, 12), (500, 1, 10), (5, 2, 4), (50, 2, 5),
                                   (500, 2, 6), (50, 3, 4), (200, 3, 3)])
def test_mxm_form_equals_nxn_posterior(N, p, n):
    pr = W.random_problem(100 + N + p, N, 17, p, n, eps=1.1, alpha=0.9, sigma2=0.02)
    mdl = O.fit(pr.X, pr.y, n, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    m2, v2 = O.posterior_nxn(pr.X, pr.y, pr.Xs, n, pr.eps, pr.alpha, pr.sigma2)
    assert O.relerr(m, m2) < 1e-10
    assert O.relerr(v, v2) < 1e-10


@pytest.mark.parametrize("N,p,n", [(30, 1, 7), (60, 2, 4)])
def test_mxm_form_equals_explicit_w_form(N, p, n):
    pr = W.random_problem(200 + N, N, 11, p, n, eps=1.0, alpha=1.0, sigma2=0.05)
    mdl = O.fit(pr.X, pr.y, n, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    m2, v2 = O.posterior_fagp_w(pr.X, pr.y, pr.Xs, n, pr.eps, pr.alpha, pr.sigma2)
    assert O.relerr(m, m2) < 1e-9
    assert O.relerr(v, v2) < 1e-9


def test_large_n_tends_to_exact_se_gp():
    pr = W.random_problem(5, 20, 15, 1, 50, eps=1.0, alpha=1.0, sigma2=0.01)
    mdl = O.fit(pr.X, pr.y, 50, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    me, ve = O.posterior_exact_se(pr.X, pr.y, pr.Xs, pr.eps, pr.sigma2)
    assert O.relerr(m, me) < 1e-8
    assert np.max(np.abs(v - ve)) < 1e-8


def test_small_noise_tends_to_least_squares():
    pr = W.random_problem(9, 2000, 50, 2, 4, sigma2=1e-12)
    mdl = O.fit(pr.X, pr.y, 4, pr.eps, pr.alpha, pr.sigma2)
    m, _ = O.predict(mdl, pr.Xs)
    P = O.phi_matrix(pr.X, 4, pr.eps, pr.alpha)
    coef = np.linalg.lstsq(P, pr.y, rcond=None)[0]
    ref = O.phi_matrix(pr.Xs, 4, pr.eps, pr.alpha) @ coef
    assert O.relerr(m, ref) < 1e-7


# ---------------------------------------------------------------- invariants

def test_posterior_variance_bounds_and_y_independence():
    pr = W.random_problem(21, 300, 40, 2, 6)
    mdl = O.fit(pr.X, pr.y, 6, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    prior = O.prior_variance(pr.Xs, 6, pr.eps, pr.alpha)
    assert np.all(v > 0) and np.all(v <= prior * (1 + 1e-12))
    mdl2 = O.fit(pr.X, 3.0 * pr.y + 1.0, 6, pr.eps, pr.alpha, pr.sigma2)
    m2, v2 = O.predict(mdl2, pr.Xs)
    np.testing.assert_allclose(v2, v, rtol=1e-12)
    mdl1 = O.fit(pr.X, np.ones_like(pr.y), 6, pr.eps, pr.alpha, pr.sigma2)
    m1, _ = O.predict(mdl1, pr.Xs)
    np.testing.assert_allclose(m2, 3.0 * m + m1, rtol=1e-10, atol=1e-12)


def test_dimension_permutation_invariance():
    pr = W.random_problem(31, 200, 25, 3, 4)
    mdl = O.fit(pr.X, pr.y, 4, pr.eps, pr.alpha, pr.sigma2)
    m, v = O.predict(mdl, pr.Xs)
    perm = [2, 0, 1]
    mdlp = O.fit(pr.X[:, perm], pr.y, 4, pr.eps, pr.alpha, pr.sigma2)
    mp, vp = O.predict(mdlp, pr.Xs[:, perm])
    np.testing.assert_allclose(mp, m, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(vp, v, rtol=1e-10)


def test_row_blocking_of_gram_is_a_plain_sum():
    pr = W.random_problem(41, 1000, 1, 2, 5)
    G1, b1 = O.gram(pr.X, pr.y, 5, 1.0, 1.0, row_block=7)
    G2, b2 = O.gram(pr.X, pr.y, 5, 1.0, 1.0, row_block=100000)
    np.testing.assert_allclose(G1, G2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(b1, b2, rtol=1e-12, atol=1e-12)


def test_clamp_only_touches_negligible_columns(monkeypatch):
    pr = W.random_problem(51, 30, 10, 1, 1100, sigma2=0.01)
    d = O.noise_diagonal(1100, 1, pr.eps, pr.alpha, pr.sigma2)
    assert d.max() == O.CLAMP_D and np.isfinite(d).all()
    m1, v1 = O.predict(O.fit(pr.X, pr.y, 1100, pr.eps, pr.alpha, pr.sigma2), pr.Xs)
    monkeypatch.setattr(O, "CLAMP_D", 1e150)
    m2, v2 = O.predict(O.fit(pr.X, pr.y, 1100, pr.eps, pr.alpha, pr.sigma2), pr.Xs)
    assert O.relerr(m2, m1) < 1e-12 and O.relerr(v2, v1) < 1e-12


def test_workload_generators_shapes_and_determinism():
    a = W.workload1()
    b = W.workload1()
    np.testing.assert_array_equal(a.X, b.X)
    assert a.X.shape == (1000, 1) and a.Xs.shape == (1000, 1) and a.M == 10
    w2 = W.workload2(N=1000, Ns=100)
    assert w2.X.shape == (1000, 2) and w2.M == 400 and w2.alpha == 0.8
    w3 = W.workload3(N=100, Ns=10)
    assert w3.M == 4096 and w3.eps == 1.2
    w4 = W.workload4(count=16, Ns=4)
    assert all(pr.M <= 1024 and 1 <= pr.p <= 4 and pr.n >= 2 for pr in w4)


def test_single_point_posterior_sensitivity_to_gram_errors():
    # Pins the amplification used for the N = 1 mixed-precision tolerance in
    # the GPU parity test: a relative perturbation r of G moves the mean by
    # about 30 r for this problem.
    pr = W.random_problem(23, 1, 7, 2, 3)
    ref = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
    mo, _ = O.predict(ref, pr.Xs)
    rng = np.random.Generator(np.random.PCG64(0))
    G = ref["G"] * (1 + 1e-6 * rng.standard_normal(ref["G"].shape))
    G = (G + G.T) / 2
    L = np.linalg.cholesky(G + np.diag(ref["d"]))
    import scipy.linalg as sla
    c = sla.cho_solve((L, True), ref["b"])
    m = O.phi_matrix(pr.Xs, pr.n, pr.eps, pr.alpha) @ c
    amp = O.relerr(m, mo) / 1e-6
    assert 10 < amp < 40


# ---- log marginal likelihood (hyperparameter learning, the paper's future work)

@pytest.mark.parametrize("N,p,n", [(5, 1, 8), (40, 1, 6), (150, 2, 4), (60, 2, 9), (30, 1, 60)])
def test_log_marginal_likelihood_equals_the_nxn_definition(N, p, n):
    # includes M > N (the truncated kernel is then full rank in y's space) and
    # n = 60, where the smallest eigenvalues hit the clamp of d
    rng = np.random.default_rng(N + 10 * p + n)
    X = rng.uniform(-1.0, 1.0, size=(N, p))
    y = np.sin(2.0 * X).sum(axis=1) + 0.1 * rng.standard_normal(N)
    eps, rho, s2 = 0.9, 1.1, 0.02
    mdl = O.fit(X, y, n, eps, rho, s2)
    got = O.log_marginal_likelihood(mdl, y)
    ref = O.log_marginal_likelihood_nxn(X, y, n, eps, rho, s2)
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)


def test_log_marginal_likelihood_rank_one_closed_form():
    # p = 1, n = 1: K = lambda phi phi^T. |s2 I + lambda phi phi^T| =
    # s2^N (1 + lambda |phi|^2 / s2), and by Sherman-Morrison
    # y^T (s2 I + lambda phi phi^T)^{-1} y = (|y|^2 - lambda (phi.y)^2 / (s2 + lambda |phi|^2)) / s2
    rng = np.random.default_rng(7)
    N, eps, rho, s2 = 25, 1.3, 0.7, 0.05
    X = rng.uniform(-1.0, 1.0, size=(N, 1))
    y = rng.standard_normal(N)
    phi = O.eigenfunctions_1d(X[:, 0], 1, eps, rho)[:, 0]
    lam = float(np.exp(O.log_eigenvalues_1d(1, eps, rho)[0]))
    pp, py = float(phi @ phi), float(phi @ y)
    quad = (float(y @ y) - lam * py * py / (s2 + lam * pp)) / s2
    logdet = N * math.log(s2) + math.log1p(lam * pp / s2)
    ref = -0.5 * (quad + logdet + N * math.log(2.0 * math.pi))
    got = O.log_marginal_likelihood(O.fit(X, y, 1, eps, rho, s2), y)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def test_log_marginal_likelihood_peaks_near_the_generating_noise():
    # data drawn from the truncated-kernel prior with noise variance 0.04:
    # the likelihood over sigma^2 is largest near the generating value
    rng = np.random.default_rng(11)
    N, n, eps, rho = 400, 6, 1.0, 1.0
    X = rng.uniform(-1.0, 1.0, size=(N, 1))
    Phi = O.eigenfunctions_1d(X[:, 0], n, eps, rho)
    lam = np.exp(O.log_eigenvalues_1d(n, eps, rho))
    y = Phi @ (np.sqrt(lam) * rng.standard_normal(n)) + 0.2 * rng.standard_normal(N)
    grid = [0.01, 0.02, 0.04, 0.08, 0.16]
    vals = [O.log_marginal_likelihood(O.fit(X, y, n, eps, rho, s2), y) for s2 in grid]
    assert int(np.argmax(vals)) == 2, vals


@pytest.mark.parametrize("N,p,n", [(40, 1, 6), (150, 2, 4), (30, 1, 60)])
def test_log_marginal_likelihood_sigma2_gradient_matches_finite_differences(N, p, n):
    # central differences of the pinned log p(y) (n = 60 includes clamped d)
    rng = np.random.default_rng(3 * N + p + n)
    X = rng.uniform(-1.0, 1.0, size=(N, p))
    y = np.cos(1.5 * X).sum(axis=1) + 0.1 * rng.standard_normal(N)
    eps, rho, s2 = 1.1, 0.9, 0.03
    g = O.log_marginal_likelihood_dsigma2(O.fit(X, y, n, eps, rho, s2), y)
    h = 1e-6 * s2
    lp = O.log_marginal_likelihood(O.fit(X, y, n, eps, rho, s2 + h), y)
    lm = O.log_marginal_likelihood(O.fit(X, y, n, eps, rho, s2 - h), y)
    fd = (lp - lm) / (2 * h)
    assert abs(g - fd) <= 1e-5 * max(1.0, abs(fd)), (g, fd)


def test_log_marginal_likelihood_sigma2_gradient_vanishes_at_the_maximum():
    # on a fine grid of sigma^2 the gradient changes sign where log p(y) peaks
    rng = np.random.default_rng(11)
    N, n, eps, rho = 400, 6, 1.0, 1.0
    X = rng.uniform(-1.0, 1.0, size=(N, 1))
    Phi = O.eigenfunctions_1d(X[:, 0], n, eps, rho)
    lam = np.exp(O.log_eigenvalues_1d(n, eps, rho))
    y = Phi @ (np.sqrt(lam) * rng.standard_normal(n)) + 0.2 * rng.standard_normal(N)
    grid = np.geomspace(0.01, 0.16, 21)
    vals = [O.log_marginal_likelihood(O.fit(X, y, n, eps, rho, s2), y) for s2 in grid]
    grads = [O.log_marginal_likelihood_dsigma2(O.fit(X, y, n, eps, rho, s2), y) for s2 in grid]
    k = int(np.argmax(vals))
    assert 0 < k < len(grid) - 1
    assert grads[k - 1] > 0 > grads[k + 1]


def test_predictive_covariance_block_equals_the_nxn_route():
    # Eq. 12's full Sigma_* (the f2 row's quantity): the M x M form against
    # the dense N x N posterior covariance with the truncated kernel, its
    # diagonal against predict(), symmetry and positive semidefiniteness
    rng = np.random.default_rng(21)
    N, p, n, eps, rho, s2 = 80, 2, 5, 0.9, 1.1, 0.02
    X = rng.uniform(-1.0, 1.0, size=(N, p))
    y = np.sin(2.0 * X).sum(axis=1) + 0.1 * rng.standard_normal(N)
    Xs = rng.uniform(-1.0, 1.0, size=(15, p))
    mdl = O.fit(X, y, n, eps, rho, s2)
    S = O.predict_covariance(mdl, Xs)
    Kxx = O.kernel_approx(X, X, n, eps, rho) + s2 * np.eye(N)
    Ksx = O.kernel_approx(Xs, X, n, eps, rho)
    ref = O.kernel_approx(Xs, Xs, n, eps, rho) - Ksx @ np.linalg.solve(Kxx, Ksx.T)
    assert np.max(np.abs(S - ref)) <= 1e-10 * np.max(np.abs(ref))
    _, var = O.predict(mdl, Xs)
    np.testing.assert_allclose(np.diag(S), var, rtol=1e-12)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=1e-15 * np.max(np.abs(S)))
    assert np.linalg.eigvalsh(S).min() > -1e-12 * np.max(np.abs(S))


# ---- ARD (Eq. 17): eps and rho per input dimension (the f1 row's oracle)

def test_ard_with_equal_parameters_is_the_isotropic_model():
    pr = W.random_problem(41, 300, 40, 2, 6, eps=0.9, alpha=1.1, sigma2=0.02)
    iso = O.predict(O.fit(pr.X, pr.y, pr.n, 0.9, 1.1, 0.02), pr.Xs)
    ard = O.predict(O.fit(pr.X, pr.y, pr.n, [0.9, 0.9], [1.1, 1.1], 0.02), pr.Xs)
    for a, b in zip(iso, ard):
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)


def test_ard_mercer_sum_converges_to_the_anisotropic_se_kernel():
    rng = np.random.default_rng(5)
    X = rng.uniform(-1.0, 1.0, size=(12, 2))
    eps, rho = [0.6, 1.4], [1.0, 0.8]
    K = O.kernel_approx(X, X, 40, eps, rho)
    ref = O.kernel_se(X, X, eps)
    assert np.max(np.abs(K - ref)) < 1e-10
    # the per-dimension factors are really different: the isotropic kernels miss it
    assert np.max(np.abs(O.kernel_se(X, X, 0.6) - ref)) > 1e-2


def test_ard_dimension_permutation_invariance():
    rng = np.random.default_rng(8)
    X = rng.uniform(-1.0, 1.0, size=(200, 3))
    y = np.sin(2.0 * X).sum(axis=1) + 0.1 * rng.standard_normal(200)
    Xs = rng.uniform(-1.0, 1.0, size=(30, 3))
    eps, rho = np.array([0.5, 1.0, 1.5]), np.array([0.9, 1.0, 1.2])
    perm = [2, 0, 1]
    a = O.predict(O.fit(X, y, 4, eps, rho, 0.03), Xs)
    b = O.predict(O.fit(X[:, perm], y, 4, eps[perm], rho[perm], 0.03), Xs[:, perm])
    for u, v in zip(a, b):
        np.testing.assert_allclose(u, v, rtol=1e-10, atol=1e-14)


def test_ard_mxm_form_equals_the_nxn_posterior():
    rng = np.random.default_rng(9)
    X = rng.uniform(-1.0, 1.0, size=(60, 2))
    y = np.cos(3.0 * X[:, 0]) * np.sin(X[:, 1]) + 0.05 * rng.standard_normal(60)
    Xs = rng.uniform(-1.0, 1.0, size=(20, 2))
    eps, rho, s2 = [0.7, 1.6], [1.2, 0.9], 0.01
    mean, var = O.predict(O.fit(X, y, 7, eps, rho, s2), Xs)
    m2, v2 = O.posterior_nxn(X, y, Xs, 7, eps, rho, s2)
    assert O.relerr(mean, m2) < 1e-10 and O.relerr(var, v2) < 1e-8
    with pytest.raises(ValueError):
        O.phi_matrix(X, 7, [0.7, 1.6, 1.0], rho)  # one value per dimension


# ---------------------------------------------------------------- likelihood gradient (eps, rho, sigma^2)

def _lml_at(pr, n, eps, rho, s2):
    return O.log_marginal_likelihood(O.fit(pr.X, pr.y, n, eps, rho, s2), pr.y)


@pytest.mark.parametrize("N,p,n,eps,rho,s2", [(60, 1, 6, 1.1, 0.9, 0.02), (80, 2, 4, 0.8, 1.3, 0.05),
                                              (50, 3, 3, 1.3, 1.0, 0.03), (40, 1, 120, 1.0, 1.0, 0.01)])
def test_log_marginal_likelihood_gradient_matches_central_differences(N, p, n, eps, rho, s2):
    """The analytic gradient (chain rule through beta, delta^2, gamma_i, the
    Hermite argument and the eigenvalues; dense N x N trace formula) against
    central differences of the M x M log-likelihood (itself pinned to the dense
    definition), including n > 100 (the normalised-recurrence branch)."""
    pr = W.random_problem(9, N, 1, p, n, eps=eps, alpha=rho, sigma2=s2)
    g = O.log_marginal_likelihood_grad(pr.X, pr.y, n, eps, rho, s2)
    h = 1e-5
    fd = ((_lml_at(pr, n, eps + h, rho, s2) - _lml_at(pr, n, eps - h, rho, s2)) / (2 * h),
          (_lml_at(pr, n, eps, rho + h, s2) - _lml_at(pr, n, eps, rho - h, s2)) / (2 * h),
          (_lml_at(pr, n, eps, rho, s2 * (1 + h)) - _lml_at(pr, n, eps, rho, s2 * (1 - h))) / (2 * h * s2))
    for a, b in zip(g, fd):
        assert abs(a - b) <= 1e-5 * max(1.0, abs(b)), (g, fd)
    # the sigma^2 component equals the M x M closed form used on the device
    ds = O.log_marginal_likelihood_dsigma2(O.fit(pr.X, pr.y, n, eps, rho, s2), pr.y)
    assert abs(g[2] - ds) <= 1e-8 * abs(ds)


@pytest.mark.parametrize("theta", ["eps", "rho"])
def test_eigenfunction_derivative_matches_central_differences(theta):
    x = np.linspace(-2.0, 2.0, 41)
    for n in (8, 130):
        d = O.eigenfunctions_1d_grad(x, n, 1.2, 0.9, theta)
        h = 1e-6
        if theta == "eps":
            fd = (O.eigenfunctions_1d(x, n, 1.2 + h, 0.9) - O.eigenfunctions_1d(x, n, 1.2 - h, 0.9)) / (2 * h)
        else:
            fd = (O.eigenfunctions_1d(x, n, 1.2, 0.9 + h) - O.eigenfunctions_1d(x, n, 1.2, 0.9 - h)) / (2 * h)
        np.testing.assert_allclose(d, fd, rtol=1e-6, atol=1e-8)


def test_dropped_term_in_delta_derivative_is_caught(monkeypatch):
    """Planted mistake: d delta^2 / d rho without its rho (beta^2 - 1) term
    makes the rho component disagree with central differences."""
    good = O.se_constants_grad

    def bad(eps, rho):
        out = good(eps, rho)
        db, dd, drb = out["rho"]
        beta, _ = O.se_constants(eps, rho)
        out["rho"] = (db, dd - rho * (beta ** 2 - 1.0), drb)
        return out

    monkeypatch.setattr(O, "se_constants_grad", bad)
    pr = W.random_problem(9, 60, 1, 1, 6, eps=1.1, alpha=0.9, sigma2=0.02)
    g = O.log_marginal_likelihood_grad(pr.X, pr.y, 6, 1.1, 0.9, 0.02)
    h = 1e-5
    fd = (_lml_at(pr, 6, 1.1, 0.9 + h, 0.02) - _lml_at(pr, 6, 1.1, 0.9 - h, 0.02)) / (2 * h)
    assert abs(g[1] - fd) > 1e-3 * max(1.0, abs(fd))
