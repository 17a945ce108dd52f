"""Plain FP64 CPU oracle for the decomposed-kernel (FAGP) Gaussian process.

TEST INFRASTRUCTURE ONLY. This module is the slow, obviously correct
definition that the CUDA path is checked against. Only the test suite, the
package's ``smoke()`` check and the CPU-baseline leg of the benchmark may
import it; the library itself never does, and this module imports nothing
from the library.

Everything is float64 numpy. Library primitives used as single steps: the
matrix product (numpy ``@``), the Cholesky factorisation
(``numpy.linalg.cholesky``), triangular solves (``scipy.linalg``) and the
symmetric tridiagonal eigenvalues (``numpy.linalg.eigvalsh``, for Golub-Welsch).

Notation follows the paper: eps = epsilon (SE shape parameter, Eq. 13),
rho = the global scale factor of the eigen-decomposition (Eq. 14-16; the
library's ``alpha`` argument), sigma2 = sigma^2 (noise variance, Eq. 1),
n eigenfunctions per input dimension, p input dimensions, M = n**p
tensor-product columns (Eq. 19-20).

Readings of the paper taken here (each is pinned by a test):
  * delta^2 = rho^2 (beta^2 - 1) / 2.  Eq. 14 prints rho/2 (beta^2 - 1); only
    the rho^2 form makes the Mercer sum (Eq. 5) converge to the SE kernel and
    the eigenfunctions orthonormal when rho != 1.
  * H_k in Eq. 15 are the physicists' Hermite polynomials (H_1(t) = 2t); only
    those are normalised by the gamma_i of Eq. 14.
  * The multi-index set of Eq. 18 is the full grid {0..n-1}^p; column
    m = sum_j m_j n^(p-1-j) (last dimension fastest).
  * The predictive variance is the diagonal of Sigma_* of Eq. 12 (latent f,
    no added noise), with prior mean zero (Sec. 2.1).
  * sigma^2 / lambda_m is clamped at 1e200 (CLAMP_D) so that eigenvalues
    that underflow stay finite; columns that hit the clamp contribute below
    1e-180 relative.
"""
from __future__ import annotations

import math
from typing import Dict, Optional

import numpy as np
import scipy.linalg as sla

# Degree up to which the eigenfunctions are evaluated with the literal
# physicists' Hermite recurrence times gamma_i (Eq. 14-15). Beyond it H_k(t)
# overflows float64, and the algebraically identical normalised recurrence
# (see eigenfunctions_1d) is used instead.
LITERAL_MAX_N = 100

# Upper bound on sigma^2 / lambda_m (reading A5).
CLAMP_D = 1e200


# --------------------------------------------------------------------------
# Sec. 2.3: one-dimensional SE eigenpairs
# --------------------------------------------------------------------------

def se_constants(eps: float, rho: float):
    """beta and delta^2 of Eq. 14 (delta^2 with the rho^2 reading)."""
    beta = (1.0 + (2.0 * eps / rho) ** 2) ** 0.25
    delta2 = rho ** 2 / 2.0 * (beta ** 2 - 1.0)
    return beta, delta2


def gamma_coeffs(n: int, beta: float) -> np.ndarray:
    """gamma_i = sqrt(beta / (2^(i-1) Gamma(i))), i = 1..n (Eq. 14).

    Evaluated through log-gamma so that large i does not overflow.
    """
    i = np.arange(1, n + 1, dtype=np.float64)
    lg = np.array([math.lgamma(v) for v in i])
    return np.exp(0.5 * (math.log(beta) - (i - 1.0) * math.log(2.0) - lg))


def hermite_phys(n: int, t: np.ndarray) -> np.ndarray:
    """Physicists' Hermite polynomials H_0..H_{n-1} at t, shape t.shape + (n,).

    Three-term recurrence H_0 = 1, H_1 = 2t, H_{k+1} = 2t H_k - 2k H_{k-1}.
    """
    t = np.asarray(t, dtype=np.float64)
    H = np.empty(t.shape + (n,), dtype=np.float64)
    H[..., 0] = 1.0
    if n > 1:
        H[..., 1] = 2.0 * t
    for k in range(1, n - 1):
        H[..., k + 1] = 2.0 * t * H[..., k] - 2.0 * k * H[..., k - 1]
    return H


def eigenvalues_1d(n: int, eps: float, rho: float) -> np.ndarray:
    """lambda_i, i = 1..n, of Eq. 16 (may underflow to 0 for large i)."""
    return np.exp(log_eigenvalues_1d(n, eps, rho))


def log_eigenvalues_1d(n: int, eps: float, rho: float) -> np.ndarray:
    """log lambda_i of Eq. 16:
    lambda_i = sqrt(rho^2 / D) * (eps^2 / D)^(i-1),  D = rho^2 + delta^2 + eps^2.
    """
    _, delta2 = se_constants(eps, rho)
    D = rho ** 2 + delta2 + eps ** 2
    i = np.arange(1, n + 1, dtype=np.float64)
    return 0.5 * math.log(rho ** 2 / D) + (i - 1.0) * math.log(eps ** 2 / D)


def eigenfunctions_1d(x: np.ndarray, n: int, eps: float, rho: float) -> np.ndarray:
    """phi_i(x) = gamma_i exp(-delta^2 x^2) H_{i-1}(rho beta x), i = 1..n (Eq. 15).

    Returns shape x.shape + (n,). For n <= LITERAL_MAX_N the literal product
    gamma_i * H_{i-1} is used. For larger n, gamma_i H_{i-1}(t) is computed by
    the recurrence it satisfies (divide the Hermite recurrence by
    sqrt(2^k k!)): with q_k = gamma_{k+1} H_k(t),
        q_0 = sqrt(beta), q_1 = sqrt(2) t q_0,
        q_{k+1} = sqrt(2/(k+1)) t q_k - sqrt(k/(k+1)) q_{k-1},
    which is the same quantity without the overflow of H_k.
    """
    x = np.asarray(x, dtype=np.float64)
    beta, delta2 = se_constants(eps, rho)
    t = rho * beta * x
    env = np.exp(-delta2 * x * x)
    if n <= LITERAL_MAX_N:
        q = hermite_phys(n, t) * gamma_coeffs(n, beta)
    else:
        q = np.empty(x.shape + (n,), dtype=np.float64)
        q[..., 0] = math.sqrt(beta)
        if n > 1:
            q[..., 1] = math.sqrt(2.0) * t * q[..., 0]
        for k in range(1, n - 1):
            q[..., k + 1] = (math.sqrt(2.0 / (k + 1)) * t * q[..., k]
                             - math.sqrt(k / (k + 1.0)) * q[..., k - 1])
    return q * env[..., None]


# --------------------------------------------------------------------------
# Sec. 2.3: tensor-product (multi-index) eigenpairs, Eq. 18-20
# --------------------------------------------------------------------------

def multi_index(n: int, p: int) -> np.ndarray:
    """All n^p multi-indices (m_1..m_p), 0-based, as an (M, p) int array.

    Row m holds the digits of m in base n, most significant first, so the
    last dimension varies fastest.
    """
    grids = np.indices((n,) * p).reshape(p, -1).T
    return np.ascontiguousarray(grids, dtype=np.int64)


def per_dimension(v, p: int) -> np.ndarray:
    """eps or rho for each of the p dimensions: a scalar applies to all (the
    isotropic kernel, Eq. 13), a length-p sequence gives the ARD kernel's
    eps_j (Eq. 17) and a scale factor per dimension."""
    a = np.asarray(v, dtype=np.float64)
    if a.ndim == 0:
        return np.full(p, float(a))
    if a.shape != (p,):
        raise ValueError(f"expected a scalar or {p} values, got shape {a.shape}")
    return a


def log_eigenvalues(n: int, p: int, eps, rho) -> np.ndarray:
    """log lambda_m = sum_j log lambda^{(j)}_{m_j} (Eq. 20; with ARD, Eq. 17,
    dimension j has its own eps_j and rho_j)."""
    e, r = per_dimension(eps, p), per_dimension(rho, p)
    idx = multi_index(n, p)
    out = np.zeros(idx.shape[0])
    for j in range(p):
        out += log_eigenvalues_1d(n, float(e[j]), float(r[j]))[idx[:, j]]
    return out


def phi_matrix(X: np.ndarray, n: int, eps, rho) -> np.ndarray:
    """Phi[i, m] = prod_j phi^{(j)}_{m_j}(x_ij) (Eq. 19), shape (N, n^p); eps
    and rho scalar or per dimension (ARD, Eq. 17)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    N, p = X.shape
    e, r = per_dimension(eps, p), per_dimension(rho, p)
    idx = multi_index(n, p)
    Phi = np.ones((N, idx.shape[0]), dtype=np.float64)
    for j in range(p):
        E = eigenfunctions_1d(X[:, j], n, float(e[j]), float(r[j]))      # (N, n)
        Phi *= E[:, idx[:, j]]
    return Phi


def kernel_approx(X1: np.ndarray, X2: np.ndarray, n: int, eps: float, rho: float) -> np.ndarray:
    """Truncated Mercer kernel Phi(X1) Lambda Phi(X2)^T (Eq. 6-7)."""
    P1 = phi_matrix(X1, n, eps, rho)
    P2 = phi_matrix(X2, n, eps, rho)
    p = np.atleast_2d(X1).shape[1]
    lam = np.exp(log_eigenvalues(n, p, eps, rho))
    return (P1 * lam) @ P2.T


def kernel_se(X1: np.ndarray, X2: np.ndarray, eps) -> np.ndarray:
    """The SE kernel exp(-sum_j eps_j^2 (x_j - x'_j)^2) (Eq. 13; Eq. 17, ARD,
    with eps per dimension)."""
    X1 = np.atleast_2d(X1)
    X2 = np.atleast_2d(X2)
    e = per_dimension(eps, X1.shape[1])
    d2 = (((X1[:, None, :] - X2[None, :, :]) * e) ** 2).sum(axis=2)
    return np.exp(-d2)


# --------------------------------------------------------------------------
# Sec. 2.2: fit and predict in the M x M (Woodbury) form
# --------------------------------------------------------------------------

def noise_diagonal(n: int, p: int, eps: float, rho: float, sigma2: float) -> np.ndarray:
    """d_m = sigma^2 / lambda_m, clamped at CLAMP_D (the sigma^2 Lambda^{-1} of A)."""
    logd = math.log(sigma2) - log_eigenvalues(n, p, eps, rho)
    return np.where(logd >= math.log(CLAMP_D), CLAMP_D,
                    np.exp(np.minimum(logd, math.log(CLAMP_D))))


def gram(X: np.ndarray, y: np.ndarray, n: int, eps: float, rho: float,
         row_block: int = 16384):
    """G = Phi^T Phi and b = Phi^T y.

    Both are sums over training points (G = sum_i phi(x_i) phi(x_i)^T), taken
    here over consecutive blocks of rows so that Phi need not be held whole.
    """
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    N, p = X.shape
    M = n ** p
    G = np.zeros((M, M), dtype=np.float64)
    b = np.zeros(M, dtype=np.float64)
    for r0 in range(0, N, row_block):
        P = phi_matrix(X[r0:r0 + row_block], n, eps, rho)
        G += P.T @ P
        b += P.T @ y[r0:r0 + row_block]
    return G, b


def fit(X: np.ndarray, y: np.ndarray, n: int, eps: float, rho: float, sigma2: float,
        row_block: int = 16384) -> Dict[str, np.ndarray]:
    """Fit in the M x M form derived from Eq. 10-12.

    With Sigma_n = sigma^2 I, Lambda-bar = Lambda^{-1} + Phi^T Phi / sigma^2
    (Sec. 2.2). Multiplying by sigma^2 gives A = sigma^2 Lambda-bar
    = Phi^T Phi + sigma^2 Lambda^{-1}. Substituting into W of Eq. 11 reduces
    it to W = Phi_* A^{-1} Phi^T, so mu_* = Phi_* c with c = A^{-1} Phi^T y.
    A is symmetric positive definite, so it is factored A = L L^T.
    """
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    N, p = X.shape
    G, b = gram(X, y, n, eps, rho, row_block)
    d = noise_diagonal(n, p, eps, rho, sigma2)
    A = G + np.diag(d)
    L = np.linalg.cholesky(A)
    w = sla.solve_triangular(L, b, lower=True)
    c = sla.solve_triangular(L.T, w, lower=False)
    return dict(G=G, b=b, d=d, A=A, L=L, c=c, n=n, p=p, eps=eps, rho=rho, sigma2=sigma2)


def predict(model: Dict[str, np.ndarray], Xs: np.ndarray, row_block: int = 16384):
    """Predictive mean and variance at Xs (Eq. 11-12 in the M x M form).

    mu_* = Phi_* c.  The diagonal of Sigma_* of Eq. 12 reduces, with the
    substitution used in ``fit``, to sigma^2 Phi_* A^{-1} Phi_*^T, so
    var_i = sigma^2 |L^{-1} phi(x*_i)|^2.
    """
    Xs = np.atleast_2d(np.asarray(Xs, dtype=np.float64))
    Ns = Xs.shape[0]
    mean = np.empty(Ns)
    var = np.empty(Ns)
    for r0 in range(0, Ns, row_block):
        Ps = phi_matrix(Xs[r0:r0 + row_block], model["n"], model["eps"], model["rho"])
        mean[r0:r0 + row_block] = Ps @ model["c"]
        V = sla.solve_triangular(model["L"], Ps.T, lower=True)
        var[r0:r0 + row_block] = model["sigma2"] * np.sum(V * V, axis=0)
    return mean, var


def predict_covariance(model: Dict[str, np.ndarray], Xs: np.ndarray) -> np.ndarray:
    """The full predictive covariance block Sigma_* of Eq. 12 (latent f,
    N_* x N_*) in the M x M form: Sigma_* = sigma^2 Phi_* A^{-1} Phi_*^T =
    sigma^2 V^T V with V = L^{-1} Phi_*^T. Its diagonal is ``predict``'s
    variance. Only for small N_*."""
    Ps = phi_matrix(np.atleast_2d(np.asarray(Xs, dtype=np.float64)), model["n"], model["eps"], model["rho"])
    V = sla.solve_triangular(model["L"], Ps.T, lower=True)
    return model["sigma2"] * (V.T @ V)


def log_marginal_likelihood(model: Dict[str, np.ndarray], y: np.ndarray) -> float:
    """log p(y) of the truncated-kernel GP, K = Phi Lambda Phi^T (Eq. 7-9),
    from the fitted M x M factors (the quantity that hyperparameter learning,
    named as future work in Sec. 4, maximises).

    The definition is log N(y; 0, K + sigma^2 I) (Eq. 1-2). By the matrix
    determinant lemma, |K + sigma^2 I| = sigma^(2N) |Lambda| |A| / sigma^(2M),
    and sigma^(2M) / |Lambda| = prod_m d_m with d_m = sigma^2 / lambda_m; by
    the Woodbury identity (Eq. 10), y^T (K + sigma^2 I)^{-1} y =
    (y^T y - b^T c) / sigma^2 with b = Phi^T y, c = A^{-1} b. So
      log p(y) = -1/2 [ (y^T y - b^T c) / sigma^2 + N log sigma^2
                        + log|A| - sum_m log d_m + N log 2 pi ],
    log|A| = 2 sum_j log L_jj. Clamped d_m stand for eigenvalues below
    1e-200 sigma^2, whose columns add nothing measurable to K.
    """
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    s2 = model["sigma2"]
    quad = (y @ y - model["b"] @ model["c"]) / s2
    logdet = N * math.log(s2) + 2.0 * np.sum(np.log(np.diag(model["L"]))) - np.sum(np.log(model["d"]))
    return -0.5 * (quad + logdet + N * math.log(2.0 * math.pi))


def log_marginal_likelihood_dsigma2(model: Dict[str, np.ndarray], y: np.ndarray) -> float:
    """d log p(y) / d sigma^2 at fixed eps, rho (the noise part of the
    gradient that hyperparameter learning follows).

    A = G + diag(d) with d_m = sigma^2 / lambda_m (clamped at CLAMP_D, where
    d no longer moves), so dA / dsigma^2 = E = diag(e), e_m = d_m / sigma^2 on
    unclamped columns and 0 on clamped ones. Differentiating the terms of
    ``log_marginal_likelihood``: d(b^T c) = -c^T E c, d log|A| = tr(A^{-1} E),
    d sum log d_m = (unclamped count) / sigma^2, so
      d log p / d sigma^2 = -1/2 [ c^T E c / sigma^2 - (y^T y - b^T c) / sigma^4
                                   + N / sigma^2 + tr(A^{-1} E) - n_u / sigma^2 ].
    """
    y = np.asarray(y, dtype=np.float64)
    N = y.shape[0]
    s2 = model["sigma2"]
    d, c, b, L = model["d"], model["c"], model["b"], model["L"]
    free = d < CLAMP_D
    e = np.where(free, d / s2, 0.0)
    Linv = sla.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    diag_Ainv = np.sum(Linv * Linv, axis=0)  # (A^{-1})_mm = sum_k (L^{-1})_km^2
    return -0.5 * (c @ (e * c) / s2 - (y @ y - b @ c) / s2 ** 2 + N / s2
                   + e @ diag_Ainv - np.count_nonzero(free) / s2)


def se_constants_grad(eps: float, rho: float):
    """Partial derivatives of beta, delta^2 and rho beta (Eq. 14, delta^2 with
    the rho^2 reading) with respect to eps and rho, by the chain rule:
      beta = (1 + 4 eps^2 / rho^2)^(1/4):
        d beta / d eps = 2 eps / (rho^2 beta^3),  d beta / d rho = -2 eps^2 / (rho^3 beta^3);
      delta^2 = rho^2 (beta^2 - 1) / 2:
        d delta^2 / d eps = rho^2 beta d beta / d eps,
        d delta^2 / d rho = rho (beta^2 - 1) + rho^2 beta d beta / d rho.
    Returns {theta: (d beta, d delta^2, d (rho beta))} for theta in 'eps', 'rho'."""
    beta, _ = se_constants(eps, rho)
    db_de = 2.0 * eps / (rho ** 2 * beta ** 3)
    db_dr = -2.0 * eps ** 2 / (rho ** 3 * beta ** 3)
    dd_de = rho ** 2 * beta * db_de
    dd_dr = rho * (beta ** 2 - 1.0) + rho ** 2 * beta * db_dr
    return {"eps": (db_de, dd_de, rho * db_de), "rho": (db_dr, dd_dr, beta + rho * db_dr)}


def eigenfunctions_1d_grad(x: np.ndarray, n: int, eps: float, rho: float, theta: str) -> np.ndarray:
    """d phi_i(x) / d theta for theta in 'eps', 'rho' (Eq. 15), shape x.shape + (n,).

    phi_i = gamma_i e^{-delta^2 x^2} H_{i-1}(t), t = rho beta x, gamma_i^2 =
    beta / (2^{i-1} (i-1)!). The product rule gives
      d phi_i = phi_i (d log gamma_i - x^2 d delta^2) + gamma_i e^{-delta^2 x^2} H'_{i-1}(t) x d(rho beta),
    with d log gamma_i = (d beta) / (2 beta) and H'_k = 2k H_{k-1}, so that
    gamma_i H'_{i-1} = sqrt(2 (i-1)) (gamma_{i-1} H_{i-2}) -- the previous
    column of the same eigenfunction table without its envelope.
    """
    x = np.asarray(x, dtype=np.float64)
    beta, delta2 = se_constants(eps, rho)
    dbeta, ddelta2, drb = se_constants_grad(eps, rho)[theta]
    phi = eigenfunctions_1d(x, n, eps, rho)
    env = np.exp(-delta2 * x * x)[..., None]
    q = phi / env                                   # gamma_i H_{i-1}(t)
    dq = np.zeros_like(q)                           # gamma_i H'_{i-1}(t)
    k = np.arange(1, n, dtype=np.float64)
    dq[..., 1:] = np.sqrt(2.0 * k) * q[..., :-1]
    xx = x[..., None]
    return phi * (0.5 * dbeta / beta - xx * xx * ddelta2) + env * dq * xx * drb


def log_eigenvalues_grad(n: int, p: int, eps: float, rho: float, theta: str) -> np.ndarray:
    """d log lambda_m / d theta for the tensor-product eigenvalues (Eq. 16, 20):
    log lambda_k = 1/2 log(rho^2 / D) + k log(eps^2 / D), D = rho^2 + delta^2 + eps^2,
    differentiated through D (and delta^2), summed over the dimensions."""
    _, delta2 = se_constants(eps, rho)
    _, ddelta2, _ = se_constants_grad(eps, rho)[theta]
    D = rho ** 2 + delta2 + eps ** 2
    if theta == "eps":
        dD = ddelta2 + 2.0 * eps
        dl0 = -0.5 * dD / D
        dr = 2.0 / eps - dD / D
    else:
        dD = 2.0 * rho + ddelta2
        dl0 = 1.0 / rho - 0.5 * dD / D
        dr = -dD / D
    dk = dl0 + np.arange(n, dtype=np.float64) * dr  # d log lambda_k, k = 0..n-1
    idx = multi_index(n, p)
    return dk[idx].sum(axis=1)


def log_marginal_likelihood_grad(X, y, n: int, eps: float, rho: float, sigma2: float):
    """Gradient (d/d eps, d/d rho, d/d sigma^2) of log p(y) = log N(y; 0, K +
    sigma^2 I), K = Phi Lambda Phi^T (Eq. 1-2, 7-9), the objective of the
    hyperparameter learning named as future work in Sec. 4.

    For a parameter theta of K, d log p / d theta = 1/2 a^T (dK) a - 1/2
    tr(Ky^{-1} dK) with Ky = K + sigma^2 I and a = Ky^{-1} y; dK = dPhi Lambda
    Phi^T + Phi dLambda Phi^T + Phi Lambda dPhi^T, with dPhi from
    eigenfunctions_1d_grad through the tensor product (Eq. 19) and dLambda =
    Lambda diag(d log lambda). For sigma^2, dK = I. Dense N x N; only for
    small N. (Clamped eigenvalues are not treated: the test problems keep
    sigma^2 / lambda_m below the clamp.)"""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    y = np.asarray(y, dtype=np.float64)
    N, p = X.shape
    idx = multi_index(n, p)
    Phi = phi_matrix(X, n, eps, rho)
    lam = np.exp(log_eigenvalues(n, p, eps, rho))
    Ky = (Phi * lam) @ Phi.T + sigma2 * np.eye(N)
    Kinv = np.linalg.inv(Ky)
    a = Kinv @ y
    out = []
    for theta in ("eps", "rho"):
        E = [eigenfunctions_1d(X[:, j], n, eps, rho) for j in range(p)]
        dE = [eigenfunctions_1d_grad(X[:, j], n, eps, rho, theta) for j in range(p)]
        dPhi = np.zeros_like(Phi)
        for j in range(p):
            term = np.ones_like(Phi)
            for i in range(p):
                term *= (dE[i] if i == j else E[i])[:, idx[:, i]]
            dPhi += term
        dlam = lam * log_eigenvalues_grad(n, p, eps, rho, theta)
        dK = (dPhi * lam) @ Phi.T + (Phi * dlam) @ Phi.T + (Phi * lam) @ dPhi.T
        out.append(0.5 * a @ dK @ a - 0.5 * np.sum(Kinv * dK.T))
    out.append(0.5 * a @ a - 0.5 * np.trace(Kinv))
    return tuple(out)


# --------------------------------------------------------------------------
# Other routes to the same posterior (used to pin the M x M form)
# --------------------------------------------------------------------------

def posterior_nxn(X, y, Xs, n, eps, rho, sigma2):
    """Eq. 8-9 directly: the N x N GP posterior with the truncated kernel.

    K = Phi Lambda Phi^T + sigma^2 I is N x N; only for small N.
    Returns (mean, diagonal of Sigma_*).
    """
    Kxx = kernel_approx(X, X, n, eps, rho)
    Ksx = kernel_approx(Xs, X, n, eps, rho)
    Kss = kernel_approx(Xs, Xs, n, eps, rho)
    Kt = Kxx + sigma2 * np.eye(Kxx.shape[0])
    mean = Ksx @ np.linalg.solve(Kt, y)
    cov = Kss - Ksx @ np.linalg.solve(Kt, Ksx.T)
    return mean, np.diag(cov).copy()


def posterior_fagp_w(X, y, Xs, n, eps, rho, sigma2):
    """Eq. 11-12 with the explicit W and Lambda-bar of Sec. 2.2 (Woodbury, Eq. 10).

    Forms the N_* x N matrix W; only for small sizes.
    """
    X = np.atleast_2d(X)
    p = X.shape[1]
    Phi = phi_matrix(X, n, eps, rho)
    Phis = phi_matrix(Xs, n, eps, rho)
    lam = np.exp(log_eigenvalues(n, p, eps, rho))
    Lam = np.diag(lam)
    N = Phi.shape[0]
    Sinv = np.eye(N) / sigma2                       # Sigma_N^{-1}
    Lbar = np.diag(1.0 / lam) + Phi.T @ Sinv @ Phi  # Lambda-bar
    W = Phis @ Lam @ Phi.T @ (Sinv - Sinv @ Phi @ np.linalg.solve(Lbar, Phi.T @ Sinv))
    mean = W @ y
    cov = Phis @ Lam @ Phis.T - W @ Phi @ Lam @ Phis.T
    return mean, np.diag(cov).copy()


def log_marginal_likelihood_nxn(X, y, n, eps, rho, sigma2) -> float:
    """log N(y; 0, K + sigma^2 I) with the N x N truncated kernel, by a dense
    log-determinant and solve; only for small N."""
    K = kernel_approx(X, X, n, eps, rho) + sigma2 * np.eye(np.atleast_2d(X).shape[0])
    sign, logdet = np.linalg.slogdet(K)
    assert sign > 0
    y = np.asarray(y, dtype=np.float64)
    return -0.5 * (y @ np.linalg.solve(K, y) + logdet + y.shape[0] * math.log(2.0 * math.pi))


def posterior_exact_se(X, y, Xs, eps, sigma2):
    """Eq. 3-4 with the true SE kernel (no truncation), zero prior mean."""
    K = kernel_se(X, X, eps) + sigma2 * np.eye(np.atleast_2d(X).shape[0])
    Ks = kernel_se(Xs, X, eps)
    Kss = kernel_se(Xs, Xs, eps)
    mean = Ks @ np.linalg.solve(K, y)
    cov = Kss - Ks @ np.linalg.solve(K, Ks.T)
    return mean, np.diag(cov).copy()


def prior_variance(Xs, n, eps, rho):
    """diag(Phi_* Lambda Phi_*^T): the truncated prior variance (first term of Eq. 12)."""
    Xs = np.atleast_2d(Xs)
    Ps = phi_matrix(Xs, n, eps, rho)
    lam = np.exp(log_eigenvalues(n, Xs.shape[1], eps, rho))
    return (Ps * Ps) @ lam


# --------------------------------------------------------------------------
# Gauss-Hermite quadrature by Golub-Welsch (used to check orthonormality)
# --------------------------------------------------------------------------

def gauss_hermite(K: int):
    """Nodes and weights of K-point Gauss-Hermite quadrature (weight e^{-t^2}).

    Golub-Welsch: the nodes are the eigenvalues of the symmetric tridiagonal
    Jacobi matrix of the monic Hermite recurrence (zero diagonal, off-diagonal
    sqrt(k/2), k = 1..K-1). The weights are the Christoffel numbers
    w_k = 1 / sum_{j<K} p_j(t_k)^2 with p_j the orthonormal Hermite
    polynomials (p_j = H_j / sqrt(sqrt(pi) 2^j j!)); this equals sqrt(pi)
    times the squared first eigenvector component, but keeps full relative
    accuracy for the tiny outer weights.
    """
    J = np.zeros((K, K))
    for k in range(1, K):
        J[k - 1, k] = J[k, k - 1] = math.sqrt(k / 2.0)
    t = np.linalg.eigvalsh(J)
    # orthonormal recurrence: p_0 = pi^{-1/4}, p_1 = sqrt(2) t p_0,
    # p_{j+1} = sqrt(2/(j+1)) t p_j - sqrt(j/(j+1)) p_{j-1}
    s = np.zeros_like(t)
    pm1 = np.zeros_like(t)
    pj = np.full_like(t, math.pi ** -0.25)
    for j in range(K):
        s += pj * pj
        pn = math.sqrt(2.0 / (j + 1)) * t * pj - math.sqrt(j / (j + 1.0)) * pm1
        pm1, pj = pj, pn
    return t, 1.0 / s


def relerr(a: np.ndarray, ref: np.ndarray) -> float:
    """Relative L2 error |a - ref|_2 / |ref|_2."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.linalg.norm(ref))
    return float(np.linalg.norm(a - ref)) / (den if den > 0 else 1.0)
