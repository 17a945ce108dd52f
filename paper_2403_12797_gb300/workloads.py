"""Seeded synthetic inputs for the decomposed-kernel GP.

This module only draws random numbers: it holds none of the method's
arithmetic (no eigenfunctions, no kernel, no solve), so both the CUDA path
and the CPU oracle can consume the same arrays without sharing any code
that computes a result.

Every generator uses numpy's PCG64 with a fixed seed per workload and role:
train inputs use seed 1000+k, test inputs 2000+k, noise 3000+k, where k is
the workload number below.

Workloads (all regression data follow the model y = f(x) + noise of Sec. 2.1):

  1  p=1, n=10,  N=1,000     x~U[-1,1],     y=sin(3x)+0.1*xi,  test: 1,000-point grid on [-1,1]
  2  p=2, n=20,  N=200,000   x~U[-1,1]^2,   y=sin(3x1)cos(2x2)+0.05*xi, 50,000 test points ~U[-1,1]^2
  3  p=3, n=16,  N=2,000,000 x~N(0,0.5^2 I), y=exp(-|x|^2)+sum_i sin(2x_i)+0.05*xi, 200,000 test points, same law
  4  256 independent problems of uneven N, p, n (batched fit)
  5  64 resident models plus a Poisson stream of predict / refit requests (serving)
  6  the paper's own sweep workload (Sec. 3): N=10,000, y=sum_i cos(x_i)+nu

The sizes of workloads 1-3 may be reduced through the ``N``/``Ns`` arguments
(used by tests that must finish in seconds); the defaults are the full sizes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Problem:
    """One GP regression problem: training set, test set and hyperparameters.

    ``alpha`` is the SE eigen-decomposition's global scale factor (rho in
    Sec. 2.3), ``eps`` the kernel's shape parameter (epsilon in Sec. 2.3) and
    ``sigma2`` the noise variance (sigma^2 in Sec. 2.1).
    """

    name: str
    X: np.ndarray          # (N, p) float64, row-major
    y: np.ndarray          # (N,)   float64
    Xs: np.ndarray         # (Ns, p) float64, row-major
    n: int                 # eigenfunctions per dimension; M = n**p
    eps: float
    alpha: float
    sigma2: float

    @property
    def N(self) -> int:
        return int(self.X.shape[0])

    @property
    def p(self) -> int:
        return int(self.X.shape[1])

    @property
    def Ns(self) -> int:
        return int(self.Xs.shape[0])

    @property
    def M(self) -> int:
        return int(self.n) ** int(self.p)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _c(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def workload1(N: int = 1000, Ns: int = 1000) -> Problem:
    k = 1
    X = _rng(1000 + k).uniform(-1.0, 1.0, size=(N, 1))
    noise = _rng(3000 + k).standard_normal(N)
    y = np.sin(3.0 * X[:, 0]) + 0.1 * noise
    Xs = np.linspace(-1.0, 1.0, Ns).reshape(Ns, 1)
    return Problem("w1_p1_n10", _c(X), _c(y), _c(Xs), 10, 1.0, 1.0, 0.01)


def workload2(N: int = 200_000, Ns: int = 50_000) -> Problem:
    k = 2
    X = _rng(1000 + k).uniform(-1.0, 1.0, size=(N, 2))
    noise = _rng(3000 + k).standard_normal(N)
    y = np.sin(3.0 * X[:, 0]) * np.cos(2.0 * X[:, 1]) + 0.05 * noise
    Xs = _rng(2000 + k).uniform(-1.0, 1.0, size=(Ns, 2))
    return Problem("w2_p2_n20", _c(X), _c(y), _c(Xs), 20, 1.0, 0.8, 0.0025)


def workload3(N: int = 2_000_000, Ns: int = 200_000) -> Problem:
    k = 3
    X = _rng(1000 + k).normal(0.0, 0.5, size=(N, 3))
    noise = _rng(3000 + k).standard_normal(N)
    y = np.exp(-np.sum(X * X, axis=1)) + np.sum(np.sin(2.0 * X), axis=1) + 0.05 * noise
    Xs = _rng(2000 + k).normal(0.0, 0.5, size=(Ns, 3))
    return Problem("w3_p3_n16", _c(X), _c(y), _c(Xs), 16, 1.2, 1.0, 0.0025)


def iroot(v: int, p: int) -> int:
    """Largest integer r with r**p <= v (exact, no floating point)."""
    r = int(round(v ** (1.0 / p)))
    while r ** p > v:
        r -= 1
    while (r + 1) ** p <= v:
        r += 1
    return r


def workload4(count: int = 256, Ns: int = 256, n_lo: int = 2,
              N_lo: int = 1_000, N_hi: int = 200_000, M_max: int = 1024,
              seed_offset: int = 0) -> List[Problem]:
    """Batched-fit workload: ``count`` independent problems of uneven shape.

    N is log-uniform on [N_lo, N_hi]; p uniform on {1,2,3,4}; n uniform on
    {n_lo .. floor(M_max**(1/p))}; x ~ U[-1,1]^p; y is a random sum of four
    sinusoids a_k sin(w_k . x + phi_k) with a_k ~ U[0.5,1.5], w_k ~ U[-3,3]^p,
    phi_k ~ U[0, 2 pi], plus 0.1 * N(0,1) noise; eps and alpha are
    log-uniform on [0.5, 2]; sigma2 = 0.01.
    """
    k = 4
    rs = _rng(1000 + k + seed_offset)
    rn = _rng(3000 + k + seed_offset)
    rt = _rng(2000 + k + seed_offset)
    out = []
    for i in range(count):
        N = int(round(math.exp(rs.uniform(math.log(N_lo), math.log(N_hi)))))
        p = int(rs.integers(1, 5))
        n_hi = max(n_lo, iroot(M_max, p))
        n = int(rs.integers(n_lo, n_hi + 1))
        eps = float(math.exp(rs.uniform(math.log(0.5), math.log(2.0))))
        alpha = float(math.exp(rs.uniform(math.log(0.5), math.log(2.0))))
        X = rs.uniform(-1.0, 1.0, size=(N, p))
        a = rs.uniform(0.5, 1.5, size=4)
        w = rs.uniform(-3.0, 3.0, size=(4, p))
        ph = rs.uniform(0.0, 2.0 * math.pi, size=4)
        y = np.sin(X @ w.T + ph) @ a + 0.1 * rn.standard_normal(N)
        Xs = rt.uniform(-1.0, 1.0, size=(Ns, p))
        out.append(Problem(f"w4_{i}", _c(X), _c(y), _c(Xs), n, eps, alpha, 0.01))
    return out


def workload6(p: int, n: int, N: int = 10_000, Ns: int = 1_000, sigma_n: float = 0.1) -> Problem:
    """The paper's sweep workload (Sec. 3): y = sum_i cos(x_i) + nu, N = 10,000.

    The paper states neither the input law nor sigma_n; x ~ U[-1,1]^p and
    sigma_n = 0.1 are this module's choice.
    """
    k = 6
    X = _rng(1000 + k + 10 * p).uniform(-1.0, 1.0, size=(N, p))
    y = np.sum(np.cos(X), axis=1) + sigma_n * _rng(3000 + k + 10 * p).standard_normal(N)
    Xs = _rng(2000 + k + 10 * p).uniform(-1.0, 1.0, size=(Ns, p))
    return Problem(f"w6_p{p}_n{n}", _c(X), _c(y), _c(Xs), n, 1.0, 1.0, sigma_n ** 2)


def random_problem(seed: int, N: int, Ns: int, p: int, n: int, eps: float = 1.0,
                   alpha: float = 1.0, sigma2: float = 0.01, law: str = "uniform",
                   scale: float = 1.0) -> Problem:
    """A small problem with arbitrary shape, for parity and edge-case tests."""
    r = _rng(seed)
    if law == "uniform":
        X = r.uniform(-scale, scale, size=(N, p))
        Xs = r.uniform(-scale, scale, size=(Ns, p))
    else:
        X = r.normal(0.0, scale, size=(N, p))
        Xs = r.normal(0.0, scale, size=(Ns, p))
    y = np.sin(2.0 * X).sum(axis=1) + 0.1 * r.standard_normal(N)
    return Problem(f"rand_{seed}", _c(X), _c(y), _c(Xs), n, eps, alpha, sigma2)


@dataclasses.dataclass
class Request:
    """One serving request: a predict against a resident model, or a refit."""

    t_arrive: float        # seconds from the start of the stream
    kind: str              # "predict" or "refit"
    model: int             # resident model slot
    Xs: Optional[np.ndarray] = None       # predict: (Ns, p)
    refit: Optional[Problem] = None       # refit: the new training set


def workload5_models(count: int = 64, N_max: int = 500_000, M_max: int = 2048,
                     N_lo: int = 10_000) -> List[Problem]:
    """Resident models of the serving workload: p in {2,3,4}, M <= M_max."""
    k = 5
    rs = _rng(1000 + k)
    rn = _rng(3000 + k)
    out = []
    for i in range(count):
        p = int(rs.integers(2, 5))
        n = int(rs.integers(2, iroot(M_max, p) + 1))
        N = int(round(math.exp(rs.uniform(math.log(N_lo), math.log(N_max)))))
        X = rs.uniform(-1.0, 1.0, size=(N, p))
        y = np.sin(3.0 * X[:, 0]) * np.cos(2.0 * X[:, 1 % p]) + 0.05 * rn.standard_normal(N)
        eps = float(math.exp(rs.uniform(math.log(0.5), math.log(2.0))))
        alpha = float(math.exp(rs.uniform(math.log(0.5), math.log(2.0))))
        out.append(Problem(f"w5_m{i}", _c(X), _c(y), np.zeros((0, p)), n, eps, alpha, 0.0025))
    return out


def workload5_stream(models: List[Problem], count: int, rate_hz: float,
                     refit_frac: float = 0.05, Ns_max: int = 65_536,
                     N_refit_lo: int = 10_000, N_refit_hi: int = 500_000,
                     seed: int = 0) -> List[Request]:
    """A Poisson stream of requests against ``models``.

    Inter-arrival times are exponential with mean 1/rate_hz; predict sizes are
    log-uniform on [1, Ns_max]; a fraction ``refit_frac`` of requests are
    refits with N log-uniform on [N_refit_lo, N_refit_hi].
    """
    k = 5
    r = _rng(2000 + k + seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(r.exponential(1.0 / rate_hz))
        m = int(r.integers(0, len(models)))
        p = models[m].p
        if r.uniform() < refit_frac:
            N = int(round(math.exp(r.uniform(math.log(N_refit_lo), math.log(N_refit_hi)))))
            X = r.uniform(-1.0, 1.0, size=(N, p))
            y = np.sin(3.0 * X[:, 0]) * np.cos(2.0 * X[:, 1 % p]) + 0.05 * r.standard_normal(N)
            base = models[m]
            prob = Problem(base.name + "_refit", _c(X), _c(y), np.zeros((0, p)), base.n,
                           base.eps, base.alpha, base.sigma2)
            out.append(Request(t, "refit", m, refit=prob))
        else:
            Ns = int(math.floor(math.exp(r.uniform(0.0, math.log(Ns_max)))))
            Ns = max(1, min(Ns, Ns_max))
            out.append(Request(t, "predict", m, Xs=_c(r.uniform(-1.0, 1.0, size=(Ns, p)))))
    return out
