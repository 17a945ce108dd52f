"""The full predictive covariance block (Eq. 12) through gp_predict_cov_ex.

Every element is compared with the FP64 oracle's Sigma_* = sigma^2 V^T V,
V = L^{-1} Phi_*^T, on test sets that span several 128-point tiles with a
ragged tail. Covariances between distant points are small next to the
variances, so the bar is set on the correlation scale:
|cov_ij - ref_ij| <= tol * sqrt(ref_ii ref_jj). The mixed model forms
Z = Phi_* L^{-T} in bf16x3 and its Gram in bf16x3 again (float32
accumulation); the float64 model stays in float64.

Exact properties checked as well: symmetry (both triangles are written from
one product), the noisy diagonal (+sigma^2, the covariance of y*), the mean
equal to gp_predict_ex's mean, the diagonal equal to gp_predict_ex's
variance within the mode's rounding, and positive semi-definiteness up to
rounding.
"""
import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (name, problem, Ns)
CASES = [
    ("p2n12", lambda: W.random_problem(61, 6_000, 300, 2, 12, eps=0.9, alpha=1.1, sigma2=0.01)),
    ("p1n40", lambda: W.random_problem(62, 3_000, 129, 1, 40, eps=1.0, alpha=1.0, sigma2=0.02)),
    ("p3n12_m1728", lambda: W.random_problem(63, 20_000, 385, 3, 12, eps=1.1, alpha=1.0, sigma2=0.005)),
    ("p4n5", lambda: W.random_problem(64, 8_000, 200, 4, 5, eps=0.8, alpha=1.2, sigma2=0.02)),
    ("ns1", lambda: W.random_problem(65, 2_000, 1, 2, 8, eps=1.0, alpha=0.9, sigma2=0.01)),
    ("p5n3", lambda: W.random_problem(67, 3_000, 200, 5, 3, eps=0.9, alpha=1.1, sigma2=0.02)),
]

TOL = {"fp64": 1e-11, "mixed": 2e-4}
TOL_DIAG = {"fp64": 1e-12, "mixed": 2e-4}  # |diag - var| / var against the same model's predict


def _corr_err(cov, ref):
    d = np.sqrt(np.maximum(np.diag(ref), 1e-300))
    return float(np.max(np.abs(cov - ref) / np.outer(d, d)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_covariance_block_matches_oracle(prec, case):
    name, make = CASES[case]
    pr = make()
    m = _lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    try:
        mean, cov = m.predict_cov(pr.Xs)
        mean2, var2 = m.predict(pr.Xs)
        mean_n, cov_n = m.predict_cov(pr.Xs, noisy=True)
    finally:
        m.free()
    mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
    ref = O.predict_covariance(mdl, pr.Xs)
    ref_mean, ref_var = O.predict(mdl, pr.Xs)
    assert cov.shape == (pr.Ns, pr.Ns) and np.all(np.isfinite(cov))
    assert np.array_equal(cov, cov.T), name
    err = _corr_err(cov, ref)
    assert err <= TOL[prec], (name, err)
    # the covariance's mean is the predict's mean
    assert np.array_equal(mean, mean2), name
    # the diagonal is the variance, up to the mode's rounding
    assert np.max(np.abs(np.diag(cov) - var2) / var2) <= TOL_DIAG[prec], name
    assert np.allclose(np.diag(ref), ref_var, rtol=1e-10)
    # y* adds sigma^2 on the diagonal and nothing else
    assert np.array_equal(mean_n, mean)
    off = ~np.eye(pr.Ns, dtype=bool)
    assert np.array_equal(cov_n[off], cov[off])
    assert np.allclose(np.diag(cov_n) - np.diag(cov), pr.sigma2, rtol=1e-12, atol=0)
    # positive semi-definite up to rounding: an error E with |E_ij| <= tol
    # sqrt(ref_ii ref_jj) has spectral norm <= tol * trace(ref)
    w = np.linalg.eigvalsh(cov)
    assert w.min() >= -TOL[prec] * np.trace(ref), (name, w.min(), w.max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_covariance_block_device_pointers(prec):
    torch = pytest.importorskip("torch")
    pr = W.random_problem(66, 4_000, 260, 2, 10, eps=1.0, alpha=1.0, sigma2=0.01)
    m = _lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    try:
        mh, ch = m.predict_cov(pr.Xs)
        Xd = torch.from_numpy(pr.Xs).cuda()
        md, cd = m.predict_cov(Xd)
        torch.cuda.synchronize()
        assert np.array_equal(md.cpu().numpy(), mh)
        assert np.array_equal(cd.cpu().numpy(), ch)
        # no test points: nothing to do
        m0, c0 = m.predict_cov(pr.Xs[:0])
        assert m0.shape == (0,) and c0.shape == (0, 0)
    finally:
        m.free()
