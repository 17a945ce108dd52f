"""The row-sharded fit's device path on one GPU: the packed Gram exchange
buffer that gp_gram_packed_ex writes, the fit from it (gp_fit_gram_packed_ex),
and dist.fit_sharded with the buffer in device memory (one rank, so the
all-reduce is the identity).

The packed buffer must be the lower triangle of gp_gram_ex's Gram and its b,
bit for bit; the fit from it must equal the fit from the full Gram bit for
bit; both must match the oracle within the precision mode's tolerance.
"""
import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import dist as D
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(mean=1e-10, var=1e-10), "mixed": dict(mean=1e-4, var=1e-3)}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_packed_gram_exchange_on_device(prec):
    torch = pytest.importorskip("torch")
    pr = W.random_problem(72, 30_000, 400, 3, 8, eps=1.0, alpha=0.9, sigma2=0.005)  # M = 512
    dev = torch.device("cuda", 0)
    Xd, yd = torch.from_numpy(pr.X).to(dev), torch.from_numpy(pr.y).to(dev)
    buf = _lib.gram_packed(Xd, yd, pr.n, pr.eps, pr.alpha, prec=prec)
    G, b = _lib.gram(Xd, yd, pr.n, pr.eps, pr.alpha, prec=prec)
    torch.cuda.synchronize()
    assert buf.shape[0] == D.packed_size(pr.n ** 3)
    np.testing.assert_array_equal(buf.cpu().numpy(), D.pack_lower(G.cpu().numpy(), b.cpu().numpy()))
    m1 = _lib.fit_gram_packed(buf, pr.N, 3, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    m2 = _lib.fit_gram(G.cpu().numpy(), b.cpu().numpy(), pr.N, 3, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec)
    m3 = D.fit_sharded(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec, device=dev)
    try:
        r1, r2, r3 = m1.predict(pr.Xs), m2.predict(pr.Xs), m3.predict(pr.Xs)
        for r in (r2, r3):
            np.testing.assert_array_equal(r[0], r1[0])
            np.testing.assert_array_equal(r[1], r1[1])
        mo, vo = O.predict(O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2), pr.Xs)
        assert O.relerr(r1[0], mo) < TOL[prec]["mean"]
        assert O.relerr(r1[1], vo) < TOL[prec]["var"]
    finally:
        for m in (m1, m2, m3):
            m.free()


def test_packed_fit_from_host_buffer_and_bad_length():
    pr = W.random_problem(73, 5_000, 50, 2, 9, eps=1.1, alpha=1.0, sigma2=0.01)
    buf = _lib.gram_packed(pr.X, pr.y, pr.n, pr.eps, pr.alpha, prec="fp64")
    G, b = O.gram(pr.X, pr.y, pr.n, pr.eps, pr.alpha)
    assert O.relerr(buf, D.pack_lower(G, b)) < 1e-12
    m = _lib.fit_gram_packed(buf, pr.N, 2, pr.n, pr.eps, pr.alpha, pr.sigma2, prec="fp64")
    try:
        mean, var = m.predict(pr.Xs)
        mo, vo = O.predict(O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2), pr.Xs)
        assert O.relerr(mean, mo) < 1e-10 and O.relerr(var, vo) < 1e-10
    finally:
        m.free()
    with pytest.raises(ValueError):
        _lib.fit_gram_packed(buf[:-1], pr.N, 2, pr.n, pr.eps, pr.alpha, pr.sigma2)
