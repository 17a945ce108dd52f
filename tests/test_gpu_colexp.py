"""The mixed Gram's column scales (Phi of Eq. 19, the sums of Sec. 2.2).

For every 1024-row block and column the library takes the exponent E with
the block's maximum of |Phi| in [2^(E-1), 2^E) (raised by 2^-20, floor -100),
scales the column by 2^(6 - E) and relies on |w| < 64 for its exact integer
sums. Checked here against the oracle's float64 eigenfunction columns, block
by block: an exponent one too small would break the exact sums, one too
large would cost a bit of every value. The 4096-row (CTA-pair) exponents
must be the largest of their four blocks', the global ones the largest of
all. The shapes cover the staged kernel (p = 1..4) and the general one
(p = 5, and p = 1 with n = 400, whose table chunks are too large for the
staged ring).
"""
import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    # the M = 4096 workload's input law (x ~ N(0, 0.5^2)), ragged N
    "p3n16_gauss": lambda: W.random_problem(81, 20_037, 1, 3, 16, eps=1.2, alpha=1.0, law="normal", scale=0.5),
    "p2n20_unif": lambda: W.random_problem(82, 9_000, 1, 2, 20, eps=1.0, alpha=0.8),
    "p4n6_unif": lambda: W.random_problem(83, 5_000, 1, 4, 6, eps=1.1, alpha=1.0),
    "p1n400_unif": lambda: W.random_problem(84, 3_000, 1, 1, 400, eps=1.0, alpha=1.0),
    "p5n3_unif": lambda: W.random_problem(85, 4_100, 1, 5, 3, eps=1.0, alpha=1.0),
}

SLACK = 1e-4  # float32 tables against the float64 oracle, far below a factor of 2


def _block_maxima(X, n, eps, alpha, r0, r1):
    p = X.shape[1]
    E = [O.eigenfunctions_1d(X[r0:r1, j], n, eps, alpha) for j in range(p)]
    idx = O.multi_index(n, p)
    phi = E[0][:, idx[:, 0]].copy()
    for j in range(1, p):
        phi *= E[j][:, idx[:, j]]
    return np.abs(phi).max(axis=0)


@pytest.mark.parametrize("name", sorted(CASES))
def test_column_exponents_bound_the_block_maxima(name):
    pr = CASES[name]()
    N = pr.X.shape[0]
    ebx, ebx4, colexp = _lib.debug_column_exponents(pr.X, pr.n, pr.eps, pr.alpha)
    nblk = ebx.shape[0]
    assert nblk == -(-(-(-N // 128) * 128) // 1024)
    for b in range(nblk):
        r0, r1 = b * 1024, min(N, (b + 1) * 1024)
        mx = _block_maxima(pr.X, pr.n, pr.eps, pr.alpha, r0, r1)
        E = ebx[b]
        tiny = mx < 2.0 ** -101
        assert np.all(E[tiny] == -100), (name, b)
        ok = (np.ldexp(1.0, E - 1) <= mx * (1 + SLACK)) & (mx * (1 - SLACK) < np.ldexp(1.0, E))
        bad = np.flatnonzero(~ok & ~tiny)
        assert bad.size == 0, (name, b, bad[:5], E[bad[:5]], mx[bad[:5]])
    # the CTA-pair kernel's 4096-row blocks and the global exponents
    for b4 in range(ebx4.shape[0]):
        np.testing.assert_array_equal(ebx4[b4], ebx[4 * b4:4 * b4 + 4].max(axis=0))
    np.testing.assert_array_equal(colexp, ebx.max(axis=0))
