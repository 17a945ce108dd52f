"""The allocation-free Gram entry point, gp_gram_static.

It serves callers that cannot allocate device memory during the call (a
fixed, pre-carved memory budget, a real-time loop that must not enter the
allocator, an allocator hook that must not be re-entered): its scratch is a
static device array inside the library. The test calls it through the C ABI
with device pointers and compares it with the allocating gp_gram_ex on
several calls in a row, so that contents left in the shared array by one
call cannot leak into the next, with the library's allocator armed to fail
its next allocation during each call (so any allocation would show as
GP_ENOMEM). This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the fp64 Gram tolerance of the parity tests


def _static_gram(L, X, y, N, p, n, eps, alpha):
    import torch
    M = n ** p
    G = torch.full((M, M), float("nan"), dtype=torch.float64, device=X.device)
    b = torch.full((M,), float("nan"), dtype=torch.float64, device=X.device)
    rc = L.gp_gram_static(X.data_ptr(), y.data_ptr(), N, p, n, eps, alpha, G.data_ptr(),
                          b.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, G, b


def test_static_gram_matches_allocating_gram_on_consecutive_calls():
    import torch
    from oracle import fagp as O
    from paper_2403_12797_gb300 import _lib
    from paper_2403_12797_gb300 import workloads as W
    L = _lib.lib()
    cases = [(31, 5000, 2, 12), (32, 1777, 3, 5), (31, 5000, 2, 12)]
    for seed, N, p, n in cases:
        pr = W.random_problem(seed, N, 1, p, n, eps=1.1, alpha=0.9)
        X = torch.from_numpy(pr.X).cuda()
        y = torch.from_numpy(pr.y).cuda()
        M = n ** p
        G = torch.full((M, M), float("nan"), dtype=torch.float64, device="cuda")
        b = torch.full((M,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        # the library's allocator is armed to fail its next allocation: a call
        # that allocated anything would return GP_ENOMEM
        _lib.debug_fail_alloc_after(1)
        try:
            rc = L.gp_gram_static(X.data_ptr(), y.data_ptr(), N, p, n, pr.eps, pr.alpha, G.data_ptr(),
                                  b.data_ptr(), torch.cuda.current_stream().cuda_stream)
        finally:
            _lib.debug_fail_alloc_after(0)
        assert rc == _lib.GP_OK, _lib.strerror(rc)
        Gr, br = _lib.gram(X, y, n, pr.eps, pr.alpha, prec="fp64")
        torch.cuda.synchronize()
        assert O.relerr(G.cpu().numpy(), Gr.cpu().numpy()) < TOL
        assert O.relerr(b.cpu().numpy(), br.cpu().numpy()) < TOL


def test_static_gram_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2403_12797_gb300 import _lib
    L = _lib.lib()
    N, p, n = 400_000, 2, 20     # tables alone: 2 * 20 * 400k doubles = 128 MB > 32 MiB
    X = torch.zeros((N, p), dtype=torch.float64, device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    rc, _, _ = _static_gram(L, X, y, N, p, n, 1.0, 1.0)
    assert rc == _lib.GP_EINVAL
    assert L.gp_last_error_detail() > (32 << 20)
