"""Request server: continuous batching over resident models.

Predict requests of uneven sizes against several resident models are all
submitted at once (more than there are slots), so most start while others
are on the GPU and queued predicts leave in batches (one persistent predict
launch per basis dimension); each result must equal the same request run alone through
gp_predict (bitwise: the same kernels with the same launch plans) and match
the FP64 oracle's posterior within the precision mode's tolerance. A tight
memory budget must still complete everything. A refit swaps the model in:
predicts after it equal a fresh fit of the new data.
"""
import numpy as np
import pytest

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(mean=1e-10, var=1e-10), "mixed": dict(mean=1e-4, var=1e-3)}


def _problems():
    out = []
    for k, (p, n, N) in enumerate([(2, 12, 20_000), (3, 6, 15_000), (1, 40, 8_000), (4, 4, 12_000)]):
        out.append(W.random_problem(40 + k, N, 64, p, n, eps=0.9, alpha=1.1, sigma2=0.01))
    return out


def _requests(probs, count, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        k = int(rng.integers(len(probs)))
        ns = int(np.exp(rng.uniform(0.0, np.log(6000.0))))
        Xs = rng.uniform(-1.0, 1.0, size=(ns, probs[k].X.shape[1]))
        reqs.append((k, Xs))
    return reqs


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("budget", [0, 24 << 20])
def test_mix_equals_alone(prec, budget):
    probs = _problems()
    alone = [_lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec) for pr in probs]
    served = [_lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec) for pr in probs]
    reqs = _requests(probs, 40, seed=budget % 7)
    try:
        with _lib.Server(slots=6, mem_budget=budget) as srv:
            ids = [srv.add_model(m) for m in served]
            tickets = [srv.submit_predict(ids[k], Xs) for k, Xs in reqs]
            outs = [srv.wait(t, timeout=120.0) for t in tickets]
            st = srv.stats()
        assert st["predicts_done"] == len(reqs)
        assert st["points"] == sum(Xs.shape[0] for _, Xs in reqs)
        assert 1 <= st["peak_inflight"] <= len(reqs)
        assert 1 <= st["peak_batch"] <= st["peak_inflight"]
        assert 1 <= st["batches"] <= len(reqs)
        if budget == 0:
            # 40 requests queue faster than 6 slots drain: predicts travel in batches
            assert st["peak_batch"] >= 2 and st["batches"] < len(reqs)
        assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
        oracles = [O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in probs]
        for (k, Xs), (mean, var) in zip(reqs, outs):
            m1, v1 = alone[k].predict(Xs)
            np.testing.assert_array_equal(mean, m1)
            np.testing.assert_array_equal(var, v1)
            mo, vo = O.predict(oracles[k], Xs)
            assert O.relerr(mean, mo) < TOL[prec]["mean"], (k, O.relerr(mean, mo))
            assert O.relerr(var, vo) < TOL[prec]["var"], (k, O.relerr(var, vo))
    finally:
        for m in alone:
            m.free()


def test_refit_swaps_model():
    probs = _problems()[:2]
    new = W.random_problem(77, 9_000, 64, probs[0].X.shape[1], probs[0].n, eps=probs[0].eps,
                           alpha=probs[0].alpha, sigma2=probs[0].sigma2)
    ref = _lib.fit(new.X, new.y, new.n, new.eps, new.alpha, new.sigma2)
    try:
        with _lib.Server(slots=4) as srv:
            ids = [srv.add_model(_lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)) for pr in probs]
            before = srv.submit_predict(ids[0], new.Xs)
            t = srv.submit_refit(ids[0], new.X, new.y)
            other = srv.submit_predict(ids[1], probs[1].Xs)
            srv.wait(before, timeout=120.0)
            srv.wait(t, timeout=120.0)
            srv.wait(other, timeout=120.0)
            after = srv.wait(srv.submit_predict(ids[0], new.Xs), timeout=120.0)
            assert srv.stats()["refits_done"] == 1
        m1, v1 = ref.predict(new.Xs)
        np.testing.assert_array_equal(after[0], m1)
        np.testing.assert_array_equal(after[1], v1)
    finally:
        ref.free()
