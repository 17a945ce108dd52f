"""Batched fit (one captured graph; the mixed Grams of all problems in one
launch per p; an autotuned plan with an on-disk cache) and batched predict.

The batch is a small instance of the uneven-shape batched workload (p in
1..4, M <= 256, N log-uniform up to 20,000) plus one member at M = 1024. Every batched model is checked
against the FP64 oracle with the precision mode's tolerances, batched
predicts against single predicts bitwise, and a failing member against its
index.
"""
import numpy as np
import pytest
import torch

from oracle import fagp as O
from paper_2403_12797_gb300 import _lib
from paper_2403_12797_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(mean=1e-10, var=1e-10), "mixed": dict(mean=1e-4, var=1e-3)}


def _batch(count=16, seed_offset=0, with_m1024=False):
    out = W.workload4(count=count, Ns=300, N_hi=20_000, M_max=256, seed_offset=seed_offset)
    if with_m1024:
        # one member at the batched workload's largest M (p = 2, n = 32)
        out.append(W.random_problem(61, 20_000, 300, 2, 32, eps=1.0, alpha=0.9, sigma2=0.01))
    return out


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_fit_batch_matches_oracle(prec):
    probs = _batch(with_m1024=True)
    models = _lib.fit_batch([(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in probs], prec=prec)
    used_graph, k = _lib.batch_info()
    plan = _lib.batch_plan()
    assert k == plan["k"] and k in ((1, 2, 4) if prec == "mixed" else (0,))
    assert plan["streams"] in (8, 16, 17) and plan["tuned_ms"] > 0
    assert used_graph in (0, 1)
    try:
        for pr, m in zip(probs, models):
            assert m is not None
            mean, var = m.predict(pr.Xs)
            mdl = O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2)
            mo, vo = O.predict(mdl, pr.Xs)
            assert O.relerr(mean, mo) < TOL[prec]["mean"], (pr.name, O.relerr(mean, mo))
            assert O.relerr(var, vo) < TOL[prec]["var"], (pr.name, O.relerr(var, vo))
    finally:
        for m in models:
            m.free()


def test_fit_batch_agrees_with_single_fits():
    probs = _batch(count=6, seed_offset=7)
    models = _lib.fit_batch([(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in probs], prec="fp64")
    try:
        for pr, m in zip(probs, models):
            s = _lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec="fp64")
            try:
                # same arithmetic up to the order of the Gram's split sums
                assert O.relerr(m.read("L"), s.read("L")) < 1e-12
                assert O.relerr(m.read("c"), s.read("c")) < 1e-9
            finally:
                s.free()
    finally:
        for m in models:
            m.free()


def test_fit_batch_reports_failing_member():
    probs = _batch(count=5, seed_offset=3)
    bad = 2
    ys = [pr.y.copy() for pr in probs]
    ys[bad][7] = np.nan
    with pytest.raises(_lib.GPError) as ei:
        _lib.fit_batch([(pr.X, y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr, y in zip(probs, ys)])
    assert ei.value.status == _lib.GP_EINVAL
    assert ei.value.detail == bad


def test_predict_batch_bitwise_equals_single():
    probs = _batch(count=3, seed_offset=11)
    dev = torch.device("cuda", 0)
    for prec in ("mixed", "fp64"):
        models = [_lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec) for pr in probs]
        try:
            reqs, singles = [], []
            rng = np.random.default_rng(5)
            for r in range(9):
                m, pr = models[r % 3], probs[r % 3]
                ns = int(rng.choice([1, 17, 129, 300]))
                Xs = torch.from_numpy(pr.Xs[:ns].copy()).to(dev)
                mo = torch.empty(ns, dtype=torch.float64, device=dev)
                vo = torch.empty(ns, dtype=torch.float64, device=dev)
                reqs.append((m, Xs, mo, vo))
                singles.append(m.predict(pr.Xs[:ns]))
            _lib.predict_batch(reqs)
            torch.cuda.synchronize()
            for (m, Xs, mo, vo), (ms, vs) in zip(reqs, singles):
                np.testing.assert_array_equal(mo.cpu().numpy(), ms)
                np.testing.assert_array_equal(vo.cpu().numpy(), vs)
        finally:
            for m in models:
                m.free()


def test_predict_batch_mixed_dimensions_and_modes():
    """One gp_predict_batch over models of p = 1..5 in both precision modes
    (one persistent predict launch per p for the mixed models), requests
    with and without the variance, sizes from 1 point to several tiles with
    ragged tails: each result bitwise equal to the request alone, and within
    the mode's tolerance of the oracle."""
    shapes = [(1, 30, 5_000), (2, 12, 8_000), (3, 7, 6_000), (4, 4, 6_000), (2, 20, 12_000), (3, 10, 9_000),
              (5, 3, 4_000)]
    probs = [W.random_problem(90 + k, N, 700, p, n, eps=0.9 + 0.1 * k, alpha=1.0, sigma2=0.01)
             for k, (p, n, N) in enumerate(shapes)]
    dev = torch.device("cuda", 0)
    models, precs = [], []
    for k, pr in enumerate(probs):
        for prec in ("mixed", "fp64"):
            models.append((_lib.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2, prec=prec), k, prec))
    try:
        rng = np.random.default_rng(9)
        reqs, meta = [], []
        for r in range(30):
            m, k, prec = models[int(rng.integers(len(models)))]
            ns = int(rng.choice([1, 5, 127, 128, 129, 300, 700]))
            with_var = bool(rng.integers(4))
            Xs = torch.from_numpy(probs[k].Xs[:ns].copy()).to(dev)
            mo = torch.empty(ns, dtype=torch.float64, device=dev)
            vo = torch.empty(ns, dtype=torch.float64, device=dev) if with_var else None
            reqs.append((m, Xs, mo, vo))
            meta.append((k, prec, ns))
        _lib.predict_batch(reqs)
        torch.cuda.synchronize()
        oracles = [O.fit(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in probs]
        for (m, Xs, mo, vo), (k, prec, ns) in zip(reqs, meta):
            ms, vs = m.predict(probs[k].Xs[:ns])
            np.testing.assert_array_equal(mo.cpu().numpy(), ms)
            if vo is not None:
                np.testing.assert_array_equal(vo.cpu().numpy(), vs)
            mref, vref = O.predict(oracles[k], probs[k].Xs[:ns])
            assert O.relerr(ms, mref) < TOL[prec]["mean"], (k, prec, ns)
            assert O.relerr(vs, vref) < TOL[prec]["var"], (k, prec, ns)
    finally:
        for m, _, _ in models:
            m.free()


_CACHE_PROBE = r"""
import json, sys
sys.path.insert(0, {root!r})
from paper_2403_12797_gb300 import _lib, workloads as W
probs = W.workload4(count=12, Ns=1, N_hi=20_000, M_max=256, seed_offset=21)
ms = _lib.fit_batch([(pr.X, pr.y, pr.n, pr.eps, pr.alpha, pr.sigma2) for pr in probs])
print(json.dumps(_lib.batch_plan()))
for m in ms:
    m.free()
"""


def test_batch_plan_cache_persists_across_processes(tmp_path):
    """The first process times the candidates and appends the winner to
    GPFAGP_TUNE_CACHE; a second process with the same batch reads it back
    and runs the same plan without tuning."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.tsv"
    env = dict(os.environ, GPFAGP_TUNE_CACHE=str(cache))
    code = _CACHE_PROBE.format(root=root)
    runs = []
    for _ in range(2):
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        runs.append(json.loads(r.stdout.strip().splitlines()[-1]))
    assert not runs[0]["from_cache"] and runs[1]["from_cache"]
    assert [runs[1][k] for k in ("streams", "k", "factor_ctas")] == [runs[0][k] for k in ("streams", "k", "factor_ctas")]
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and lines[0].startswith("batch/")
