"""The row-sharded fit's host logic on CPU: partition, packing, and
fit_sharded itself across gloo ranks -- each rank's Gram (the oracle's, in
the exchange layout, injected in place of the library's) of its row block,
one all-reduce of the buffer with the row count, the empty shard, and the
hand-off to the fit step."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import fagp as O
from paper_2403_12797_gb300 import dist as D
from paper_2403_12797_gb300 import workloads as W


@pytest.mark.parametrize("N,world,granule", [(1000, 2, 1), (1000, 3, 512), (7, 4, 1), (0, 2, 1),
                                             (200_000, 8, 512), (513, 2, 512)])
def test_row_partition_covers_rows_once(N, world, granule):
    blocks = [D.row_partition(N, world, r, granule) for r in range(world)]
    assert blocks[0][0] == 0 and blocks[-1][1] == N
    for (a0, a1), (b0, b1) in zip(blocks, blocks[1:]):
        assert a1 == b0 and a0 <= a1
    sizes = [b - a for a, b in blocks]
    assert max(sizes) - min(sizes) <= granule
    for a, _ in blocks[:-1]:
        assert a % granule == 0


def test_pack_roundtrip():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((9, 9))
    G = B @ B.T
    b = rng.standard_normal(9)
    buf = D.pack_lower(G, b)
    assert buf.size == 9 * 10 // 2 + 9
    G2, b2 = D.unpack_lower(buf, 9)
    np.testing.assert_array_equal(G2, G2.T)
    np.testing.assert_allclose(G2, G, rtol=0, atol=0)
    np.testing.assert_array_equal(b2, b)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_path, N, local):
    """One gloo rank: fit_sharded with the oracle's packed Gram injected and a
    fit step that returns what it was handed (the summed buffer and N)."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    calls = []

    def gram(Xl, yl, out):
        calls.append(int(Xl.shape[0]))
        return D.pack_lower(*O.gram(Xl, yl, 6, 1.0, 0.9))

    def fit_gram(buf, N_):
        return buf.numpy().copy(), N_

    if local:  # each rank holds its own rows
        pr = W.random_problem(100 + rank, N + 37 * rank, 1, 2, 6, eps=1.0, alpha=0.9)
    else:      # every rank holds the whole set
        pr = W.random_problem(5, N, 1, 2, 6, eps=1.0, alpha=0.9)
    buf, Ntot = D.fit_sharded(pr.X, pr.y, 6, 1.0, 0.9, 0.01, group=None, local=local, gram=gram,
                              fit_gram=fit_gram)
    np.savez(out_path + f".{rank}.npz", buf=buf, N=Ntot, calls=np.array(calls, dtype=np.int64))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("N,world,local", [(3001, 2, False), (700, 3, False), (1500, 2, True)])
def test_fit_sharded_exchange(tmp_path, N, world, local):
    """The summed exchange buffer on every rank is the packed Gram of all rows
    (one all-reduce), the row count is the total, an empty shard (world 3,
    700 rows in 512-row granules) contributes zeros without a Gram call,
    and every rank hands the same buffer to the fit step."""
    out = str(tmp_path / "x")
    mp.spawn(_rank_main, args=(world, _free_port(), out, N, local), nprocs=world, join=True)
    res = [np.load(out + f".{r}.npz") for r in range(world)]
    if local:
        parts = [W.random_problem(100 + r, N + 37 * r, 1, 2, 6, eps=1.0, alpha=0.9) for r in range(world)]
        X = np.concatenate([q.X for q in parts])
        y = np.concatenate([q.y for q in parts])
    else:
        pr = W.random_problem(5, N, 1, 2, 6, eps=1.0, alpha=0.9)
        X, y = pr.X, pr.y
    ref = D.pack_lower(*O.gram(X, y, 6, 1.0, 0.9))
    for r, z in enumerate(res):
        assert int(z["N"]) == X.shape[0]
        assert O.relerr(z["buf"], ref) < 1e-13
        np.testing.assert_array_equal(z["buf"], res[0]["buf"])
        if not local:
            i0, i1 = D.row_partition(N, world, r, granule=512)
            assert list(z["calls"]) == ([i1 - i0] if i1 > i0 else [])
    G, b = D.unpack_lower(res[0]["buf"], 36)
    np.testing.assert_array_equal(G, G.T)
