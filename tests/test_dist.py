"""The row-sharded fit's host logic on CPU: partition, packing, and the one
all-reduce of the Gram across two gloo ranks (each rank's partial Gram is the
oracle's Gram of its row block; their sum must be the Gram of all rows)."""
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


def _rank_main(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = W.random_problem(5, 3001, 1, 2, 6, eps=1.0, alpha=0.9)
    i0, i1 = D.row_partition(pr.N if hasattr(pr, "N") else pr.X.shape[0], world, rank, granule=512)
    G, b = O.gram(pr.X[i0:i1], pr.y[i0:i1], pr.n, pr.eps, pr.alpha)
    Gs, bs = D.allreduce_gram(G, b)
    if rank == 0:
        np.savez(out_path, G=Gs, b=bs)
    dist.barrier()
    dist.destroy_process_group()


def test_allreduce_gram_world2(tmp_path):
    out = str(tmp_path / "g.npz")
    mp.spawn(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True)
    r = np.load(out)
    pr = W.random_problem(5, 3001, 1, 2, 6, eps=1.0, alpha=0.9)
    Go, bo = O.gram(pr.X, pr.y, pr.n, pr.eps, pr.alpha)
    assert O.relerr(r["G"], Go) < 1e-13
    assert O.relerr(r["b"], bo) < 1e-13
    np.testing.assert_array_equal(r["G"], r["G"].T)
