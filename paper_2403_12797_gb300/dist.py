"""Row-sharded fit across processes (one GPU each): the one exchange step.

The Gram G = Phi^T Phi and b = Phi^T y are sums over training rows (Sec. 2.2,
Eq. 11), so a training set split into contiguous row blocks, one per rank,
gives per-rank partial Grams whose sum is the Gram of the whole set. One
all-reduce (sum) of the lower triangle of G and of b -- M(M+1)/2 + M float64
values -- is the only collective; every rank then factors the same A and
holds the same model, and prediction shards the test points with no
collective at all.

Functions here are host logic: the partition, the packing of the lower
triangle, and the all-reduce through torch.distributed (NCCL on GPUs, gloo
on CPUs); the Gram and the factorisation are the library's (gp_gram_ex,
gp_fit_gram_ex).
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def row_partition(N: int, world: int, rank: int, granule: int = 1) -> Tuple[int, int]:
    """Contiguous row block [start, stop) of `rank`: blocks of whole granules,
    sizes differing by at most one granule, covering 0..N exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    units = (N + granule - 1) // granule
    base, extra = divmod(units, world)
    # the last `extra` ranks take one more granule, so the partial last
    # granule falls on a rank that has a whole one more than the first ranks
    first_big = world - extra
    u0 = rank * base + max(0, rank - first_big)
    u1 = u0 + base + (1 if rank >= first_big else 0)
    return min(N, u0 * granule), min(N, u1 * granule)


def pack_lower(G: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The lower triangle of G (row by row) followed by b, as one float64 vector."""
    M = G.shape[0]
    il = np.tril_indices(M)
    return np.concatenate([G[il], b]).astype(np.float64)


def unpack_lower(buf: np.ndarray, M: int) -> Tuple[np.ndarray, np.ndarray]:
    """Inverse of pack_lower: the full symmetric G and b."""
    il = np.tril_indices(M)
    nl = il[0].size
    G = np.zeros((M, M))
    G[il] = buf[:nl]
    G = G + np.tril(G, -1).T
    return G, np.array(buf[nl:nl + M], dtype=np.float64)


def allreduce_gram(G: np.ndarray, b: np.ndarray, group=None, device=None) -> Tuple[np.ndarray, np.ndarray]:
    """Sum (G, b) over the ranks of `group` with one all-reduce of the packed lower triangle."""
    import torch
    import torch.distributed as dist

    buf = torch.from_numpy(pack_lower(G, b))
    if device is not None:
        buf = buf.to(device)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return unpack_lower(buf.cpu().numpy(), G.shape[0])


def fit_sharded(X: np.ndarray, y: np.ndarray, n: int, eps: float, alpha: float, sigma2: float,
                prec: str = "mixed", group=None, device=None):
    """Fit on the whole (X, y) held by every rank, each rank contracting its own
    row block: local Gram on this rank's GPU, one all-reduce, then the same
    factorisation on every rank. Returns this rank's (identical) model."""
    import torch.distributed as dist

    from . import _lib

    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    N = X.shape[0]
    i0, i1 = row_partition(N, world, rank, granule=512)
    Xl = np.ascontiguousarray(X[i0:i1] if i1 > i0 else X[:1] * 0.0)
    yl = np.ascontiguousarray(y[i0:i1] if i1 > i0 else y[:1] * 0.0)
    G, b = _lib.gram(Xl, yl, n, eps, alpha, prec=prec)
    if i1 <= i0:  # an empty shard contributes nothing
        G, b = np.zeros_like(G), np.zeros_like(b)
    if world > 1:
        G, b = allreduce_gram(G, b, group=group, device=device)
    return _lib.fit_gram(G, b, N, X.shape[1] if X.ndim > 1 else 1, n, eps, alpha, sigma2, prec=prec)
