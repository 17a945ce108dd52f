"""Row-sharded fit across processes (one GPU each): the one exchange step.

The Gram G = Phi^T Phi and b = Phi^T y are sums over training rows (Sec. 2.2,
Eq. 11), so a training set split into contiguous row blocks, one per rank,
gives per-rank partial Grams whose sum is the Gram of the whole set. One
all-reduce (sum) of the lower triangle of G and of b -- M(M+1)/2 + M float64
values -- is the only collective; every rank then factors the same A and
holds the same model, and prediction shards the test points with no
collective at all.

On GPUs the exchange never leaves device memory: the library writes the
rank's packed Gram into a device buffer (gp_gram_packed_ex), NCCL sums the
buffers in place, and the library fits from the sum (gp_fit_gram_packed_ex).
This module holds the host logic around that: the row partition, the empty
shard, the row count that travels with the buffer, and the all-reduce
through torch.distributed (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

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


def packed_size(M: int) -> int:
    """Length of the exchange buffer: the lower triangle of an M x M Gram, then b."""
    return M * (M + 1) // 2 + M


def pack_lower(G: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The exchange layout on the host: the lower triangle of G (row by row,
    entry (i, j) at i (i + 1) / 2 + j) followed by b, as one float64 vector
    (the layout gp_gram_packed_ex writes on the device)."""
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


def fit_sharded(X, y, n: int, eps: float, alpha: float, sigma2: float, prec: str = "mixed",
                group=None, device=None, local: bool = False,
                gram: Optional[Callable] = None, fit_gram: Optional[Callable] = None):
    """Fit one GP on a training set whose rows are spread over the ranks of
    `group`: each rank's Gram of its own rows, one all-reduce, then the same
    factorisation on every rank. Returns this rank's (identical) model.

    X, y: the whole training set on every rank (local=False: each rank takes
    its row_partition block, in granules of 512 rows), or this rank's own
    rows (local=True: the total row count is summed with the exchange).
    device: this rank's CUDA device -- rows, Gram, all-reduce (NCCL) and fit
    stay in its memory; None: host buffers (gloo).
    gram(Xl, yl, out) -> packed Gram of the rows (written into the view
    `out` of the exchange buffer, or returned) and
    fit_gram(buf, N) -> model default to the library's gram_packed and
    fit_gram_packed; they are parameters so that the host logic can be
    exercised on CPU ranks.
    """
    import torch
    import torch.distributed as dist

    if gram is None or fit_gram is None:
        from . import _lib
        if gram is None:
            def gram(Xl, yl, out):
                return _lib.gram_packed(Xl, yl, n, eps, alpha, prec=prec, out=out)
        if fit_gram is None:
            p_ = X.shape[1] if X.ndim > 1 else 1

            def fit_gram(buf, N_):
                return _lib.fit_gram_packed(buf, N_, p_, n, eps, alpha, sigma2, prec=prec)

    on = dist.is_available() and dist.is_initialized()
    world = dist.get_world_size(group) if on else 1
    rank = dist.get_rank(group) if on else 0
    p = X.shape[1] if X.ndim > 1 else 1
    size = packed_size(int(n) ** p)
    if local:
        Xl, yl = X, y
    else:
        i0, i1 = row_partition(int(X.shape[0]), world, rank, granule=512)
        Xl, yl = X[i0:i1], y[i0:i1]
    nloc = int(Xl.shape[0])
    # the exchange buffer: packed Gram of this rank's rows, then its row count
    buf = torch.zeros(size + 1, dtype=torch.float64, device=device if device is not None else "cpu")
    if nloc > 0:  # an empty shard contributes zeros
        if device is not None and not torch.is_tensor(Xl):
            Xl = torch.from_numpy(np.ascontiguousarray(Xl, dtype=np.float64)).to(device)
            yl = torch.from_numpy(np.ascontiguousarray(yl, dtype=np.float64)).to(device)
        view = buf[:size]
        part = gram(Xl, yl, view)
        if part is not view:
            if not torch.is_tensor(part):
                part = torch.from_numpy(np.ascontiguousarray(part))
            view.copy_(part.reshape(-1))
    buf[size] = float(nloc)
    if world > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    N = int(round(float(buf[size].item())))
    if N < 1:
        raise ValueError("no training rows on any rank")
    return fit_gram(buf[:size], N)
