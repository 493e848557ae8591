"""Row-sharded rLU-/rQR-CholeskyQR over several processes or GPUs.

This is the parallel scheme of Section 2.4 (its communication is Section
2.5's table), laid out for GPUs:

* each shard holds a contiguous block of A's rows (global rows row0 ..
  row0 + m_local - 1);
* it computes its partial sketch (rxr_sketch_part: Omega's columns follow the
  global rows, so no random numbers travel) and its partial Grams with the
  library's kernels;
* the shards exchange these s x n and n x n partials with one allgather per
  stage and sum them on the device in rank order (rxr_sum_parts), so that every
  shard holds the same sketch, the same Grams and the same R, and runs the
  small factorisations (XR of the sketch, Cholesky, R accumulation) itself:
  there is no broadcast;
* Q's rows never leave their shard.

That makes 1 + P allgathers of s x n or n x n doubles per factorisation for P
CholeskyQR passes (the paper counts 3 to 4 collectives).  This module only
sequences the library calls and the collectives: every arithmetic step runs
in librxr's kernels (or, for the CPU tests, in the oracle).
"""
from __future__ import annotations

from typing import Callable, Optional

__all__ = ["LibraryOps", "cholqr_sharded", "torch_allgather"]


class LibraryOps:
    """The steps one shard runs, on the GPU through librxr (a Handle)."""

    def __init__(self, handle, stream=None):
        self.h = handle
        self.stream = stream

    def sketch_part(self, A, s, seed, row0, prec):
        return self.h.sketch_part(A, s, seed=seed, row0=row0, prec=prec, stream=self.stream)

    def sum_parts(self, parts):
        # parts[k] is shard k's column-major matrix stored as its transpose
        # (see torch_allgather): the fixed-order device sum, back to (rows, cols)
        return self.h.sum_parts(parts, stream=self.stream).t()

    def xr_factor(self, Y, variant):
        return self.h.xr_factor(Y, variant, stream=self.stream, raise_on_error=False)

    def precond_gram(self, A, R, prec, X=None):
        return self.h.precond_gram(A, R, X=X, prec=prec, stream=self.stream)

    def cholesky(self, G):
        return self.h.cholesky(G, stream=self.stream, raise_on_error=False)

    def trmm_upper(self, A, B):
        return self.h.trmm_upper(A, B, stream=self.stream)

    def apply_rinv(self, X, R, prec):
        return self.h.apply_rinv(X, R, prec=prec, stream=self.stream)


def cholqr_sharded(ops, A, row0: int, allgather: Callable, variant: str = "qr", s: Optional[int] = None,
                   seed: int = 0, passes: int = 2, prec: str = "fp64"):
    """Factorise the matrix whose rows row0 .. row0 + m_local - 1 this shard
    holds in A (m_local x n, m_local >= n).  allgather(t) returns every
    shard's t in rank order, in the layout ops.sum_parts takes (for
    LibraryOps: torch_allgather's stack of transposes).  Returns
    (Q_local, R, status): Q_local the shard's rows of Q (m_local x n), R the
    n x n factor (the same bits on every shard), status 0 or an RXR_ERR_*
    code (the same on every shard: they factorise the same sums)."""
    n = A.shape[1]
    s = 2 * n if s is None else int(s)
    # steps 1-2 of Algorithms 4/5: Y = Omega A over all shards, R_s = XR(Y)
    Y = ops.sum_parts(allgather(ops.sketch_part(A, s, seed, row0, prec)))
    Rs, code = ops.xr_factor(Y, variant)
    if code:
        return None, None, code
    # step 3: X = A R_s^{-1} on the shard's rows (into Q), with its Gram share
    Q, G = ops.precond_gram(A, Rs, prec)
    R = Rs
    # CholeskyQR passes (Algorithm 2): the Gram summed over shards, R_p by
    # every shard, X <- X R_p^{-1} in place with the next Gram share
    for p in range(1, passes + 1):
        G = ops.sum_parts(allgather(G))
        Rp, code = ops.cholesky(G)
        if code:
            return Q, None, code
        R = ops.trmm_upper(Rp, R)
        if p == passes:
            ops.apply_rinv(Q, Rp, prec)
        else:
            Q, G = ops.precond_gram(Q, Rp, prec, X=Q)
    return Q, R, 0


def torch_allgather(group=None) -> Callable:
    """allgather over a torch.distributed process group (NCCL for CUDA
    tensors, gloo for CPU tensors).  t: a column-major matrix (rows x cols,
    stride (1, ld)); returns a contiguous (world, cols, rows) tensor whose block
    k is rank k's matrix transposed, i.e. its column-major data: the layout
    LibraryOps.sum_parts sums."""
    import torch.distributed as dist

    def gather(t):
        import torch

        world = dist.get_world_size(group)
        flat = t.t().contiguous()  # (cols, rows): the column-major data of t
        outs = [torch.empty_like(flat) for _ in range(world)]
        dist.all_gather(outs, flat, group=group)
        return torch.stack(outs)

    return gather
