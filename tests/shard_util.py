"""Test helpers for the row-sharded factorisation: the shard steps done by
the CPU oracle (so the orchestrator's protocol runs on gloo ranks without a
GPU), a gather over gloo for numpy shards, and an in-process gather for
shards run as threads."""
import threading

import numpy as np

import oracle as o


class OracleOps:
    """One shard's steps (sketch share, XR, substitution + Gram, Cholesky, R
    product, apply) by the oracle's routines, on numpy arrays."""

    def sketch_part(self, A, s, seed, row0, prec):
        return o.sketch(A, s, seed, row0=row0)

    def sum_parts(self, parts):
        # parts: (shards, cols, rows), block k = shard k's column-major data
        out = np.array(parts[0], dtype=np.float64)
        for k in range(1, len(parts)):
            out = out + parts[k]
        return np.asfortranarray(out.T)

    def xr_factor(self, Y, variant):
        R = o.geqr_r(Y) if variant == "qr" else o.getrf_u(Y)[0]
        R = o.sign_normalise(R)
        return R, o.check_factor(R)

    def precond_gram(self, A, R, prec, X=None):
        Xn = o.trsm_right_upper(A, R)
        return Xn, o.gram(Xn)

    def cholesky(self, G):
        R, info = o.potrf_u(G)
        return R, (2 if info else 0)

    def trmm_upper(self, A, B):
        return o.trmm_upper(A, B)

    def apply_rinv(self, X, R, prec):
        X[...] = o.trsm_right_upper(X, R)
        return X


def gloo_gather_numpy():
    """allgather of a numpy matrix over the default gloo group, in the layout
    OracleOps.sum_parts takes."""
    import torch

    from paper_2111_11148_gb300.sharded import torch_allgather

    g = torch_allgather()
    return lambda a: g(torch.from_numpy(np.asfortranarray(a))).numpy()


class ThreadGather:
    """allgather among `world` threads of one process: each thread hands in
    its block, waits for the others, and gets every block in rank order (for
    CUDA tensors a copy, for numpy an array), in the layout the ops take."""

    def __init__(self, world, stack):
        self.world = world
        self.stack = stack
        self.slots = [None] * world
        self.barrier = threading.Barrier(world)

    def for_rank(self, rank):
        def gather(t):
            self.slots[rank] = t
            self.barrier.wait()
            out = self.stack(list(self.slots))
            self.barrier.wait()  # every rank has read the slots before they are reused
            return out

        return gather


def shard_bounds(m, world):
    """Contiguous row blocks of near-equal size, rank order."""
    return [(m * r // world, m * (r + 1) // world) for r in range(world)]
