"""Seeded synthetic inputs for randomized XR-preconditioned CholeskyQR.

This module builds the test matrices only; it holds none of the method's
arithmetic.  Both the CUDA path's tests/benchmark and the CPU oracle take their
inputs from here, so the two sides see the same bytes.

Construction (Section 4.1 of Fan, Guo & Lin): A = U diag(sigma) V^T with U an
m x n matrix with orthonormal columns, V an n x n orthogonal matrix and
sigma_i = kappa^{-(i-1)/(n-1)}, so that ||A||_2 = 1 and cond_2(A) = kappa.
The paper takes U and V from the SVD of a random matrix; here U is the
Householder-orthonormalised (LAPACK) Q factor of a seeded N(0,1) m x n matrix
and V is Haar-distributed (QR of a seeded Gaussian with the signs of diag(R)
moved into Q), which gives the same distribution of singular subspaces.

Random bits come from numpy's Philox counter-based generator, keyed by
(seed, stream): stream 1 feeds U and stream 2 feeds V.  Stream 0 is reserved
for the sketch matrix Omega, which the method draws itself.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["sigma_profile", "usv_matrix", "batch_specs", "BatchSpec"]


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Philox key = seed, counter offset chosen by stream: independent streams.
    return np.random.Generator(np.random.Philox(key=[int(seed) & (2**64 - 1), int(stream)]))


def sigma_profile(n: int, kappa: float) -> np.ndarray:
    """sigma_i = kappa^{-(i-1)/(n-1)}, i = 1..n (log-spaced from 1 to 1/kappa)."""
    if n == 1:
        return np.ones(1)
    e = np.arange(n, dtype=np.float64) / (n - 1)
    return np.power(float(kappa), -e)


def _householder_q(g: np.ndarray) -> np.ndarray:
    """Orthonormal Q of the thin Householder QR of g (LAPACK geqrf/orgqr).  For
    large matrices the multithreaded LAPACK behind torch is used; numpy's
    otherwise."""
    if g.shape[0] * g.shape[1] >= 2**20:
        try:
            import torch

            q, _ = torch.linalg.qr(torch.from_numpy(np.ascontiguousarray(g)))
            return q.numpy()
        except ImportError:
            pass
    q, _ = np.linalg.qr(g)
    return q


def _haar(n: int, rng: np.random.Generator) -> np.ndarray:
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def usv_matrix(m: int, n: int, kappa: float, seed: int = 0, *, order: str = "F",
                lda: int | None = None) -> np.ndarray:
    """Return A = U diag(sigma) V^T (float64, column-major by default).

    With ``lda`` > m the result is an (lda x n) column-major buffer whose first
    m rows hold A and whose padding rows hold NaN (so that a reader that
    touches the padding is caught).  Use ``A[:m]`` for the matrix itself.
    """
    if m < n or n < 1:
        raise ValueError("need m >= n >= 1")
    g = _rng(seed, 1).standard_normal((m, n))
    u = _householder_q(g)
    v = _haar(n, _rng(seed, 2))
    sig = sigma_profile(n, kappa)
    a = (u * sig) @ v.T
    a = np.asfortranarray(a) if order == "F" else np.ascontiguousarray(a)
    if lda is not None and lda > m:
        buf = np.full((lda, n), np.nan, order="F")
        buf[:m] = a
        return buf
    return a


class BatchSpec:
    """Shape/conditioning of one matrix of the batched workload."""

    __slots__ = ("m", "n", "kappa", "seed")

    def __init__(self, m: int, n: int, kappa: float, seed: int):
        self.m, self.n, self.kappa, self.seed = int(m), int(n), float(kappa), int(seed)

    def __repr__(self) -> str:
        return f"BatchSpec(m={self.m}, n={self.n}, kappa={self.kappa:.3g}, seed={self.seed})"


def batch_specs(count: int = 512, seed: int = 0, *, log2m=(12, 18), ns=(8, 16, 32, 64, 128),
                log10k=(2, 12)) -> list[BatchSpec]:
    """Shapes for a batch of independent tall-skinny problems, as block Krylov,
    LOBPCG or randomized SVD produce them: m log-uniform in [2^a, 2^b], n drawn
    uniformly from ``ns`` and kappa log-uniform in [10^c, 10^d]; matrix i uses
    seed i."""
    rng = _rng(seed, 3)
    out = []
    for i in range(count):
        m = int(round(2.0 ** rng.uniform(*log2m)))
        n = int(ns[int(rng.integers(0, len(ns)))])
        m = max(m, n)
        kappa = 10.0 ** rng.uniform(*log10k)
        out.append(BatchSpec(m, n, kappa, i))
    return out
