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
for the sketch matrix Omega, which the method draws itself.  Stream 3 feeds
the batch shapes, stream 4 the randomized SVD's starting block and streams 5-6
the sparse operators.

Sparse operators for the randomized SVD of Section 5.1 (the paper's test
matrices come from the SuiteSparse collection, which is not available here):
``sparse_operator`` draws square matrices with the row-length statistics of
that table (a nonzero diagonal plus Poisson-distributed off-diagonal entries
at uniform random columns, N(0,1) values), and ``planted_operator`` builds a
sparse matrix with a prescribed spectrum (randomly permuted b x b blocks
U_j diag(sigma_j) V_j^T, Haar U_j and V_j), whose singular values are known.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["sigma_profile", "usv_factors", "usv_matrix", "batch_specs", "BatchSpec", "Csr", "sparse_operator",
           "planted_operator", "start_block"]


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


def usv_factors(n: int, kappa: float, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(sigma, V) of ``usv_matrix(m, n, kappa, seed)``: the singular values and
    the n x n orthogonal factor, the same for every m."""
    return sigma_profile(n, kappa), _haar(n, _rng(seed, 2))


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


class Csr:
    """A sparse m x n matrix in compressed sparse row form (indptr int64[m+1],
    indices int32[nnz] sorted within each row, data float64[nnz]), together
    with the same form of its transpose: the randomized SVD multiplies by both
    A and A^T."""

    __slots__ = ("m", "n", "indptr", "indices", "data", "t_indptr", "t_indices", "t_data")

    def __init__(self, m, n, indptr, indices, data):
        self.m, self.n = int(m), int(n)
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.data = np.ascontiguousarray(data, dtype=np.float64)
        # transpose by a stable counting sort on the column index
        order = np.argsort(self.indices, kind="stable")
        rows = np.repeat(np.arange(self.m, dtype=np.int64), np.diff(self.indptr))
        counts = np.bincount(self.indices, minlength=self.n)
        self.t_indptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.t_indices = rows[order].astype(np.int32)
        self.t_data = self.data[order]

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.data, self.indices, self.indptr), shape=(self.m, self.n))

    def dense(self) -> np.ndarray:
        a = np.zeros((self.m, self.n), order="F")
        rows = np.repeat(np.arange(self.m), np.diff(self.indptr))
        a[rows, self.indices] = self.data
        return a


def _csr_from_coo(m, n, rows, cols, vals) -> Csr:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    keep = np.ones(rows.size, dtype=bool)
    keep[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])  # first of each duplicate
    rows, cols, vals = rows[keep], cols[keep], vals[keep]
    indptr = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=m))])
    return Csr(m, n, indptr, cols, vals)


def sparse_operator(m: int, nnz_per_row: float, seed: int = 0) -> Csr:
    """Square m x m sparse matrix: a diagonal entry in every row plus
    Poisson(nnz_per_row - 1) off-diagonal entries at uniform random columns
    (duplicates merged), all values N(0,1)."""
    if m < 1 or nnz_per_row < 1:
        raise ValueError("need m >= 1 and nnz_per_row >= 1")
    rng = _rng(seed, 5)
    extra = rng.poisson(nnz_per_row - 1.0, m)
    rows = np.concatenate([np.arange(m, dtype=np.int64), np.repeat(np.arange(m, dtype=np.int64), extra)])
    cols = np.concatenate([np.arange(m, dtype=np.int64), rng.integers(0, m, int(extra.sum()))])
    vals = rng.standard_normal(rows.size)
    return _csr_from_coo(m, m, rows, cols, vals)


def planted_operator(sigma, block: int = 4, seed: int = 0) -> Csr:
    """Square sparse matrix with singular values ``sigma`` (length a multiple
    of ``block``): the values are shuffled into blocks of ``block``, block j is
    U_j diag(sigma_j) V_j^T with Haar U_j, V_j, and the rows and columns of
    the block-diagonal matrix are then permuted at random."""
    sigma = np.asarray(sigma, dtype=np.float64)
    n = sigma.size
    if n % block:
        raise ValueError("len(sigma) must be a multiple of block")
    rng = _rng(seed, 6)
    vals = sigma[rng.permutation(n)].reshape(-1, block)
    nb = n // block
    g = rng.standard_normal((2, nb, block, block))
    qu, ru = np.linalg.qr(g[0])
    qv, rv = np.linalg.qr(g[1])
    qu = qu * np.sign(np.diagonal(ru, axis1=1, axis2=2))[:, None, :]
    qv = qv * np.sign(np.diagonal(rv, axis1=1, axis2=2))[:, None, :]
    blocks = np.einsum("jab,jb,jcb->jac", qu, vals, qv)  # U_j diag(s_j) V_j^T
    pr, pc = rng.permutation(n), rng.permutation(n)
    j, a, c = np.meshgrid(np.arange(nb), np.arange(block), np.arange(block), indexing="ij")
    rows = pr[j * block + a].ravel()
    cols = pc[j * block + c].ravel()
    return _csr_from_coo(n, n, rows, cols, blocks.ravel())


def start_block(n: int, k: int, seed: int = 0) -> np.ndarray:
    """The randomized SVD's starting block X (n x k, column-major, N(0,1))."""
    return np.asfortranarray(_rng(seed, 4).standard_normal((n, k)))
