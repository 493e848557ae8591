"""Pins for the oracle's randomized SVD with power iteration (Algorithm 7,
Section 5.1) and for the sparse operators it runs on.  The checks come from
the mathematics, not from the oracle: an operator of rank k is recovered
exactly; the computed singular values never exceed the true ones (they are
those of Y^T A) and converge at the power method's rate; the rank-k error is
at least sigma_{k+1} (Eckart-Young); the final Y spans the Krylov-type block
(A A^T)^K A X; the factors satisfy A^T U = V diag(S) and U^T A V = diag(S);
and replacing Householder QR by rQR-CholeskyQR2 (the replacement Section 5.1
makes) leaves the result unchanged up to rounding."""
import numpy as np
import pytest

import oracle as o
from paper_2111_11148_gb300.inputs import planted_operator, sparse_operator, start_block


def _spd(sig, seed=1):
    P = planted_operator(sig, 4, seed)
    return P, P.scipy(), P.dense()


# ---- the operators ---------------------------------------------------------

def test_planted_operator_has_the_prescribed_spectrum():
    sig = np.geomspace(1.0, 1e-6, 120)
    P, _, D = _spd(sig, 3)
    assert np.allclose(np.linalg.svd(D, compute_uv=False), np.sort(sig)[::-1], rtol=0, atol=1e-14)
    assert P.nnz == 120 * 4  # b x b blocks, b = 4
    # rows and columns are permuted: the block structure is not diagonal in index order
    assert np.count_nonzero(np.diag(D)) < 120


def test_sparse_operator_structure():
    P = sparse_operator(5000, 3.81, seed=2)
    D = P.dense()
    assert np.all(np.diag(D) != 0)
    assert abs(P.nnz / P.m - 3.81) < 0.1  # duplicates are rare at this density
    for i in range(0, P.m, 97):
        c = P.indices[P.indptr[i]:P.indptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    T = np.zeros((P.n, P.m))
    rows = np.repeat(np.arange(P.n), np.diff(P.t_indptr))
    T[rows, P.t_indices] = P.t_data
    assert np.array_equal(T, D.T)


# ---- the method --------------------------------------------------------------

@pytest.mark.parametrize("K", [0, 2])
@pytest.mark.parametrize("orth", ["rxr", "householder"])
def test_rank_k_operator_recovered_exactly(K, orth):
    k = 12
    sig = np.concatenate([np.geomspace(1.0, 1e-3, k), np.zeros(388)])
    _, A, D = _spd(sig)
    r = o.rsvd(A, start_block(400, k, 0), K, orth=orth)
    assert r.status == 0
    assert np.max(np.abs(r.S - sig[:k])) <= 1e-14
    assert np.linalg.norm(D - (r.U * r.S) @ r.V.T) <= 1e-14 * np.linalg.norm(D)
    assert o.orth_error(r.U) <= 1e-13 and o.orth_error(r.V) <= 1e-13


def test_singular_values_interlace_and_converge():
    # S_i <= sigma_i (the singular values of Y^T A, Y orthonormal); the error of
    # the leading ones shrinks like (sigma_{k+1} / sigma_i)^{2(2K+1)}
    n, k = 400, 10
    sig = 0.8 ** np.arange(n)
    _, A, D = _spd(sig, 4)
    X = start_block(n, k, 1)
    errs = []
    for K in range(5):
        r = o.rsvd(A, X, K)
        assert r.status == 0
        assert np.all(r.S <= sig[:k] * (1 + 1e-13))
        errs.append(np.max((sig[:5] - r.S[:5]) / sig[:5]))
        # Eckart-Young: no rank-k matrix is closer to A than sigma_{k+1}
        assert np.linalg.norm(D - (r.U * r.S) @ r.V.T, 2) >= sig[k] * (1 - 1e-12)
    assert errs[0] > errs[1] > errs[2] and errs[4] <= 1e-9, errs


@pytest.mark.parametrize("K", [0, 1, 2])
def test_final_block_spans_the_power_iterates(K):
    # span(Y) = span((A A^T)^K A X): a loop that multiplied by A where A^T
    # belongs (A is square here) or skipped an orth-product pair fails this
    n, k = 600, 8
    P = sparse_operator(n, 6.0, seed=5)
    A, D = P.scipy(), P.dense()
    X = start_block(n, k, 2)
    r = o.rsvd(A, X, K)
    assert r.status == 0 and r.calls == 2 * K + 1
    Z = D @ X
    for _ in range(K):
        Z = D @ (D.T @ Z)
    Zq, _ = np.linalg.qr(Z)
    cos = np.linalg.svd(Zq.T @ r.Q, compute_uv=False)
    assert cos.min() >= 1 - 1e-10, cos.min()


def test_factors_satisfy_the_svd_identities():
    n, k = 800, 16
    P = sparse_operator(n, 10.0, seed=6)
    A, D = P.scipy(), P.dense()
    r = o.rsvd(A, start_block(n, k, 3), 2)
    assert r.status == 0
    nrm = r.S[0]
    assert np.all(np.diff(r.S) <= 0) and r.S[-1] > 0
    # U S V^T = Y Y^T A (the projection of A onto span(Y))
    assert np.linalg.norm((r.U * r.S) @ r.V.T - r.Q @ (r.Q.T @ D)) <= 1e-13 * np.linalg.norm(D)
    assert np.max(np.abs(D.T @ r.U - r.V * r.S)) <= 1e-13 * nrm
    assert np.max(np.abs(r.U.T @ D @ r.V - np.diag(r.S))) <= 1e-13 * nrm


@pytest.mark.parametrize("variant", [o.VARIANT_QR, o.VARIANT_LU])
def test_rxr_orth_matches_householder(variant):
    # Section 5.1 replaces the QR inside Algorithm 7 by randomized CholeskyQR:
    # the iteration depends only on the subspaces, so the results agree
    n, k = 3000, 20
    P = sparse_operator(n, 5.0, seed=7)
    X = start_block(n, k, 4)
    a = o.rsvd(P.scipy(), X, 2, variant=variant)
    b = o.rsvd(P.scipy(), X, 2, orth="householder")
    assert a.status == b.status == 0
    assert np.max(np.abs(a.S - b.S)) <= 1e-12 * b.S[0]
    # planted spectrum with a gap after k: the subspaces agree as well
    sig = np.concatenate([np.linspace(2.0, 1.0, k), 0.1 * np.linspace(1.0, 0.5, 380)])
    _, A, _ = _spd(sig, 8)
    X = start_block(400, k, 5)
    a = o.rsvd(A, X, 1, variant=variant)
    b = o.rsvd(A, X, 1, orth="householder")
    for Ua, Ub in ((a.U, b.U), (a.V, b.V)):
        cos = np.linalg.svd(Ua.T @ Ub, compute_uv=False)
        assert cos.min() >= 1 - 1e-12


def test_dense_and_sparse_operator_agree():
    P = sparse_operator(1000, 4.0, seed=9)
    X = start_block(1000, 10, 6)
    a = o.rsvd(P.scipy(), X, 1)
    b = o.rsvd(P.dense(), X, 1)
    assert a.status == b.status == 0
    assert np.max(np.abs(a.S - b.S)) <= 1e-13 * b.S[0]


def test_seeds_advance_per_orthonormalisation():
    # call j uses seed + j: the same Y from rsvd(seed) and a hand-run first step
    n, k = 500, 6
    P = sparse_operator(n, 4.0, seed=10)
    A = P.scipy()
    X = start_block(n, k, 7)
    r = o.rsvd(A, X, 1, seed=40)
    q0 = o.rxr_cholqr(np.asfortranarray(A @ X), o.VARIANT_QR, 2 * k, 40).Q
    q1 = o.rxr_cholqr(np.asfortranarray(A.T @ q0), o.VARIANT_QR, 2 * k, 41).Q
    q2 = o.rxr_cholqr(np.asfortranarray(A @ q1), o.VARIANT_QR, 2 * k, 42).Q
    assert np.array_equal(r.Q, q2)
