"""Parity of the randomized SVD with power iteration (Algorithm 7, Section
5.1; every orthonormalisation by rQR-/rLU-CholeskyQR2) with the CPU oracle on
seeded sparse operators: the singular values agree with the oracle's within
rounding of sigma_1 and, where the spectrum has a gap after k, so do the
singular subspaces; an operator of rank k is recovered exactly; the factors
satisfy A^T U = V diag(S) with orthonormal U and V.  Odd k (a Jacobi round
with a sitting-out column), k above 112 (V_r outside shared memory), the
widest k = 128, rectangular operators, out-of-range CSR entries and a rank
below k are covered."""
import numpy as np
import pytest

import oracle as o
from gpu_util import to_dev, to_host
from paper_2111_11148_gb300.inputs import Csr, planted_operator, sparse_operator, start_block

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402

OV = {"qr": o.VARIANT_QR, "lu": o.VARIANT_LU}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


def _gpu(h, P, k, iters, xseed=0, **kw):
    A = rxr.DeviceCsr.from_host(P)
    U, S, V, code = h.rsvd(A, to_dev(start_block(P.n, k, xseed)), iters, raise_on_error=False, **kw)
    return to_host(U), S.cpu().numpy(), to_host(V), code


def _identities(P, U, S, V, tol):
    # A^T U = V diag(S) and U^T U = V^T V = I (the construction's identities)
    AtU = P.scipy().T @ U
    assert np.max(np.abs(AtU - V * S)) <= tol * S[0]
    assert o.orth_error(U) <= 1e-12 and o.orth_error(V) <= 1e-12
    assert np.all(np.diff(S) <= 0) and S[-1] >= 0


def _rows_of(P, m):
    # the first m rows of P as an m x n operator (rectangular, m < n)
    nnz = int(P.indptr[m])
    return Csr(m, P.n, P.indptr[:m + 1], P.indices[:nnz], P.data[:nnz])


def _transpose(P):
    return Csr(P.n, P.m, P.t_indptr, P.t_indices, P.t_data)


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("iters", [0, 2])
def test_rank_k_operator_recovered_exactly(h, prec, iters):
    k = 12
    sig = np.concatenate([np.geomspace(1.0, 1e-3, k), np.zeros(1024 - k)])
    P = planted_operator(sig, 4, seed=1)
    U, S, V, code = _gpu(h, P, k, iters, prec=prec)
    assert code == 0
    assert np.max(np.abs(S - sig[:k])) <= 1e-13
    D = P.dense()
    assert np.linalg.norm(D - (U * S) @ V.T) <= 1e-13 * np.linalg.norm(D)


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("m,d,k,iters", [(3000, 3.81, 20, 2), (2000, 44.36, 8, 1), (5000, 4.83, 50, 0),
                                         (4000, 69.85, 7, 1)])
def test_matches_oracle_on_sparse_operators(h, prec, variant, m, d, k, iters):
    P = sparse_operator(m, d, seed=m)
    U, S, V, code = _gpu(h, P, k, iters, xseed=1, variant=variant, seed=9, prec=prec)
    assert code == 0
    ref = o.rsvd(P.scipy(), start_block(m, k, 1), iters, variant=OV[variant], seed=9)
    assert ref.status == 0
    assert np.max(np.abs(S - ref.S)) <= 1e-12 * ref.S[0], np.max(np.abs(S - ref.S)) / ref.S[0]
    _identities(P, U, S, V, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_subspaces_match_oracle_across_a_gap(h, prec):
    k = 16
    sig = np.concatenate([np.linspace(3.0, 1.0, k), 0.05 * np.linspace(1.0, 0.1, 4096 - k)])
    P = planted_operator(sig, 4, seed=2)
    U, S, V, code = _gpu(h, P, k, 1, xseed=2, prec=prec)
    assert code == 0
    ref = o.rsvd(P.scipy(), start_block(P.n, k, 2), 1)
    assert np.max(np.abs(S - ref.S)) <= 1e-12 * ref.S[0]
    for G, R in ((U, ref.U), (V, ref.V)):
        cos = np.linalg.svd(G.T @ R, compute_uv=False)
        assert cos.min() >= 1 - 1e-10
    # the leading singular values are the planted ones to the power method's accuracy
    assert np.max(np.abs(S[:8] - sig[:8]) / sig[:8]) <= 1e-6


@pytest.mark.parametrize("k", [1, 7, 80, 113, 128])
def test_block_widths(h, k):
    P = sparse_operator(1500, 6.0, seed=k)
    U, S, V, code = _gpu(h, P, k, 1, xseed=3)
    assert code == 0
    ref = o.rsvd(P.scipy(), start_block(P.n, k, 3), 1)
    assert np.max(np.abs(S - ref.S)) <= 1e-12 * ref.S[0]
    _identities(P, U, S, V, 1e-12)


@pytest.mark.parametrize("shape", ["wide", "tall"])
def test_rectangular_operators(h, shape):
    P = _rows_of(sparse_operator(3000, 5.0, seed=4), 1800)
    if shape == "tall":
        P = _transpose(P)
    k = 24
    U, S, V, code = _gpu(h, P, k, 2, xseed=4)
    assert code == 0 and U.shape == (P.m, k) and V.shape == (P.n, k)
    ref = o.rsvd(P.scipy(), start_block(P.n, k, 4), 2)
    assert np.max(np.abs(S - ref.S)) <= 1e-12 * ref.S[0]
    _identities(P, U, S, V, 1e-12)


def test_medium_operator_matches_oracle(h):
    # 2^18 rows of the sparsest stand-in (3.81 nonzeros per row), k = 20
    P = sparse_operator(1 << 18, 3.81, seed=0)
    U, S, V, code = _gpu(h, P, 20, 1, prec="split")
    assert code == 0
    ref = o.rsvd(P.scipy(), start_block(P.n, 20, 0), 1)
    assert np.max(np.abs(S - ref.S)) <= 1e-12 * ref.S[0]
    _identities(P, U, S, V, 1e-12)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_rank_below_k_fails(h, prec):
    # a scaled permutation of rank 4 and k = 16: the first sketch is rank
    # deficient and its XR factorisation reports it, as the oracle does
    sig = np.concatenate([np.ones(4), np.zeros(508)])
    P = planted_operator(sig, 1, seed=3)
    _, _, _, code = _gpu(h, P, 16, 0, xseed=3, prec=prec)
    assert code in (rxr.SKETCH_SINGULAR, rxr.CHOL_BREAKDOWN)
    assert o.rsvd(P.scipy(), start_block(512, 16, 3), 0).status != 0


@pytest.mark.parametrize("what", ["column", "negative", "rowptr"])
def test_out_of_range_csr_entries_are_reported(h, what):
    P = sparse_operator(800, 4.0, seed=5)
    A = rxr.DeviceCsr.from_host(P)
    if what == "column":
        A.indices[17] = P.n
    elif what == "negative":
        A.indices[0] = -1
    else:
        A.indptr[3] = P.nnz + 5
    X = to_dev(start_block(P.n, 8, 0))
    _, _, _, code = h.rsvd(A, X, 1, raise_on_error=False)
    assert code == rxr.BAD_SPARSE
    # the handle stays usable
    A = rxr.DeviceCsr.from_host(P)
    _, _, _, code = h.rsvd(A, X, 1, raise_on_error=False)
    assert code == 0


def test_argument_errors(h):
    P = sparse_operator(300, 4.0, seed=6)
    A = rxr.DeviceCsr.from_host(P)
    X = to_dev(start_block(300, 8, 0))
    U = rxr.empty_colmajor(300, 8)
    V = rxr.empty_colmajor(300, 8)
    S = torch.empty(8, dtype=torch.float64, device="cuda")
    lib = rxr.load()
    p = lambda t: t.data_ptr()
    st = torch.cuda.current_stream().cuda_stream

    def call(m=300, n=300, nnz=P.nnz, ldx=300, k=8, iters=1, variant=rxr.QR, s=16, passes=2, prec=rxr.FP64,
             ldu=300, ldv=300, x=None):
        return lib.rxr_rsvd(h._h, m, n, p(A.indptr), p(A.indices), p(A.data), p(A.t_indptr), p(A.t_indices),
                            p(A.t_data), nnz, p(X) if x is None else x, ldx, k, iters, variant, s, 0, passes, prec,
                            p(U), ldu, p(S), p(V), ldv, st)

    assert call(m=0) == -2
    assert call(n=0) == -3
    assert call(nnz=-1) == -10
    assert call(x=0) == -11
    assert call(ldx=299) == -12
    assert call(k=0) == -13
    assert call(k=301) == -13
    assert call(iters=-1) == -14
    assert call(variant=9) == -15
    assert call(s=7) == -16
    assert call(passes=0) == -18
    assert call(prec=5) == -19
    assert call(ldu=299) == -21
    assert call(ldv=299) == -24
    assert call(k=129, s=258) == rxr.UNSUPPORTED
    assert call() == 0
