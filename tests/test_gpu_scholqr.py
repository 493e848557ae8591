"""Parity of the shifted CholeskyQR3 comparator (Section 2.1; RXR_SHIFTED) with
the CPU oracle: the device estimates ||A||_2^2 by power iteration for the shift
eps = 1e-15 ||A||_2^2 (the paper's experimental choice), the oracle takes the
exact norm; both reach the same unique thin QR factorisation within the
forward-error bound, and the shift keeps the first Cholesky alive where
unshifted CholeskyQR breaks down."""
import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, U, r_rel, to_dev, to_host
from paper_2111_11148_gb300.inputs import usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("m,n,kappa", [(5000, 16, 1e8), (5000, 16, 1e12), (3000, 64, 1e15), (2100, 100, 1e10),
                                       (1, 1, 1.0), (700, 9, 1e3)])
def test_scholqr3_matches_oracle(h, prec, m, n, kappa):
    A = usv_matrix(m, n, kappa, seed=n + 1)
    Q, R, code = h.cholqr(to_dev(A), variant="shifted", passes=3, prec=prec)
    assert code == 0
    ref = o.scholqr(A, 1e-15 * np.linalg.norm(A, 2) ** 2, passes=3)
    assert ref.status == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    rel = np.linalg.norm(Rg - ref.R) / np.linalg.norm(ref.R)
    assert rel <= R_TOL, rel


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_shift_keeps_first_cholesky_alive(h, prec):
    A = usv_matrix(3000, 16, 1e12, seed=5)
    _, _, code = h.cholqr(to_dev(A), variant="none", passes=2, prec=prec, raise_on_error=False)
    assert code == rxr.CHOL_BREAKDOWN
    _, _, code = h.cholqr(to_dev(A), variant="shifted", passes=3, prec=prec)
    assert code == 0


def test_batched_shifted_runs_each_problem_as_the_single_call(h):
    As = [to_dev(usv_matrix(m, n, 1e10, seed=m)) for m, n in [(500, 8), (4000, 33)]]
    Qs, Rs, st = h.cholqr_batched(As, variant="shifted", passes=3)
    assert np.all(st == 0)
    for A, Qb, Rb in zip(As, Qs, Rs):
        Q, R, _ = h.cholqr(A, variant="shifted", passes=3)
        assert torch.equal(Q, Qb) and torch.equal(R, Rb)


@pytest.mark.parametrize("m,n,kappa,passes", [(5000, 16, 1e6, 2), ((1 << 17) + 5, 48, 1e7, 2), (2100, 100, 1e5, 2),
                                              (900, 64, 1e3, 3)])
def test_choleskyqr_split_matches_oracle(h, m, n, kappa, passes):
    # unpreconditioned CholeskyQR2/3 on the split path: X_0 = A, first Gram on
    # the tensor cores at FP64 grade
    A = usv_matrix(m, n, kappa, seed=n + 2)
    Q, R, code = h.cholqr(to_dev(A), variant="none", passes=passes, prec="split")
    assert code == 0
    ref = o.rxr_cholqr(A, o.VARIANT_NONE, n, seed=0, passes=passes)
    assert ref.status == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    rel = np.linalg.norm(Rg - ref.R) / np.linalg.norm(ref.R)
    assert rel <= R_TOL, rel


@pytest.mark.parametrize("variant,n", [("none", 16), ("none", 100), ("shifted", 32)])
def test_nan_reported_without_a_sketch(h, variant, n):
    A = usv_matrix(3000, n, 1e3, seed=3)
    A[1234, n - 1] = np.inf
    for prec in ("fp64", "split"):
        _, _, code = h.cholqr(to_dev(A), variant=variant, passes=3 if variant == "shifted" else 2, prec=prec,
                              raise_on_error=False)
        assert code == rxr.NONFINITE, (prec, code)
