"""Parity of the row-extraction sketch (Section 2.3; Theorem 3.2's
equal-probability case) with the CPU oracle: the sketch itself is a gather of
the drawn rows and must match bit for bit (the draws are integer work); the
factorisations it preconditions must meet the accuracy targets and agree with
the oracle's R within the forward-error bound; the coherent [I; 0] case must
report a singular sketch, and NaN in a row the sketch never draws must still
be reported."""
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

OVR = {"lu-rows": o.VARIANT_LU | o.SKETCH_ROWS, "qr-rows": o.VARIANT_QR | o.SKETCH_ROWS}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


@pytest.mark.parametrize("m,n,s,seed,ld_pad", [(1, 1, 1, 0, 0), (1, 3, 5, 1, 3), (1000, 7, 2000, 2, 0),
                                                (4097, 64, 128, 3, 1), ((1 << 22) + 1, 16, 32, 7, 0),
                                                (300, 130, 260, 9, 2)])
def test_sketch_rows_bit_exact(h, m, n, s, seed, ld_pad):
    A = usv_matrix(m, n, 10.0, seed=n) if m >= n else np.asfortranarray(
        np.random.default_rng(m).standard_normal((m, n)))
    Ad = to_dev(A, ld=m + ld_pad) if ld_pad else to_dev(A)
    Y = to_host(h.sketch_rows(Ad, s, seed=seed))
    idx = o.row_indices(seed, s, m)
    assert idx.min() >= 0 and idx.max() < m
    assert np.array_equal(Y, A[idx])
    if m * n <= 1 << 20:
        assert np.array_equal(Y, o.sketch_rows(A, s, seed))


def _check(A, Qg, Rg, ref, kappa):
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    rel = np.linalg.norm(Rg - ref.R) / np.linalg.norm(ref.R)
    assert rel <= R_TOL, rel


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("variant", ["qr-rows", "lu-rows"])
@pytest.mark.parametrize("m,n,kappa", [(5000, 16, 1e4), (5000, 16, 1e12), (3000, 64, 1e15), (2100, 100, 1e8),
                                       (1 << 17, 48, 1e10)])
def test_cholqr_rows_matches_oracle(h, prec, variant, m, n, kappa):
    A = usv_matrix(m, n, kappa, seed=n)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=2 * n, seed=5, passes=2, prec=prec)
    assert code == 0
    ref = o.rxr_cholqr(A, OVR[variant], 2 * n, seed=5, passes=2)
    assert ref.status == 0
    _check(A, to_host(Q), to_host(R), ref, kappa)


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_coherent_matrix_gives_singular_sketch(h, prec):
    m, n, s = 1000, 8, 16
    A = np.zeros((m, n), order="F")
    A[:n, :n] = np.eye(n)
    _, _, code = h.cholqr(to_dev(A), variant="qr-rows", s=s, seed=0, prec=prec, raise_on_error=False)
    assert code == rxr.SKETCH_SINGULAR
    assert o.rxr_cholqr(A, OVR["qr-rows"], s, seed=0).status == o.SKETCH_SINGULAR


@pytest.mark.parametrize("prec,n", [("fp64", 16), ("split", 16), ("split", 100)])
def test_nan_outside_the_drawn_rows_is_reported(h, prec, n):
    m, s, seed = 4000, 2 * n, 3
    A = usv_matrix(m, n, 1e3, seed=1)
    drawn = set(o.row_indices(seed, s, m).tolist())
    row = next(i for i in range(m) if i not in drawn)
    A[row, n // 2] = np.nan
    _, _, code = h.cholqr(to_dev(A), variant="qr-rows", s=s, seed=seed, prec=prec, raise_on_error=False)
    assert code == rxr.NONFINITE
    assert o.rxr_cholqr(A, OVR["qr-rows"], s, seed=seed).status == o.NONFINITE


def test_host_entry_point_rows(h):
    A = usv_matrix(20000, 32, 1e9, seed=2)
    Qh, Rh = h.cholqr_host(A, variant="qr-rows", seed=4, prec="split")
    Q, R, _ = h.cholqr(to_dev(A), variant="qr-rows", seed=4, prec="split")
    assert np.array_equal(Qh, to_host(Q)) and np.array_equal(Rh, to_host(R))


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_batched_rows_runs_each_problem_as_the_single_call(h, prec):
    # the row-extraction sketch in a batch: every problem's own launch sequence
    # (the single call's kernels and partition), so the same bits
    As = [to_dev(usv_matrix(m, n, 1e6, seed=m)) for m, n in [(500, 8), (3000, 40), (20000, 100)]]
    Qs, Rs, st = h.cholqr_batched(As, variant="qr-rows", seeds=[4, 5, 6], prec=prec)
    assert np.all(st == 0)
    for A, Qb, Rb, seed in zip(As, Qs, Rs, [4, 5, 6]):
        Q, R, _ = h.cholqr(A, variant="qr-rows", seed=seed, prec=prec)
        assert torch.equal(Q, Qb) and torch.equal(R, Rb)
