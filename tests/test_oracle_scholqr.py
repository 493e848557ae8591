"""Pins for the oracle's shifted CholeskyQR3 (the comparator of Section 2.1:
R_1 = chol(A^T A + eps I), then two CholeskyQR steps): the shift enters the
first Gram's diagonal only, the first Q's condition number obeys the bound
quoted from Fukaya et al. in Section 2.1, the three steps reach rounding level
up to kappa = 1e15 with the paper's experimental shift, a zero shift reduces
to CholeskyQR3, and the result is the unique thin QR factorisation."""
import math

import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, r_rel
from paper_2111_11148_gb300.inputs import usv_matrix

U = 2.0**-53


def test_shift_enters_first_gram_diagonal():
    # R_1^T R_1 = A^T A + eps I (a shift large enough to dominate rounding)
    A = usv_matrix(2000, 12, 1e3, seed=1)
    nrm2 = np.linalg.norm(A, 2) ** 2
    eps = 1e-3 * nrm2
    r = o.scholqr(A, eps, passes=1)
    assert r.status == 0
    D = r.R.T @ r.R - A.T @ A
    assert np.allclose(np.diag(D), eps, rtol=1e-9)
    assert np.max(np.abs(D - np.diag(np.diag(D)))) <= 1e-12 * nrm2


@pytest.mark.parametrize("kappa", [1e8, 1e12, 1e15])
def test_first_step_condition_bound(kappa):
    # cond(Q_1) <= 2 sqrt(3) sqrt(1 + (eps / ||A||^2) kappa^2) (Section 2.1)
    A = usv_matrix(3000, 16, kappa, seed=2)
    alpha = 1e-15
    r = o.scholqr(A, alpha * np.linalg.norm(A, 2) ** 2, passes=1)
    assert r.status == 0
    assert np.linalg.cond(r.Q) <= 2 * math.sqrt(3) * math.sqrt(1 + alpha * kappa**2)


@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12, 1e15])
def test_three_steps_reach_rounding_level(kappa):
    m, n = 4000, 16
    A = usv_matrix(m, n, kappa, seed=3)
    r = o.scholqr(A, 1e-15 * np.linalg.norm(A, 2) ** 2, passes=3)
    assert r.status == 0
    assert o.orth_error(r.Q) <= 1e-13
    assert o.resid_error(A, r.Q, r.R) <= 1e-14
    _, Rh = o.householder_qr(A)
    assert r_rel(r.R, Rh) <= R_TOL


def test_zero_shift_is_choleskyqr3():
    A = usv_matrix(1500, 10, 1e4, seed=4)
    r = o.scholqr(A, 0.0, passes=3)
    c = o.rxr_cholqr(A, o.VARIANT_NONE, s=10, seed=0, passes=3)
    assert r.status == c.status == 0
    assert np.array_equal(r.Q, c.Q) and np.array_equal(r.R, c.R)


def test_unshifted_choleskyqr2_breaks_down_where_the_shift_does_not():
    # Section 2.1: CholeskyQR2's first Cholesky breaks down near cond(A) ~ u^-1/2
    A = usv_matrix(3000, 16, 1e12, seed=5)
    assert o.rxr_cholqr(A, o.VARIANT_NONE, s=16, seed=0, passes=2).status == o.CHOL_BREAKDOWN
    assert o.scholqr(A, 1e-15 * np.linalg.norm(A, 2) ** 2, passes=3).status == 0
