"""Pins for the oracle's dense building blocks against closed forms, exact
rational arithmetic and LAPACK (a library routine reached independently of
the oracle's code).  Each test is chosen so that a plausible slip in the
oracle -- a dropped term, a wrong sign or index, a transposed operand --
fails it."""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

import oracle as o

U = 2.0**-53


def _rand(m, n, seed):
    return np.asfortranarray(np.random.default_rng(seed).standard_normal((m, n)))


def _signfix_r(R):
    d = np.sign(np.diag(R))
    d[d == 0] = 1
    return d[:, None] * R


# ---------------------------------------------------------------- Householder
def test_geqr_r_n1_is_the_norm():
    x = _rand(9, 1, 0)
    R = o.sign_normalise(o.geqr_r(x))
    assert R.shape == (1, 1)
    assert abs(R[0, 0] - np.linalg.norm(x)) <= 4 * U * np.linalg.norm(x)


def test_geqr_r_n2_closed_form():
    a, b = _rand(7, 1, 1)[:, 0], _rand(7, 1, 2)[:, 0]
    R = o.sign_normalise(o.geqr_r(np.column_stack([a, b])))
    r11 = np.linalg.norm(a)
    r12 = a @ b / r11
    r22 = np.linalg.norm(b - (a @ b) / (a @ a) * a)
    np.testing.assert_allclose([R[0, 0], R[0, 1], R[1, 1]], [r11, r12, r22], rtol=1e-14)
    assert R[1, 0] == 0.0


def test_geqr_r_matches_lapack():
    W = _rand(40, 12, 3)
    R = o.sign_normalise(o.geqr_r(W))
    Rl = _signfix_r(np.linalg.qr(W, mode="r"))
    np.testing.assert_allclose(R, Rl, rtol=0, atol=1e-13 * np.abs(Rl).max())
    assert np.all(np.tril(R, -1) == 0)


def test_geqr_r_orthogonal_times_diagonal():
    Q0, _ = np.linalg.qr(_rand(30, 5, 4))
    D = np.diag([3.0, 0.5, 2.0, 1e-3, 7.0])
    R = o.sign_normalise(o.geqr_r(Q0 @ D))
    np.testing.assert_allclose(R, D, atol=1e-14 * 7)


def test_geqr_r_triangle_on_top_of_zeros():
    T = np.triu(_rand(6, 6, 5)) + 4 * np.eye(6)
    T = _signfix_r(T)
    R = o.sign_normalise(o.geqr_r(np.vstack([T, np.zeros((5, 6))])))
    np.testing.assert_allclose(R, T, rtol=0, atol=1e-14 * np.abs(T).max())


# ---------------------------------------------------------------- LU
def test_getrf_matches_scipy_partial_pivoting():
    W = _rand(50, 10, 6)
    U_, L, piv = o.getrf_u(W)
    P, Ls, Us = sla.lu(W)
    np.testing.assert_allclose(U_, Us[:10], rtol=0, atol=1e-13 * np.abs(Us).max())
    assert np.all(np.abs(L) <= 1.0)


def test_getrf_reconstructs_permuted_input():
    W = _rand(20, 6, 7)
    U_, L, piv = o.getrf_u(W)
    Wp = W.copy()
    for k, p in enumerate(piv):
        Wp[[k, p]] = Wp[[p, k]]
    np.testing.assert_allclose(L @ U_, Wp, atol=1e-14 * 20)


def test_getrf_tie_breaks_to_lowest_row():
    W = np.asfortranarray([[1.0, 2.0], [-3.0, 1.0], [3.0, 5.0], [2.0, 0.0]])
    _, _, piv = o.getrf_u(W)
    assert piv[0] == 1           # |-3| == |3|: the lower index wins


# ---------------------------------------------------------------- Cholesky
def test_potrf_matches_lapack_and_reconstructs():
    X = _rand(60, 9, 8)
    G = X.T @ X
    R, info = o.potrf_u(G)
    assert info == 0
    np.testing.assert_allclose(R, np.linalg.cholesky(G).T, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(R.T @ R, G, rtol=1e-13, atol=1e-12)
    assert np.all(np.tril(R, -1) == 0) and np.all(np.diag(R) > 0)


def test_potrf_reads_upper_triangle_only():
    X = _rand(30, 5, 9)
    G = X.T @ X
    Gu = np.triu(G) + np.tril(np.full((5, 5), 1e300), -1)
    R1, _ = o.potrf_u(G)
    R2, _ = o.potrf_u(np.asfortranarray(Gu))
    assert np.array_equal(R1, R2)


def test_potrf_reports_breakdown_column():
    G = np.diag([4.0, 1.0, -1.0, 2.0])
    R, info = o.potrf_u(G)
    assert info == 3             # third column (1-based)
    G = np.diag([4.0, np.nan, 1.0])
    assert o.potrf_u(G)[1] == 2


# ---------------------------------------------------------------- substitution, Gram, products
def test_trsm_matches_lapack_solve():
    A = _rand(100, 8, 10)
    R = np.triu(_rand(8, 8, 11)) + 3 * np.eye(8)
    X = o.trsm_right_upper(A, R)
    Xs = sla.solve_triangular(R.T, A.T, lower=True).T     # X R = A  <=>  R^T X^T = A^T
    np.testing.assert_allclose(X, Xs, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(X @ R, A, rtol=1e-13, atol=1e-13)


def test_trsm_is_backward_stable_for_ill_conditioned_r():
    # rows x of X satisfy x (R + dR) = a with |dR| <= n u |R|: residual small
    # relative to |x||R| even when cond(R) = 1e14 (the R_s of a bad A)
    n = 10
    Rs = np.triu(_rand(n, n, 12)) @ np.diag(np.logspace(0, -14, n))
    Rs += np.diag(np.logspace(0, -14, n))
    A = _rand(200, n, 13)
    X = o.trsm_right_upper(A, Rs)
    res = np.abs(X @ Rs - A)
    bound = 4 * n * U * (np.abs(X) @ np.abs(Rs))
    assert np.all(res <= bound + 1e-300)


def test_gram_matches_definition():
    X = _rand(1000, 7, 14)
    np.testing.assert_allclose(o.gram(X), X.T @ X, rtol=1e-13, atol=1e-12)
    G = o.gram(X)
    assert np.array_equal(G, G.T)


def test_trmm_upper():
    A = np.triu(_rand(6, 6, 15))
    B = np.triu(_rand(6, 6, 16))
    np.testing.assert_allclose(o.trmm_upper(A, B), A @ B, rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- Householder thin QR (definition)
def test_householder_qr_matches_lapack_and_is_orthonormal():
    A = _rand(300, 12, 17)
    Q, R = o.householder_qr(A)
    Ql, Rl = np.linalg.qr(A)
    d = np.sign(np.diag(Rl))
    np.testing.assert_allclose(R, d[:, None] * Rl, atol=1e-13 * np.abs(Rl).max())
    np.testing.assert_allclose(Q, Ql * d, atol=1e-13)
    assert np.linalg.norm(Q.T @ Q - np.eye(12)) < 1e-14
    assert np.all(np.diag(R) > 0)


def test_householder_qr_n2_closed_form():
    A = _rand(11, 2, 18)
    a, b = A[:, 0], A[:, 1]
    _, R = o.householder_qr(A)
    r11 = np.linalg.norm(a)
    np.testing.assert_allclose(R[0], [r11, a @ b / r11], rtol=1e-14)
    np.testing.assert_allclose(R[1, 1], np.linalg.norm(b - (a @ b) / (a @ a) * a), rtol=1e-13)


# ---------------------------------------------------------------- Dot2 and the accuracy measures
def _exact_dot(x, y):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))


def test_dot2_is_twice_working_precision():
    # ill-conditioned dot products (cond ~ 1e20): naive FP64 loses every digit,
    # Dot2 stays within a few ulp of the exact rational result
    rng = np.random.default_rng(19)
    for t in range(20):
        x = rng.standard_normal(50) * 10.0 ** rng.integers(-8, 9, 50)
        y = rng.standard_normal(50)
        x = np.concatenate([x, -x, [1.0]])
        y = np.concatenate([y, y * (1 + 2.0**-40), [1e-3]])
        ex = _exact_dot(x, y)
        got = o.dot2(x, y)
        assert abs(Fraction(got) - ex) <= 4 * U * abs(ex) + Fraction(1, 10**300)


def test_orth_and_resid_measures_against_exact_rationals():
    rng = np.random.default_rng(20)
    Q = np.asfortranarray(np.linalg.qr(rng.standard_normal((7, 3)))[0] + 1e-9 * rng.standard_normal((7, 3)))
    F = [[sum(Fraction(Q[i, j]) * Fraction(Q[i, l]) for i in range(7)) - (1 if j == l else 0)
          for l in range(3)] for j in range(3)]
    exact = math.sqrt(float(sum(v * v for row in F for v in row)))
    assert abs(o.orth_error(Q) - exact) <= 1e-12 * exact
    A = np.asfortranarray(rng.standard_normal((7, 3)))
    R = np.triu(rng.standard_normal((3, 3)))
    num = sum((Fraction(A[i, j]) - sum(Fraction(Q[i, k]) * Fraction(R[k, j]) for k in range(j + 1))) ** 2
              for i in range(7) for j in range(3))
    den = sum(Fraction(A[i, j]) ** 2 for i in range(7) for j in range(3))
    exact_r = math.sqrt(float(num)) / math.sqrt(float(den))
    assert abs(o.resid_error(A, Q, R) - exact_r) <= 1e-12 * exact_r


def test_orth_measure_resolves_tiny_errors():
    # an exactly orthonormal Q (a signed permutation) has measure 0, and a
    # perturbation of 1e-15 in one entry is seen at that size
    Q = np.zeros((50, 4), order="F")
    for j in range(4):
        Q[3 * j + 1, j] = -1.0 if j % 2 else 1.0
    assert o.orth_error(Q) == 0.0
    Q2 = Q.copy(order="F")
    Q2[40, 2] = 1e-15
    # (Q^T Q)_22 = 1 + 1e-30 exactly; every other entry is exact
    assert abs(o.orth_error(Q2) - 1e-30) <= 1e-44
