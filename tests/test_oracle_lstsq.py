"""Pins for the oracle's least-squares solver preconditioned by the sketch's R
factor (Section 5.2): consistent systems recover the exact solution within
the conditioning bound, inconsistent ones agree with LAPACK's least-squares
solution, columns of a multi-right-hand-side call are independent solves, and
power-of-two scaling of b passes through exactly."""
import numpy as np
import pytest

import oracle as o
from paper_2111_11148_gb300.inputs import usv_matrix

U = 2.0**-53


@pytest.mark.parametrize("variant", [o.VARIANT_QR, o.VARIANT_LU, o.VARIANT_QR | o.SKETCH_ROWS])
@pytest.mark.parametrize("kappa", [1e2, 1e8, 1e12])
def test_consistent_system_recovered(variant, kappa):
    m, n = 3000, 20
    A = usv_matrix(m, n, kappa, seed=2)
    xt = np.random.default_rng(3).standard_normal(n)
    x, st = o.lstsq(A, A @ xt, variant=variant, seed=1)
    assert st == 0
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 10 * n * kappa * U


@pytest.mark.parametrize("kappa", [1e3, 1e6])
def test_inconsistent_system_matches_lapack(kappa):
    m, n = 2000, 12
    A = usv_matrix(m, n, kappa, seed=4)
    rng = np.random.default_rng(5)
    b = A @ rng.standard_normal(n) + 1e-6 * rng.standard_normal(m)
    x, st = o.lstsq(A, b, seed=2)
    assert st == 0
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    # forward-error bound of the LS problem: kappa u + kappa^2 u ||r|| / (||A|| ||x||)
    r = np.linalg.norm(b - A @ xr)
    bound = 100 * n * (kappa * U + kappa**2 * U * r / (np.linalg.norm(A, 2) * np.linalg.norm(xr)))
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= bound


def test_multiple_right_hand_sides_are_independent_solves():
    A = usv_matrix(1500, 10, 1e5, seed=6)
    B = np.asfortranarray(np.random.default_rng(7).standard_normal((1500, 3)))
    X, st = o.lstsq(A, B, seed=3)
    assert st == 0
    for j in range(3):
        xj, _ = o.lstsq(A, np.ascontiguousarray(B[:, j]), seed=3)
        assert np.array_equal(X[:, j], xj)


def test_power_of_two_scaling_of_b_is_exact():
    A = usv_matrix(1000, 8, 1e4, seed=8)
    b = np.random.default_rng(9).standard_normal(1000)
    x1, _ = o.lstsq(A, b, seed=4)
    x2, _ = o.lstsq(A, 8.0 * b, seed=4)
    assert np.array_equal(8.0 * x1, x2)


def test_nonfinite_b_reported():
    A = usv_matrix(500, 5, 10.0, seed=1)
    b = np.ones(500)
    b[7] = np.nan
    assert o.lstsq(A, b)[1] == o.NONFINITE
