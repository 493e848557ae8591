"""Pins for the oracle's row-extraction sketch (Section 2.3; Theorem 3.2's
equal-probability case): draws are uniform on the m rows, independent and with
replacement; the sketch is a gather of those rows; Theorem 3.2's identity
cond(X) = cond(Q_1) holds for the preconditioned X; the extreme case the paper
discusses before Theorem 3.2 (A = [I; 0]) leaves the sketch rank-deficient;
and on incoherent A the full factorisation meets the accuracy targets."""
import math

import numpy as np
import pytest

import oracle as o
from paper_2111_11148_gb300.inputs import usv_matrix

ROWS_QR = o.VARIANT_QR | o.SKETCH_ROWS
ROWS_LU = o.VARIANT_LU | o.SKETCH_ROWS


def test_draws_uniform_small_m():
    # every row equally likely: counts within 5 sigma of l / m
    m, l = 7, 70000
    idx = o.row_indices(11, l, m)
    assert idx.min() >= 0 and idx.max() < m
    counts = np.bincount(idx, minlength=m)
    sigma = math.sqrt(l * (1 / m) * (1 - 1 / m))
    assert np.all(np.abs(counts - l / m) < 5 * sigma), counts


def test_draws_range_and_mean_large_m():
    # m beyond 2^32: the 64-bit draw scaled by m stays in range, mean m / 2
    m, l = (1 << 40) + 3, 20000
    idx = o.row_indices(5, l, m)
    assert idx.min() >= 0 and idx.max() < m
    mean = idx.astype(np.float64).mean() / m
    assert abs(mean - 0.5) < 5 * math.sqrt(1 / 12 / l)
    # both halves of the range and the low bits are used
    assert 0.45 < np.mean(idx < m // 2) < 0.55
    assert 0.45 < np.mean(idx & 1) < 0.55


def test_draws_independent():
    # successive draws uncorrelated (|corr| < 5 / sqrt(l))
    m, l = 1 << 20, 50000
    x = o.row_indices(2, l, m).astype(np.float64)
    c = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(l)


def test_draws_deterministic_and_seeded():
    a = o.row_indices(3, 100, 12345)
    assert np.array_equal(a, o.row_indices(3, 100, 12345))
    assert not np.array_equal(a, o.row_indices(4, 100, 12345))
    # draw k does not depend on l (a prefix of a longer run)
    assert np.array_equal(a[:40], o.row_indices(3, 40, 12345))


def test_with_replacement_inclusion_probability():
    # m = 10, l = 6 draws with replacement: P(rows 0 and 1 both drawn)
    # = 1 - 2 (9/10)^6 + (8/10)^6 by inclusion-exclusion
    p = 1 - 2 * 0.9**6 + 0.8**6
    trials = 5000
    hit = 0
    for seed in range(trials):
        s = set(o.row_indices(seed, 6, 10).tolist())
        hit += (0 in s and 1 in s)
    f = hit / trials
    assert abs(f - p) < 5 * math.sqrt(p * (1 - p) / trials), (f, p)


def test_sketch_is_gather():
    A = usv_matrix(500, 7, 1e3, seed=2)
    idx = o.row_indices(9, 30, 500)
    Y = o.sketch_rows(A, 30, 9)
    assert np.array_equal(Y, A[idx])


@pytest.mark.parametrize("seed", [6, 7])
def test_theorem_3_2_identity(seed):
    # cond(X) = cond(Q_1), X = A R_s^{-1} with R_s the R factor of the sketch
    # (rQR, as in Theorem 3.2), Q_1 the sampled rows of A's Q factor
    m, n, l = 2000, 10, 40
    A = usv_matrix(m, n, 1e6, seed=3)
    r = o.rxr_cholqr(A, ROWS_QR, s=l, seed=seed, passes=1)
    assert r.status == 0
    X = o.trsm_right_upper(A, r.Rs)
    Q, _ = np.linalg.qr(A)
    Q1 = Q[o.row_indices(seed, l, m)]
    assert abs(np.linalg.cond(X) / np.linalg.cond(Q1) - 1) < 1e-6


@pytest.mark.parametrize("variant", [ROWS_QR, ROWS_LU])
@pytest.mark.parametrize("kappa", [1e4, 1e10, 1e15])
def test_full_factorisation_accurate_on_incoherent_A(variant, kappa):
    # A = U Sigma V^T with Gaussian-based U: m theta(Q) = O(n), so l = 2n rows
    # precondition well (Theorem 3.2) and CholeskyQR2 reaches rounding level
    m, n = 4000, 16
    A = usv_matrix(m, n, kappa, seed=4)
    r = o.rxr_cholqr(A, variant, s=2 * n, seed=1, passes=2)
    assert r.status == 0
    assert o.orth_error(r.Q) <= 1e-13
    assert o.resid_error(A, r.Q, r.R) <= 1e-14
    Qh, Rh = o.householder_qr(A)
    assert np.linalg.norm(r.R - Rh) / np.linalg.norm(Rh) <= 50 * kappa * 2.0**-53 * n


def test_coherent_identity_block_breaks_the_sketch():
    # the extreme case before Theorem 3.2: A = [I_n; 0], theta(Q) = 1; l draws
    # miss some of the first n rows with probability ~1 - (l/m)^n, the sketch
    # is rank-deficient and the XR step reports it
    m, n, l = 1000, 8, 16
    A = np.zeros((m, n), order="F")
    A[:n, :n] = np.eye(n)
    missed = 0
    for seed in range(200):
        missed += not set(range(n)) <= set(o.row_indices(seed, l, m).tolist())
    assert missed == 200
    for variant in (ROWS_QR, ROWS_LU):
        assert o.rxr_cholqr(A, variant, s=l, seed=0).status == o.SKETCH_SINGULAR
