"""Pins for the oracle's rLU-/rQR-CholeskyQR (Algorithms 4 and 5, with the
repeated CholeskyQR pass of Algorithm 2) against what the paper and the
mathematics fix: the thin QR factorisation is unique with diag(R) > 0
(footnote to Algorithm 1), Proposition 3.1's identity, Theorem 3.4's bound,
the CholeskyQR2 orthogonality bound of Section 2.1, the accuracy measures of
Section 4.2, the breakdown of unpreconditioned CholeskyQR, and invariances of
the QR factorisation."""
import math

import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, r_rel
from paper_2111_11148_gb300.inputs import usv_matrix

U = 2.0**-53
VARIANTS = [o.VARIANT_LU, o.VARIANT_QR]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kappa", [1e2, 1e5, 1e8, 1e12, 1e15])
def test_accuracy_independent_of_kappa(variant, kappa):
    # Section 4.2: orthogonality and residual stay at rounding level up to 1e15
    m, n = 3000, 16
    A = usv_matrix(m, n, kappa, seed=1)
    r = o.rxr_cholqr(A, variant, 2 * n, seed=0, passes=2)
    assert r.status == 0
    assert o.orth_error(r.Q) <= 1e-13
    assert o.resid_error(A, r.Q, r.R) <= 1e-14
    # CholeskyQR2 orthogonality bound 6 (m + n + 1) n u (Section 2.1)
    assert o.orth_error(r.Q) <= 6 * (m + n + 1) * n * U
    assert np.all(np.diag(r.R) > 0) and np.all(np.tril(r.R, -1) == 0)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("kappa", [1e3, 1e8, 1e12])
def test_r_agrees_with_householder_definition(variant, kappa):
    # the computed R is the unique R factor with positive diagonal, up to the
    # R-factor perturbation bound c * kappa * u
    A = usv_matrix(2000, 12, kappa, seed=2)
    r = o.rxr_cholqr(A, variant, 24, seed=3)
    Qh, Rh = o.householder_qr(A)
    rel = np.linalg.norm(r.R - Rh) / np.linalg.norm(Rh)
    assert rel <= R_TOL, rel
    if kappa <= 1e8:
        assert np.linalg.norm(r.Q - Qh) <= 100 * kappa * U * math.sqrt(12)


def test_seed_invariance_of_the_factorisation():
    A = usv_matrix(1500, 10, 1e6, seed=4)
    r0 = o.rxr_cholqr(A, o.VARIANT_QR, 20, seed=0)
    r1 = o.rxr_cholqr(A, o.VARIANT_QR, 20, seed=1)
    assert not np.array_equal(r0.Rs, r1.Rs)          # different sketches ...
    assert r_rel(r1.R, r0.R) <= R_TOL   # ... same QR


def test_scaling_and_column_scaling_and_row_permutation():
    A = usv_matrix(1200, 8, 1e4, seed=5)
    base = o.rxr_cholqr(A, o.VARIANT_QR, 16, seed=0)
    a = o.rxr_cholqr(np.asfortranarray(4.0 * A), o.VARIANT_QR, 16, seed=0)      # power of 2: exact
    np.testing.assert_allclose(a.R, 4.0 * base.R, rtol=0, atol=1e-14 * np.abs(base.R).max() * 4)
    np.testing.assert_allclose(a.Q, base.Q, atol=1e-14)
    D = np.array([1.0, 3.0, 0.5, 10.0, 2.0, 1.0, 7.0, 0.1])
    c = o.rxr_cholqr(np.asfortranarray(A * D), o.VARIANT_QR, 16, seed=0)       # A D = Q (R D)
    np.testing.assert_allclose(c.R, base.R * D, rtol=0, atol=1e-11 * np.abs(base.R * D).max())
    perm = np.random.default_rng(0).permutation(1200)
    p = o.rxr_cholqr(np.asfortranarray(A[perm]), o.VARIANT_QR, 16, seed=0)     # Pi A = (Pi Q) R
    np.testing.assert_allclose(p.R, base.R, rtol=0, atol=1e-11 * np.abs(base.R).max())
    np.testing.assert_allclose(p.Q, base.Q[perm], atol=1e-10)


@pytest.mark.parametrize("kappa", [1e2, 1e6])
def test_proposition_3_1_identity(kappa):
    # cond(A R_s^{-1}) = cond(Omega Q_A) for A = Q_A R_A, R_s = R factor of Omega A
    m, n, s = 600, 8, 16
    A = usv_matrix(m, n, kappa, seed=6)
    r = o.rxr_cholqr(A, o.VARIANT_QR, s, seed=9, passes=1)
    X = o.trsm_right_upper(A, r.Rs)
    Qa, _ = np.linalg.qr(A)
    Om = o.omega(seed=9, s=s, m=m)
    cx = np.linalg.cond(X)
    cq = np.linalg.cond(Om @ Qa)
    assert abs(cx - cq) <= 1e3 * kappa * U * cq


def test_sketch_matches_explicit_omega_product():
    m, n, s = 700, 5, 11
    A = usv_matrix(m, n, 1e3, seed=7)
    Y = o.sketch(A, s, seed=4)
    Om = o.omega(seed=4, s=s, m=m)
    np.testing.assert_allclose(Y, Om @ A, rtol=0, atol=1e-14 * np.abs(Om).sum(1).max() * np.abs(A).max())


@pytest.mark.parametrize("row0", [1, 256, 1000, 2**32 + 5])
def test_shard_sketch_is_its_share_of_the_whole(row0):
    # Omega's columns follow the global rows (Section 2.4's row blocks): a shard
    # holding rows row0 .. row0 + m - 1 takes columns row0 .. of the same Omega
    m, n, s = 613, 4, 9
    A = usv_matrix(m, n, 1e3, seed=8)
    Y = o.sketch(A, s, seed=6, row0=row0)
    z = o.omega_z(6, s, row0, m).astype(np.float64)         # (rows, s): z of rows row0 ..
    Om = (1.0 / np.sqrt(float(s))) * z.T
    np.testing.assert_allclose(Y, Om @ A, rtol=0, atol=1e-14 * np.abs(Om).sum(1).max() * np.abs(A).max())
    # the shards of a split matrix add up to the whole sketch (to rounding)
    B = usv_matrix(1500, n, 1e3, seed=9)
    parts = o.sketch(B[:700], s, 6) + o.sketch(B[700:], s, 6, row0=700)
    np.testing.assert_allclose(parts, o.sketch(B, s, 6), rtol=0, atol=1e-13 * np.abs(B).max() * 1500)


def _cond_x(n, s, seed, m=None, kappa=1e3, variant=o.VARIANT_QR):
    m = m or 20 * s
    A = usv_matrix(m, n, kappa, seed=100 + seed)
    r = o.rxr_cholqr(A, variant, s, seed=seed, passes=1)
    X = o.trsm_right_upper(A, r.Rs)
    sv = np.linalg.svd(X, compute_uv=False)
    return sv[0] / sv[-1], sv


@pytest.mark.slow
def test_theorem_3_4_gaussian_bound():
    # P[cond(X) >= (3 + sqrt(n/l)) / (1 - sqrt(n/l))] <= 2 exp(-(sqrt(l) - sqrt(n))^2 / 8)
    n, s = 64, 128
    thr = (3 + math.sqrt(n / s)) / (1 - math.sqrt(n / s))
    pb = 2 * math.exp(-((math.sqrt(s) - math.sqrt(n)) ** 2) / 8)
    conds, smax, smin = [], [], []
    for seed in range(40):
        c, sv = _cond_x(n, s, seed, m=2000)
        conds.append(c)
    frac = np.mean(np.array(conds) >= thr)
    assert frac <= pb + 3 * math.sqrt(pb * (1 - pb) / 40)
    # with N(0, 1/s) entries, the singular values of Omega Q sit near
    # 1 +- sqrt(n/s) (Marchenko-Pastur edges), so cond(X) is near 5.8 here
    assert 4.0 < np.median(conds) < thr


def test_sampling_rate_sweep():
    # Section 4.5: cond(X) falls steeply as l/n moves away from 1
    n = 24
    med = {}
    for ratio in (1.0, 1.25, 2.0, 4.0):
        s = int(round(ratio * n))
        med[ratio] = np.median([_cond_x(n, s, sd, m=1500)[0] for sd in range(12)])
    assert med[1.0] > 5 * med[1.25] > 5 * 1.0
    assert med[1.25] > med[2.0] > med[4.0] > 1.0
    # Remark 3.5: with l > 1.1 n the bound (3 + sqrt(n/l)) / (1 - sqrt(n/l)) is below 100
    assert (3 + math.sqrt(1 / 1.1)) / (1 - math.sqrt(1 / 1.1)) < 100


def test_unpreconditioned_choleskyqr_breaks_down_where_rxr_does_not():
    # Section 2.1 / 4.2: CholeskyQR(2) breaks down once cond(A)^2 > 1/u
    A = usv_matrix(2000, 10, 1e12, seed=8)
    plain = o.rxr_cholqr(A, o.VARIANT_NONE, 20, seed=0, passes=2)
    assert plain.status == o.CHOL_BREAKDOWN and plain.info[0] == 1
    for v in VARIANTS:
        r = o.rxr_cholqr(A, v, 20, seed=0, passes=2)
        assert r.status == 0 and o.orth_error(r.Q) < 1e-13


def test_single_pass_orthogonality_is_u_cond_squared():
    # one CholeskyQR pass (Algorithms 4/5 as printed): error ~ cond(X)^2 u,
    # with cond(X) small after preconditioning; the second pass reaches u
    A = usv_matrix(3000, 16, 1e10, seed=9)
    r1 = o.rxr_cholqr(A, o.VARIANT_QR, 32, seed=0, passes=1)
    r2 = o.rxr_cholqr(A, o.VARIANT_QR, 32, seed=0, passes=2)
    c, _ = _cond_x(16, 32, 0, m=3000, kappa=1e10)
    assert o.orth_error(r1.Q) < 50 * c * c * 16 * U
    assert o.orth_error(r2.Q) < o.orth_error(r1.Q) or o.orth_error(r1.Q) < 1e-15


def test_failure_statuses():
    A = usv_matrix(500, 6, 1e3, seed=10)
    B = A.copy(order="F")
    B[3, 2] = np.nan
    assert o.rxr_cholqr(B, o.VARIANT_QR, 12).status == o.NONFINITE
    Z = A.copy(order="F")
    Z[:, 4] = 0.0                                          # rank deficient
    for v in VARIANTS:
        assert o.rxr_cholqr(Z, v, 12).status == o.SKETCH_SINGULAR


def test_appendix_a_perturbation_bound():
    # cond(X^) <= (1 + g) / (1 - g) cond(X), g = ||X - X^||_2 / ||X||_2, with X the
    # exact A R_s^{-1} (here in 60-digit arithmetic) and X^ the oracle's
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    m, n = 60, 4
    A = usv_matrix(m, n, 1e10, seed=11)
    r = o.rxr_cholqr(A, o.VARIANT_QR, 8, seed=0, passes=1)
    Xh = o.trsm_right_upper(A, r.Rs)
    Am = mp.matrix(A.tolist())
    Rm = mp.matrix(r.Rs.tolist())
    Xm = Am * mp.inverse(Rm)
    D = Xm - mp.matrix(Xh.tolist())
    sv_x = mp.svd_r(Xm, compute_uv=False)
    g = float(max(mp.svd_r(D, compute_uv=False)) / max(sv_x))
    cond_x = float(max(sv_x) / min(sv_x))
    assert g * cond_x < 1
    assert np.linalg.cond(Xh) <= (1 + g) / (1 - g) * cond_x * (1 + 1e-12)
    assert g < 1e3 * 1e10 * U                              # beta-stability of the substitution


def test_quantised_sketch_matches_explicit_product_and_is_close_to_gaussian():
    # Omega' = rint(4096 z)/4096/sqrt(s): every entry is an integer multiple of
    # 2^-12/sqrt(s) within 2^-13/sqrt(s) of Omega, and the oracle's Y' equals Omega' A
    m, n, s = 900, 6, 13
    A = usv_matrix(m, n, 1e4, seed=21)
    Oq = o.omega_quantised(3, s, m)
    Om = o.omega(3, s, m)
    k = Oq * math.sqrt(s) * 4096.0          # integers up to the rounding of the 1/sqrt(s) scale
    assert np.max(np.abs(k - np.rint(k))) < 1e-9
    assert np.max(np.abs(Oq - Om)) <= 2.0**-13 / math.sqrt(s) * (1 + 1e-9)   # ties are exactly 2^-13 away
    Yq = o.sketch_quantised(A, s, seed=3)
    np.testing.assert_allclose(Yq, Oq @ A, rtol=0, atol=1e-14 * np.abs(Oq).sum(1).max() * np.abs(A).max())
    # Proposition 3.1 holds for any sketch matrix: cond(A R^{-1}) = cond(Omega' Q_A)
    Rq = o.sign_normalise(o.geqr_r(Yq))
    X = o.trsm_right_upper(A, Rq)
    Qa, _ = np.linalg.qr(A)
    assert abs(np.linalg.cond(X) - np.linalg.cond(Oq @ Qa)) <= 1e-8 * np.linalg.cond(X)


@pytest.mark.parametrize("variant", [o.VARIANT_QR, o.VARIANT_LU, o.VARIANT_QR | o.SKETCH_ROWS])
def test_openmp_build_returns_the_same_bits(variant):
    # the multi-core build parallelises only independent row blocks and rows and
    # combines the blocks' partial sums in the serial order
    A = usv_matrix(70001, 24, 1e9, seed=8)
    r1 = o.rxr_cholqr(A, variant, 48, seed=3, passes=2)
    rp = o.rxr_cholqr(A, variant, 48, seed=3, passes=2, parallel=True)
    assert r1.status == rp.status == 0
    assert np.array_equal(r1.Q, rp.Q) and np.array_equal(r1.R, rp.R) and np.array_equal(r1.Y, rp.Y)
    assert o.threads(parallel=False) == 1 and o.threads(parallel=True) >= 1
