"""Parity of the split-precision (tcgen05 tensor-core) contractions with the
CPU oracle.

The split sketch computes Y' = Omega' A with Omega' the same Philox draws on
the 2^-12 grid (the oracle's sketch_quantised); its digit decomposition of A
is exact up to 2^-55 of each column's largest entry per 512-row window, and its
tensor-memory sums are exact integers, so it must meet the FP64 sketch bound
plus that truncation term.  The split Gram cuts each column into seven exact
8-bit digits (FP64 grade: the FP64 Gram bound plus 2^-52 m colmax_j colmax_l);
the preconditioning placement's BF16x3 Gram keeps three 8-bit significand
chunks per entry and accumulates in FP32 (truncating) over 24 tensor-core
accumulations per 64-row tile before each FP64 drain: its bound is
2^-17 (|X|^T |X|) entrywise.  End to end, the split path must reach the same
accuracy targets as the FP64 path for every kappa."""
import math

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

OV = {"lu": o.VARIANT_LU, "qr": o.VARIANT_QR}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


@pytest.mark.parametrize("m,n,s,kappa", [(1, 1, 1, 1.0), (700, 5, 13, 1e3), (1500, 64, 128, 1e12),
                                         (2049, 70, 140, 1e6), (1100, 128, 256, 1e15), (513, 16, 33, 1e8)])
def test_split_sketch_parity(h, m, n, s, kappa):
    A = usv_matrix(m, n, kappa, seed=m + 3)
    Y = to_host(h.sketch(to_dev(A), s, seed=5, prec="split"))
    ref = o.sketch_quantised(A, s, seed=5)
    Oq = o.omega_quantised(5, s, m)
    colmax = np.abs(A).max(axis=0)
    bound = 8 * (math.log2(m) + 4) * U * (np.abs(Oq) @ np.abs(A)) + \
        2.0**-54 * np.abs(Oq).sum(axis=1)[:, None] * colmax[None, :]
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)


@pytest.mark.parametrize("m,n", [(1, 1), (600, 8), (5000, 64), (3000, 100), (2100, 128), (511, 17)])
def test_split_gram_parity(h, m, n):
    A = usv_matrix(m, n, 1e3, seed=n)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=1, passes=1).Rs
    X, G = h.precond_gram(to_dev(A), to_dev(R), prec="split")
    Xg, Gg = to_host(X), to_host(G)
    Go = o.gram(Xg)
    cm = np.abs(Xg).max(axis=0)
    bound = 8 * (m + 2) * U * (np.abs(Xg).T @ np.abs(Xg)) + 2.0**-52 * m * np.outer(cm, cm)
    assert np.all(np.abs(Gg - Go) <= bound), np.max(np.abs(Gg - Go) / bound)
    assert np.array_equal(Gg, Gg.T)


@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e12, 1e15])
def test_split_cholqr_accuracy(h, variant, kappa):
    m, n = 6000, 32
    A = usv_matrix(m, n, kappa, seed=2)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=64, seed=0, passes=2, prec="split")
    assert code == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    ref = o.rxr_cholqr(A, OV[variant], 64, seed=0, passes=2)
    assert r_rel(Rg, ref.R) <= R_TOL, r_rel(Rg, ref.R)


def test_split_matches_fp64_factorisation(h):
    A = to_dev(usv_matrix(20000, 64, 1e10, seed=4))
    Qs, Rs, _ = h.cholqr(A, variant="qr", seed=0, prec="split")
    Qf, Rf, _ = h.cholqr(A, variant="qr", seed=0, prec="fp64")
    rel = (torch.linalg.norm(Rs - Rf) / torch.linalg.norm(Rf)).item()
    assert rel <= R_TOL, rel
    assert h.orth_error(Qs) <= 1e-13


@pytest.mark.parametrize("m,n,kappa", [(1, 1, 1.0), (700, 8, 1e2), (5000, 64, 1e6), (3000, 100, 1e12), (2100, 128, 1e3),
                                       (129, 65, 1e15), (700, 200, 1e8), (600, 512, 1e3), (200003, 128, 1e8),
                                       (262176, 120, 1e12), (76 * 32 * 9 + 64, 96, 1e4)])
def test_ozaki_gram_is_fp64_grade(h, m, n, kappa):
    # exact 7-digit splitting: G = X^T X to FP64 accuracy, entrywise within the
    # FP64 Gram bound plus the digit truncation 2^-54 * colmax_j * colmax_l * m
    X = usv_matrix(m, n, kappa, seed=m)
    Gs = to_host(h.gram(to_dev(X), prec="split"))
    Go = o.gram(X)
    cm = np.abs(X).max(axis=0)
    bound = 8 * (m + 2) * U * (np.abs(X).T @ np.abs(X)) + 2.0**-52 * m * np.outer(cm, cm)
    assert np.all(np.abs(Gs - Go) <= bound), np.max(np.abs(Gs - Go) / bound)
    if n <= 128:
        Gf = to_host(h.gram(to_dev(X), prec="fp64"))
        assert np.all(np.abs(Gf - Go) <= 8 * (m + 2) * U * (np.abs(X).T @ np.abs(X)))
    assert np.array_equal(Gs, Gs.T)


@pytest.mark.parametrize("m,n,kappa", [(3000, 64, 1e12), (1000, 17, 1e6), (2500, 128, 1e15), (900, 200, 1e10),
                                       (700, 512, 1e8), (129, 33, 1e3)])
def test_blocked_substitution_is_backward_stable(h, m, n, kappa):
    # split mode solves X R = A by column blocks (FP64 diagonal blocks, tensor-core
    # trailing updates): the backward error ||X R - A|| / (||X|| ||R||) must stay
    # at FP64 rounding level however ill-conditioned R is
    A = usv_matrix(m, n, kappa, seed=n + 1)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=3, passes=1).Rs    # cond(R) ~ kappa
    X, G = h.precond_gram(to_dev(A), to_dev(R), prec="split")
    Xg = to_host(X)
    back = np.linalg.norm(Xg @ R - A) / (np.linalg.norm(Xg) * np.linalg.norm(R))
    assert back <= 64 * n * U, back
    Xo = o.trsm_right_upper(A, R)
    back_o = np.linalg.norm(Xo @ R - A) / (np.linalg.norm(Xo) * np.linalg.norm(R))
    assert back <= 64 * max(back_o, n * U)


@pytest.mark.parametrize("m,n,kappa", [(1, 1, 1.0), (130, 16, 1e4), (4097, 48, 1e13), (1000, 63, 1e9),
                                       (128 * 152 * 2 + 77, 64, 1e11)])
def test_fused_substitution_edges(h, m, n, kappa):
    # the fused kernel (n <= 64): one block, whole blocks, a narrow last block,
    # a ragged last tile and more tiles than CTAs; backward error at FP64
    # rounding level, and an even leading dimension (TMA) must give the same
    # bits as an odd one (plain loads and stores)
    A = usv_matrix(m, n, kappa, seed=m + n)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=5, passes=1).Rs
    X, _ = h.precond_gram(to_dev(A), to_dev(R), prec="split")
    Xg = to_host(X)
    back = np.linalg.norm(Xg @ R - A) / max(np.linalg.norm(Xg) * np.linalg.norm(R), 1e-300)
    assert back <= 64 * n * U, back
    Xodd, _ = h.precond_gram(to_dev(A, ld=m + 1), to_dev(R), X=rxr.empty_colmajor(m, n, ld=m + 1), prec="split")
    assert np.array_equal(to_host(Xodd), Xg)


def test_fused_substitution_first_block_is_plain_substitution(h):
    # the first 16 columns see no trailing update: they must equal the FP64
    # path's substitution bit for bit (same FMA order, same 1 / R_jj)
    m, n = 3000, 40
    A = usv_matrix(m, n, 1e8, seed=9)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=1, passes=1).Rs
    Xs, _ = h.precond_gram(to_dev(A), to_dev(R), prec="split")
    Xf, _ = h.precond_gram(to_dev(A), to_dev(R), prec="fp64")
    assert np.array_equal(to_host(Xs)[:, :16], to_host(Xf)[:, :16])


@pytest.mark.parametrize("m,n", [(64 * 152 * 5 + 13, 64), (4100, 33), (300, 1), (32 * 152 * 9 + 6, 128), (70001, 97)])
def test_ozaki_gram_column_scales(h, m, n):
    # columns scaled across the whole FP64 range, one column zero: the Gram must
    # stay FP64-grade column-normwise (the digit scale of each column is its own
    # largest exponent over all rows)
    rng = np.random.default_rng(m)
    X = usv_matrix(m, n, 1e4, seed=m + 1) * np.ldexp(1.0, rng.integers(-400, 400, size=n))[None, :]
    if n > 2:
        X[:, 2] = 0.0
    Gs = to_host(h.gram(to_dev(X), prec="split"))
    Go = o.gram(X)
    cm = np.abs(X).max(axis=0)
    bound = 8 * (m + 2) * U * (np.abs(X).T @ np.abs(X)) + 2.0**-52 * m * np.outer(cm, cm)
    assert np.all(np.abs(Gs - Go) <= bound), np.nanmax(np.abs(Gs - Go) / np.where(bound > 0, bound, 1))
    assert np.array_equal(Gs, Gs.T)


@pytest.mark.parametrize("m,n,kappa", [(65, 65, 1e3), (3001, 80, 1e12), (128 * 152 + 5, 127, 1e14), (5000, 128, 1e15)])
def test_fused128_substitution(h, m, n, kappa):
    # the 64 < n <= 128 fused kernel (records of R streamed per column block):
    # a narrow last block, a ragged last tile, more tiles than CTAs; backward
    # error at FP64 rounding level, and TMA (even ld) and plain (odd ld) staging
    # give the same bits
    A = usv_matrix(m, n, kappa, seed=m + 7)
    R = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=2, passes=1).Rs
    X, _ = h.precond_gram(to_dev(A), to_dev(R), prec="split")
    Xg = to_host(X)
    back = np.linalg.norm(Xg @ R - A) / (np.linalg.norm(Xg) * np.linalg.norm(R))
    assert back <= 64 * n * U, back
    Xodd, _ = h.precond_gram(to_dev(A, ld=m + 1), to_dev(R), X=rxr.empty_colmajor(m, n, ld=m + 1), prec="split")
    assert np.array_equal(to_host(Xodd), Xg)
    # against the oracle's substitution (for n > 64 the FP64 path splits each
    # row's sums over two lanes, so bit equality is not expected)
    Xo = o.trsm_right_upper(A, R)
    assert np.linalg.norm(Xg - Xo) <= 64 * n * U * np.linalg.cond(R) * np.linalg.norm(Xo)


@pytest.mark.parametrize("s_factor,kappa", [(2, 1e12), (1, 1e6), (1, 1e10)])
def test_middle_pass_selection(h, s_factor, kappa):
    # above 2^17 rows the middle CholeskyQR pass multiplies by the explicit
    # inverse of R_1 on the tensor cores when its estimated condition number is
    # at most 16, else substitutes; a square sketch (s = n) leaves X_1 worse
    # conditioned than s = 2n.  Either way the factorisation meets the targets.
    m, n = 1 << 17, 48
    A = usv_matrix(m, n, kappa, seed=int(kappa) % 97 + s_factor)
    Q, R, code = h.cholqr(to_dev(A), variant="qr", s=s_factor * n, seed=4, passes=2, prec="split")
    assert code == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert np.all(np.diag(Rg) > 0)


def _upper(n, rng, eps):
    """I + eps F with F upper triangular, standard normal entries."""
    return np.asfortranarray(np.eye(n) + eps * np.triu(rng.standard_normal((n, n))))


def _row_rel_err(Qg, Qo, T):
    """max over rows of |Qg - Qo|_2 / (|x_row|_2 |T|_2), x_row = Qo_row R."""
    den = np.linalg.norm(Qo, axis=1) * np.linalg.norm(T, 2) * max(1.0, np.linalg.cond(T))
    return float(np.max(np.linalg.norm(Qg - Qo, axis=1) / np.maximum(den, 1e-300)))


@pytest.mark.parametrize("m,n,eps", [(1, 1, 1e-14), (677, 7, 1e-14), (128 * 9 + 37, 33, 1e-15),
                                     (4096 + 5, 64, 1e-13), (900, 64, 1e-12), (900, 64, 1e-11),
                                     (900, 48, 0.3), (3000, 64, 0.05), (250, 1, 0.5),
                                     (128 * 9 + 37, 100, 1e-15), (1000, 128, 1e-13), (700, 65, 1e-14),
                                     (900, 128, 1e-11), (2000, 97, 0.3), (333, 128, 0.05)])
def test_apply_rinv_split(h, m, n, eps):
    # X <- X R^{-1}, n <= 128: with R - I at most about 2^-38 the correction
    # X (R^{-1} - I) is formed in FP32 (error below 2^-55 |X| per term); a
    # larger R - I (eps = 1e-11 lies above 2^-38 after inversion, 0.05 .. 0.5
    # far above) takes the FP64-grade tensor-core product (n <= 64) or the fused
    # substitution (64 < n <= 128).  Each must match the oracle's substitution
    # to FP64 accuracy, far below what an FP32 product of X and R^{-1} reaches
    # (about 1e-7).
    rng = np.random.default_rng(m + n)
    X = usv_matrix(m, n, 10.0, seed=n)
    R = _upper(n, rng, eps)
    Qo = o.trsm_right_upper(X, R)
    Xd = to_dev(X)
    h.apply_rinv(Xd, to_dev(R), prec="split")
    Qg = to_host(Xd)
    T = np.linalg.inv(R)
    err = _row_rel_err(Qg, Qo, T)
    assert err <= 64 * U, err


@pytest.mark.parametrize("n", [64, 128])
def test_apply_rinv_split_odd_ld_and_large(h, n):
    # a leading dimension that is not a multiple of the tile, and 2^20 + 77 rows
    # (sampled rows against the oracle): the FP32-correction form
    m = (1 << 20) + 77
    rng = np.random.default_rng(5)
    R = _upper(n, rng, 2e-15)
    X = np.asfortranarray(rng.standard_normal((m + 3, n)))
    Xfull = to_dev(X)
    Xd = Xfull[:m]
    assert Xd.stride() == (1, m + 3)
    h.apply_rinv(Xd, to_dev(R), prec="split")
    Qg = to_host(Xd)
    rows = np.concatenate([np.arange(0, 300), rng.integers(0, m, 2000), np.arange(m - 300, m)])
    Qo = o.trsm_right_upper(np.asfortranarray(X[rows]), R)
    assert _row_rel_err(Qg[rows], Qo, np.linalg.inv(R)) <= 64 * U
    # the padding rows are not touched
    assert np.array_equal(to_host(Xfull)[m:], X[m:])


@pytest.mark.parametrize("prec,m,n", [("fp64", 700, 20), ("fp64", 3000, 100), ("split", 2100, 100),
                                      ("split", 999, 128)])
def test_apply_rinv_other_forms(h, prec, m, n):
    rng = np.random.default_rng(n)
    X = usv_matrix(m, n, 10.0, seed=n + 1)
    R = _upper(n, rng, 0.1)
    Qo = o.trsm_right_upper(X, R)
    Xd = to_dev(X)
    h.apply_rinv(Xd, to_dev(R), prec=prec)
    assert _row_rel_err(to_host(Xd), Qo, np.linalg.inv(R)) <= 64 * U


# ------------------------------------------------------------------ RXR_SPLIT_PRECOND
@pytest.mark.parametrize("m,n", [(1, 1), (700, 8), (5000, 33), (6000, 64), (3000, 100), (2100, 128), (65, 17)])
def test_precond_mode_gram_parity(h, m, n):
    # the first-pass Gram of the preconditioning placement: BF16x3 on the tensor
    # cores, three 8-bit significand chunks per entry, FP32 sums drained every 64
    # rows; bound 2^-17 (|X|^T |X|) entrywise, as for the n > 64 split Gram
    A = usv_matrix(m, n, 1e3, seed=n + 2)
    X = o.rxr_cholqr(A, o.VARIANT_QR, 2 * n, seed=1, passes=1).Q
    G = to_host(h.gram(to_dev(X), prec="split_precond"))
    Go = o.gram(X)
    bound = 2.0**-17 * (np.abs(X).T @ np.abs(X))
    assert np.all(np.abs(G - Go) <= bound), np.max(np.abs(G - Go) / bound)
    assert np.array_equal(G, G.T)


@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("m,n,kappa", [(6000, 1, 1.0), (6000, 8, 1e15), (5000, 33, 1e12), (6000, 64, 1e15),
                                       (3000, 100, 1e10), (2100, 128, 1e14), (1100, 200, 1e13), (4001, 48, 1e8)])
def test_precond_mode_cholqr_parity(h, variant, m, n, kappa):
    # only the sketch and the first Gram leave FP64; the FP64 second pass brings
    # Q and R to the same accuracy as the FP64 path
    A = usv_matrix(m, n, kappa, seed=n + 5)
    Q, R, code = h.cholqr(to_dev(A), variant=variant, s=2 * n, seed=2, passes=2, prec="split_precond")
    assert code == 0
    Qg, Rg = to_host(Q), to_host(R)
    assert o.orth_error(Qg) <= 1e-13
    assert o.resid_error(A, Qg, Rg) <= 1e-14
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    ref = o.rxr_cholqr(A, OV[variant], 2 * n, seed=2, passes=2)
    assert r_rel(Rg, ref.R) <= R_TOL, r_rel(Rg, ref.R)


def test_precond_mode_reports_nonfinite_and_matches_host_entry(h):
    A = usv_matrix(3000, 40, 1e6, seed=3)
    Qh, Rh = h.cholqr_host(A, variant="qr", seed=4, prec="split_precond")
    Q, R, code = h.cholqr(to_dev(A), variant="qr", seed=4, prec="split_precond")
    assert code == 0
    assert np.array_equal(Qh, to_host(Q)) and np.array_equal(Rh, to_host(R))
    B = A.copy(order="F")
    B[1234, 7] = np.inf
    _, _, code = h.cholqr(to_dev(B), variant="qr", seed=4, prec="split_precond", raise_on_error=False)
    assert code == rxr.NONFINITE
