"""Parity with the oracle at the shapes and conditionings that the workload
configurations name, on the kernels those shapes select (each case checked
element by element against the oracle's rQR-/rLU-CholeskyQR2, Algorithms 4/5
with the repeated pass of Algorithm 2, on the same seeded A):

* the split-precision Gaussian path at n = 128: the sketch on the tensor cores,
  the per-block records of R_s, the fused substitution for 64 < n <= 128, the
  BF16x3 first Gram and the FP64-grade second Gram, for kappa in {1e6, 1e12,
  1e14} with rLU and rQR, at m = 2^17 + 77 (many 128-row tiles, a ragged tail);
* n = 64 at m = 2^17 + 77 with kappa in {1e4, 1e10, 1e15}: there the split
  path's middle pass chooses on the device between the explicit inverse on the
  tensor cores and the fused substitution, and its last pass between the FP32
  correction and the FP64-grade product; both paths, both variants;
* the batched form, each problem's Q and R against the oracle's own.

R is compared with the oracle's R within R_TOL (100 times the spread measured
between independent FP64 implementations), Q with the oracle's Q within ten
times that spread where kappa <= 1e12; Q and R meet Section 4.2's measures."""
import numpy as np
import pytest

import oracle as o
from gpu_util import R_TOL, r_rel, to_dev, to_host
from paper_2111_11148_gb300.inputs import batch_specs, usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402

OV = {"lu": o.VARIANT_LU, "qr": o.VARIANT_QR}
M17 = (1 << 17) + 77


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


def _check(A, Q, R, ref, what):
    Qg, Rg = to_host(Q), to_host(R)
    orth, resid = o.orth_error(Qg), o.resid_error(A, Qg, Rg)
    assert orth <= 1e-13 and resid <= 1e-14, (what, orth, resid)
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    rel = r_rel(Rg, ref.R)
    assert rel <= R_TOL, (what, rel)
    # Q against the oracle's Q: Q = A R^{-1} carries R's conditioning, and the
    # spread measured between independent FP64 implementations grows with
    # kappa and stays below sqrt(n) kappa u (n = 16, 64; kappa = 1e2 .. 1e15),
    # so the check binds where that is small
    n = Rg.shape[0]
    kappa = what[1] if isinstance(what[1], float) else None
    if kappa is not None and kappa <= 1e12:
        dq = np.linalg.norm(Qg - ref.Q)
        assert dq <= 10 * np.sqrt(n) * max(kappa, 10.0) * 2.0**-53, (what, dq)
    return rel, orth, resid


@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("kappa", [1e6, 1e12, 1e14])
def test_split_gaussian_n128(h, variant, kappa):
    n = 128
    A = usv_matrix(M17, n, kappa, seed=11)
    ref = o.rxr_cholqr(A, OV[variant], 2 * n, seed=0, passes=2)
    assert ref.status == 0
    for prec in ("split", "split_precond", "fp64"):
        Q, R, code = h.cholqr(to_dev(A), variant=variant, s=2 * n, seed=0, passes=2, prec=prec)
        assert code == 0
        rel, orth, resid = _check(A, Q, R, ref, (variant, kappa, prec))
        print(f"n=128 m={M17} {variant} kappa={kappa:.0e} {prec}: R vs oracle {rel:.2e} orth {orth:.2e} "
              f"resid {resid:.2e}")


@pytest.mark.parametrize("variant", ["qr", "lu"])
@pytest.mark.parametrize("kappa", [1e4, 1e10, 1e15])
def test_n64_above_2p17_rows(h, variant, kappa):
    n = 64
    A = usv_matrix(M17, n, kappa, seed=12)
    ref = o.rxr_cholqr(A, OV[variant], 2 * n, seed=5, passes=2)
    assert ref.status == 0
    for prec in ("split", "split_precond", "fp64"):
        Q, R, code = h.cholqr(to_dev(A), variant=variant, s=2 * n, seed=5, passes=2, prec=prec)
        assert code == 0
        rel, orth, resid = _check(A, Q, R, ref, (variant, kappa, prec))
        print(f"n=64 m={M17} {variant} kappa={kappa:.0e} {prec}: R vs oracle {rel:.2e} orth {orth:.2e} "
              f"resid {resid:.2e}")


def test_batched_against_oracle(h):
    # 48 problems with the batched workload's distribution of shapes and
    # conditionings (m capped at 2^15 so that the oracle runs in seconds)
    specs = batch_specs(48, seed=0, log2m=(7, 15))
    As_np = [usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed) for sp in specs]
    As = [to_dev(a) for a in As_np]
    seeds = [sp.seed for sp in specs]
    Qs, Rs, st = h.cholqr_batched(As, variant="qr", seeds=seeds)
    assert np.all(st == 0)
    worst = 0.0
    for i, sp in enumerate(specs):
        ref = o.rxr_cholqr(As_np[i], o.VARIANT_QR, 2 * sp.n, seed=sp.seed, passes=2)
        assert ref.status == 0
        rel, _, _ = _check(As_np[i], Qs[i], Rs[i], ref, ("batched", sp.kappa, i))
        worst = max(worst, rel)
    print(f"batched: worst R vs oracle {worst:.2e} over {len(specs)} problems")


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_plain_load_path_repeated(h, prec):
    # an odd leading dimension rules TMA out, so every panel is staged by plain
    # loads, each thread loading entries that other warps then read: at n = 8
    # the substitution starts right after the loads (a missing barrier there
    # once left 32-row blocks of one odd column stale in about one call in ten)
    m, n = 40001, 8
    A_full = usv_matrix(m, n, 1e4, seed=77, lda=m + 1)
    A = A_full[:m]
    ref = o.rxr_cholqr(np.asfortranarray(A), o.VARIANT_QR, 2 * n, seed=2, passes=2)
    Ad = to_dev(A_full)[:m]
    assert Ad.stride() == (1, m + 1)
    for _ in range(12):
        Q, R, code = h.cholqr(Ad, variant="qr", s=2 * n, seed=2, passes=2, prec=prec)
        assert code == 0
        _check(np.asfortranarray(A), Q, R, ref, ("plain", 1e4, prec))


@pytest.mark.parametrize("n,s_factor", [(128, 2), (128, 1), (100, 2), (100, 1)])
def test_split_middle_pass_branches_n128(h, n, s_factor):
    # 64 < n <= 128, m >= 2^17: the middle pass multiplies by R_1^{-1} in 64-column
    # blocks on the tensor cores when the device's estimate of cond_2(R_1) is at
    # most 16 (s = 2n: Theorem 3.4's well-conditioned X), else substitutes (s = n
    # leaves cond(X) far larger); both against the oracle
    A = usv_matrix(M17, n, 1e12, seed=n + s_factor)
    s = s_factor * n
    ref = o.rxr_cholqr(A, o.VARIANT_QR, s, seed=7, passes=2)
    assert ref.status == 0
    X1 = np.linalg.solve(ref.Rs.T, A.T).T
    cond_r1 = np.linalg.cond(X1)
    Q, R, code = h.cholqr(to_dev(A), variant="qr", s=s, seed=7, passes=2, prec="split")
    assert code == 0
    rel, orth, resid = _check(A, Q, R, ref, ("middle", 1e12, n, s))
    print(f"n={n} s={s}: cond(X_1) {cond_r1:.1f}, R vs oracle {rel:.2e}, orth {orth:.2e}, resid {resid:.2e}")
