"""The workloads at their full sizes, in the launch configuration bench.py
times, on both paths: m = 2^22, n = 64, s = 128 with kappa in {1e4, 1e10, 1e15}
(rQR and rLU), and m = 2^23, n = 128, s = 256 with kappa = 1e14, seed 0,
CholeskyQR2.  The oracle cannot factorise millions of rows in a test's time, so
the checks are sampled outputs and properties that hold at any size:

* every sketch entry against the oracle's sketch, built from the oracle's own
  Omega draws chunk by chunk (the quantised draws for the split path), within
  the sketch's rounding bound;
* Q = A R^{-1} on sampled rows (each row one triangular solve on the host);
* R against the Householder R of LAPACK (the unique thin QR), within 100 times
  the spread measured between independent FP64 implementations;
* the accuracy measures of Section 4.2 on the full Q and R's structure."""
import math
import time

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

M, N, S, KAPPA, SEED = 1 << 22, 64, 128, 1e10, 0
CHUNK = 1 << 19
# (m, n, kappa): the scale configuration at three conditionings, and the
# split-precision configuration at its hardest conditioning
FULL = [(1 << 22, 64, 1e4), (1 << 22, 64, 1e10), (1 << 22, 64, 1e15), (1 << 23, 128, 1e14)]


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


_cache = {}


def _matrix(m, n, kappa):
    """A = U Sigma V^T of the configuration, its device copy and LAPACK's
    Householder R with diag > 0; one configuration kept at a time."""
    key = (m, n, kappa)
    if key not in _cache:
        _cache.clear()
        torch.cuda.empty_cache()
        A = usv_matrix(m, n, kappa, seed=SEED)
        Rh = np.linalg.qr(A, mode="r")
        Rh = np.sign(np.diag(Rh))[:, None] * Rh
        _cache[key] = (A, to_dev(A), Rh)
    return _cache[key]


def _sketch_refs(A):
    """Oracle's Y = Omega A and Y' = Omega' A (quantised draws) with |Omega| |A|,
    accumulated over 2^19-row chunks of Omega's columns."""
    Y = np.zeros((S, N))
    Yq = np.zeros((S, N))
    absY = np.zeros((S, N))
    absYq = np.zeros((S, N))
    absq_rows = np.zeros(S)
    c = 1.0 / math.sqrt(S)
    for i0 in range(0, M, CHUNK):
        z = o.omega_z(SEED, S, i0, CHUNK).astype(np.float64)  # (rows, s)
        Ac = A[i0:i0 + CHUNK]
        om = c * z
        omq = c * (np.rint(z * 4096.0) / 4096.0)
        Y += om.T @ Ac
        Yq += omq.T @ Ac
        absY += np.abs(om).T @ np.abs(Ac)
        absYq += np.abs(omq).T @ np.abs(Ac)
        absq_rows += np.abs(omq).sum(axis=0)
    return Y, Yq, absY, absYq, absq_rows


def test_fullsize_sketch_entries(h):
    A, Ad, _ = _matrix(M, N, KAPPA)
    Y, Yq, absY, absYq, absq_rows = _sketch_refs(A)
    bound = 8 * (math.log2(M) + 4) * U * absY
    Yg = to_host(h.sketch(Ad, S, seed=SEED, prec="fp64"))
    assert np.all(np.abs(Yg - Y) <= bound), np.max(np.abs(Yg - Y) / bound)
    colmax = np.abs(A).max(axis=0)
    boundq = 8 * (math.log2(M) + 4) * U * absYq + 2.0**-54 * absq_rows[:, None] * colmax[None, :]
    Yqg = to_host(h.sketch(Ad, S, seed=SEED, prec="split"))
    assert np.all(np.abs(Yqg - Yq) <= boundq), np.max(np.abs(Yqg - Yq) / boundq)


@pytest.mark.parametrize("m,n,kappa", FULL, ids=[f"m{m}-n{n}-k{k:.0e}" for m, n, k in FULL])
def test_fullsize_factorisation(h, m, n, kappa):
    A, Ad, Rh = _matrix(m, n, kappa)
    rng = np.random.default_rng(1)
    rows = np.concatenate([np.arange(64), rng.integers(0, m, 4000), np.arange(m - 64, m)])
    for variant in ("qr", "lu"):
        for prec in ("split", "split_precond", "fp64"):
            t0 = time.perf_counter()
            Q, R, code = h.cholqr(Ad, variant=variant, s=2 * n, seed=SEED, passes=2, prec=prec)
            assert code == 0, (variant, prec)
            Rg = to_host(R)
            assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
            # Section 4.2's measures on the whole Q (the library's Dot2 evaluators,
            # pinned against exact arithmetic at small sizes; the CPU oracle's would
            # take minutes at millions of rows)
            orth, resid = h.orth_error(Q), h.resid_error(Ad, Q, R)
            assert orth <= 1e-13 and resid <= 1e-14, (variant, prec, orth, resid)
            # Q = A R^{-1} on sampled rows (each row one triangular solve on the host)
            Qs = np.linalg.solve(Rg.T, A[rows].T).T
            Qg = Q[torch.from_numpy(rows).to(Q.device)].cpu().numpy()
            err = np.linalg.norm(Qs - Qg, axis=1) / np.maximum(np.linalg.norm(Qs, axis=1), 1e-300)
            assert np.max(err) <= 1e3 * kappa * U, (variant, prec, np.max(err))
            # R against LAPACK's Householder R (the unique thin QR)
            rel = r_rel(Rg, Rh)
            assert rel <= R_TOL, (variant, prec, rel)
            print(f"fullsize m={m} n={n} kappa={kappa:.0e} {variant} {prec}: orth {orth:.2e} resid {resid:.2e} "
                  f"R vs Householder {rel:.2e} ({time.perf_counter() - t0:.1f} s with checks)")
            del Q, R
