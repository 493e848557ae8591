"""The benchmark workload at its full size (m = 2^22, n = 64, s = 128,
kappa = 1e10, seed 0, rQR-CholeskyQR2), in the launch configuration bench.py
times, on both paths.  The oracle cannot factorise 2^22 rows in a test's time,
so the checks are sampled outputs and properties that hold at any size:

* every sketch entry against the oracle's sketch, built from the oracle's own
  Omega draws chunk by chunk (the quantised draws for the split path), within
  the sketch's rounding bound;
* Q = A R^{-1} on sampled rows (each row one triangular solve on the host);
* R against the Householder R of LAPACK (the unique thin QR, forward error
  ~ kappa u);
* the accuracy measures of Section 4.2 on the full Q and R's structure."""
import math

import numpy as np
import pytest

import oracle as o
from gpu_util import U, to_dev, to_host
from paper_2111_11148_gb300.inputs import usv_matrix

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2111_11148_gb300 import rxr  # noqa: E402

M, N, S, KAPPA, SEED = 1 << 22, 64, 128, 1e10, 0
CHUNK = 1 << 19


@pytest.fixture(scope="module")
def setup():
    A = usv_matrix(M, N, KAPPA, seed=SEED)
    with rxr.Handle(0) as h:
        yield h, A, to_dev(A)


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


def test_fullsize_sketch_entries(setup):
    h, A, Ad = setup
    Y, Yq, absY, absYq, absq_rows = _sketch_refs(A)
    bound = 8 * (math.log2(M) + 4) * U * absY
    Yg = to_host(h.sketch(Ad, S, seed=SEED, prec="fp64"))
    assert np.all(np.abs(Yg - Y) <= bound), np.max(np.abs(Yg - Y) / bound)
    colmax = np.abs(A).max(axis=0)
    boundq = 8 * (math.log2(M) + 4) * U * absYq + 2.0**-54 * absq_rows[:, None] * colmax[None, :]
    Yqg = to_host(h.sketch(Ad, S, seed=SEED, prec="split"))
    assert np.all(np.abs(Yqg - Yq) <= boundq), np.max(np.abs(Yqg - Yq) / boundq)


@pytest.mark.parametrize("prec", ["split", "fp64"])
def test_fullsize_factorisation(setup, prec):
    h, A, Ad = setup
    Q, R, code = h.cholqr(Ad, variant="qr", s=S, seed=SEED, passes=2, prec=prec)
    assert code == 0
    Rg = to_host(R)
    assert np.all(np.diag(Rg) > 0) and np.all(np.tril(Rg, -1) == 0)
    # Section 4.2's measures on the whole Q (the library's Dot2 evaluators,
    # pinned against exact arithmetic at small sizes; the CPU oracle's would
    # take minutes at 2^22 rows)
    assert h.orth_error(Q) <= 1e-13
    assert h.resid_error(Ad, Q, R) <= 1e-14
    Qg = to_host(Q)
    # Q = A R^{-1} on sampled rows
    rng = np.random.default_rng(1)
    rows = np.concatenate([np.arange(64), rng.integers(0, M, 4000), np.arange(M - 64, M)])
    Qs = np.linalg.solve(Rg.T, A[rows].T).T
    err = np.linalg.norm(Qs - Qg[rows], axis=1) / np.maximum(np.linalg.norm(Qs, axis=1), 1e-300)
    assert np.max(err) <= 1e3 * KAPPA * U
    # R against LAPACK's Householder R (the unique thin QR)
    Rh = np.linalg.qr(A, mode="r")
    Rh = np.sign(np.diag(Rh))[:, None] * Rh
    assert np.linalg.norm(Rg - Rh) / np.linalg.norm(Rh) <= 100 * KAPPA * U
