"""Parity of the least-squares solver of Section 5.2 (rxr_lstsq) with the CPU
oracle: both solve the normal equations of B = A R_s^{-1} with the same sketch,
so both recover a consistent system's solution within the conditioning bound
and agree with each other on inconsistent ones; several right-hand sides,
n = 1, the wide (n > 128) FP64 path, the split path above and below n = 64,
row extraction, and NaN in b are covered."""
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

OV = {"qr": o.VARIANT_QR, "lu": o.VARIANT_LU, "qr-rows": o.VARIANT_QR | o.SKETCH_ROWS}


@pytest.fixture(scope="module")
def h():
    with rxr.Handle(0) as hh:
        yield hh


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("m,n,k,kappa,variant", [(3000, 20, 1, 1e8, "qr"), (5000, 64, 3, 1e12, "lu"),
                                                 (2100, 100, 2, 1e6, "qr"), (777, 1, 1, 1.0, "qr"),
                                                 ((1 << 17) + 3, 32, 64, 1e10, "qr-rows"), (1200, 200, 1, 1e4, "qr")])
def test_lstsq_consistent_and_matches_oracle(h, prec, m, n, k, kappa, variant):
    A = usv_matrix(m, n, kappa, seed=n)
    rng = np.random.default_rng(m + n)
    Xt = rng.standard_normal((n, k))
    Bm = np.asfortranarray(A @ Xt)
    x, code = h.lstsq(to_dev(A), to_dev(Bm), variant=variant, seed=2, prec=prec)
    assert code == 0
    xg = to_host(x)
    assert np.linalg.norm(xg - Xt) / np.linalg.norm(Xt) <= 10 * max(n, 4) * kappa * U
    xo, st = o.lstsq(A, Bm, variant=OV[variant], seed=2)
    assert st == 0
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 20 * max(n, 4) * kappa * U


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_lstsq_inconsistent_matches_oracle(h, prec):
    m, n, kappa = 4000, 24, 1e5
    A = usv_matrix(m, n, kappa, seed=1)
    rng = np.random.default_rng(2)
    b = A @ rng.standard_normal(n) + 1e-6 * rng.standard_normal(m)
    x, code = h.lstsq(to_dev(A), torch.from_numpy(b).cuda(), seed=5, prec=prec)
    assert code == 0
    xo, st = o.lstsq(A, b, seed=5)
    xr = np.linalg.lstsq(A, b, rcond=None)[0]
    r = np.linalg.norm(b - A @ xr)
    bound = 200 * n * (kappa * U + kappa**2 * U * r / (np.linalg.norm(A, 2) * np.linalg.norm(xr)))
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= bound


def test_lstsq_nan_in_b(h):
    A = usv_matrix(1000, 8, 10.0, seed=3)
    b = np.ones(1000)
    b[500] = np.nan
    _, code = h.lstsq(to_dev(A), torch.from_numpy(b).cuda(), raise_on_error=False)
    assert code == rxr.NONFINITE
