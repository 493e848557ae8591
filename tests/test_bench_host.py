"""Host-side pieces of bench.py that need no GPU: the reference R factor it
compares every run against (the R factor of diag(sigma) V^T, which for
A = U diag(sigma) V^T with orthonormal U is A's own), the configuration table,
the CPU baseline's use of the oracle's OpenMP build, the device input
builder's recipe (run here on torch's CPU device: its singular values are the
construction's sigma and its R factor the construction's) and the launch
count the bench line claims.""" 
import numpy as np
import pytest

import bench
from gpu_util import r_rel
from paper_2111_11148_gb300.inputs import usv_matrix


@pytest.mark.parametrize("m,n,kappa", [(3000, 8, 1e4), (5000, 24, 1e12), (4000, 64, 1e15)])
def test_construction_r_is_the_r_factor_of_a(m, n, kappa):
    A = usv_matrix(m, n, kappa, seed=3)
    Rl = np.linalg.qr(A, mode="r")
    Rl = np.sign(np.diag(Rl))[:, None] * Rl
    Rc = bench.construction_r(n, kappa, 3)
    assert np.all(np.diag(Rc) > 0) and np.allclose(np.tril(Rc, -1), 0.0)
    assert r_rel(Rc, Rl) <= 1e-14


def test_configurations_match_the_workloads():
    assert bench.CONFIGS["c3"] == {"m": 2**23, "n": 128, "kappa": 1e12, "variant": "qr", "label": "m=2^23"}
    assert bench.CONFIGS["c2"]["m"] == 2**22 and bench.CONFIGS["c2"]["n"] == 64
    assert bench.CONFIGS["c1"]["m"] == 20000 and bench.CONFIGS["c1"]["variant"] == "lu"
    bench.set_config("c3")
    assert (bench.M, bench.N, bench.S) == (2**23, 128, 256)
    assert bench.b_alg(bench.M, bench.N, 2) == 8.0 * 2**23 * 128 * 5


def test_cpu_baseline_reports_both_builds(monkeypatch):
    monkeypatch.setenv("RXR_BENCH_ORACLE_ROWS", "3000")
    bench.set_config("c1")
    A = usv_matrix(4000, bench.N, 1e4, seed=0)
    line = bench.cpu_baseline(A, "lu")
    assert line["kind"] == "oracle" and line["cores"] >= 1 and line["value"] > 0
    assert line["single_thread"]["cores"] == 1
    bench.set_config("c3")


@pytest.mark.parametrize("m,n,kappa", [(4096, 16, 1e6), (3000, 40, 1e12)])
def test_device_input_recipe(m, n, kappa):
    torch = pytest.importorskip("torch")
    from paper_2111_11148_gb300.inputs import sigma_profile

    saved = (bench.M, bench.N, bench.KAPPA, bench.SEED)
    try:
        bench.M, bench.N, bench.KAPPA, bench.SEED = m, n, kappa, 5
        A = bench.make_input_device(torch.device("cpu"))
    finally:
        bench.M, bench.N, bench.KAPPA, bench.SEED = saved
    assert A.shape == (m, n) and A.stride() == (1, m)  # column-major
    a = A.numpy()
    sv = np.linalg.svd(a, compute_uv=False)
    # the computed singular values are within the SVD's own absolute error
    # (a few u ||A||, ||A|| = 1) of sigma
    assert np.all(np.abs(sv - sigma_profile(n, kappa)) <= 8 * n * 2.0**-53)
    R = np.linalg.qr(a, mode="r")
    R = np.sign(np.diag(R))[:, None] * R
    assert r_rel(R, bench.construction_r(n, kappa, 5)) <= 1e-13


def test_launch_count_of_the_split_factorisation():
    # m = 2^23, n = 128: sketch + reduce, blocked XR (4 panels, 3 V^T C, 3 updates,
    # finish), record prep + fused substitution, Gram + reduce, blocked Cholesky
    # (init, 4 diagonal, 3 panel, 3 update, R product) twice, the middle pass's
    # inverse, estimate, three products and fallback pair, Gram + reduce, the last
    # pass's inverse, selection, correction and fallback pair, copy
    assert bench.launches_per_step("split", 128, 2**23) == 2 + 11 + 2 + 2 + 12 + 7 + 2 + 12 + 5 + 1
    assert bench.launches_per_step("split", 64, 2**22) == 19
    assert bench.launches_per_step("fp64", 64, 2**22) == 11
