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


def test_bench_line_carries_the_contract_keys(capsys):
    import json
    import types

    bench.set_config("c3")
    stages = {"sketch": 23.0, "precond_subst": 55.0, "pass_subst": 21.0, "last_apply": 8.5, "gram1_tensor": 14.0,
              "gram2_tensor": 14.0, "xr_factor": 1.3}
    path = {"ms": 138.0, "stages_ms": stages, "accuracy": {"orth": 3e-15, "resid": 2e-15},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}}
    fp64 = dict(path, ms=1084.0, stages_ms={"precond_subst": 254.0})
    main = {"ms": 138.0, "value": bench.job_value(138.0, 1), "paths": {"split": path, "fp64": fp64},
            "generation_s": 7.0, "preconditioner": {"cond_Rs": 1e12, "cond_R1": 5.5},
            "e2e": {"value": 210.0, "unit": "GB/s", "h2d_bytes_per_step": 8 * bench.M * bench.N,
                    "d2h_bytes_per_step": 8 * bench.M * bench.N + 8 * bench.N ** 2},
            "cpu_baseline": {"value": 1.1, "unit": "GB/s", "cores": 16, "kind": "oracle", "sample": "rows"}}
    args = types.SimpleNamespace(steps=10, warmup=3, variant="qr", prec="split")
    cfg = {"m": bench.M, "n": bench.N, "s": bench.S, "kappa": bench.KAPPA}
    bench._emit(args, 1, main, cfg, 1.25, {})
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline"):
        assert key in line, key
    assert line["metric"] == bench.METRIC and line["unit"] == "GB/s" and line["higher_is_better"] is True
    assert line["gpu_launches"] == 56 * 10 and line["config"]["workload"].startswith("rQR-CholeskyQR2 m=2^23")
    rl = line["roofline"]
    assert rl["bound"] == "alu" and 0 < rl["frac"] == rl["achieved"] / rl["peak"]
    assert rl["traffic"] == bench.TRAFFIC[("split", 128)][0] * bench.M / bench.TRAFFIC[("split", 128)][1]
    assert abs(line["speedup_vs_fp64"] - 1084.0 / 138.0) < 1e-12
