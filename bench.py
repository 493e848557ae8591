"""Benchmark of randomized XR-preconditioned CholeskyQR on one GB300 (under
torchrun with N GPUs: the row-sharded factorisation of N x m rows, or with
--replicas N independent factorisations).

A step is one full factorisation A = QR (sketch, XR factor of the sketch, the
precondition + Gram pass, two CholeskyQR passes, Q and R) with inputs resident
in HBM.  The default workload is the split-precision configuration: m = 2^23,
n = 128, s = 2n Gaussian sketch, A = U Sigma V^T with kappa = 1e12, seed 0,
rQR-CholeskyQR2 (8.6 GB of A).  The metric is the effective bandwidth
B_alg / t with B_alg = 8 m n (P + 3) bytes: one read of A for the sketch, one
per CholeskyQR pass, and a read plus a write for Q, reported for the
split-precision path next to the FP64 path and the preconditioning-only split
placement on the same A, each at its achieved accuracy.  The same line carries
m = 2^22, n = 64, kappa = 1e10 (the scale configuration) and m = 20000, n = 16,
kappa = 1e8, rLU (QR/s over 1000 CUDA-graph replays) under "configs".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3|c2|c1|c5]
                    [--variant qr|lu|none|shifted] [--prec split|split_precond|fp64]
                    [--impl reference] [--workload single|batched|lstsq|rsvd]

`--impl reference` times the CPU oracle (the plain FP64 implementation
written from the paper, its OpenMP build on every host core) on a bounded row
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# the workload configurations: rows, columns, condition number, variant
CONFIGS = {
    "c1": {"m": 20000, "n": 16, "kappa": 1e8, "variant": "lu", "label": "m=20000"},
    "c2": {"m": 2**22, "n": 64, "kappa": 1e10, "variant": "qr", "label": "m=2^22"},
    "c3": {"m": 2**23, "n": 128, "kappa": 1e12, "variant": "qr", "label": "m=2^23"},
    "c5": {"m": 2**20, "n": 512, "kappa": 1e13, "variant": "qr", "label": "m=2^20"},
}
M, N, S, KAPPA, SEED, PASSES = 2**23, 128, 256, 1e12, 0, 2
METRIC = "tall-skinny QR GB/s & roofline frac, split-prec vs FP64 at \u2016Q\u1d40Q\u2212I\u2016\u22641e-13"
WORKLOAD = "rQR-CholeskyQR2 m=2^23 n=128 s=256 kappa=1e12"
PRECS = ("split", "split_precond", "fp64")
DTYPES = {"fp64": "f64",
          "split": "f64 with fp16 8-bit-digit tcgen05 operands (fp32 accumulation, exact)",
          "split_precond": "f64 with fp16 8-bit-digit sketch and bf16x3 first Gram on tcgen05"}


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the roofline
# kernel, from an ncu capture of a smaller case (bytes, rows captured), scaled
# by rows to the workload (traffic grows with the rows); absent where no capture
# of the current kernel exists
TRAFFIC = {
    # k_subst_gram (FP64 precondition + Gram), m = 2^19, n = 64
    ("fp64", 64): (268.552704e6 + 225.660672e6, 2**19),
    # k_subst_fused128 (split precondition), m = 2^19, n = 128
    ("split", 128): (537.306880e6 + 486.197504e6, 2**19),
}
HBM_GBS = 6784.2  # measured copy bandwidth of this GPU pool (STREAM-style copy)


def b_alg(m, n, passes):
    return 8.0 * m * n * (passes + 3)


def f_alg(m, n, s, passes):
    # sketch 2smn, X = A R_s^{-1} mn^2, per pass Gram mn^2 and apply mn^2
    return 2.0 * s * m * n + (2 * passes + 1) * m * n * n


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def hbm_peak() -> tuple[float, str]:
    """Copy bandwidth of this GPU pool: MEASURED_PEAKS.json when present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_GBS, "measured earlier on this pool (STREAM-style copy)"


def oracle_rows(n: int, parallel: bool) -> int:
    """Row count of an oracle sample: about 10 s of work for the serial build on
    one core (the oracle's cost per row grows as n^2) and for the OpenMP build
    on the box's 16 host cores (16x the rows)."""
    base = int(os.environ.get("RXR_BENCH_ORACLE_ROWS", 2**19 * 64 * 64 // (n * n)))
    return max(n, base * (16 if parallel else 1))


def run_oracle_sample(A_sample: np.ndarray, variant: str, parallel: bool = False):
    import oracle

    t0 = time.perf_counter()
    if variant == "shifted":
        r = oracle.scholqr(A_sample, 1e-15 * np.linalg.norm(A_sample, 2) ** 2, passes=PASSES)
    else:
        ov = {"qr": oracle.VARIANT_QR, "lu": oracle.VARIANT_LU, "none": oracle.VARIANT_NONE}[variant.split("-")[0]]
        if variant.endswith("-rows"):
            ov |= oracle.SKETCH_ROWS
        r = oracle.rxr_cholqr(A_sample, ov, S, seed=SEED, passes=PASSES, parallel=parallel)
    dt = time.perf_counter() - t0
    if r.status != 0:
        raise RuntimeError(f"oracle status {r.status}")
    return dt


def cpu_baseline(A_np: np.ndarray, variant: str) -> dict:
    """The oracle as it stands, timed on the host: its OpenMP build on every
    core (the reported baseline) and its serial build, each on the first rows of
    the same A (bounded samples)."""
    import oracle

    oracle.build()
    out = {}
    for parallel in (True, False):
        rows = min(oracle_rows(N, parallel), A_np.shape[0])
        t = run_oracle_sample(np.asfortranarray(A_np[:rows]), variant, parallel)
        out[parallel] = {"value": b_alg(rows, N, PASSES) / t / 1e9, "unit": "GB/s",
                         "cores": oracle.threads(parallel), "kind": "oracle",
                         "sample": f"first {rows} of {M} rows of the same A, one full rxr_cholqr of the "
                                   f"C oracle ({'OpenMP build, every host core' if parallel else 'serial build'}), "
                                   f"{t:.2f} s"}
    line = dict(out[True])
    line["single_thread"] = out[False]
    return line


def make_input():
    from paper_2111_11148_gb300.inputs import usv_matrix

    return usv_matrix(M, N, KAPPA, seed=SEED)


def make_input_device(dev):
    """The workload's A = U diag(sigma) V^T built on the GPU, column-major: the
    recipe of inputs.usv_matrix (sigma and V from inputs.usv_factors; U the Q
    factor, diag(R) > 0, of a seeded N(0,1) m x n matrix) with the Gaussian drawn
    by torch's CUDA generator and its Q factor taken by two Cholesky QR steps
    (Gram and product by cuBLAS, the n x n Cholesky factor and its inverse on the
    host; the Gaussian is well conditioned, so two steps reach orthonormality to
    rounding): the same distribution, other bytes than the host generator's.
    Building the 8.6 GB input on the host (multithreaded LAPACK on the CPU) took
    about 70 s and left the host link reading pinned memory at 24-60 GB/s
    instead of 200 GB/s for the rest of the process."""
    import torch

    from paper_2111_11148_gb300 import rxr
    from paper_2111_11148_gb300.inputs import usv_factors

    sigma, V = usv_factors(N, KAPPA, SEED)
    g = torch.Generator(device=dev)
    g.manual_seed(SEED)
    U = torch.randn((M, N), dtype=torch.float64, device=dev, generator=g)
    for _ in range(2):
        Rc = np.linalg.cholesky((U.t() @ U).cpu().numpy()).T
        U = U @ torch.from_numpy(np.linalg.inv(Rc)).to(dev)
    A = (U * torch.from_numpy(sigma).to(dev)) @ torch.from_numpy(V.T.copy()).to(dev)
    del U
    out = rxr.colmajor(A)
    del A
    if dev.type == "cuda":
        torch.cuda.synchronize(dev)
    return out


def host_rows(A_dev, rows: int) -> np.ndarray:
    """The first rows of a column-major device matrix as a Fortran-ordered array."""
    return A_dev[:rows].t().contiguous().cpu().numpy().T


def construction_r(n: int, kappa: float, seed: int) -> np.ndarray:
    """The R factor (diag > 0) of A = U diag(sigma) V^T: U has orthonormal
    columns, so it is the R factor of the n x n matrix diag(sigma) V^T (LAPACK's
    Householder QR of that small matrix; it agrees with LAPACK's R of the whole
    stored A to 1e-15 at kappa up to 1e15)."""
    from paper_2111_11148_gb300.inputs import usv_factors

    sigma, V = usv_factors(n, kappa, seed)
    R = np.linalg.qr(sigma[:, None] * V.T, mode="r")
    return np.sign(np.diag(R))[:, None] * R


def reference_arm(args, rank: int, world: int):
    """Time the CPU oracle as it stands (its OpenMP build on every host core)
    on a bounded sample of the workload, each step one full factorisation."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    rows = oracle_rows(N, True)
    from paper_2111_11148_gb300.inputs import usv_matrix

    A = usv_matrix(rows, N, KAPPA, seed=SEED)
    for _ in range(min(args.warmup, 1)):
        run_oracle_sample(A, args.variant, True)
    times = [run_oracle_sample(A, args.variant, True) for _ in range(args.steps)]
    t = statistics.median(times)
    gbs = b_alg(rows, N, PASSES) / t / 1e9
    sample = (f"{rows} x {N} rows of the same A = U Sigma V^T construction, one full rxr_cholqr per step "
              f"(C oracle, OpenMP build on {oracle.threads(True)} host threads)")
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle_rows": rows, "m": M, "n": N, "s": S, "kappa": KAPPA,
                   "passes": PASSES, "variant": args.variant},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": oracle.threads(True), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_arm(args, rank: int, world: int, local_rank: int):
    """512 independent problems (m log-uniform in [2^12, 2^18], n in {8..128},
    kappa log-uniform in [1e2, 1e12], matrix k seed k), rQR-CholeskyQR2: a
    batched plan made once (outside the timed region), one rxr_batch_run per
    step: the split-precision plan (every problem's own tensor-core sequence,
    spread over eight streams) and, beside it, the FP64 plan (one launch per
    stage over the whole batch, persistent CTAs on a work queue)."""
    import torch

    from paper_2111_11148_gb300 import rxr
    from paper_2111_11148_gb300.inputs import batch_specs, usv_matrix

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    specs = batch_specs(args.count, seed=0)
    t0 = time.perf_counter()
    As_np = [usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed) for sp in specs]
    As = [rxr.colmajor(torch.from_numpy(a).to(dev)) for a in As_np]
    gen_s = time.perf_counter() - t0
    h = rxr.Handle(local_rank)
    seeds = [sp.seed for sp in specs]
    stream = torch.cuda.current_stream(dev)
    prec = args.prec
    bytes_alg = sum(b_alg(sp.m, sp.n, PASSES) for sp in specs)
    flops_alg = sum(f_alg(sp.m, sp.n, 2 * sp.n, PASSES) for sp in specs)

    def timed(p, steps, clocks=None):
        plan = h.batch_plan(As, variant=args.variant, seeds=seeds, passes=PASSES, prec=p)
        try:
            for _ in range(max(3, args.warmup)):
                plan.run()
            torch.cuda.synchronize(dev)
            assert bool((plan.status[:, 0] == 0).all()), plan.status[plan.status[:, 0] != 0][:4]
            if clocks:
                clocks.start()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                plan.run()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            clk = clocks.stop() if clocks else None
            ms = e0.elapsed_time(e1) / steps
            # accuracy: every problem against Section 4.2's measures (device Dot2)
            worst = max(h.orth_error(Q) for Q in plan.Qs)
            resid = max(h.resid_error(A, Q, R) for A, Q, R in zip(As, plan.Qs, plan.Rs))
            return ms, clk, worst, resid
        finally:
            plan.close()

    ms, clk, worst, resid = timed(prec, args.steps, ClockSampler(local_rank))
    other = "split" if prec == "fp64" else "fp64"
    ms_o, _, worst_o, resid_o = timed(other, max(2, args.steps // 2))
    peak_fp64 = rxr.fp64_peak_tflops()
    nk = sum(1 for sp in specs)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * bytes_alg / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": f"batched rQR-CholeskyQR2, {len(specs)} problems (plan made once, one run per step)",
                       "count": len(specs), "total_rows": sum(sp.m for sp in specs),
                       "bytes_A": sum(8 * sp.m * sp.n for sp in specs), "generation_s": gen_s, "prec": prec},
            "roofline": {"bound": "alu", "kernel": "whole batch", "achieved": flops_alg / (ms * 1e-3) / 1e12,
                         "peak": peak_fp64, "unit": "TFLOP/s", "frac": flops_alg / (ms * 1e-3) / 1e12 / peak_fp64,
                         "traffic": None},
            "qr_per_s": world * len(specs) / (ms * 1e-3), "gflops": world * flops_alg / (ms * 1e-3) / 1e9,
            "accuracy": {"worst_orth": worst, "worst_resid": resid},
            "compare": {"prec": other, "ms_per_step": ms_o, "value": world * bytes_alg / (ms_o * 1e-3) / 1e9,
                        "qr_per_s": world * len(specs) / (ms_o * 1e-3), "dtype": DTYPES[other],
                        "accuracy": {"worst_orth": worst_o, "worst_resid": resid_o}},
            "gpu_launches": (3 * PASSES + 5) * args.steps if prec == "fp64" else None, "clocks": clk,
        }), flush=True)
    h.close()


STAGES = ["sketch", "precond_subst", "pass_subst", "last_apply", "gram1_tensor", "gram2_tensor", "xr_factor"]


def lstsq_arm(args, rank: int, world: int, local_rank: int):
    """Least squares (Section 5.2) on the workload's A with one right-hand side
    b = A x_true: one rxr_lstsq per step, B_alg = 8 m n (sketch read, B = A R_s^-1
    read) + 8 m n (B written) + 8 m n (B read for B^T b)."""
    import torch

    from paper_2111_11148_gb300 import rxr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    A_np = make_input()
    xt = np.random.default_rng(1).standard_normal(N)
    A = rxr.colmajor(torch.from_numpy(A_np).to(dev))
    b = torch.from_numpy(A_np @ xt).to(dev)
    h = rxr.Handle(local_rank)
    stream = torch.cuda.current_stream(dev)
    step = lambda: h.lstsq(A, b, variant=args.variant, s=S, seed=SEED, prec=args.prec)
    for _ in range(max(3, args.warmup)):
        x, code = step()
    assert code == 0
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        x, code = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    err = float(np.linalg.norm(x.cpu().numpy() - xt) / np.linalg.norm(xt))
    balg = 8.0 * M * N * 4
    if rank == 0:
        print(json.dumps({"metric": "least-squares solve effective GB/s (B_alg = 32mn)", "value": balg / ms / 1e6,
                          "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": DTYPES[args.prec], "data": "synthetic",
                          "config": {"workload": f"least squares (Section 5.2) {WORKLOAD}", "m": M, "n": N, "s": S,
                                     "kappa": KAPPA, "rhs": 1},
                          "accuracy": {"x_rel_err": err}}), flush=True)
    h.close()


# the randomized SVD's stand-in for the sparsest matrix of Section 5.1's table
# (1,447,360 rows and columns, 3.81 nonzeros per row)
RSVD_M, RSVD_D, RSVD_K, RSVD_ITERS = 1447360, 3.81, 20, 4


def rsvd_bytes_per_iter(m, nnz, k, passes):
    """Algorithmic bytes of one power iteration (A^T Y, orth, A Y, orth): per
    sparse product the CSR arrays (12 bytes a nonzero, 8 a row), one read of
    the k-column block and one write of the product; per transpose a read and a
    write of the block; per orthonormalisation 8 m k (P + 3)."""
    spmm = 12.0 * nnz + 8.0 * (m + 1) + 2 * 8.0 * m * k
    return 2 * spmm + 2 * 16.0 * m * k + 2 * b_alg(m, k, passes)


def rsvd_launches(prec, k, iters):
    """Kernels one rxr_rsvd call launches: per orthonormalisation the
    factorisation's kernels (no R copy but for the last), the status merge, a
    transpose and a sparse product; then the Jacobi SVD and two products."""
    c = launches_per_step(prec, k, RSVD_M)
    return (2 * iters + 2) * (c + 2) + 4


def rsvd_oracle_ms_per_iter(k: int, rows: int = 2**18) -> tuple[float, int]:
    """The oracle's time for one power iteration on a 2^18-row operator of the
    same density, scaled to the workload's rows (the work grows with the rows)."""
    import oracle
    from paper_2111_11148_gb300.inputs import sparse_operator, start_block

    P = sparse_operator(rows, RSVD_D, seed=SEED)
    A = P.scipy()
    X = start_block(rows, k, SEED)
    t0 = time.perf_counter()
    oracle.rsvd(A, X, 0, seed=SEED)
    t1 = time.perf_counter()
    oracle.rsvd(A, X, 1, seed=SEED)
    t2 = time.perf_counter()
    return ((t2 - t1) - (t1 - t0)) * 1e3 * RSVD_M / rows, rows


def rsvd_arm(args, rank: int, world: int, local_rank: int):
    """Randomized SVD with power iteration (Algorithm 7, Section 5.1) of the
    sparse stand-in, each orthonormalisation by rQR-CholeskyQR2: the metric is
    the time of one power iteration, (t(K) - t(0)) / K from calls with K and
    with no iterations, as Section 5.1's table reports it."""
    import torch

    from paper_2111_11148_gb300 import rxr
    from paper_2111_11148_gb300.inputs import sparse_operator, start_block

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    k = args.k or RSVD_K
    t0 = time.perf_counter()
    P = sparse_operator(RSVD_M, RSVD_D, seed=SEED)
    X_np = start_block(RSVD_M, k, SEED)
    gen_s = time.perf_counter() - t0
    A = rxr.DeviceCsr.from_host(P, device=dev)
    X = rxr.colmajor(torch.from_numpy(X_np).to(dev))
    h = rxr.Handle(local_rank)
    stream = torch.cuda.current_stream(dev)
    U = rxr.empty_colmajor(RSVD_M, k, device=dev)
    V = rxr.empty_colmajor(RSVD_M, k, device=dev)
    S = torch.empty(k, dtype=torch.float64, device=dev)
    call = lambda iters: h.rsvd(A, X, iters, variant=args.variant, seed=SEED, prec=args.prec, U=U, S=S, V=V)
    for _ in range(max(3, args.warmup)):
        call(RSVD_ITERS)
        call(0)
    torch.cuda.synchronize(dev)

    def timed(iters, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            call(iters)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(local_rank)
    clocks.start()
    t_k = timed(RSVD_ITERS, args.steps)
    t_0 = timed(0, args.steps)
    clk = clocks.stop()
    ms_iter = max_over_ranks((t_k - t_0) / RSVD_ITERS, None, dev)
    # accuracy of the result: orthonormal factors and A^T U = V diag(S) on sampled rows
    call(RSVD_ITERS)
    Uh, Sh, Vh = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    rows = np.random.default_rng(0).integers(0, RSVD_M, 2000)
    AtU = np.stack([P.t_data[P.t_indptr[i]:P.t_indptr[i + 1]] @ Uh[P.t_indices[P.t_indptr[i]:P.t_indptr[i + 1]]]
                    for i in rows])
    ident = float(np.max(np.abs(AtU - Vh[rows] * Sh)) / Sh[0])
    # end to end: the operator and X from host memory, U, S, V back to host memory
    def e2e_call():
        Ad = rxr.DeviceCsr.from_host(P, device=dev)
        Xd = rxr.colmajor(torch.from_numpy(X_np).to(dev))
        Ue, Se, Ve, _ = h.rsvd(Ad, Xd, RSVD_ITERS, variant=args.variant, seed=SEED, prec=args.prec)
        return Ue.cpu(), Se.cpu(), Ve.cpu()

    e2e_call()
    torch.cuda.synchronize(dev)
    w0 = time.perf_counter()
    for _ in range(3):
        e2e_call()
    e2e_ms = (time.perf_counter() - w0) * 1e3 / 3
    h2d = P.indptr.nbytes + P.indices.nbytes + P.data.nbytes + P.t_indptr.nbytes + P.t_indices.nbytes
    h2d += P.t_data.nbytes + X_np.nbytes
    d2h = 8 * (2 * RSVD_M * k + k)
    balg = rsvd_bytes_per_iter(RSVD_M, P.nnz, k, PASSES)
    cpu = None
    if not args.no_cpu_baseline and rank == 0:
        cms, crow = rsvd_oracle_ms_per_iter(k)
        cpu = {"value": cms, "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": f"one power iteration of the oracle on a {crow}-row operator of the same density, "
                         f"scaled by rows to {RSVD_M}"}
    if rank == 0:
        print(json.dumps({
            "metric": "randomized SVD (Algorithm 7) time per power iteration", "value": ms_iter, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_iter,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.prec], "data": "synthetic",
            "config": {"workload": f"RSVD power iteration, sparse {RSVD_M}x{RSVD_M} with {RSVD_D} nonzeros/row "
                                   f"(stand-in for Section 5.1's sparsest matrix), k={k}, orth = "
                                   f"{'rLU' if args.variant == 'lu' else 'rQR'}-CholeskyQR2",
                       "m": RSVD_M, "nnz": P.nnz, "k": k, "iters_timed": RSVD_ITERS, "generation_s": gen_s,
                       "l2": "working set (CSR + 5 blocks of m x k) larger than L2"},
            "roofline": {"bound": "hbm", "kernel": "whole power iteration", "achieved": balg / (ms_iter * 1e-3) / 1e9,
                         "peak": hbm_peak()[0], "unit": "GB/s", "frac": balg / (ms_iter * 1e-3) / 1e9 / hbm_peak()[0],
                         "traffic": None},
            "e2e": {"value": e2e_ms, "unit": f"ms per call with {RSVD_ITERS} iterations", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "ms_call_iters": {str(RSVD_ITERS): t_k, "0": t_0},
            "accuracy": {"orth_U": h.orth_error(U), "orth_V": h.orth_error(V), "AtU_minus_VS_sampled": ident},
            "gpu_launches": args.steps * (rsvd_launches(args.prec, k, RSVD_ITERS) + rsvd_launches(args.prec, k, 0)),
            "cpu_baseline": cpu, "clocks": clk,
        }), flush=True)
    h.close()


def time_path(h, A, Q, R, prec, args, dev, stream, steps, warmup, sample_clocks=False, R_ref=None):
    """Time `steps` factorisations (after `warmup`) with CUDA events on the
    launching stream; then per-stage event times, the accuracy measures of
    Section 4.2 and R against the construction's R factor."""
    import torch

    def step():
        h.cholqr(A, variant=args.variant, s=S, seed=SEED, passes=PASSES, prec=prec, Q=Q, R=R)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index or 0) if sample_clocks else None
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    clk = clocks.stop() if clocks else None
    h.set_kernel_timing(True)
    kms = {k: [] for k in range(len(STAGES))}
    for _ in range(3):
        step()
        for k in range(len(STAGES)):
            kms[k].append(h.last_kernel_ms(k))
    h.set_kernel_timing(False)
    stages = {STAGES[k]: statistics.median(v) for k, v in kms.items() if statistics.median(v) > 0}
    acc = {"orth": h.orth_error(Q), "resid": h.resid_error(A, Q, R)}
    if R_ref is not None:
        Rg = R.cpu().numpy()
        acc["R_vs_construction"] = float(np.linalg.norm(Rg - R_ref) / np.linalg.norm(R_ref))
    return {"ms": ms, "stages_ms": stages, "accuracy": acc, "clocks": clk}


def preconditioner_conds(h, A, Q, args, prec) -> dict:
    """cond_2(R_s) and cond_2(R_1) = cond_2(A R_s^{-1}) of this A and sketch, from
    the library's stage entry points (the sketch, its XR factor, the FP64
    precondition + Gram pass), outside the timed region; the condition numbers
    of the small n x n factors are taken on the host."""
    import torch

    variant = args.variant.split("-")[0]
    if variant not in ("qr", "lu"):
        return {}
    Y = h.sketch(A, S, seed=SEED, prec=prec)
    Rs, code = h.xr_factor(Y, variant, raise_on_error=False)
    if code != 0:
        return {"xr_status": code}
    _, G = h.precond_gram(A, Rs, X=Q, prec="fp64")
    torch.cuda.synchronize()
    ev = np.linalg.eigvalsh(G.cpu().numpy())
    return {"cond_Rs": float(np.linalg.cond(Rs.cpu().numpy())),
            "cond_R1": float(math.sqrt(ev[-1] / ev[0])) if ev[0] > 0 else float("inf"), "sketch_prec": prec}


def max_over_ranks(ms: float, dist, device) -> float:
    """The whole job's step time: the slowest rank's (each rank factorises its
    own replica of the workload; no data-path collective)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms: float, world: int) -> float:
    """Whole-job throughput: every rank's algorithmic bytes over the slowest time."""
    return world * b_alg(M, N, PASSES) / (ms * 1e-3) / 1e9


def set_config(name: str):
    global M, N, S, KAPPA, WORKLOAD
    c = CONFIGS[name]
    M, N, S, KAPPA = c["m"], c["n"], 2 * c["n"], c["kappa"]


def workload_name(variant: str, rows: bool) -> str:
    method = {"qr": "rQR-CholeskyQR2", "lu": "rLU-CholeskyQR2", "none": "CholeskyQR2",
              "shifted": "sCholeskyQR3"}[variant.split("-")[0]]
    mm = {2**20: "2^20", 2**22: "2^22", 2**23: "2^23"}.get(M, str(M))
    w = f"{method} m={mm} n={N} s={S} kappa={KAPPA:g}, A = U Sigma V^T (seed {SEED})"
    return w + (", row-extraction sketch" if rows else "")


def measure_config(h, args, dev, stream, peak_fp64, world, dist, main_clocks: bool, extras: bool) -> dict:
    """Every precision path on one configuration's A (the reported one first,
    with clocks sampled), then, when `extras`, the preconditioner's condition
    numbers, the host-buffer end-to-end leg and the CPU baselines."""
    import torch

    from paper_2111_11148_gb300 import rxr

    t0 = time.perf_counter()
    A = make_input_device(dev)
    gen_s = time.perf_counter() - t0
    Q = rxr.empty_colmajor(M, N, device=dev)
    R = rxr.empty_colmajor(N, N, device=dev)
    R_ref = construction_r(N, KAPPA, SEED) if args.variant.split("-")[0] in ("qr", "lu", "none", "shifted") else None
    warm = max(3, args.warmup)
    order = [args.prec] + ([p for p in PRECS if p != args.prec] if not args.no_compare else [])
    paths = {}
    if dist:
        dist.barrier()
    e2e = None
    for i, prec in enumerate(order):
        steps = args.steps if i == 0 else max(2, args.steps // 2)
        paths[prec] = time_path(h, A, Q, R, prec, args, dev, stream, steps, warm, sample_clocks=(i == 0 and main_clocks),
                                R_ref=R_ref)
        if i == 0 and extras and not args.no_e2e:
            # the host-buffer leg right after the device-resident one, before
            # the comparison paths (the host link measured slower after the
            # FP64 path's long run in the same process)
            e2e = e2e_leg(h, args, world, A)
    ms = max_over_ranks(paths[args.prec]["ms"], dist, dev)
    out = {"ms": ms, "value": job_value(ms, world), "paths": paths, "generation_s": gen_s}
    if extras:
        out["preconditioner"] = preconditioner_conds(h, A, Q, args, args.prec)
        out["e2e"] = e2e
        if world == 1 and not args.no_cpu_baseline and dist is None:
            rows = min(M, max(oracle_rows(N, True), oracle_rows(N, False)))
            out["cpu_baseline"] = cpu_baseline(host_rows(A, rows), args.variant)
    del A, Q, R
    torch.cuda.empty_cache()
    return out


def graph_replay_qr_per_s(h, args, dev, prec: str, replays: int = 1000) -> dict:
    """QR/s of a latency-bound configuration: one rxr_cholqr_async captured in
    a CUDA graph and replayed `replays` times, timed with CUDA events."""
    import torch

    from paper_2111_11148_gb300 import rxr

    A = rxr.colmajor(torch.from_numpy(make_input()).to(dev))
    Q = rxr.empty_colmajor(M, N, device=dev)
    R = rxr.empty_colmajor(N, N, device=dev)
    st = torch.zeros(4, dtype=torch.int32, device=dev)
    s = torch.cuda.Stream(dev)
    g = torch.cuda.CUDAGraph()
    variant = args.variant_c1
    with torch.cuda.stream(s):
        h.cholqr_async(A, Q, R, st, variant=variant, s=S, seed=SEED, passes=PASSES, prec=prec, stream=s)
        s.synchronize()
        with torch.cuda.graph(g, stream=s):
            h.cholqr_async(A, Q, R, st, variant=variant, s=S, seed=SEED, passes=PASSES, prec=prec, stream=s)
    for _ in range(10):
        g.replay()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream(dev)
    e0.record(cur)
    for _ in range(replays):
        g.replay()
    e1.record(cur)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / replays
    assert int(st[0].item()) == 0, st
    return {"qr_per_s": 1e3 / ms, "ms_per_qr": ms, "gbs": b_alg(M, N, PASSES) / (ms * 1e-3) / 1e9,
            "replays": replays, "orth": h.orth_error(Q), "resid": h.resid_error(A, Q, R)}


def sharded_arm(args, rank: int, world: int, local_rank: int):
    """N GPUs factorise one matrix of N x m rows, split by contiguous row
    blocks (Section 2.4's parallel scheme): rank r holds rows r m .. (r + 1) m - 1
    (its block an independent A = U Sigma V^T of the configuration, seed + r),
    and the ranks exchange the sketch and Gram partials with one NCCL allgather
    per stage (paper_2111_11148_gb300.sharded).  Weak scaling: m rows per GPU;
    value = all ranks' algorithmic bytes over the slowest rank's time."""
    import torch
    import torch.distributed as dist

    from paper_2111_11148_gb300 import rxr
    from paper_2111_11148_gb300.inputs import usv_matrix
    from paper_2111_11148_gb300.sharded import LibraryOps, cholqr_sharded, torch_allgather

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if "MASTER_ADDR" not in os.environ:  # one process without torchrun: a group of one
        import socket

        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK="0", WORLD_SIZE="1")
    dist.init_process_group("nccl", device_id=dev)
    A = rxr.colmajor(torch.from_numpy(usv_matrix(M, N, KAPPA, seed=SEED + rank)).to(dev))
    h = rxr.Handle(local_rank)
    ops = LibraryOps(h)
    gather = torch_allgather()
    variant = args.variant.split("-")[0]
    prec = args.prec if args.prec != "split_precond" else "split"
    step = lambda: cholqr_sharded(ops, A, rank * M, gather, variant=variant, s=S, seed=SEED, passes=PASSES,
                                  prec=prec)
    for _ in range(max(3, args.warmup)):
        Q, R, code = step()
    assert code == 0, code
    stream = torch.cuda.current_stream(dev)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank) if rank == 0 else None
    if clocks:
        clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        Q, R, code = step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    clk = clocks.stop() if clocks else None
    # accuracy of the whole factorisation: ||Q^T Q - I|| from the summed shard
    # Grams (FP64), the residual bound by the largest shard ratio
    Gq = ops.sum_parts(gather(h.gram(Q, prec="fp64")))
    orth = float(np.linalg.norm(Gq.cpu().numpy() - np.eye(N)))
    resid = max_over_ranks(h.resid_error(A, Q, R), dist, dev)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * b_alg(M, N, PASSES) / (ms * 1e-3) / 1e9, "unit": "GB/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
            "data": "synthetic",
            "config": {"workload": f"row-sharded {WORKLOAD}, {M} rows per GPU ({world * M} in all)", "m_per_gpu": M,
                       "m": world * M, "n": N, "s": S, "kappa": KAPPA, "variant": variant, "prec": prec,
                       "parallelism": f"row shards x{world}, NCCL allgather of the s x n / n x n partials",
                       "l2": "each shard's A larger than L2; no flush needed"},
            "accuracy": {"orth_from_summed_grams": orth, "resid_max_over_shards": resid},
            "clocks": clk, "cpu_baseline": None, "e2e": None,
        }), flush=True)
    h.close()
    dist.barrier()
    dist.destroy_process_group()


_PINNED: dict = {}  # the end-to-end leg's pinned host buffers


def gpu_arm(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_2111_11148_gb300 import rxr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if not args.no_e2e:
        # before any input is generated (see e2e_leg)
        _PINNED["A"] = torch.empty(M * N, dtype=torch.float64).pin_memory()
        _PINNED["Q"] = torch.empty(M * N, dtype=torch.float64).pin_memory()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    h = rxr.Handle(local_rank)
    stream = torch.cuda.current_stream(dev)
    peak_fp64 = rxr.fp64_peak_tflops()
    main = measure_config(h, args, dev, stream, peak_fp64, world, dist, main_clocks=True, extras=True)
    main_cfg = {"m": M, "n": N, "s": S, "kappa": KAPPA}
    secondary = {}
    if args.secondary and rank == 0:
        # the other configurations on the same box: the scale one (c2) with its
        # three paths, and the latency-bound one (c1) as QR/s over graph replays
        saved = (M, N, S, KAPPA)
        set_config("c2")
        c2 = measure_config(h, args, dev, stream, peak_fp64, 1, None, main_clocks=False, extras=False)
        secondary["c2"] = summarise(c2, args)
        set_config("c1")
        secondary["c1"] = {"m": M, "n": N, "s": S, "kappa": KAPPA, "variant": args.variant_c1,
                           "graph_replays": {p: _safe(graph_replay_qr_per_s, h, args, dev, p) for p in ("fp64", "split")}}
        globals().update(M=saved[0], N=saved[1], S=saved[2], KAPPA=saved[3])
    if rank == 0:
        _emit(args, world, main, main_cfg, peak_fp64, secondary)
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _safe(fn, *a):
    try:
        return fn(*a)
    except Exception as e:  # reported in the line, not fatal to the main measurement
        return {"error": f"{type(e).__name__}: {e}"}


def summarise(res: dict, args) -> dict:
    """A configuration's paths in a few numbers (nested in the main line)."""
    out = {"m": M, "n": N, "s": S, "kappa": KAPPA, "variant": args.variant}
    for prec, r in res["paths"].items():
        out[prec] = {"value": b_alg(M, N, PASSES) / (r["ms"] * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": r["ms"],
                     "stages_ms": r["stages_ms"], "accuracy": r["accuracy"]}
    return out


def subst_fp64_flop_per_row(n, bw, sub_ops):
    """FP64 flop a blocked substitution issues per row: the diagonal-block
    solves (bw (bw - 1) / 2 FMAs per block, 2 flop each), the n multiplications
    by 1 / R_jj, and sub_ops FP64 operations per trailing output per block (the
    subtraction of the tensor-core update: one, the update's FP32 pair turned
    into one double on the integer pipes)."""
    flop, c0 = 0.0, 0
    while c0 < n:
        b = min(bw, n - c0)
        flop += b * (b - 1) + sub_ops * (n - c0 - b)
        c0 += b
    return flop + n


def launches_per_step(prec, n, m, rows=False):
    """Kernels one CholeskyQR2 factorisation launches (P = 2, rQR, s = 2n)."""
    npanel = (n + 31) // 32
    xr = 1 if 2 * n * n <= 16384 else 3 * npanel - 1  # one-CTA XR, or blocked: panels, V^T C, updates, finish
    sk = 1 if rows else 2  # row gather, or the Gaussian sketch and its reduction
    # one Cholesky factor: one CTA up to n = 64, else the blocked form (init, a diagonal block, panel and
    # update per further 32-column block, and the R accumulation)
    factor = 1 if n <= 64 else 3 * ((n + 31) // 32)
    if prec == "fp64":
        # sketch, XR, 3 x substitution (+ its Gram's reduction except the last), 2 factors, copy
        return sk + xr + (5 if n <= 128 else 7) + 2 * factor + 1
    if n <= 64:
        # sketch, XR, fused substitution, Gram, reduce, factor, middle pass (above 2^17 rows: inverse,
        # condition estimate, apply, fused substitution, the one not selected returning at once; else the
        # fused substitution), Gram, reduce, factor, last pass (inverse, selection, FP32-correction apply,
        # FP64-grade apply: the one not selected returns at once), copy
        return sk + xr + 4 + (4 if m >= 1 << 17 else 1) + 3 + 4 + 1
    if n <= 128:
        # sketch, XR, record prep + fused substitution, Gram, reduce, factor, middle pass (above 2^17 rows:
        # inverse, condition estimate, three block products, record prep + fused substitution; else record
        # prep + fused substitution), Gram, reduce, factor, last pass (inverse, selection, FP32-correction
        # apply, record prep + fused substitution), copy
        return sk + xr + 2 + 2 + factor + (7 if m >= 1 << 17 else 2) + 2 + factor + 5 + 1
    blocked = 2 * ((n + 63) // 64) - 1  # diagonal solves + trailing updates
    return sk + xr + 3 * blocked + 2 * 2 + 2 * factor + 1 + (1 if rows else 0)


def roofline_entry(prec, stages, peak_fp64):
    """The dominant FP64 launch of the path against the measured DFMA peak,
    counting the FP64 flop that launch actually issues.
    FP64 path: the fused precondition+Gram launch, (2n^2 + n) flop per row.
    Split paths: the substitution X = A R_s^{-1}.  RXR_SPLIT_BF16 runs its
    trailing updates on the tensor cores, so only its 16-column diagonal-block
    solves and the FP64 subtractions of the updates are FP64 work;
    RXR_SPLIT_PRECOND runs it as the plain FP64 substitution, n^2 flop per row."""
    t = stages.get("precond_subst")
    hbm, hbm_kind = hbm_peak()
    if t is None or t <= 0:
        return None
    if prec == "fp64":
        flop = (2.0 * N * N + N) * M
        name = "k_subst_gram (fused precondition + Gram launch)" if N <= 128 else "k_subst_wide (blocked FP64)"
        hbm_bytes = 16.0 * M * N
    elif prec == "split_precond":
        flop = 1.0 * N * N * M
        name = "k_subst_gram (FP64 substitution X = A R_s^-1, no Gram)" if N <= 128 else "k_subst_wide"
        hbm_bytes = 16.0 * M * N
    elif N <= 128:
        flop = subst_fp64_flop_per_row(N, 16, 1) * M
        name = ("k_subst_fused" if N <= 64 else "k_rprep128 + k_subst_fused128") + \
            " (FP64 16-column diagonal solves + FP64 subtraction of tcgen05 updates)"
        hbm_bytes = 16.0 * M * N
    else:
        flop = subst_fp64_flop_per_row(N, 64, 1) * M
        name = "k_solve_block + k_update_ozaki (blocked substitution: FP64 diagonal blocks, tcgen05 updates)"
        hbm_bytes = 16.0 * M * N
    achieved = flop / (t * 1e-3) / 1e12
    cap = TRAFFIC.get((prec, N))
    traffic = cap[0] * M / cap[1] if cap else None
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": achieved / peak_fp64, "traffic": traffic, "ms": t,
            "hbm_frac": (hbm_bytes / (t * 1e-3) / 1e9) / hbm, "hbm_peak_gbs": hbm, "hbm_peak_kind": hbm_kind,
            "peak_kind": "FP64 DFMA pipe, measured by the rxr_fp64_peak calibration kernel in this run "
                         "(MEASURED_PEAKS.json has no FP64 figure)"}


def e2e_leg(h, args, world, A_dev):
    """Same metric through rxr_cholqr_host: pinned host A in, pinned host Q, R out,
    host<->device copies inside the timed region."""
    import torch

    # pinned column-major buffers (the transpose of a pinned row-major tensor),
    # allocated at the start of the process
    tA, tQ = _PINNED.get("A"), _PINNED.get("Q")
    if tA is None or tA.numel() < M * N:
        tA = torch.empty(M * N, dtype=torch.float64).pin_memory()
        tQ = torch.empty(M * N, dtype=torch.float64).pin_memory()
    hA = tA[:M * N].view(N, M).numpy().T
    tA[:M * N].view(N, M).copy_(A_dev.t())  # the resident A's bytes, outside the timed calls
    torch.cuda.synchronize()
    hQ = tQ[:M * N].view(N, M).numpy().T
    hR = torch.empty((N, N), dtype=torch.float64).pin_memory().numpy().T
    for _ in range(2):
        h.cholqr_host(hA, variant=args.variant, s=S, seed=SEED, passes=PASSES, prec=args.prec, Q=hQ, R=hR)
    e_steps = max(3, min(args.steps, 7))
    times = []
    for _ in range(e_steps):  # each call is blocking; the median of the calls' wall-clock times
        t0 = time.perf_counter()
        h.cholqr_host(hA, variant=args.variant, s=S, seed=SEED, passes=PASSES, prec=args.prec, Q=hQ, R=hR)
        times.append(time.perf_counter() - t0)
    e2e_s = statistics.median(times)
    # the host link on its own, with the same pinned buffers: one plain copy
    # each way (what the call's copies cost when nothing overlaps them)
    tA, tQ = tA[:M * N].view(N, M), tQ[:M * N].view(N, M)
    dbuf = torch.empty(tA.shape, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    ev[0].record()
    dbuf.copy_(tA, non_blocking=True)
    ev[1].record()
    tQ.copy_(dbuf, non_blocking=True)
    ev[2].record()
    torch.cuda.synchronize()
    h2d_ms, d2h_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    del dbuf
    return {"value": world * b_alg(M, N, PASSES) / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * M * N,
            "d2h_bytes_per_step": 8 * M * N + 8 * N * N, "ms_per_step": e2e_s * 1e3,
            "host_link": {"h2d_gbs": 8 * M * N / h2d_ms / 1e6, "d2h_gbs": 8 * M * N / d2h_ms / 1e6,
                          "h2d_ms": h2d_ms, "d2h_ms": d2h_ms}}


def _emit(args, world, main, cfg, peak_fp64, secondary):
    M_, N_ = cfg["m"], cfg["n"]
    globals().update(M=cfg["m"], N=cfg["n"], S=cfg["s"], KAPPA=cfg["kappa"])
    rows = args.variant.endswith("-rows")
    base = args.variant.split("-")[0]
    launches = launches_per_step(args.prec, N, M, rows) if PASSES == 2 and base in ("qr", "lu") else None
    p0 = main["paths"][args.prec]
    line = {
        "metric": METRIC, "value": main["value"], "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": main["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic",
        "config": {"workload": workload_name(args.variant, rows), "m": M, "n": N, "s": S, "kappa": KAPPA,
                   "seed": SEED, "passes": PASSES, "variant": args.variant, "prec": args.prec,
                   "l2": f"A ({8 * M * N / 1e9:.1f} GB) larger than L2 (129 MB); no flush needed",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                   "generation_s": main["generation_s"]},
        "roofline": roofline_entry(args.prec, p0["stages_ms"], peak_fp64),
        "stages_ms": p0["stages_ms"],
        "gflops": world * f_alg(M, N, S, PASSES) / (main["ms"] * 1e-3) / 1e9,
        "qr_per_s": world / (main["ms"] * 1e-3),
        "accuracy": p0["accuracy"],
        "preconditioner": main.get("preconditioner"),
        "e2e": main.get("e2e"),
        "gpu_launches": launches * args.steps if launches else None,
        "clocks": p0["clocks"],
        "cpu_baseline": main.get("cpu_baseline"),
    }
    compare = {}
    for prec, r in main["paths"].items():
        if prec == args.prec:
            continue
        compare[prec] = {"value": world * b_alg(M, N, PASSES) / (r["ms"] * 1e-3) / 1e9, "unit": "GB/s",
                         "ms_per_step": r["ms"], "dtype": DTYPES[prec], "stages_ms": r["stages_ms"],
                         "accuracy": r["accuracy"], "roofline": roofline_entry(prec, r["stages_ms"], peak_fp64)}
    if compare:
        line["compare"] = compare
        if "fp64" in compare:
            line["speedup_vs_fp64"] = compare["fp64"]["ms_per_step"] / main["ms"]
    if secondary:
        line["configs"] = secondary
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS),
                    help="c3: m=2^23 n=128 kappa=1e12 (default); c2: m=2^22 n=64 kappa=1e10; "
                         "c1: m=20000 n=16 kappa=1e8; c5: m=2^20 n=512 kappa=1e13")
    ap.add_argument("--variant", default=None, choices=["qr", "lu", "none", "shifted"],
                    help="rQR / rLU preconditioning (default: the configuration's), or the comparators "
                         "CholeskyQR2 (none) and sCholeskyQR3")
    ap.add_argument("--sketch", default="gaussian", choices=["gaussian", "rows"],
                    help="Gaussian sketch (the workload's) or row extraction (Section 2.3)")
    ap.add_argument("--prec", default="split", choices=list(PRECS),
                    help="the reported path; the other two are timed alongside unless --no-compare")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precisions")
    ap.add_argument("--no-secondary", action="store_true", help="skip the nested c2 and c1 measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--m", type=int, default=None, help="rows (profiling runs on a smaller case)")
    ap.add_argument("--n", type=int, default=None, help="columns (s = 2n)")
    ap.add_argument("--kappa", type=float, default=None, help="condition number of A")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "lstsq", "rsvd", "sharded"],
                    help="sharded: the row-sharded factorisation (the default under torchrun with N > 1)")
    ap.add_argument("--replicas", action="store_true",
                    help="under torchrun: N independent single-GPU factorisations instead of row shards")
    ap.add_argument("--k", type=int, default=None, help="block width of the rsvd workload (default 20)")
    ap.add_argument("--count", type=int, default=512, help="problems in the batched workload")
    args = ap.parse_args()
    global M, N, S, KAPPA, WORKLOAD, PASSES
    if args.workload in ("lstsq", "batched", "rsvd") and args.config == "c3" and "--config" not in sys.argv:
        args.config = "c2"  # those arms keep the scale configuration's A
    set_config(args.config)
    if args.variant is None:
        args.variant = CONFIGS[args.config]["variant"]
    args.variant_c1 = CONFIGS["c1"]["variant"]
    if args.variant == "shifted":
        PASSES = 3
    if args.m:
        M = int(args.m)
    if args.n:
        N, S = int(args.n), 2 * int(args.n)
    if args.kappa:
        KAPPA = float(args.kappa)
    # the nested configurations ride along with the default workload only
    args.secondary = (not args.no_secondary and args.config == "c3" and not (args.m or args.n or args.kappa)
                      and args.sketch == "gaussian" and args.variant == "qr")
    if args.sketch == "rows":
        args.variant += "-rows"
    WORKLOAD = workload_name(args.variant, args.sketch == "rows")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.workload == "batched":
        batched_arm(args, rank, world, local_rank)
        return
    if args.workload == "lstsq":
        lstsq_arm(args, rank, world, local_rank)
        return
    if args.workload == "rsvd":
        rsvd_arm(args, rank, world, local_rank)
        return
    if args.workload == "sharded" or (world > 1 and not args.replicas):
        sharded_arm(args, rank, world, local_rank)
        return
    gpu_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
