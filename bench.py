"""Benchmark of randomized XR-preconditioned CholeskyQR on one GB300 (or N
independent replicas, one per GPU, under torchrun).

A step is one full factorisation A = QR (sketch, XR factor of the sketch, the
fused precondition+Gram pass, two CholeskyQR passes, Q and R) of the
tall-skinny workload m = 2^22, n = 64 (A = U Sigma V^T, kappa = 1e10, s = 2n
Gaussian sketch, seed 0) with inputs resident in HBM.  The metric is the
effective bandwidth B_alg / t with B_alg = 8 m n (P + 3) bytes: one read of A
for the sketch, one per CholeskyQR pass, and a read plus a write for Q.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant qr|lu]
                    [--prec fp64|split] [--impl reference]

`--impl reference` times the CPU oracle (the plain FP64 implementation
written from the paper) on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, S, KAPPA, SEED, PASSES = 2**22, 64, 128, 1e10, 0, 2
METRIC = "tall-skinny QR effective GB/s (B_alg = 8mn(P+3)) at ||Q^T Q - I||_F <= 1e-13"
WORKLOAD = "rQR-CholeskyQR2 m=2^22 n=64 s=128 kappa=1e10 FP64"


# dram__bytes_read.sum + dram__bytes_write.sum of one precondition+Gram launch,
# ncu capture at m = 2^19 scaled by 8 rows-for-rows (profiles/k_subst_gram_precond_m524288_n64.md)
TRAFFIC_PG = (268.552704e6 + 225.660672e6) * 8
# DRAM bytes (read + write) of one k_subst_fused launch at m = 2^22, n = 64: the ncu capture at
# m = 2^19 (268.58 MB read + 216.93 MB written) scaled by the 8x rows (traffic grows with the rows)
TRAFFIC_SUBST = (268.584960e6 + 216.926208e6) * 8
HBM_GBS = 6795.5  # measured copy bandwidth of this GPU pool (STREAM-style copy)


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


def cpu_cores() -> int:
    return 1


def oracle_rows(target_s: float = 15.0) -> int:
    """Row count of the oracle sample: about `target_s` seconds of single-core work."""
    return int(os.environ.get("RXR_BENCH_ORACLE_ROWS", 2**19))


def run_oracle_sample(A_sample: np.ndarray, variant: str):
    import oracle

    t0 = time.perf_counter()
    if variant == "shifted":
        r = oracle.scholqr(A_sample, 1e-15 * np.linalg.norm(A_sample, 2) ** 2, passes=PASSES)
    else:
        ov = {"qr": oracle.VARIANT_QR, "lu": oracle.VARIANT_LU, "none": oracle.VARIANT_NONE}[variant.split("-")[0]]
        if variant.endswith("-rows"):
            ov |= oracle.SKETCH_ROWS
        r = oracle.rxr_cholqr(A_sample, ov, S, seed=SEED, passes=PASSES)
    dt = time.perf_counter() - t0
    if r.status != 0:
        raise RuntimeError(f"oracle status {r.status}")
    return dt


def make_input():
    from paper_2111_11148_gb300.inputs import usv_matrix

    return usv_matrix(M, N, KAPPA, seed=SEED)


def reference_arm(args, rank: int, world: int):
    """Time the CPU oracle as it stands on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle

    oracle.build()
    rows = oracle_rows()
    from paper_2111_11148_gb300.inputs import usv_matrix

    A = usv_matrix(rows, N, KAPPA, seed=SEED)
    for _ in range(args.warmup if args.warmup < 1 else 1):
        run_oracle_sample(A, args.variant)
    times = [run_oracle_sample(A, args.variant) for _ in range(args.steps)]
    t = statistics.median(times)
    gbs = b_alg(rows, N, PASSES) / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle_rows": rows, "m": M, "n": N, "s": S, "passes": PASSES,
                   "variant": args.variant},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{rows} x {N} rows of the same A = U Sigma V^T construction, full "
                                   f"rxr_cholqr per step (single-threaded C oracle)"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_arm(args, rank: int, world: int, local_rank: int):
    """512 independent problems (m log-uniform in [2^12, 2^18], n in {8..128},
    kappa log-uniform in [1e2, 1e12], matrix k seed k), one rxr_cholqr_batched per
    step: every stage is one launch over the whole batch."""
    import torch

    from paper_2111_11148_gb300 import rxr
    from paper_2111_11148_gb300.inputs import batch_specs, usv_matrix

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    specs = batch_specs(args.count, seed=0)
    t0 = time.perf_counter()
    As = [rxr.colmajor(torch.from_numpy(usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed)).to(dev)) for sp in specs]
    gen_s = time.perf_counter() - t0
    h = rxr.Handle(local_rank)
    seeds = [sp.seed for sp in specs]
    stream = torch.cuda.current_stream(dev)

    def step():
        return h.cholqr_batched(As, variant=args.variant, seeds=seeds, passes=PASSES)

    for _ in range(max(3, args.warmup)):
        Qs, Rs, st = step()
    assert (st[:, 0] == 0).all(), st[st[:, 0] != 0][:4]
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local_rank)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    bytes_alg = sum(b_alg(sp.m, sp.n, PASSES) for sp in specs)
    flops_alg = sum(f_alg(sp.m, sp.n, 2 * sp.n, PASSES) for sp in specs)
    worst_orth = max(h.orth_error(Q) for Q in Qs[:: max(1, len(Qs) // 32)])
    peak_fp64 = rxr.fp64_peak_tflops()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": world * bytes_alg / (ms * 1e-3) / 1e9, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched rQR-CholeskyQR2, {len(specs)} problems", "count": len(specs),
                       "total_rows": sum(sp.m for sp in specs), "bytes_A": sum(8 * sp.m * sp.n for sp in specs),
                       "generation_s": gen_s},
            "roofline": {"bound": "alu", "kernel": "whole batch", "achieved": flops_alg / (ms * 1e-3) / 1e12,
                         "peak": peak_fp64, "unit": "TFLOP/s", "frac": flops_alg / (ms * 1e-3) / 1e12 / peak_fp64,
                         "traffic": None},
            "qr_per_s": world * len(specs) / (ms * 1e-3), "gflops": world * flops_alg / (ms * 1e-3) / 1e9,
            "accuracy": {"worst_orth_sampled": worst_orth}, "gpu_launches": 12 * args.steps, "clocks": clk,
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
                          "dtype": "f64+bf16" if args.prec == "split" else "f64", "data": "synthetic",
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
        cpu = {"value": cms, "unit": "ms", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"one power iteration of the oracle on a {crow}-row operator of the same density, "
                         f"scaled by rows to {RSVD_M}"}
    if rank == 0:
        print(json.dumps({
            "metric": "randomized SVD (Algorithm 7) time per power iteration", "value": ms_iter, "unit": "ms",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_iter,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64+bf16" if args.prec == "split" else "f64", "data": "synthetic",
            "config": {"workload": f"RSVD power iteration, sparse {RSVD_M}x{RSVD_M} with {RSVD_D} nonzeros/row "
                                   f"(stand-in for Section 5.1's sparsest matrix), k={k}, orth = "
                                   f"{'rLU' if args.variant == 'lu' else 'rQR'}-CholeskyQR2",
                       "m": RSVD_M, "nnz": P.nnz, "k": k, "iters_timed": RSVD_ITERS, "generation_s": gen_s,
                       "l2": "working set (CSR + 5 blocks of m x k) larger than L2"},
            "roofline": {"bound": "hbm", "kernel": "whole power iteration", "achieved": balg / (ms_iter * 1e-3) / 1e9,
                         "peak": HBM_GBS, "unit": "GB/s", "frac": balg / (ms_iter * 1e-3) / 1e9 / HBM_GBS,
                         "traffic": None},
            "e2e": {"value": e2e_ms, "unit": f"ms per call with {RSVD_ITERS} iterations", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "ms_call_iters": {str(RSVD_ITERS): t_k, "0": t_0},
            "accuracy": {"orth_U": h.orth_error(U), "orth_V": h.orth_error(V), "AtU_minus_VS_sampled": ident},
            "gpu_launches": args.steps * (rsvd_launches(args.prec, k, RSVD_ITERS) + rsvd_launches(args.prec, k, 0)),
            "cpu_baseline": cpu, "clocks": clk,
        }), flush=True)
    h.close()


def time_path(h, A, Q, R, prec, args, dev, stream, steps, warmup, sample_clocks=False):
    """Time `steps` factorisations (after `warmup`) with CUDA events on the
    launching stream; then per-stage event times and the accuracy."""
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
    return {"ms": ms, "stages_ms": stages, "orth": h.orth_error(Q), "resid": h.resid_error(A, Q, R), "clocks": clk}


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


def gpu_arm(args, rank: int, world: int, local_rank: int):
    import torch

    from paper_2111_11148_gb300 import rxr

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    A_np = make_input()
    A = rxr.colmajor(torch.from_numpy(A_np).to(dev))
    Q = rxr.empty_colmajor(M, N, device=dev)
    R = rxr.empty_colmajor(N, N, device=dev)
    h = rxr.Handle(local_rank)
    stream = torch.cuda.current_stream(dev)
    peak_fp64 = rxr.fp64_peak_tflops()
    warm = max(3, args.warmup)

    # the reported path, timed with clocks sampled; then the other precision
    other = "fp64" if args.prec == "split" else "split"
    if dist:
        dist.barrier()
    main = time_path(h, A, Q, R, args.prec, args, dev, stream, args.steps, warm, sample_clocks=True)
    ref = None if args.no_compare else time_path(h, A, Q, R, other, args, dev, stream, max(2, args.steps // 2), warm)
    ms = max_over_ranks(main["ms"], dist, dev)
    value = job_value(ms, world)

    e2e = None if args.no_e2e else e2e_leg(h, A_np, args, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        rows = min(oracle_rows(), M)
        t_or = run_oracle_sample(np.asfortranarray(A_np[:rows]), args.variant)
        cpu = {"value": b_alg(rows, N, PASSES) / t_or / 1e9, "unit": "GB/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"first {rows} of {M} rows of the same A, one full rxr_cholqr (single-threaded C oracle), "
                         f"{t_or:.2f} s"}
    if rank == 0:
        _emit(args, world, ms, value, peak_fp64, main, ref, other, e2e, cpu)
    h.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def subst_fp64_flop_per_row(n, bw, sub_ops):
    """FP64 flop a blocked substitution issues per row: the diagonal-block
    solves (bw (bw - 1) / 2 FMAs per block, 2 flop each), the n multiplications
    by 1 / R_jj, and sub_ops FP64 operations per trailing output per block (the
    subtraction of the tensor-core update)."""
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
    if prec == "fp64":
        # sketch, XR, 3 x (substitution [+ wide Gram] + reduce except last), 2 factors, copy
        return sk + (8 if n <= 128 else 10) + xr
    if n <= 64:
        # sketch, XR, fused substitution, Gram, reduce, factor, middle pass (above 2^17 rows: inverse,
        # condition estimate, apply, fused substitution, the one not selected returning at once; else the
        # fused substitution), Gram, reduce, factor, last pass (inverse, selection, FP32-correction apply,
        # FP64-grade apply: the one not selected returns at once), copy
        return sk + xr + 4 + (4 if m >= 1 << 17 else 1) + 3 + 4 + 1
    if n <= 128:
        # sketch, XR, 3 x (record prep, fused substitution), 2 x (Gram, reduce), 2 factors, copy
        return sk + xr + 3 * 2 + 2 * 2 + 2 + 1 + (1 if rows else 0)
    blocked = 2 * ((n + 63) // 64) - 1  # diagonal solves + trailing updates
    return sk + xr + 3 * blocked + 2 * 2 + 2 + 1 + (1 if rows else 0)


def roofline_entry(prec, stages, peak_fp64):
    """The dominant FP64 launch of the path against the measured DFMA peak,
    counting the FP64 flop that launch actually issues.
    FP64 path: the fused precondition+Gram launch, (2n^2 + n) flop per row.
    Split path: the substitution X = A R_s^{-1}; its trailing updates run on the
    tensor cores, so only its diagonal-block solves and the FP64 subtractions
    of the updates are FP64 work."""
    if prec == "fp64":
        t = stages.get("precond_subst")
        flop = (2.0 * N * N + N) * M
        name = "k_subst_gram (fused precondition + Gram launch)"
        traffic = TRAFFIC_PG if (M == 2**22 and N == 64) else None
        hbm_bytes = 16.0 * M * N
    elif N <= 128:
        t = stages.get("precond_subst")
        flop = subst_fp64_flop_per_row(N, 16, 2) * M
        name = ("k_subst_fused" if N <= 64 else "k_subst_fused128") + \
            " (FP64 16-column diagonal solves + FP64 subtraction of tcgen05 updates)"
        traffic = TRAFFIC_SUBST if (M == 2**22 and N == 64) else None
        hbm_bytes = 16.0 * M * N
    else:
        t = stages.get("precond_subst")
        flop = subst_fp64_flop_per_row(N, 64, 3) * M
        name = "k_solve_block + k_update_ozaki (blocked substitution: FP64 diagonal blocks, tcgen05 updates)"
        traffic = None
        hbm_bytes = 16.0 * M * N
    achieved = flop / (t * 1e-3) / 1e12
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": achieved / peak_fp64, "traffic": traffic,
            "hbm_frac": (hbm_bytes / (t * 1e-3) / 1e9) / HBM_GBS,
            "peak_kind": "FP64 DFMA pipe, measured by the rxr_fp64_peak calibration kernel in this run"}


def e2e_leg(h, A_np, args, world):
    """Same metric through rxr_cholqr_host: pinned host A in, pinned host Q, R out,
    host<->device copies inside the timed region."""
    import torch

    hA = torch.from_numpy(A_np).pin_memory().numpy()
    hA = np.asfortranarray(hA) if not hA.flags["F_CONTIGUOUS"] else hA
    hQ = torch.empty((N, M), dtype=torch.float64).pin_memory().numpy().T
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
    return {"value": world * b_alg(M, N, PASSES) / e2e_s / 1e9, "unit": "GB/s", "h2d_bytes_per_step": 8 * M * N,
            "d2h_bytes_per_step": 8 * M * N + 8 * N * N}


def _emit(args, world, ms, value, peak_fp64, main, ref, other, e2e, cpu):
    launches = (launches_per_step(args.prec, N, M, args.variant.endswith("-rows"))
                if PASSES == 2 and args.variant.split("-")[0] in ("qr", "lu") else None)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f64+bf16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "m": M, "n": N, "s": S, "kappa": KAPPA, "seed": SEED, "passes": PASSES,
                   "variant": args.variant, "prec": args.prec,
                   "l2": f"A ({8 * M * N / 1e9:.1f} GB) larger than L2 (129 MB); no flush needed",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": roofline_entry(args.prec, main["stages_ms"], peak_fp64),
        "stages_ms": main["stages_ms"],
        "gflops": world * f_alg(M, N, S, PASSES) / (ms * 1e-3) / 1e9,
        "qr_per_s": world / (ms * 1e-3),
        "accuracy": {"orth": main["orth"], "resid": main["resid"]},
        "e2e": e2e,
        "gpu_launches": launches * args.steps if launches else None,
        "clocks": main["clocks"],
        "cpu_baseline": cpu,
    }
    if ref is not None:
        line["compare"] = {
            "prec": other, "value": world * b_alg(M, N, PASSES) / (ref["ms"] * 1e-3) / 1e9, "unit": "GB/s",
            "ms_per_step": ref["ms"], "stages_ms": ref["stages_ms"],
            "accuracy": {"orth": ref["orth"], "resid": ref["resid"]},
            "roofline": roofline_entry(other, ref["stages_ms"], peak_fp64),
        }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--variant", default="qr", choices=["qr", "lu", "none", "shifted"],
                    help="rQR / rLU preconditioning, or the comparators CholeskyQR2 (none) and sCholeskyQR3")
    ap.add_argument("--sketch", default="gaussian", choices=["gaussian", "rows"],
                    help="Gaussian sketch (the workload's) or row extraction (Section 2.3)")
    ap.add_argument("--prec", default="split", choices=["fp64", "split"],
                    help="the reported path; the other precision is timed alongside unless --no-compare")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--m", type=int, default=None, help="rows (profiling runs on a smaller case)")
    ap.add_argument("--n", type=int, default=None, help="columns (s = 2n)")
    ap.add_argument("--kappa", type=float, default=None, help="condition number of A")
    ap.add_argument("--workload", default="single", choices=["single", "batched", "lstsq", "rsvd"])
    ap.add_argument("--k", type=int, default=None, help="block width of the rsvd workload (default 20)")
    ap.add_argument("--count", type=int, default=512, help="problems in the batched workload")
    args = ap.parse_args()
    global M, N, S, KAPPA, WORKLOAD, PASSES
    if args.variant == "shifted":
        PASSES = 3
    if args.m:
        M = int(args.m)
    if args.n:
        N, S = int(args.n), 2 * int(args.n)
    if args.kappa:
        KAPPA = float(args.kappa)
    method = {"qr": "rQR-CholeskyQR2", "lu": "rLU-CholeskyQR2", "none": "CholeskyQR2",
              "shifted": "sCholeskyQR3"}[args.variant]
    WORKLOAD = (f"{method} m={'2^22' if M == 2**22 else M} n={N} "
                f"s={S} kappa={KAPPA:g} {'FP64' if args.prec == 'fp64' else 'split BF16 sketch+Gram1, FP64 rest'}")
    if args.sketch == "rows":
        WORKLOAD += ", row-extraction sketch"
        args.variant += "-rows"
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
    gpu_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
