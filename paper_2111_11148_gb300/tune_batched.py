"""Tune the batched form's row chunking on this GPU and write
csrc/batched_tuning.h (then rebuild the library).

The FP64 batched plan splits every problem's rows into chunks of about
total_rows / (c * SMs) rows, where c (CTAs per SM per stage) comes from a
table indexed by the problem's n (buckets n <= 8, 16, 32, 64, 128).  More
chunks balance the persistent kernels' work queue better; fewer chunks leave
fewer partial sums to reduce.  This script times plan runs of the batched
workload (512 problems, m log-uniform in [2^12, 2^18], n from {8, ..., 128},
kappa log-uniform in [1e2, 1e12], rQR-CholeskyQR2) with CUDA events: first
one c for every bucket, then each bucket in turn with the others held (one
round of coordinate descent), over the candidates 4, 8, 16, 32, 64, 128.

    python -m paper_2111_11148_gb300.tune_batched [--count 512] [--write]
"""
from __future__ import annotations

import argparse
import os
import time

CANDIDATES = (4, 8, 16, 32, 64, 128)
BUCKETS = (8, 16, 32, 64, 128)
HEADER = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "batched_tuning.h")


def time_plan(h, As, seeds, table, runs=2) -> float:
    import torch

    from . import rxr

    for b, c in enumerate(table):
        h.set_test_hook(rxr.HOOK_BATCH_CTAS, (b << 8) | c)
    plan = h.batch_plan(As, variant="qr", seeds=seeds, prec="fp64")
    try:
        plan.run()
        torch.cuda.synchronize()
        if not bool((plan.status[:, 0] == 0).all()):
            raise RuntimeError("a problem of the batch failed")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(runs):
            plan.run()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / runs
    finally:
        plan.close()
        for b in range(len(table)):
            h.set_test_hook(rxr.HOOK_BATCH_CTAS, b << 8)


def write_header(table, ms, note, path=HEADER):
    with open(path, "w") as f:
        f.write(f"""// batched_tuning.h -- row-chunk table of the batched form, written by
// paper_2111_11148_gb300/tune_batched.py from timings on a GB300 (rerun it on
// another part).  The persistent stage kernels split each problem's rows into
// chunks of about total_rows / (ctas_per_sm * SMs) rows (at least one 128-row
// panel): more chunks balance the work queue better, fewer chunks mean fewer
// partial sums to reduce.  Entry i applies to problems whose n lies in
// (kBatchTuneN[i-1], kBatchTuneN[i]].  {note}: {ms:.1f} ms per run.
#pragma once

namespace rxr {{
constexpr int kBatchTuneBuckets = {len(BUCKETS)};
constexpr int kBatchTuneN[kBatchTuneBuckets] = {{{", ".join(str(b) for b in BUCKETS)}}};
constexpr int kBatchCtasPerSm[kBatchTuneBuckets] = {{{", ".join(str(c) for c in table)}}};
}}  // namespace rxr
""")


def main():
    import torch

    from . import rxr
    from .inputs import batch_specs, usv_matrix

    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--write", nargs="*", default=None,
                    help="write the table to csrc/batched_tuning.h (and to any paths given)")
    args = ap.parse_args()
    specs = batch_specs(args.count, seed=0)
    t0 = time.perf_counter()
    As = [rxr.colmajor(torch.from_numpy(usv_matrix(sp.m, sp.n, sp.kappa, seed=sp.seed)).cuda()) for sp in specs]
    print(f"generated {len(As)} problems in {time.perf_counter() - t0:.1f} s", flush=True)
    seeds = [sp.seed for sp in specs]
    with rxr.Handle(0) as h:
        best = None
        for c in CANDIDATES:
            ms = time_plan(h, As, seeds, [c] * len(BUCKETS))
            print(f"uniform c = {c}: {ms:.1f} ms", flush=True)
            if best is None or ms < best[0]:
                best = (ms, [c] * len(BUCKETS))
        ms_best, table = best
        for b in range(len(BUCKETS)):
            for c in CANDIDATES:
                if c == table[b]:
                    continue
                trial = list(table)
                trial[b] = c
                ms = time_plan(h, As, seeds, trial)
                print(f"bucket n <= {BUCKETS[b]} c = {c}: {ms:.1f} ms", flush=True)
                if ms < ms_best * 0.99:
                    ms_best, table = ms, trial
        print(f"table {table}: {ms_best:.1f} ms per run", flush=True)
        if args.write is not None:
            for path in [HEADER] + list(args.write):
                write_header(table, ms_best, f"{args.count} problems, rQR-CholeskyQR2, FP64", path)


if __name__ == "__main__":
    main()
