// batched_tuning.h -- row-chunk table of the batched form, written by
// paper_2111_11148_gb300/tune_batched.py from timings on a GB300 (rerun it on
// another part).  The persistent stage kernels split each problem's rows into
// chunks of about total_rows / (ctas_per_sm * SMs) rows (at least one 128-row
// panel): more chunks balance the work queue better, fewer chunks mean fewer
// partial sums to reduce.  Entry i applies to problems whose n lies in
// (kBatchTuneN[i-1], kBatchTuneN[i]].  512 problems, rQR-CholeskyQR2, FP64: 1319.5 ms per run.
#pragma once

namespace rxr {
constexpr int kBatchTuneBuckets = 5;
constexpr int kBatchTuneN[kBatchTuneBuckets] = {8, 16, 32, 64, 128};
constexpr int kBatchCtasPerSm[kBatchTuneBuckets] = {32, 32, 32, 32, 32};
}  // namespace rxr
