// split_kernels.cu -- split-precision (BF16 slices on tcgen05 tensor cores)
// forms of the two contractions that only shape the preconditioner.
#include "rxr_internal.cuh"

namespace rxr {

size_t split_workspace_bytes(int64_t, int64_t, int64_t, int) { return 0; }

int split_sketch_enqueue(Plan &, const double *, int64_t, uint64_t, cudaStream_t) { return RXR_ERR_UNSUPPORTED; }

int split_gram_enqueue(Plan &, const double *, int64_t, cudaStream_t) { return RXR_ERR_UNSUPPORTED; }

}  // namespace rxr
