// Test helper: Philox4x32-10 outputs from cuRAND's device API, to pin the
// library's own Philox against an independent implementation.  For each i the
// state is initialised with curand_init(seed, subsequence, offset) and one
// curand4() call is made; the words land in out[4*i .. 4*i+3].
#include <curand_kernel.h>
#include <stdint.h>

__global__ void k_curand_philox(uint64_t seed, const unsigned long long *subseq, const unsigned long long *offset,
                                int count, uint4 *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed, subseq[i], offset[i], &st);
    out[i] = curand4(&st);
}

extern "C" int curand_philox_outputs(uint64_t seed, const unsigned long long *d_subseq,
                                     const unsigned long long *d_offset, int count, unsigned int *d_out)
{
    if (count <= 0) return 0;
    k_curand_philox<<<(count + 127) / 128, 128>>>(seed, d_subseq, d_offset, count, (uint4 *)d_out);
    return (int)cudaDeviceSynchronize();
}
