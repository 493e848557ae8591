// noalloc.cu -- rxr_sketch_noalloc: the sketch Y = Omega A for callers that must
// not allocate device memory.
//
// The ordinary entry points keep their scratch (per-chunk partial sums of the
// sketch and the status word) in a workspace that the handle allocates with
// cudaMalloc or that the caller hands over.  Some callers can do neither:
// processes whose device memory is entirely reserved by another allocator
// (a framework's caching pool that owns the whole GPU), or loops that forbid
// any allocation after start-up because cudaMalloc may synchronise the device
// or take an unbounded time.  This entry point serves them: its scratch is the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "rxr_internal.cuh"

namespace rxr {
__global__ void k_sketch_fp64(const __grid_constant__ CUtensorMap, int, const double *, int64_t, int64_t, int, int,
                              uint64_t, int64_t, int64_t, int, double *, RxrStatus *, int64_t);
__global__ void k_reduce_parts(const double *, int, int64_t, int, int, double, int, double *, int64_t, RxrStatus *);
}  // namespace rxr

using namespace rxr;

namespace {

// 256 bytes for the status word, then the partial sums: 2^21 doubles (16 MiB).
constexpr int64_t kNoallocPartials = (int64_t)RXR_NOALLOC_SCRATCH_BYTES / 8 - 32;
// every admissible request (s <= RXR_MAX_S, n <= 128) has room for at least one
// row chunk's s x n partial sum, so no size that passes the argument checks is
// refused for lack of scratch
static_assert((int64_t)RXR_MAX_S * 128 <= kNoallocPartials, "scratch array below one chunk's partial sum");
static __device__ __align__(256) double g_noalloc_scratch[RXR_NOALLOC_SCRATCH_BYTES / 8];

constexpr int kMaxDevices = 64;
constexpr int kSkP = 64, kSkSTile = 128, kSkNTile = 64;
std::mutex g_setup_mu;
double *g_scratch_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in) and the shared-memory
// opt-in of the sketch kernel.
int setup_device(int dev, double **scratch, int *sms)
{
    if (dev < 0 || dev >= kMaxDevices) return RXR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (g_scratch_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            return RXR_ERR_CUDA;
        }
        const int smem = (kSkNTile * kSkP + kSkP * kSkSTile) * (int)sizeof(double);
        if (cudaFuncSetAttribute(k_sketch_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
            (void)cudaGetLastError();
            return RXR_ERR_CUDA;
        }
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            (void)cudaGetLastError();
            return RXR_ERR_CUDA;
        }
        g_sms[dev] = v;
        g_scratch_ptr[dev] = (double *)p;
    }
    *scratch = g_scratch_ptr[dev];
    *sms = g_sms[dev];
    return 0;
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

extern "C" RXR_API int rxr_sketch_noalloc(const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                                          double *Y, int64_t ldy, void *stream)
{
    if (A == nullptr) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1) return -3;
    if (lda < m) return -4;
    if (s < 1 || s > RXR_MAX_S) return -5;
    if (Y == nullptr) return -7;
    if (ldy < s) return -8;
    if (n > 128 || m > ((int64_t)1 << 31)) return RXR_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    double *scratch = nullptr;
    int sms = 0;
    if (int e = setup_device(dev, &scratch, &sms)) return e;
    RxrStatus *st_word = reinterpret_cast<RxrStatus *>(scratch);
    double *parts = scratch + 32;

    // the same launch geometry as the workspace path, with the number of row
    // chunks also capped by what the scratch array can hold
    const int64_t gy = cdiv(s, kSkSTile) * cdiv(n, kSkNTile);
    const int64_t panels = cdiv(m, kSkP);
    int64_t gx = std::max<int64_t>(1, cdiv(2 * (int64_t)sms, gy));
    gx = std::min<int64_t>(gx, panels);
    gx = std::min<int64_t>(gx, kNoallocPartials / (s * n));
    const int64_t ppc = cdiv(panels, gx);
    gx = cdiv(panels, ppc);

    cudaStream_t st = (cudaStream_t)stream;
    // the status word starts at zero; the partial sums are overwritten in full
    if (cudaMemsetAsync(st_word, 0, sizeof(RxrStatus), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    CUtensorMap unused;
    memset(&unused, 0, sizeof(unused));
    const int box_cols = (int)std::min<int64_t>(n, kSkNTile);
    const size_t smem = (size_t)(kSkNTile * kSkP + kSkP * kSkSTile) * sizeof(double);
    k_sketch_fp64<<<dim3((unsigned)gx, (unsigned)gy), RXR_THREADS, smem, st>>>(
        unused, 0, A, lda, m, (int)n, (int)s, seed, panels, ppc, box_cols, parts, st_word, (int64_t)0);
    k_reduce_parts<<<(int)cdiv(s * n, 256), 256, 0, st>>>(parts, (int)gx, s * n, (int)s, (int)n,
                                                          1.0 / sqrt((double)s), 0, Y, ldy, st_word);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    int code = 0;
    if (cudaMemcpyAsync(&code, st_word, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    return code;
}
