// api.cu -- host side of librxr: argument checking, workspace, TMA descriptors,
// and the launch sequence of rLU-/rQR-CholeskyQR (Algorithms 4 and 5 with the
// repeated CholeskyQR pass of Algorithm 2) behind the C ABI of include/rxr.h.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "batched_tuning.h"
#include "rxr_internal.cuh"

namespace rxr {
// stream_kernels.cu
__global__ void k_omega(uint64_t, int64_t, int64_t, int64_t, float *);
__global__ void k_sketch_fp64(const __grid_constant__ CUtensorMap, int, const double *, int64_t, int64_t, int, int,
                              uint64_t, int64_t, int64_t, int, double *, RxrStatus *, int64_t);
__global__ void k_reduce_parts(const double *, int, int64_t, int, int, double, int, double *, int64_t, RxrStatus *);
cudaError_t launch_subst_gram(int maxt, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap &map, int use_tma,
                              const double *src, int64_t lds, int64_t m, int n, const double *R, int64_t ldr,
                              int unit_r, double *dst, int64_t ldd, int do_gram, double *Gpart, int64_t panels_total,
                              int64_t panels_per_cta, int check_finite, RxrStatus *status);
cudaError_t set_subst_gram_smem(int bytes);
cudaError_t set_batched_smem(int bytes);
cudaError_t set_wide_smem();
__global__ void k_subst_wide(const double *, int64_t, int64_t, int, const double *, int64_t, double *, int64_t, int64_t,
                             int64_t, RxrStatus *);
__global__ void k_gram_tiles(const double *, int64_t, int64_t, int, int64_t, int64_t, double *, RxrStatus *);
__global__ void k_sketch_rows(const double *, int64_t, int64_t, int, int64_t, uint64_t, double *, int64_t, RxrStatus *);
__global__ void k_check_finite(const double *, int64_t, int64_t, int, RxrStatus *);
__global__ void k_sketch_fp64_batched(const SketchJob *, const int *, int, int, int *);
__global__ void k_reduce_parts_batched(const ReduceJob *, const int *, int, int, int *);
__global__ void k_subst_gram_batched(const SubstJob *, const int *, int, int, int, int *);
__global__ void k_xr_factor_batched(const XrJob *);
__global__ void k_factor_batched(const FactorJob *, int);
__global__ void k_finish_batched(const FinishJob *);
cudaError_t set_split_smem();
// small_kernels.cu
__global__ void k_xr_factor(const double *, int, int, int64_t, int, double *, double *, int64_t, RxrStatus *);
__global__ void k_factor(const double *, int, int64_t, double *, double *, double *, int, int, RxrStatus *);
__global__ void k_copy_upper(const double *, int, double *, int64_t, const RxrStatus *);
__global__ void k_identity(double *, int);
__global__ void k_shift_gram(double *, int, int64_t, double, RxrStatus *);
__global__ void k_ls_btb(const double *, int64_t, int64_t, int, const double *, int64_t, int, int64_t, double *,
                         RxrStatus *);
__global__ void k_ls_solve(const double *, const double *, int, int, const double *, double *, int64_t, RxrStatus *);
__global__ void k_status_out(const RxrStatus *, int *);
__global__ void k_orth_partial(const double *, int64_t, int, int64_t, int64_t, int, double *);
__global__ void k_orth_final(const double *, int, int, double *);
__global__ void k_resid_partial(const double *, int64_t, const double *, int64_t, const double *, int64_t, int64_t,
                                int, double *);
__global__ void k_resid_final(const double *, int, double *);
__global__ void k_fp64_peak(double *, int, double, double);
__global__ void k_trmm_upper(const double *, const double *, double *, int, RxrStatus *);
}  // namespace rxr

using namespace rxr;

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
// per-stage event slots: 0 sketch, 1 precondition (+ fused Gram), 2 middle
// passes (+ fused Gram), 3 last apply, 4 tensor-core first Gram, 5 tensor-core
// later Gram, 6 XR factorisation of the sketch
constexpr int kTimers = 7;
// row chunks of the _host entry point's copies (overlapped with the sketch
// and with the last apply)
constexpr int kIoChunks = kSketchChunks;
// shifted CholeskyQR3's shift, relative to ||A||_2^2 (the paper's experiments, Section 4.1)
constexpr double kShiftCoef = 1e-15;

struct rxr_ctx {
    int device = 0;
    int sms = 152;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool ws_owned = true;
    int *h_status = nullptr;  // pinned, 4 ints
    int last_pass = -1, last_col = -1;
    bool timing = false;
    cudaEvent_t ev[kTimers][2] = {};
    float last_ms[kTimers] = {};
    bool ev_recorded[kTimers] = {};
    // device staging for the _host entry point
    double *dA = nullptr, *dQ = nullptr, *dR = nullptr;
    size_t dA_bytes = 0, dQ_bytes = 0, dR_bytes = 0;
    double *eval_buf = nullptr;
    size_t eval_bytes = 0;
    double *ls_buf = nullptr;  // least squares: B^T b partial sums and c
    size_t ls_bytes = 0;
    double *sv_buf = nullptr;  // randomized SVD: the blocks, the row-major copy and the k x k factors
    size_t sv_bytes = 0;
    void *h_stage = nullptr;  // pinned host staging of batched job tables
    size_t h_stage_bytes = 0;
    // the _host entry point's copy stream and its chunk events
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t io_ev[2 * kIoChunks + 2] = {};
    // test hooks (rxr_set_test_hook)
    int test_stall = 0;
    int jacobi_sweeps = 0;                      // 0: the default bound
    int batch_ctas[kBatchTuneBuckets] = {};     // 0: the tuned table
};

namespace {

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                    const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled get_encode()
{
    static std::once_flag once;
    static PFN_encodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
        else
            (void)cudaGetLastError();
    });
    return fn;
}

// 2-D tiled descriptor of a column-major FP64 matrix (rows x cols, leading
// dimension ld) with box (box_rows x box_cols).  Returns false where TMA's
// rules are not met (16-byte aligned base, ld * 8 a multiple of 16, box sizes
// in range); the kernels then stage panels with plain coalesced loads.
bool encode_2d(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
               int box_cols, bool swizzle128 = false)
{
    memset(map, 0, sizeof(*map));
    PFN_encodeTiled enc = get_encode();
    if (!enc || ptr == nullptr) return false;
    if (((uintptr_t)ptr) % 16 != 0 || (ld * 8) % 16 != 0 || (box_rows * 8) % 16 != 0) return false;
    if (box_rows < 1 || box_rows > 256 || box_cols < 1 || box_cols > 256) return false;
    if (rows < 1 || cols < 1 || rows > (int64_t)1 << 31 || ld >= ((int64_t)1 << 37)) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    cuuint64_t gstride[1] = {(cuuint64_t)(ld * 8)};
    cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(ptr), gdim, gstride, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            (void)cudaGetLastError();
            prev = -1;
        }
        ok = (cudaSetDevice(dev) == cudaSuccess);
        if (!ok) (void)cudaGetLastError();
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

namespace rxr {
bool encode_tile_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     int box_cols, bool swizzle128)
{
    if (swizzle128 && box_rows * 8 > 128) return false;  // the swizzle span is one 128-byte row of the box
    return encode_2d(map, ptr, rows, cols, ld, box_rows, box_cols, swizzle128);
}

// Row chunks for a grid of gx x gy CTAs on `slots` resident CTA slots: the gx
// (at most max_gx) whose last wave is fullest, preferring fewer chunks, so a
// grid that overflows one wave by a few CTAs does not pay a second full wave.
int64_t balanced_chunks(int64_t gy, int64_t slots, int64_t max_gx)
{
    max_gx = std::max<int64_t>(1, max_gx);
    const int64_t lo = std::min(max_gx, std::max<int64_t>(1, slots / gy));
    const int64_t hi = std::min(max_gx, std::max<int64_t>(lo, 8 * slots / gy));
    int64_t best = lo;
    double best_eff = -1.0;
    for (int64_t gx = lo; gx <= hi; ++gx) {
        const int64_t ctas = gx * gy;
        const double eff = (double)ctas / (double)(cdiv(ctas, slots) * slots);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = gx;
        }
        if (eff > 0.97) break;
    }
    return best;
}
}  // namespace rxr

namespace {

constexpr int kSkP = 64, kSkSTile = 128, kSkNTile = 64, kSgP = 128;
constexpr int kMaxStreamN = RXR_MAX_N;  // n > 128 uses the column-blocked kernels
constexpr int kNarrowN = 128;            // up to here R lives in shared memory
constexpr int kWP = 128, kWB = 64;

}  // namespace


namespace {

void make_plan(Plan &p, int64_t m, int64_t n, int64_t s, int prec, int sms, int64_t max_chunks = INT64_MAX)
{
    p.m = m;
    p.n = n;
    p.s = s;
    p.prec = prec;
    p.row0 = 0;
    p.sms = sms;
    const int64_t s_tiles = cdiv(s, kSkSTile), n_tiles = cdiv(n, kSkNTile);
    p.sk_gy = (int)(s_tiles * n_tiles);
    p.sk_panels = cdiv(m, kSkP);
    int64_t gx = balanced_chunks(p.sk_gy, 2 * (int64_t)sms, std::min(p.sk_panels, std::max<int64_t>(1, max_chunks)));
    p.sk_ppc = cdiv(p.sk_panels, gx);
    p.sk_gx = (int)cdiv(p.sk_panels, p.sk_ppc);
    p.yslots = p.sk_gx;
    if (prec != RXR_FP64) {  // the sketch on the tensor cores
        int64_t sgx, spc;
        split_sketch_grid(p, &sgx, &spc);
        p.yslots = std::max<int64_t>(p.yslots, sgx);
    }

    p.wide = n > kNarrowN;
    if (p.wide) {
        // one CTA per SM for the blocked substitution; Gram over 64 x 64 block pairs
        const int64_t panels = cdiv(m, kWP);
        p.sg_panels = panels;
        p.sg_ppc = cdiv(panels, std::min<int64_t>(std::min<int64_t>(sms, panels), std::max<int64_t>(1, max_chunks)));
        p.sg_gx = (int)cdiv(panels, p.sg_ppc);
        p.sg_smem = (size_t)(2 * kWB * kWP + kWB * kWB + kWB) * sizeof(double);
        p.sg_maxt = 3;
        const int64_t nb = cdiv(n, kWB);
        p.gt_gy = (int)(nb * (nb + 1) / 2);
        int64_t cg = balanced_chunks(p.gt_gy, sms, panels);  // one CTA per SM (128 KB of shared memory)
        p.gt_ppc = cdiv(panels, cg);
        p.gt_gx = (int)cdiv(panels, p.gt_ppc);
    }
    const int64_t n4 = (n + 3) & ~3;
    if (!p.wide) p.sg_smem = (size_t)(n4 * kSgP + n * (n + 1) / 2 + n) * sizeof(double);
    if (!p.wide) {
        const int per_sm = (p.sg_smem <= 110 * 1024) ? 2 : 1;
        p.sg_panels = cdiv(m, kSgP);
        int64_t g2 = std::min<int64_t>(std::min<int64_t>((int64_t)sms * per_sm, p.sg_panels),
                                       std::max<int64_t>(1, max_chunks));
        p.sg_ppc = cdiv(p.sg_panels, g2);
        p.sg_gx = (int)cdiv(p.sg_panels, p.sg_ppc);
        // Gram tile list: off-diagonal tiles, then the diagonal ones from the next
        // multiple of 32 (see k_subst_gram)
        const int64_t NT = n4 / 4, n_off = NT * (NT - 1) / 2, d0 = (n_off + 31) & ~(int64_t)31;
        p.sg_maxt = (int)cdiv(d0 + NT, RXR_THREADS);
        p.gt_gx = p.gt_gy = 0;
        p.gt_ppc = 0;
    }

    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_status = take(sizeof(RxrStatus));
    const size_t o_ypart = take((size_t)p.yslots * s * n * 8);
    const size_t o_y = take((size_t)s * n * 8);
    const size_t o_w = take((size_t)s * n * 8);
    const size_t o_gpart = take((size_t)std::max(p.sg_gx, p.gt_gx) * n * n * 8);
    const size_t o_g = take((size_t)n * n * 8);
    const size_t o_rs = take((size_t)n * n * 8);
    const size_t o_rp = take((size_t)n * n * 8);
    const size_t o_racc = take((size_t)n * n * 8);
    const size_t o_c = take((size_t)n * n * 8);
    size_t o_split = off;
    if (prec != RXR_FP64) o_split = take(split_workspace_bytes(m, n, s, sms));
    p.bytes = off;
    p.base = nullptr;
    p.status = nullptr;
    (void)o_status;
    p.Ypart = (double *)(uintptr_t)o_ypart;
    p.Y = (double *)(uintptr_t)o_y;
    p.W = (double *)(uintptr_t)o_w;
    p.Gpart = (double *)(uintptr_t)o_gpart;
    p.G = (double *)(uintptr_t)o_g;
    p.Rs = (double *)(uintptr_t)o_rs;
    p.Rp = (double *)(uintptr_t)o_rp;
    p.Racc = (double *)(uintptr_t)o_racc;
    p.C = (double *)(uintptr_t)o_c;
    p.split = (char *)(uintptr_t)o_split;
}

void bind_plan(Plan &p, void *ws)
{
    char *b = (char *)ws;
    p.base = b;
    p.status = (RxrStatus *)b;
    p.Ypart = (double *)(b + (uintptr_t)p.Ypart);
    p.Y = (double *)(b + (uintptr_t)p.Y);
    p.W = (double *)(b + (uintptr_t)p.W);
    p.Gpart = (double *)(b + (uintptr_t)p.Gpart);
    p.G = (double *)(b + (uintptr_t)p.G);
    p.Rs = (double *)(b + (uintptr_t)p.Rs);
    p.Rp = (double *)(b + (uintptr_t)p.Rp);
    p.Racc = (double *)(b + (uintptr_t)p.Racc);
    p.C = (double *)(b + (uintptr_t)p.C);
    p.split = b + (uintptr_t)p.split;
}

int device_sms(int dev)
{
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 152;
    }
    return v;
}

int ensure_ws(rxr_handle h, size_t bytes)
{
    if (h->ws_bytes >= bytes) return 0;
    if (!h->ws_owned) return RXR_ERR_NOMEM;
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
    if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_NOMEM;
    }
    h->ws_bytes = bytes;
    return 0;
}

int grow(void **ptr, size_t *have, size_t need)
{
    if (*have >= need) return 0;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *have = 0;
    if (cudaMalloc(ptr, need) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_NOMEM;
    }
    *have = need;
    return 0;
}

bool kernel_attrs_set = false;
std::mutex attr_mu;

int set_kernel_attrs()
{
    std::lock_guard<std::mutex> lk(attr_mu);
    if (kernel_attrs_set) return 0;
    // dynamic shared memory above 48 KB must be opted into; leave room for the
    // kernels' static shared memory under the 227 KB per-block limit
    const int big = 220 * 1024;
    const cudaError_t es[] = {
        cudaFuncSetAttribute(k_sketch_fp64, cudaFuncAttributeMaxDynamicSharedMemorySize, big),
        set_subst_gram_smem(big),
        cudaFuncSetAttribute(k_orth_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, big),
        cudaFuncSetAttribute(k_resid_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, big),
        set_split_smem(),
        set_batched_smem(big),
        set_wide_smem(),
        set_small_smem(),
        set_rsvd_smem(),
    };
    for (cudaError_t e : es)
        if (e != cudaSuccess) {
            fprintf(stderr, "librxr: cudaFuncSetAttribute failed: %s\n", cudaGetErrorString(e));
            (void)cudaGetLastError();
            return RXR_ERR_CUDA;
        }
    kernel_attrs_set = true;
    return 0;
}

int launch_ok()
{
    cudaError_t e = cudaGetLastError();
    return (e == cudaSuccess) ? 0 : RXR_ERR_CUDA;
}

// one substitution(+Gram) pass
int enqueue_subst(const Plan &p, const double *src, int64_t lds, const double *R, int unit_r, double *dst,
                  int64_t ldd, bool gram, bool check_finite, cudaStream_t st)
{
    if (p.wide) {
        // column-blocked substitution writes X, then the tiled Gram reads it back
        if (unit_r || dst == nullptr) return RXR_ERR_UNSUPPORTED;
        k_subst_wide<<<p.sg_gx, RXR_THREADS, p.sg_smem, st>>>(src, lds, p.m, (int)p.n, R, p.n, dst, ldd, p.sg_panels,
                                                              p.sg_ppc, p.status);
        if (launch_ok()) return RXR_ERR_CUDA;
        if (gram) {
            k_gram_tiles<<<dim3(p.gt_gx, p.gt_gy), RXR_THREADS, 2 * kWB * kWP * sizeof(double), st>>>(
                dst, ldd, p.m, (int)p.n, p.sg_panels, p.gt_ppc, p.Gpart, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
            const int64_t nn = p.n * p.n;
            k_reduce_parts<<<(int)cdiv(nn, 256), 256, 0, st>>>(p.Gpart, p.gt_gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G,
                                                               p.n, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
        }
        return 0;
    }
    CUtensorMap map;
    const int use_tma = encode_2d(&map, src, p.m, p.n, lds, kSgP, (int)p.n) ? 1 : 0;
    if (launch_subst_gram(p.sg_maxt, dim3(p.sg_gx), p.sg_smem, st, map, use_tma, src, lds, p.m, (int)p.n, R, p.n,
                          unit_r, dst, ldd, gram ? 1 : 0, p.Gpart, p.sg_panels, p.sg_ppc, check_finite ? 1 : 0,
                          p.status) != cudaSuccess)
        return RXR_ERR_CUDA;
    if (launch_ok()) return RXR_ERR_CUDA;
    if (gram) {
        const int64_t nn = p.n * p.n;
        k_reduce_parts<<<(int)cdiv(nn, 256), 256, 0, st>>>(p.Gpart, p.sg_gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G, p.n,
                                                           p.status);
        if (launch_ok()) return RXR_ERR_CUDA;
    }
    return 0;
}

int enqueue_sketch(const Plan &p, const double *A, int64_t lda, uint64_t seed, cudaStream_t st)
{
    if (p.prec != RXR_FP64) return split_sketch_enqueue(const_cast<Plan &>(p), A, lda, seed, st);
    CUtensorMap map;
    const int box_cols = (int)std::min<int64_t>(p.n, kSkNTile);
    const int use_tma = encode_2d(&map, A, p.m, p.n, lda, kSkP, box_cols) ? 1 : 0;
    const size_t smem = (size_t)(kSkNTile * kSkP + kSkP * kSkSTile) * sizeof(double);
    k_sketch_fp64<<<dim3(p.sk_gx, p.sk_gy), RXR_THREADS, smem, st>>>(map, use_tma, A, lda, p.m, (int)p.n, (int)p.s,
                                                                     seed, p.sk_panels, p.sk_ppc, box_cols, p.Ypart,
                                                                     p.status, p.row0);
    if (launch_ok()) return RXR_ERR_CUDA;
    const int64_t sn = p.s * p.n;
    const int64_t threads = (p.sk_gx >= kReduceWarpParts) ? 32 * sn : sn;
    k_reduce_parts<<<(int)cdiv(threads, 256), 256, 0, st>>>(p.Ypart, p.sk_gx, sn, (int)p.s, (int)p.n,
                                                       1.0 / sqrt((double)p.s), 0, p.Y, p.s, p.status);
    return launch_ok();
}

// Split-path substitution X = B R^{-1}: up to n = 64 one fused pass (FP64
// diagonal blocks and tensor-core trailing updates on tiles held in shared
// memory); wider panels take the column-blocked form, one launch per block.
// colexp_out (n <= 128, nullable): also record the column exponents of X for
// the FP64-grade Gram that follows.
int split_subst(const Plan &p, const double *src, int64_t lds, const double *R, double *dst, int64_t ldd,
                cudaStream_t st, int *colexp_out = nullptr)
{
    if (colexp_out && p.n <= 128 &&
        cudaMemsetAsync(colexp_out, 0, (p.n <= 64 ? 64 : p.n) * sizeof(int), st) != cudaSuccess)
        return RXR_ERR_CUDA;
    if (p.n <= 64) return fused_subst_enqueue(const_cast<Plan &>(p), src, lds, R, p.n, dst, ldd, colexp_out, st);
    if (p.n <= 128)
        return fused128_subst_enqueue(const_cast<Plan &>(p), src, lds, R, p.n, dst, ldd, st, nullptr, colexp_out);
    return blocked_subst_enqueue(const_cast<Plan &>(p), src, lds, R, p.n, dst, ldd, st);
}

// XR factorisation of the sketch Y (s x n, ld ldy) into R_s: rQR of sketches
// above 16K entries by the blocked multi-CTA Householder QR (its scratch is the
// sketch partials, free by now), smaller ones and rLU by the one-CTA kernel
// (measured: 128 x 64 one CTA 0.48 ms vs blocked 0.56 ms; 1024 x 512: 74 vs
// 12 ms).
int enqueue_xr(const Plan &p, const double *Y, int64_t ldy, int variant, double *Rs, int64_t ldrs, cudaStream_t st)
{
    if (variant == RXR_QR && p.s * p.n > 16384 && blocked_qr_scratch_doubles(p.s, p.n) <= (size_t)p.sk_gx * p.s * p.n)
        return blocked_qr_enqueue(Y, (int)p.s, (int)p.n, ldy, p.W, Rs, ldrs, p.Ypart, p.status, st);
    k_xr_factor<<<1, 512, xr_smem_bytes(p.s, p.n), st>>>(Y, (int)p.s, (int)p.n, ldy, variant, p.W, Rs, ldrs,
                                                         p.status);
    return launch_ok();
}

struct Timer {
    rxr_handle h;
    int id;
    cudaStream_t st;
    Timer(rxr_handle h_, int id_, cudaStream_t st_) : h(h_), id(id_), st(st_)
    {
        if (h && h->timing) cudaEventRecord(h->ev[id][0], st);
    }
    ~Timer()
    {
        if (h && h->timing) {
            cudaEventRecord(h->ev[id][1], st);
            h->ev_recorded[id] = true;
        }
    }
};

// The whole factorisation, stream-ordered, no host synchronisation.
// Host buffers of the _host entry point: A arrives in row chunks on the copy
// stream while the split sketch works on the chunks already in, and Q leaves
// in row chunks as the split path's last apply finishes them.  Other paths
// copy whole matrices before and after.
struct HostIO {
    const double *hA;
    int64_t lda;
    double *hQ;
    int64_t ldq;
    cudaStream_t cs;
    cudaEvent_t *ev;  // 2 kIoChunks + 2
};

int enqueue_cholqr(rxr_handle h, const Plan &p, const double *A, int64_t lda, int variant, uint64_t seed, int passes,
                   double *Q, int64_t ldq, double *R, int64_t ldr, cudaStream_t st, bool timed,
                   const HostIO *io = nullptr)
{
    rxr_handle th = timed ? h : nullptr;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (h && h->test_stall && cudaMemsetAsync(&p.status->flags, kFlagStall, 1, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    const int n = (int)p.n;
    const bool rows = (variant & RXR_SKETCH_ROWS) != 0;  // row extraction instead of the Gaussian sketch
    variant &= ~RXR_SKETCH_ROWS;
    const bool shifted = variant == RXR_SHIFTED;  // sCholeskyQR3: no sketch, the first Gram shifted
    if (shifted) variant = RXR_NONE;
    // RXR_SPLIT_PRECOND without a sketch (CholeskyQR2, shifted CholeskyQR3) has
    // nothing to take off FP64: its first Gram decides breakdown on A itself
    const bool precond_only = p.prec == RXR_SPLIT_PRECOND && variant != RXR_NONE;
    const bool chunk_in = io && p.prec != RXR_FP64 && variant != RXR_NONE && !rows;
    const bool chunk_out = io && p.prec == RXR_SPLIT_BF16 && passes > 1 && p.n <= 64;
    if (io) {
        // the copy stream starts after this stream's earlier work
        if (cudaEventRecord(io->ev[2 * kIoChunks], st) != cudaSuccess ||
            cudaStreamWaitEvent(io->cs, io->ev[2 * kIoChunks], 0) != cudaSuccess)
            return RXR_ERR_CUDA;
        if (!chunk_in && cudaMemcpy2DAsync(const_cast<double *>(A), lda * 8, io->hA, io->lda * 8, p.m * 8, p.n,
                                           cudaMemcpyHostToDevice, st) != cudaSuccess)
            return RXR_ERR_CUDA;
    }
    // steps 1-2: sketch and its R factor (R_s = I without preconditioner)
    if (variant == RXR_NONE) {
        k_identity<<<(int)cdiv(p.n * p.n, 256), 256, 0, st>>>(p.Rs, n);
        if (launch_ok()) return RXR_ERR_CUDA;
    } else {
        if (rows) {
            Timer t(th, 0, st);
            k_sketch_rows<<<(int)cdiv(p.s, 8), 256, 0, st>>>(A, lda, p.m, n, p.s, seed, p.Y, p.s, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
        } else if (chunk_in) {
            // chunk c of A's rows lands on the copy stream, then its CTAs of
            // the sketch run (the same partition and partial sums as one launch)
            Timer t(th, 0, st);
            Plan &pm = const_cast<Plan &>(p);
            int64_t gx, spc;
            split_sketch_grid(p, &gx, &spc);
            const int K = (int)std::min<int64_t>(kIoChunks, gx);
            for (int c = 0; c < K; ++c) {
                const int64_t cb = gx * c / K, ce = gx * (c + 1) / K;
                const int64_t rb = std::min<int64_t>(p.m, cb * spc * 64), re = std::min<int64_t>(p.m, ce * spc * 64);
                if (re > rb && cudaMemcpy2DAsync(const_cast<double *>(A) + rb, lda * 8, io->hA + rb, io->lda * 8,
                                                 (re - rb) * 8, p.n, cudaMemcpyHostToDevice, io->cs) != cudaSuccess)
                    return RXR_ERR_CUDA;
                if (cudaEventRecord(io->ev[c], io->cs) != cudaSuccess ||
                    cudaStreamWaitEvent(st, io->ev[c], 0) != cudaSuccess)
                    return RXR_ERR_CUDA;
                if (int e = split_sketch_part_enqueue(pm, A, lda, seed, cb, ce, st)) return e;
            }
            if (int e = split_sketch_reduce_enqueue(pm, st)) return e;
        } else {
            Timer t(th, 0, st);
            if (int e = enqueue_sketch(p, A, lda, seed, st)) return e;
        }
        {
            Timer t(th, 6, st);
            if (int e = enqueue_xr(p, p.Y, p.s, variant, p.Rs, p.n, st)) return e;
        }
    }
    if (cudaMemcpyAsync(p.Racc, p.Rs, (size_t)p.n * p.n * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    // step 3: X = A R_s^{-1} into Q, fused with G_1 = X^T X
    {
        // the first Gram on the tensor cores: FP64-grade stacked digits for
        // n <= 64, BF16x3 for 64 < n <= 128, FP64-grade 128 x 64 blocks above
        if (p.prec == RXR_SPLIT_BF16 && variant != RXR_NONE) {
            // n <= 128: the substitution records X's column exponents for the
            // FP64-grade Gram that follows.  The first Gram is FP64-grade at
            // every n: R_1 then makes X_2 orthonormal to rounding level, so the
            // last pass's R_P^{-1} - I stays within 2^-38 and its apply takes
            // the FP32 correction (a BF16x3 Gram left it near 1e-5 at n = 128)
            int *cx = (p.n <= 128) ? split_colexp(p) : nullptr;
            {
                Timer t(th, 1, st);
                // a row sketch reads only the drawn rows: NaN or Inf elsewhere in A is
                // found by the Gram from X's column exponents (n <= 128) or here
                if (rows && !cx) {
                    k_check_finite<<<4 * p.sms, 256, 0, st>>>(A, lda, p.m, n, p.status);
                    if (launch_ok()) return RXR_ERR_CUDA;
                }
                if (int e = split_subst(p, A, lda, p.Rs, Q, ldq, st, cx)) return e;
            }
            Timer t(th, 4, st);
            if (int e = ozaki_gram_enqueue(const_cast<Plan &>(p), Q, ldq, st, cx != nullptr)) return e;
        } else if (precond_only) {
            // the preconditioning placement: X = A R_s^{-1} by FP64 substitution,
            // its Gram on the tensor cores (BF16x3 up to n = 128, digit slices above)
            {
                Timer t(th, 1, st);
                if (int e = enqueue_subst(p, A, lda, p.Rs, 0, Q, ldq, false, rows, st)) return e;
            }
            Timer t(th, 4, st);
            if (int e = p.wide ? ozaki_gram_enqueue(const_cast<Plan &>(p), Q, ldq, st, false)
                               : split_gram_enqueue(const_cast<Plan &>(p), Q, ldq, st))
                return e;
        } else if (p.prec == RXR_SPLIT_BF16) {
            // no preconditioner (CholeskyQR2, shifted CholeskyQR3): X_0 = A, and the
            // first Gram on the tensor cores at FP64 grade (it decides breakdown)
            {
                Timer t(th, 1, st);
                if (Q != A && cudaMemcpy2DAsync(Q, ldq * 8, A, lda * 8, p.m * 8, p.n, cudaMemcpyDeviceToDevice, st) !=
                                  cudaSuccess)
                    return RXR_ERR_CUDA;
                if (p.n > 64) {  // n <= 64: the Gram reports NaN or Inf from the column exponents
                    k_check_finite<<<4 * p.sms, 256, 0, st>>>(A, lda, p.m, n, p.status);
                    if (launch_ok()) return RXR_ERR_CUDA;
                }
            }
            Timer t(th, 4, st);
            if (int e = ozaki_gram_enqueue(const_cast<Plan &>(p), Q, ldq, st, false)) return e;
        } else {
            Timer t(th, 1, st);
            if (int e = enqueue_subst(p, A, lda, p.Rs, variant == RXR_NONE ? 1 : 0, Q, ldq, true,
                                      variant == RXR_NONE || rows, st))
                return e;
        }
    }
    // step 4: CholeskyQR passes on X
    for (int pass = 1; pass <= passes; ++pass) {
        if (shifted && pass == 1) {
            k_shift_gram<<<1, 256, 0, st>>>(p.G, n, p.n, kShiftCoef, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
        }
        if (p.n > 64) {
            if (int e = blocked_factor_enqueue(p.G, n, p.n, p.Rp, p.Racc, p.C, pass, 1, p.status, st)) return e;
        } else {
            k_factor<<<1, 512, factor_smem_bytes(p.n), st>>>(p.G, n, p.n, p.Rp, p.Racc, p.C, pass, 1, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
        }
        const bool last = (pass == passes);
        // X <- X R_p^{-1} (in place), with the next pass's Gram unless last; the
        // split path takes that Gram from the tensor cores at FP64 grade
        if (p.prec == RXR_SPLIT_BF16 && !last) {
            int *cx = (p.n <= 128) ? split_colexp(p) : nullptr;
            {
                Timer t(th, 2, st);
                // below ~2^17 rows the inverse and the estimate (~0.1 ms) cost more
                // than the product saves
                if (p.n <= 128 && p.m >= ((int64_t)1 << 17)) {
                    // R_p of a middle pass is well conditioned after the preconditioning:
                    // explicit-inverse product unless the estimate says otherwise
                    if (cx && cudaMemsetAsync(cx, 0, (p.n <= 64 ? 64 : p.n) * sizeof(int), st) != cudaSuccess)
                        return RXR_ERR_CUDA;
                    if (int e = middle_pass_enqueue(const_cast<Plan &>(p), Q, ldq, p.Rp, cx, split_select_flag(p), st))
                        return e;
                } else if (int e = split_subst(p, Q, ldq, p.Rp, Q, ldq, st, cx)) {
                    return e;
                }
            }
            Timer t(th, 5, st);
            if (int e = ozaki_gram_enqueue(const_cast<Plan &>(p), Q, ldq, st, cx != nullptr)) return e;
            continue;
        }
        Timer t(th, last ? 3 : 2, st);
        if (p.prec == RXR_SPLIT_BF16 && last && pass > 1 && p.n <= 64) {
            // the last pass's R_P is within rounding of I: Q = X + X (R_P^{-1} - I)
            // with the small correction in FP32, or (should R_P^{-1} - I exceed
            // 2^-38) the explicit inverse on the tensor cores at FP64 grade
            Plan &pm = const_cast<Plan &>(p);
            if (int e = ozaki_apply_prepare(pm, p.Rp, st)) return e;
            if (chunk_out) {
                // chunk c of Q leaves on the copy stream as soon as it is final
                const int64_t tiles = cdiv(p.m, 128);
                for (int c = 0; c < kIoChunks; ++c) {
                    const int64_t rb = std::min<int64_t>(p.m, tiles * c / kIoChunks * 128);
                    const int64_t re = std::min<int64_t>(p.m, tiles * (c + 1) / kIoChunks * 128);
                    if (re <= rb) continue;
                    if (int e = ozaki_apply_rows(pm, Q, ldq, rb, re - rb, st)) return e;
                    if (cudaEventRecord(io->ev[kIoChunks + c], st) != cudaSuccess ||
                        cudaStreamWaitEvent(io->cs, io->ev[kIoChunks + c], 0) != cudaSuccess ||
                        cudaMemcpy2DAsync(io->hQ + rb, io->ldq * 8, Q + rb, ldq * 8, (re - rb) * 8, p.n,
                                          cudaMemcpyDeviceToHost, io->cs) != cudaSuccess)
                        return RXR_ERR_CUDA;
                }
            } else if (int e = ozaki_apply_rows(pm, Q, ldq, 0, p.m, st)) {
                return e;
            }
        } else if (p.prec == RXR_SPLIT_BF16 && last && pass > 1 && p.n <= 128) {
            // 64 < n <= 128: the FP32 correction when R_P^{-1} - I is within
            // 2^-38, else the fused substitution (chosen on the device)
            if (int e = delta128_apply_enqueue(const_cast<Plan &>(p), Q, ldq, p.Rp, st)) return e;
        } else if (p.prec == RXR_SPLIT_BF16) {
            if (int e = split_subst(p, Q, ldq, p.Rp, Q, ldq, st)) return e;
        } else if (int e = enqueue_subst(p, Q, ldq, p.Rp, 0, Q, ldq, !last, false, st)) {
            return e;
        }
    }
    if (R) {
        k_copy_upper<<<(int)cdiv(p.n * p.n, 256), 256, 0, st>>>(p.Racc, n, R, ldr, p.status);
        if (launch_ok()) return RXR_ERR_CUDA;
    }
    if (io) {
        if (!chunk_out && cudaMemcpy2DAsync(io->hQ, io->ldq * 8, Q, ldq * 8, p.m * 8, p.n, cudaMemcpyDeviceToHost,
                                            st) != cudaSuccess)
            return RXR_ERR_CUDA;
        // this stream waits for every copy of the copy stream
        if (cudaEventRecord(io->ev[2 * kIoChunks + 1], io->cs) != cudaSuccess ||
            cudaStreamWaitEvent(st, io->ev[2 * kIoChunks + 1], 0) != cudaSuccess)
            return RXR_ERR_CUDA;
    }
    return 0;
}

int check_args(const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s, int passes,
               const double *Q, int64_t ldq, const double *R, int64_t ldr, int prec)
{
    if (A == nullptr) return -1;
    if (m < 1 || m < n) return -2;
    if (n < 1) return -3;
    if (lda < m) return -4;
    const int base = variant & ~RXR_SKETCH_ROWS;
    const bool sketchless = base == RXR_NONE || base == RXR_SHIFTED;
    if (base != RXR_LU && base != RXR_QR && !sketchless) return -5;
    if (sketchless && variant != base) return -5;  // no sketch to take by rows
    if (!sketchless && (s < n || s > RXR_MAX_S)) return -6;
    if (passes < 1 || passes > 3) return -8;
    if (Q == nullptr) return -9;
    if (ldq < m) return -10;
    if (R != nullptr && ldr < n) return -12;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16 && prec != RXR_SPLIT_PRECOND) return -13;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    if (n > kNarrowN && sketchless) return RXR_ERR_UNSUPPORTED;
    if (m > ((int64_t)1 << 31)) return RXR_ERR_UNSUPPORTED;
    (void)Q;
    return 0;
}

int finish_blocking(rxr_handle h, const RxrStatus *d_status, cudaStream_t st)
{
    if (cudaMemcpyAsync(h->h_status, d_status, 4 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    const int code = h->h_status[0];
    if (code == RXR_ERR_CHOL_BREAKDOWN) {
        h->last_pass = h->h_status[1];
        h->last_col = h->h_status[2];
    }
    if (h->timing)
        for (int k = 0; k < kTimers; ++k) {
            // a stage the last call did not run reads 0
            float ms = 0.f;
            if (h->ev_recorded[k] && cudaEventElapsedTime(&ms, h->ev[k][0], h->ev[k][1]) != cudaSuccess) {
                (void)cudaGetLastError();
                ms = 0.f;
            }
            h->last_ms[k] = ms;
            h->ev_recorded[k] = false;
        }
    return code;
}

}  // namespace

// ===========================================================================
// Batched form: a plan holds every problem's workspace and, for the FP64
// stage kernels, the device job tables; a run only enqueues work.
// ===========================================================================
constexpr int kBatchStreams = 8;  // streams of the per-problem form

struct rxr_batch {
    rxr_handle h = nullptr;
    int count = 0, variant = 0, passes = 2, prec = RXR_FP64;
    bool tables = false;  // FP64 stage kernels over job tables (else per-problem sequences)
    std::vector<Plan> plans;
    std::vector<const double *> A;
    std::vector<double *> Q, R;
    std::vector<int64_t> lda, ldq, ldr;
    std::vector<uint64_t> seed;
    int *d_status = nullptr;
    void *ws = nullptr;
    bool ws_owned = false;
    // job tables (device, inside ws) and the stage launch shapes
    RxrStatus *statuses = nullptr;
    const SketchJob *skj = nullptr;
    const ReduceJob *ryj = nullptr, *rgj = nullptr;
    const XrJob *xrj = nullptr;
    const SubstJob *prej = nullptr, *passj = nullptr;
    const FactorJob *fj = nullptr;
    const FinishJob *finj = nullptr;
    const int *st_sk = nullptr, *st_ry = nullptr, *st_sg = nullptr, *st_rg = nullptr;
    int tot_sk = 0, tot_ry = 0, tot_sg = 0, tot_rg = 0;
    int grid_sk = 0, grid_ry = 0, grid_sg = 0, grid_rg = 0;
    size_t sg_smem = 0;
    int *counters = nullptr;
    int ncounters = 0;
    // per-problem form: streams and the fork/join events
    cudaStream_t aux[kBatchStreams] = {};
    cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
};

namespace {

// CTAs per SM of the batch's row chunking for an n-column problem (the table
// of batched_tuning.h)
int batch_ctas_per_sm(rxr_handle h, int64_t n)
{
    int i = 0;
    while (i < kBatchTuneBuckets - 1 && n > kBatchTuneN[i]) ++i;
    return h->batch_ctas[i] > 0 ? h->batch_ctas[i] : kBatchCtasPerSm[i];
}

int occupancy_grid(const void *fn, int threads, size_t smem, int sms, int items)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    return std::max(1, std::min(items, per_sm * sms));
}

void batch_release(rxr_batch *b)
{
    if (!b) return;
    DeviceGuard g(b->h ? b->h->device : 0);
    if (b->ws_owned && b->ws) cudaFree(b->ws);
    for (cudaStream_t s : b->aux)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

// Lay the batch out: every problem's plan and workspace, and (FP64 over the
// stage kernels) the job tables, copied to the device before this returns.
// handle_ws: use the handle's workspace and pinned staging (the blocking call)
// instead of allocating the plan's own.
int batch_build(rxr_batch *b, const double *const *A, const int64_t *m, const int64_t *n, const int64_t *lda,
                const int64_t *s, const uint64_t *seed, double *const *Q, const int64_t *ldq, double *const *R,
                const int64_t *ldr, bool handle_ws, cudaStream_t st)
{
    rxr_handle h = b->h;
    const int count = b->count;
    std::vector<int64_t> sk(count);
    int64_t total_rows = 0;
    for (int k = 0; k < count; ++k) {
        const int base = b->variant & ~RXR_SKETCH_ROWS;
        sk[k] = ((base == RXR_NONE || base == RXR_SHIFTED) && s[k] < n[k]) ? n[k] : s[k];
        if (int e = check_args(A[k], m[k], n[k], lda[k], b->variant, sk[k], b->passes, Q[k], ldq[k], R[k], ldr[k],
                               b->prec))
            return e;
        if (b->tables && n[k] > kNarrowN) return RXR_ERR_UNSUPPORTED;  // the FP64 stage kernels: n <= 128
        total_rows += m[k];
    }
    b->plans.resize(count);
    std::vector<size_t> base(count);
    size_t off = align256((size_t)count * sizeof(RxrStatus));
    for (int k = 0; k < count; ++k) {
        // row chunks in proportion to each problem's rows (the tuned number of
        // CTAs per SM per stage over the whole batch)
        const int64_t target = std::max<int64_t>(kSgP, total_rows / ((int64_t)batch_ctas_per_sm(h, n[k]) * h->sms));
        make_plan(b->plans[k], m[k], n[k], sk[k], b->prec, h->sms, b->tables ? cdiv(m[k], target) : INT64_MAX);
        base[k] = off;
        off += align256(b->plans[k].bytes);
    }
    const size_t o_tables = off;
    const size_t o_skj = off;
    off += align256(count * sizeof(SketchJob));
    const size_t o_ryj = off;
    off += align256(count * sizeof(ReduceJob));
    const size_t o_xrj = off;
    off += align256(count * sizeof(XrJob));
    const size_t o_prej = off;
    off += align256(count * sizeof(SubstJob));
    const size_t o_passj = off;
    off += align256(count * sizeof(SubstJob));
    const size_t o_rgj = off;
    off += align256(count * sizeof(ReduceJob));
    const size_t o_fj = off;
    off += align256(count * sizeof(FactorJob));
    const size_t o_finj = off;
    off += align256(count * sizeof(FinishJob));
    const size_t o_starts = off;
    off += align256(4 * (size_t)(count + 1) * sizeof(int));
    const size_t o_counters = off;
    b->ncounters = 2 * b->passes + 3;
    off += align256((size_t)b->ncounters * sizeof(int));
    const size_t tables_bytes = off - o_tables;
    if (handle_ws) {
        if (int e = ensure_ws(h, off)) return e;
        b->ws = h->ws;
    } else {
        if (cudaMalloc(&b->ws, off) != cudaSuccess) {
            (void)cudaGetLastError();
            b->ws = nullptr;
            return RXR_ERR_NOMEM;
        }
        b->ws_owned = true;
    }
    char *ws = (char *)b->ws;
    b->statuses = (RxrStatus *)ws;
    b->A.assign(A, A + count);
    b->Q.assign(Q, Q + count);
    b->R.assign(R, R + count);
    b->lda.assign(lda, lda + count);
    b->ldq.assign(ldq, ldq + count);
    b->ldr.assign(ldr, ldr + count);
    b->seed.assign(seed, seed + count);
    for (int k = 0; k < count; ++k) {
        bind_plan(b->plans[k], ws + base[k]);
        b->plans[k].status = b->statuses + k;
    }
    auto dev = [&](size_t o) { return ws + o; };
    b->counters = (int *)dev(o_counters);
    if (!b->tables) return 0;

    // job tables, built on the host (pinned staging of the handle, or a
    // temporary host buffer for a plan's own copy)
    std::vector<char> host_buf;
    char *hs = nullptr;
    if (handle_ws) {
        if (h->h_stage_bytes < tables_bytes) {
            if (h->h_stage) cudaFreeHost(h->h_stage);
            h->h_stage = nullptr;
            h->h_stage_bytes = 0;
            if (cudaMallocHost(&h->h_stage, tables_bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                return RXR_ERR_NOMEM;
            }
            h->h_stage_bytes = tables_bytes;
        }
        hs = (char *)h->h_stage;
    } else {
        host_buf.resize(tables_bytes);
        hs = host_buf.data();
    }
    auto host_at = [&](size_t o) { return hs + (o - o_tables); };
    SketchJob *skj = (SketchJob *)host_at(o_skj);
    ReduceJob *ryj = (ReduceJob *)host_at(o_ryj);
    XrJob *xrj = (XrJob *)host_at(o_xrj);
    SubstJob *prej = (SubstJob *)host_at(o_prej);
    SubstJob *passj = (SubstJob *)host_at(o_passj);
    ReduceJob *rgj = (ReduceJob *)host_at(o_rgj);
    FactorJob *fj = (FactorJob *)host_at(o_fj);
    FinishJob *finj = (FinishJob *)host_at(o_finj);
    int *st_sk = (int *)host_at(o_starts);
    int *st_ry = st_sk + (count + 1);
    int *st_sg = st_ry + (count + 1);
    int *st_rg = st_sg + (count + 1);
    st_sk[0] = st_ry[0] = st_sg[0] = st_rg[0] = 0;
    b->sg_smem = 0;
    const int variant = b->variant;
    for (int k = 0; k < count; ++k) {
        Plan &p = b->plans[k];
        const int nn = (int)n[k];
        skj[k] = SketchJob{A[k], lda[k], m[k], nn, (int)sk[k], seed[k], p.sk_panels, p.sk_ppc,
                           (int)std::min<int64_t>(n[k], kSkNTile), p.sk_gx, p.Ypart, p.status};
        ryj[k] = ReduceJob{p.Ypart, p.sk_gx, sk[k] * n[k], (int)sk[k], nn, 1.0 / sqrt((double)sk[k]), 0, p.Y, sk[k],
                           p.status};
        xrj[k] = XrJob{p.Y, (int)sk[k], nn, sk[k], variant, p.W, p.Rs, p.Racc, p.status};
        prej[k] = SubstJob{A[k], lda[k], m[k], nn, p.Rs, n[k], variant == RXR_NONE ? 1 : 0, Q[k], ldq[k], 1, p.Gpart,
                           p.sg_panels, p.sg_ppc, variant == RXR_NONE ? 1 : 0, p.status};
        passj[k] = SubstJob{Q[k], ldq[k], m[k], nn, p.Rp, n[k], 0, Q[k], ldq[k], 1, p.Gpart, p.sg_panels, p.sg_ppc, 0,
                            p.status};
        rgj[k] = ReduceJob{p.Gpart, p.sg_gx, n[k] * n[k], nn, nn, 1.0, 1, p.G, n[k], p.status};
        fj[k] = FactorJob{p.G, nn, p.Rp, p.Racc, p.C, p.status};
        finj[k] = FinishJob{p.Racc, nn, R[k], ldr[k], p.status, b->d_status + 4 * k};
        st_sk[k + 1] = st_sk[k] + p.sk_gx * p.sk_gy;
        st_ry[k + 1] = st_ry[k] + (int)cdiv(sk[k] * n[k], 256);
        st_sg[k + 1] = st_sg[k] + p.sg_gx;
        st_rg[k + 1] = st_rg[k] + (int)cdiv(n[k] * n[k], 256);
        b->sg_smem = std::max(b->sg_smem, p.sg_smem);  // MAXT <= 3 tiles of n <= 128: the batched kernel's
    }
    if (handle_ws) {
        if (cudaMemcpyAsync(dev(o_tables), hs, tables_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return RXR_ERR_CUDA;
        }
    } else if (cudaMemcpy(dev(o_tables), hs, tables_bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    b->skj = (const SketchJob *)dev(o_skj);
    b->ryj = (const ReduceJob *)dev(o_ryj);
    b->xrj = (const XrJob *)dev(o_xrj);
    b->prej = (const SubstJob *)dev(o_prej);
    b->passj = (const SubstJob *)dev(o_passj);
    b->rgj = (const ReduceJob *)dev(o_rgj);
    b->fj = (const FactorJob *)dev(o_fj);
    b->finj = (const FinishJob *)dev(o_finj);
    b->st_sk = (const int *)dev(o_starts);
    b->st_ry = b->st_sk + (count + 1);
    b->st_sg = b->st_ry + (count + 1);
    b->st_rg = b->st_sg + (count + 1);
    b->tot_sk = st_sk[count];
    b->tot_ry = st_ry[count];
    b->tot_sg = st_sg[count];
    b->tot_rg = st_rg[count];
    const size_t sk_smem = (size_t)(kSkNTile * kSkP + kSkP * kSkSTile) * sizeof(double);
    b->grid_sk = occupancy_grid((const void *)k_sketch_fp64_batched, RXR_THREADS, sk_smem, h->sms, b->tot_sk);
    b->grid_ry = occupancy_grid((const void *)k_reduce_parts_batched, 256, 0, h->sms, b->tot_ry);
    b->grid_rg = occupancy_grid((const void *)k_reduce_parts_batched, 256, 0, h->sms, b->tot_rg);
    b->grid_sg = occupancy_grid((const void *)k_subst_gram_batched, RXR_THREADS, b->sg_smem, h->sms, b->tot_sg);
    return 0;
}

// Enqueue one run of the batch on `st`: no host synchronisation.
int batch_enqueue(rxr_batch *b, cudaStream_t st)
{
    const int count = b->count;
    if (!b->tables) {
        // every problem's own launch sequence, spread over kBatchStreams streams
        // that fork from and join back into st
        if (cudaEventRecord(b->fork, st) != cudaSuccess) return RXR_ERR_CUDA;
        const int K = std::min(count, kBatchStreams);
        for (int j = 0; j < K; ++j)
            if (cudaStreamWaitEvent(b->aux[j], b->fork, 0) != cudaSuccess) return RXR_ERR_CUDA;
        for (int k = 0; k < count; ++k) {
            cudaStream_t sk = b->aux[k % K];
            if (int e = enqueue_cholqr(b->h, b->plans[k], b->A[k], b->lda[k], b->variant, b->seed[k], b->passes,
                                       b->Q[k], b->ldq[k], b->R[k], b->ldr[k], sk, false))
                return e;
            k_status_out<<<1, 32, 0, sk>>>(b->plans[k].status, b->d_status + 4 * k);
            if (launch_ok()) return RXR_ERR_CUDA;
        }
        for (int j = 0; j < K; ++j)
            if (cudaEventRecord(b->join[j], b->aux[j]) != cudaSuccess ||
                cudaStreamWaitEvent(st, b->join[j], 0) != cudaSuccess)
                return RXR_ERR_CUDA;
        return 0;
    }
    if (cudaMemsetAsync(b->statuses, 0, (size_t)count * sizeof(RxrStatus), st) != cudaSuccess ||
        cudaMemsetAsync(b->counters, 0, (size_t)b->ncounters * sizeof(int), st) != cudaSuccess)
        return RXR_ERR_CUDA;
    int c = 0;  // next work-queue counter
    if (b->variant != RXR_NONE) {
        const size_t sk_smem = (size_t)(kSkNTile * kSkP + kSkP * kSkSTile) * sizeof(double);
        k_sketch_fp64_batched<<<b->grid_sk, RXR_THREADS, sk_smem, st>>>(b->skj, b->st_sk, count, b->tot_sk,
                                                                        b->counters + c++);
        k_reduce_parts_batched<<<b->grid_ry, 256, 0, st>>>(b->ryj, b->st_ry, count, b->tot_ry, b->counters + c++);
    }
    k_xr_factor_batched<<<count, 512, 0, st>>>(b->xrj);
    k_subst_gram_batched<<<b->grid_sg, RXR_THREADS, b->sg_smem, st>>>(b->prej, b->st_sg, count, -1, b->tot_sg,
                                                                      b->counters + c++);
    k_reduce_parts_batched<<<b->grid_rg, 256, 0, st>>>(b->rgj, b->st_rg, count, b->tot_rg, b->counters + c++);
    for (int pass = 1; pass <= b->passes; ++pass) {
        const bool last = (pass == b->passes);
        k_factor_batched<<<count, 512, 0, st>>>(b->fj, pass);
        k_subst_gram_batched<<<b->grid_sg, RXR_THREADS, b->sg_smem, st>>>(b->passj, b->st_sg, count, last ? 0 : 1,
                                                                          b->tot_sg, b->counters + c++);
        if (!last)
            k_reduce_parts_batched<<<b->grid_rg, 256, 0, st>>>(b->rgj, b->st_rg, count, b->tot_rg,
                                                               b->counters + c++);
    }
    k_finish_batched<<<count, 256, 0, st>>>(b->finj);
    return launch_ok();
}

// A plan for `count` problems: validated arguments, layout, tables, streams.
int batch_create(rxr_handle h, int count, const double *const *A, const int64_t *m, const int64_t *n,
                 const int64_t *lda, int variant, const int64_t *s, const uint64_t *seed, int passes,
                 double *const *Q, const int64_t *ldq, double *const *R, const int64_t *ldr, int prec,
                 int *d_status, bool handle_ws, cudaStream_t st, rxr_batch **out)
{
    *out = nullptr;
    if (count < 0) return -2;
    if (!A || !m || !n || !lda || !s || !seed || !Q || !ldq || !R || !ldr || !d_status) return -3;
    rxr_batch *b = new rxr_batch();
    b->h = h;
    b->count = count;
    b->variant = variant;
    b->passes = passes;
    b->prec = prec;
    b->d_status = d_status;
    const int base = variant & ~RXR_SKETCH_ROWS;
    b->tables = prec == RXR_FP64 && (variant & RXR_SKETCH_ROWS) == 0 && base != RXR_SHIFTED;
    if (int e = batch_build(b, A, m, n, lda, s, seed, Q, ldq, R, ldr, handle_ws, st)) {
        batch_release(b);
        return e;
    }
    if (!b->tables) {
        if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            batch_release(b);
            return RXR_ERR_CUDA;
        }
        for (int j = 0; j < kBatchStreams; ++j)
            if (cudaStreamCreateWithFlags(&b->aux[j], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&b->join[j], cudaEventDisableTiming) != cudaSuccess) {
                (void)cudaGetLastError();
                batch_release(b);
                return RXR_ERR_CUDA;
            }
    }
    *out = b;
    return 0;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int rxr_create(rxr_handle *h, int device)
{
    if (h == nullptr) return -1;
    *h = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    if (device < 0 || device >= count) return -2;
    DeviceGuard g(device);
    if (!g.ok) return RXR_ERR_CUDA;
    rxr_ctx *c = new rxr_ctx();
    c->device = device;
    c->sms = device_sms(device);
    if (cudaMallocHost(&c->h_status, 4 * sizeof(int)) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        return RXR_ERR_CUDA;
    }
    for (int k = 0; k < kTimers; ++k)
        for (int j = 0; j < 2; ++j) cudaEventCreate(&c->ev[k][j]);
    if (set_kernel_attrs()) {
        cudaFreeHost(c->h_status);
        delete c;
        return RXR_ERR_CUDA;
    }
    *h = c;
    return 0;
}

int rxr_destroy(rxr_handle h)
{
    if (h == nullptr) return 0;
    DeviceGuard g(h->device);
    if (h->ws && h->ws_owned) cudaFree(h->ws);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->dA) cudaFree(h->dA);
    if (h->dQ) cudaFree(h->dQ);
    if (h->dR) cudaFree(h->dR);
    if (h->eval_buf) cudaFree(h->eval_buf);
    if (h->ls_buf) cudaFree(h->ls_buf);
    if (h->sv_buf) cudaFree(h->sv_buf);
    if (h->h_stage) cudaFreeHost(h->h_stage);
    for (int k = 0; k < kTimers; ++k)
        for (int j = 0; j < 2; ++j)
            if (h->ev[k][j]) cudaEventDestroy(h->ev[k][j]);
    for (cudaEvent_t e : h->io_ev)
        if (e) cudaEventDestroy(e);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    delete h;
    return 0;
}

int rxr_workspace_bytes(int64_t m, int64_t n, int64_t s, int prec, size_t *bytes)
{
    if (bytes == nullptr) return -5;
    if (m < 1 || n < 1 || m < n) return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = 0;
    }
    Plan p;
    make_plan(p, m, n, std::max<int64_t>(s, n), prec, device_sms(dev));
    *bytes = p.bytes;
    return 0;
}

int rxr_set_workspace(rxr_handle h, void *d_ws, size_t bytes)
{
    if (h == nullptr) return -1;
    DeviceGuard g(h->device);
    if (h->ws && h->ws_owned) cudaFree(h->ws);
    if (d_ws == nullptr) {
        h->ws = nullptr;
        h->ws_bytes = 0;
        h->ws_owned = true;
    } else {
        h->ws = d_ws;
        h->ws_bytes = bytes;
        h->ws_owned = false;
    }
    return 0;
}

static int cholqr_common(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
                         uint64_t seed, int passes, double *Q, int64_t ldq, double *R, int64_t ldr, int prec,
                         void *stream, int *d_status, bool blocking)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if ((variant == RXR_NONE || variant == RXR_SHIFTED) && s < n) s = n;
    if (int e = check_args(A, m, n, lda, variant, s, passes, Q, ldq, R, ldr, prec)) return e;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    Plan p;
    make_plan(p, m, n, s, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    int e = enqueue_cholqr(h, p, A, lda, variant, seed, passes, Q, ldq, R, ldr, st, blocking && h->timing);
    if (e) return e;
    if (d_status) {
        k_status_out<<<1, 32, 0, st>>>(p.status, d_status);
        if (launch_ok()) return RXR_ERR_CUDA;
    }
    if (!blocking) return 0;
    return finish_blocking(h, p.status, st);
}

int rxr_cholqr(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s, uint64_t seed,
               int passes, double *Q, int64_t ldq, double *R, int64_t ldr, int prec, void *stream)
{
    return cholqr_common(h, A, m, n, lda, variant, s, seed, passes, Q, ldq, R, ldr, prec, stream, nullptr, true);
}

int rxr_cholqr_async(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
                     uint64_t seed, int passes, double *Q, int64_t ldq, double *R, int64_t ldr, int prec, void *stream,
                     int *d_status)
{
    if (d_status == nullptr) return -15;
    return cholqr_common(h, A, m, n, lda, variant, s, seed, passes, Q, ldq, R, ldr, prec, stream, d_status, false);
}

int rxr_cholqr_host(rxr_handle h, const double *hA, int64_t m, int64_t n, int64_t lda, int variant, int64_t s,
                    uint64_t seed, int passes, double *hQ, int64_t ldq, double *hR, int64_t ldr, int prec,
                    void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if ((variant == RXR_NONE || variant == RXR_SHIFTED) && s < n) s = n;
    if (int e = check_args(hA, m, n, lda, variant, s, passes, hQ, ldq, hR, ldr, prec)) return e;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    const int64_t ldd = (m + 1) & ~(int64_t)1;  // even leading dimension: TMA-compatible rows
    const size_t mat = (size_t)ldd * n * 8;
    if (grow((void **)&h->dA, &h->dA_bytes, mat) || grow((void **)&h->dQ, &h->dQ_bytes, mat) ||
        grow((void **)&h->dR, &h->dR_bytes, (size_t)n * n * 8))
        return RXR_ERR_NOMEM;
    if (h->copy_stream == nullptr) {  // first call: the copy stream and its events
        for (cudaEvent_t &e : h->io_ev)
            if (e == nullptr && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                (void)cudaGetLastError();
                e = nullptr;
                return RXR_ERR_CUDA;
            }
        if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            h->copy_stream = nullptr;
            return RXR_ERR_CUDA;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    Plan p;
    make_plan(p, m, n, s, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    const HostIO io{hA, lda, hQ, ldq, h->copy_stream, h->io_ev};
    int e = enqueue_cholqr(h, p, h->dA, ldd, variant, seed, passes, h->dQ, ldd, hR ? h->dR : nullptr, n, st,
                           h->timing, &io);
    if (e) {
        (void)cudaGetLastError();
        cudaStreamSynchronize(h->copy_stream);
        return e;
    }
    if (hR && cudaMemcpy2DAsync(hR, ldr * 8, h->dR, n * 8, n * 8, n, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    return finish_blocking(h, p.status, st);
}

int rxr_cholqr_batched(rxr_handle h, int count, const double *const *A, const int64_t *m, const int64_t *n,
                       const int64_t *lda, int variant, const int64_t *s, const uint64_t *seed, int passes,
                       double *const *Q, const int64_t *ldq, double *const *R, const int64_t *ldr, int prec,
                       void *stream, int *d_status)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (count < 0) return -2;
    if (count == 0) return 0;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    rxr_batch *b = nullptr;
    if (int e = batch_create(h, count, A, m, n, lda, variant, s, seed, passes, Q, ldq, R, ldr, prec, d_status, true,
                             st, &b))
        return e;
    int e = batch_enqueue(b, st);
    std::vector<int> hs_status((size_t)count * 4);
    if (!e && (cudaMemcpyAsync(hs_status.data(), d_status, (size_t)count * 4 * sizeof(int), cudaMemcpyDeviceToHost,
                               st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess)) {
        (void)cudaGetLastError();
        e = RXR_ERR_CUDA;
    }
    if (e) cudaStreamSynchronize(st);
    batch_release(b);
    if (e) return e;
    int code = 0;
    for (int k = 0; k < count && code == 0; ++k)
        if (hs_status[4 * k]) {
            code = hs_status[4 * k];
            if (code == RXR_ERR_CHOL_BREAKDOWN) {
                h->last_pass = hs_status[4 * k + 1];
                h->last_col = hs_status[4 * k + 2];
            }
        }
    return code;
}

int rxr_batch_create(rxr_handle h, int count, const double *const *A, const int64_t *m, const int64_t *n,
                     const int64_t *lda, int variant, const int64_t *s, const uint64_t *seed, int passes,
                     double *const *Q, const int64_t *ldq, double *const *R, const int64_t *ldr, int prec,
                     int *d_status, rxr_batch_plan *plan)
{
    if (plan == nullptr) return -17;
    *plan = nullptr;
    if (h == nullptr) return -1;
    if (count < 1) return -2;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    return batch_create(h, count, A, m, n, lda, variant, s, seed, passes, Q, ldq, R, ldr, prec, d_status, false,
                        nullptr, plan);
}

int rxr_batch_run(rxr_batch_plan plan, void *stream)
{
    if (plan == nullptr) return -1;
    DeviceGuard g(plan->h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    return batch_enqueue(plan, (cudaStream_t)stream);
}

int rxr_batch_destroy(rxr_batch_plan plan)
{
    batch_release(plan);
    return 0;
}

int rxr_set_test_hook(rxr_handle h, int hook, int value)
{
    if (h == nullptr) return -1;
    switch (hook) {
    case RXR_HOOK_STALL: h->test_stall = value != 0; return 0;
    case RXR_HOOK_JACOBI_SWEEPS:
        if (value < 0 || value > 40) return -3;
        h->jacobi_sweeps = value;
        return 0;
    case RXR_HOOK_BATCH_CTAS: {
        const int bucket = value >> 8, ctas = value & 255;
        if (bucket < 0 || bucket >= kBatchTuneBuckets) return -3;
        h->batch_ctas[bucket] = ctas;
        return 0;
    }
    default: return -2;
    }
}

int rxr_last_info(rxr_handle h, int *pass, int *column)
{
    if (h == nullptr) return -1;
    if (pass) *pass = h->last_pass;
    if (column) *column = h->last_col;
    return 0;
}

const char *rxr_status_string(int code)
{
    switch (code) {
    case RXR_OK: return "ok";
    case RXR_ERR_SKETCH_SINGULAR: return "sketch factor singular (rank-deficient sketch or A)";
    case RXR_ERR_CHOL_BREAKDOWN: return "Cholesky breakdown (non-positive pivot)";
    case RXR_ERR_NONFINITE: return "A contains NaN or Inf";
    case RXR_ERR_CUDA: return "CUDA error";
    case RXR_ERR_TIMEOUT: return "bounded device wait timed out";
    case RXR_ERR_NOMEM: return "workspace allocation failed or too small";
    case RXR_ERR_UNSUPPORTED: return "arguments outside what this build supports";
    case RXR_ERR_BAD_SPARSE: return "sparse matrix row pointer or column index out of range";
    case RXR_ERR_NO_CONVERGENCE: return "Jacobi SVD did not converge within its sweep limit";
    default: return code < 0 ? "invalid argument" : "unknown status";
    }
}

int rxr_omega(uint64_t seed, int64_t s, int64_t row0, int64_t rows, float *d_z, void *stream)
{
    if (s < 1) return -2;
    if (row0 < 0) return -3;
    if (rows < 0) return -4;
    if (d_z == nullptr && rows > 0) return -5;
    if (rows == 0) return 0;
    const int64_t calls = rows * ((s + 3) / 4);
    const int blocks = (int)std::min<int64_t>(cdiv(calls, 256), 152 * 16);
    k_omega<<<blocks, 256, 0, (cudaStream_t)stream>>>(seed, s, row0, rows, d_z);
    return launch_ok();
}

int rxr_sketch(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed, double *Y,
               int64_t ldy, int prec, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1 || m < n) return -3;
    if (n < 1) return -4;
    if (lda < m) return -5;
    if (s < 1 || s > RXR_MAX_S) return -6;
    if (Y == nullptr) return -8;
    if (ldy < s) return -9;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16 && prec != RXR_SPLIT_PRECOND) return -10;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, m, n, s, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (int e = enqueue_sketch(p, A, lda, seed, st)) return e;
    if (cudaMemcpy2DAsync(Y, ldy * 8, p.Y, s * 8, s * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_sketch_part(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                    int64_t row0, double *Y, int64_t ldy, int prec, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1) return -3;
    if (n < 1) return -4;
    if (lda < m) return -5;
    if (s < 1 || s > RXR_MAX_S) return -6;
    if (row0 < 0 || row0 > ((int64_t)1 << 62) - m) return -8;
    if (Y == nullptr) return -9;
    if (ldy < s) return -10;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16 && prec != RXR_SPLIT_PRECOND) return -11;
    if (n > kMaxStreamN || m > ((int64_t)1 << 31)) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, m, n, s, prec, h->sms);
    p.row0 = row0;
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (int e = enqueue_sketch(p, A, lda, seed, st)) return e;
    if (cudaMemcpy2DAsync(Y, ldy * 8, p.Y, s * 8, s * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_sum_parts(rxr_handle h, const double *parts, int count, int64_t len, double *out, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (parts == nullptr) return -2;
    if (count < 1) return -3;
    if (len < 1 || len > INT32_MAX) return -4;
    if (out == nullptr) return -5;
    DeviceGuard g(h->device);
    if (int e = ensure_ws(h, 256)) return e;
    RxrStatus *status = (RxrStatus *)h->ws;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    const int64_t threads = (count >= kReduceWarpParts) ? 32 * len : len;
    k_reduce_parts<<<(int)std::min<int64_t>(cdiv(threads, 256), 1 << 20), 256, 0, st>>>(parts, count, len, (int)len,
                                                                                       1, 1.0, 0, out, len, status);
    return launch_ok();
}

int rxr_trmm_upper(rxr_handle h, const double *A, int64_t lda, const double *B, int64_t ldb, int64_t n, double *C,
                   int64_t ldc, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (B == nullptr) return -4;
    if (n < 1 || n > RXR_MAX_N) return -6;
    if (lda < n) return -3;
    if (ldb < n) return -5;
    if (C == nullptr) return -7;
    if (ldc < n) return -8;
    DeviceGuard g(h->device);
    const size_t nn = (size_t)n * n * 8;
    if (int e = ensure_ws(h, 256 + 3 * align256(nn))) return e;
    char *w = (char *)h->ws;
    RxrStatus *status = (RxrStatus *)w;
    double *a = (double *)(w + 256), *b = (double *)(w + 256 + align256(nn)), *c = (double *)(w + 256 + 2 * align256(nn));
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(RxrStatus), st) != cudaSuccess ||
        cudaMemcpy2DAsync(a, n * 8, A, lda * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpy2DAsync(b, n * 8, B, ldb * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    k_trmm_upper<<<(int)cdiv(n * n, 256), 256, 0, st>>>(a, b, c, (int)n, status);
    if (launch_ok()) return RXR_ERR_CUDA;
    if (cudaMemcpy2DAsync(C, ldc * 8, c, n * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return 0;
}

int rxr_sketch_rows(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, int64_t s, uint64_t seed,
                    double *Y, int64_t ldy, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1) return -3;
    if (n < 1) return -4;
    if (lda < m) return -5;
    if (s < 1 || s > RXR_MAX_S) return -6;
    if (Y == nullptr) return -8;
    if (ldy < s) return -9;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, s, n, s, RXR_FP64, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    k_sketch_rows<<<(int)cdiv(s, 8), 256, 0, st>>>(A, lda, m, (int)n, s, seed, Y, ldy, p.status);
    if (launch_ok()) return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_xr_factor(rxr_handle h, const double *Y, int64_t s, int64_t n, int64_t ldy, int variant, double *Rs,
                  int64_t ldrs, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (Y == nullptr) return -2;
    if (n < 1) return -4;
    if (s < n || s > RXR_MAX_S) return -3;
    if (ldy < s) return -5;
    if (variant != RXR_LU && variant != RXR_QR) return -6;
    if (Rs == nullptr) return -7;
    if (ldrs < n) return -8;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, s, n, s, RXR_FP64, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (int e = enqueue_xr(p, Y, ldy, variant, Rs, ldrs, st)) return e;
    if (launch_ok()) return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_precond_gram(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *R, int64_t ldr,
                     double *X, int64_t ldx, double *G, int64_t ldg, int prec, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1 || m < n) return -3;
    if (n < 1) return -4;
    if (lda < m) return -5;
    if (R == nullptr) return -6;
    if (ldr < n) return -7;
    if (X != nullptr && ldx < m) return -9;
    if (G == nullptr) return -10;
    if (ldg < n) return -11;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16) return -12;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, m, n, n, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    // R may have any leading dimension: copy it to the packed n x n buffer
    if (cudaMemcpy2DAsync(p.Rp, n * 8, R, ldr * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    if (prec == RXR_SPLIT_BF16) {
        if (X == nullptr) return RXR_ERR_UNSUPPORTED;
        int *cx = (p.n <= 128) ? split_colexp(p) : nullptr;
        if (int e = split_subst(p, A, lda, p.Rp, X, ldx, st, cx)) return e;
        if (int e = ozaki_gram_enqueue(p, X, ldx, st, cx != nullptr)) return e;
    } else {
        if (int e = enqueue_subst(p, A, lda, p.Rp, 0, X, ldx, true, false, st)) return e;
    }
    if (cudaMemcpy2DAsync(G, ldg * 8, p.G, n * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_gram(rxr_handle h, const double *X, int64_t m, int64_t n, int64_t ldx, double *G, int64_t ldg, int prec,
             void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (X == nullptr) return -2;
    if (m < 1) return -3;
    if (n < 1) return -4;
    if (ldx < m) return -5;
    if (G == nullptr) return -6;
    if (ldg < n) return -7;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16 && prec != RXR_SPLIT_PRECOND) return -8;
    if (n > RXR_MAX_N || (n > kNarrowN && prec != RXR_SPLIT_BF16)) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, m, n, n, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (prec == RXR_SPLIT_BF16) {
        if (int e = ozaki_gram_enqueue(p, X, ldx, st)) return e;
    } else if (prec == RXR_SPLIT_PRECOND) {
        if (int e = split_gram_enqueue(p, X, ldx, st)) return e;
    } else if (int e = enqueue_subst(p, X, ldx, nullptr, 1, nullptr, m, true, false, st)) {
        return e;
    }
    if (cudaMemcpy2DAsync(G, ldg * 8, p.G, n * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_lstsq(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *b, int64_t k,
              int64_t ldb, int variant, int64_t s, uint64_t seed, double *x, int64_t ldx, int prec, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1 || m < n) return -3;
    if (n < 1) return -4;
    if (lda < m) return -5;
    if (b == nullptr) return -6;
    if (k < 1 || k > 64) return -7;
    if (ldb < m) return -8;
    const int base = variant & ~RXR_SKETCH_ROWS;
    if (base != RXR_LU && base != RXR_QR) return -9;
    if (s < n || s > RXR_MAX_S) return -10;
    if (x == nullptr) return -12;
    if (ldx < n) return -13;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16) return -14;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    const bool rows = (variant & RXR_SKETCH_ROWS) != 0;
    Plan p;
    make_plan(p, m, n, s, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    const int64_t ldB = (m + 1) & ~(int64_t)1;  // even: TMA-compatible rows
    const int64_t rpc = std::max<int64_t>(256, cdiv(m, 4 * (int64_t)h->sms));  // rows of B^T b per CTA
    const int64_t gx = cdiv(m, rpc);
    if (grow((void **)&h->dQ, &h->dQ_bytes, (size_t)ldB * n * 8) ||
        grow((void **)&h->ls_buf, &h->ls_bytes, (size_t)(gx + 1) * n * k * 8))
        return RXR_ERR_NOMEM;
    double *B = h->dQ, *parts = h->ls_buf, *c = h->ls_buf + gx * n * k;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    // the sketch's R factor
    if (rows) {
        k_sketch_rows<<<(int)cdiv(s, 8), 256, 0, st>>>(A, lda, m, (int)n, s, seed, p.Y, s, p.status);
        if (launch_ok()) return RXR_ERR_CUDA;
    } else if (int e = enqueue_sketch(p, A, lda, seed, st)) {
        return e;
    }
    if (int e = enqueue_xr(p, p.Y, s, base, p.Rs, n, st)) return e;
    // B = A R_s^{-1} with G = B^T B at FP64 grade (it sets the solution's accuracy)
    if (prec == RXR_SPLIT_BF16) {
        int *cx = (n <= 128) ? split_colexp(p) : nullptr;
        if (rows && !cx) {
            k_check_finite<<<4 * p.sms, 256, 0, st>>>(A, lda, m, (int)n, p.status);
            if (launch_ok()) return RXR_ERR_CUDA;
        }
        if (int e = split_subst(p, A, lda, p.Rs, B, ldB, st, cx)) return e;
        if (int e = ozaki_gram_enqueue(p, B, ldB, st, cx != nullptr)) return e;
    } else if (int e = enqueue_subst(p, A, lda, p.Rs, 0, B, ldB, true, rows, st)) {
        return e;
    }
    // c = B^T b, R_G = chol(G), then the three small solves
    k_ls_btb<<<(int)gx, 256, 0, st>>>(B, ldB, m, (int)n, b, ldb, (int)k, rpc, parts, p.status);
    if (launch_ok()) return RXR_ERR_CUDA;
    const int64_t nk = n * k;
    const int64_t threads = (gx >= kReduceWarpParts) ? 32 * nk : nk;
    k_reduce_parts<<<(int)cdiv(threads, 256), 256, 0, st>>>(parts, (int)gx, nk, (int)n, (int)k, 1.0, 0, c, n,
                                                           p.status);
    if (launch_ok()) return RXR_ERR_CUDA;
    if (n > 64) {
        if (int e = blocked_factor_enqueue(p.G, (int)n, n, p.Rp, p.Racc, p.C, 1, 0, p.status, st)) return e;
    } else {
        k_factor<<<1, 512, factor_smem_bytes(n), st>>>(p.G, (int)n, n, p.Rp, p.Racc, p.C, 1, 0, p.status);
        if (launch_ok()) return RXR_ERR_CUDA;
    }
    k_ls_solve<<<1, 512, 0, st>>>(p.Rp, p.Rs, (int)n, (int)k, c, x, ldx, p.status);
    if (launch_ok()) return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_rsvd(rxr_handle h, int64_t m, int64_t n, const int64_t *a_ptr, const int32_t *a_idx, const double *a_val,
             const int64_t *t_ptr, const int32_t *t_idx, const double *t_val, int64_t nnz, const double *X,
             int64_t ldx, int64_t k, int iters, int variant, int64_t s, uint64_t seed, int passes, int prec,
             double *U, int64_t ldu, double *S, double *V, int64_t ldv, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (m < 1) return -2;
    if (n < 1) return -3;
    if (a_ptr == nullptr) return -4;
    if (nnz > 0 && a_idx == nullptr) return -5;
    if (nnz > 0 && a_val == nullptr) return -6;
    if (t_ptr == nullptr) return -7;
    if (nnz > 0 && t_idx == nullptr) return -8;
    if (nnz > 0 && t_val == nullptr) return -9;
    if (nnz < 0) return -10;
    if (X == nullptr) return -11;
    if (ldx < n) return -12;
    if (k < 1 || k > m || k > n) return -13;
    if (iters < 0 || iters > 1000) return -14;
    const int base = variant & ~RXR_SKETCH_ROWS;
    if ((base == RXR_NONE || base == RXR_SHIFTED) && s < k) s = k;
    // the factorisations' own checks, for the m x k and the n x k blocks
    for (int64_t rows : {m, n}) {
        const int e = check_args(X, rows, k, rows, variant, s, passes, X, rows, nullptr, k, prec);
        if (e == -5) return -15;
        if (e == -6) return -16;
        if (e == -8) return -18;
        if (e == -13) return -19;
        if (e) return e;
    }
    if (U == nullptr) return -20;
    if (ldu < m) return -21;
    if (S == nullptr) return -22;
    if (V == nullptr) return -23;
    if (ldv < n) return -24;
    if (k > kNarrowN || n > INT32_MAX) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return RXR_ERR_CUDA;
    Plan pm, pn;
    make_plan(pm, m, k, s, prec, h->sms);
    make_plan(pn, n, k, s, prec, h->sms);
    if (int e = ensure_ws(h, std::max(pm.bytes, pn.bytes))) return e;
    bind_plan(pm, h->ws);
    bind_plan(pn, h->ws);
    // scratch: status | Y (m x k) | Q (m x k) | Z (n x k) | Q_z (n x k) | row-major
    // copy (max(m, n) x k) | R_z | U_r | V_r | V_r's Jacobi scratch (k x k each)
    const int64_t ldm = (m + 1) & ~(int64_t)1, ldn = (n + 1) & ~(int64_t)1;  // even: TMA-compatible rows
    auto al = [](int64_t d) { return (d + 31) & ~(int64_t)31; };
    const int64_t o_ym = 32, o_qm = o_ym + al(ldm * k), o_zn = o_qm + al(ldm * k), o_qn = o_zn + al(ldn * k);
    const int64_t o_xr = o_qn + al(ldn * k), o_rz = o_xr + al(std::max(m, n) * k), o_ur = o_rz + al(k * k);
    const int64_t o_vr = o_ur + al(k * k), o_vg = o_vr + al(k * k), total = o_vg + al(k * k);
    if (grow((void **)&h->sv_buf, &h->sv_bytes, (size_t)total * 8)) return RXR_ERR_NOMEM;
    double *b = h->sv_buf;
    RxrStatus *acc = (RxrStatus *)b;
    double *Ym = b + o_ym, *Qm = b + o_qm, *Zn = b + o_zn, *Qn = b + o_qn, *Xr = b + o_xr;
    double *Rz = b + o_rz, *Ur = b + o_ur, *Vr = b + o_vr, *Vg = b + o_vg;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(acc, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    const int kk = (int)k;
    int call = 0;
    // orthonormalisation `call`: Q_b = the Q factor of Y_b by CholeskyQR, seed + call
    auto orth = [&](const Plan &p, double *Yb, int64_t ld, double *Qb, double *R) -> int {
        if (int e = enqueue_cholqr(h, p, Yb, ld, variant, seed + (uint64_t)call, passes, Qb, ld, R, kk, st, false))
            return e;
        return rsvd_status_keep_enqueue(p.status, acc, call++, st);
    };
    auto a_mul = [&](const double *B, int64_t ldb) -> int {  // Y = A B, B n x k
        if (int e = rsvd_transpose_enqueue(B, ldb, n, kk, Xr, st)) return e;
        return rsvd_spmm_enqueue(a_ptr, a_idx, a_val, nnz, m, n, Xr, kk, Ym, ldm, acc, st);
    };
    auto at_mul = [&](const double *B, int64_t ldb) -> int {  // Z = A^T B, B m x k
        if (int e = rsvd_transpose_enqueue(B, ldb, m, kk, Xr, st)) return e;
        return rsvd_spmm_enqueue(t_ptr, t_idx, t_val, nnz, n, m, Xr, kk, Zn, ldn, acc, st);
    };
    if (int e = a_mul(X, ldx)) return e;
    if (int e = orth(pm, Ym, ldm, Qm, nullptr)) return e;
    for (int it = 0; it < iters; ++it) {
        if (int e = at_mul(Qm, ldm)) return e;
        if (int e = orth(pn, Zn, ldn, Qn, nullptr)) return e;
        if (int e = a_mul(Qn, ldn)) return e;
        if (int e = orth(pm, Ym, ldm, Qm, nullptr)) return e;
    }
    // B^T = A^T Y = Q_z R_z, R_z = U_r S V_r^T: Y^T A = V_r S (Q_z U_r)^T
    if (int e = at_mul(Qm, ldm)) return e;
    if (int e = orth(pn, Zn, ldn, Qn, Rz)) return e;
    if (int e = rsvd_jacobi_enqueue(Rz, k, kk, Ur, Vr, S, Vg, acc, h->jacobi_sweeps, st)) return e;
    if (int e = rsvd_right_mult_enqueue(Qm, ldm, m, kk, Vr, U, ldu, acc, st)) return e;
    if (int e = rsvd_right_mult_enqueue(Qn, ldn, n, kk, Ur, V, ldv, acc, st)) return e;
    return finish_blocking(h, acc, st);
}

int rxr_apply_rinv(rxr_handle h, double *X, int64_t m, int64_t n, int64_t ldx, const double *R, int64_t ldr, int prec,
                   void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (X == nullptr) return -2;
    if (m < 1 || m < n) return -3;
    if (n < 1) return -4;
    if (ldx < m) return -5;
    if (R == nullptr) return -6;
    if (ldr < n) return -7;
    if (prec != RXR_FP64 && prec != RXR_SPLIT_BF16) return -8;
    if (n > kMaxStreamN) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, m, n, n, prec, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (cudaMemcpy2DAsync(p.Rp, n * 8, R, ldr * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    if (prec == RXR_SPLIT_BF16 && n <= 64) {
        if (int e = ozaki_apply_enqueue(p, X, ldx, p.Rp, st)) return e;
    } else if (prec == RXR_SPLIT_BF16 && n <= 128) {
        if (int e = delta128_apply_enqueue(p, X, ldx, p.Rp, st)) return e;
    } else if (prec == RXR_SPLIT_BF16) {
        if (int e = split_subst(p, X, ldx, p.Rp, X, ldx, st)) return e;
    } else if (int e = enqueue_subst(p, X, ldx, p.Rp, 0, X, ldx, false, false, st)) {
        return e;
    }
    return finish_blocking(h, p.status, st);
}

int rxr_cholesky(rxr_handle h, const double *G, int64_t n, int64_t ldg, double *R, int64_t ldr, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (G == nullptr) return -2;
    if (n < 1) return -3;
    if (ldg < n) return -4;
    if (R == nullptr) return -5;
    if (ldr < n) return -6;
    if (n > RXR_MAX_N) return RXR_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    Plan p;
    make_plan(p, n, n, n, RXR_FP64, h->sms);
    if (int e = ensure_ws(h, p.bytes)) return e;
    bind_plan(p, h->ws);
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(p.status, 0, sizeof(RxrStatus), st) != cudaSuccess) return RXR_ERR_CUDA;
    if (n > 64) {
        if (int e = blocked_factor_enqueue(G, (int)n, ldg, p.Rp, p.Racc, p.C, 1, 0, p.status, st)) return e;
    } else {
        k_factor<<<1, 512, factor_smem_bytes(n), st>>>(G, (int)n, ldg, p.Rp, p.Racc, p.C, 1, 0, p.status);
    }
    if (launch_ok()) return RXR_ERR_CUDA;
    if (cudaMemcpy2DAsync(R, ldr * 8, p.Rp, n * 8, n * 8, n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return RXR_ERR_CUDA;
    return finish_blocking(h, p.status, st);
}

int rxr_orth_error(rxr_handle h, const double *Q, int64_t m, int64_t n, int64_t ldq, double *out, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (Q == nullptr) return -2;
    if (m < 1) return -3;
    if (n < 1 || n > RXR_MAX_N) return -4;
    if (ldq < m) return -5;
    if (out == nullptr) return -6;
    DeviceGuard g(h->device);
    const int npairs = (int)(n * (n + 1) / 2);
    const int gy = (int)cdiv(npairs, 256);
    const int64_t chunks = std::min<int64_t>(cdiv(m, 64), std::max<int64_t>(1, 2 * h->sms / gy + 1));
    const int64_t rpc = cdiv(cdiv(m, chunks), 64) * 64;
    const int64_t nch = cdiv(m, rpc);
    if (grow((void **)&h->eval_buf, &h->eval_bytes, ((size_t)nch * npairs * 2 + 8) * 8)) return RXR_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    const int evp = (n <= 128) ? 64 : 32;  // rows staged per step: evp * n doubles of shared memory
    const size_t smem = (size_t)evp * n * 8;
    k_orth_partial<<<dim3((unsigned)nch, gy), 256, smem, st>>>(Q, m, (int)n, ldq, rpc, evp, h->eval_buf);
    if (launch_ok()) return RXR_ERR_CUDA;
    double *res = h->eval_buf + (size_t)nch * npairs * 2;
    k_orth_final<<<1, 1024, 0, st>>>(h->eval_buf, (int)nch, (int)n, res);
    if (launch_ok()) return RXR_ERR_CUDA;
    if (cudaMemcpyAsync(out, res, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    return 0;
}

int rxr_resid_error(rxr_handle h, const double *A, int64_t m, int64_t n, int64_t lda, const double *Q, int64_t ldq,
                    const double *R, int64_t ldr, double *out, void *stream)
{
    if (h == nullptr) return RXR_ERR_CUDA;
    if (A == nullptr) return -2;
    if (m < 1) return -3;
    if (n < 1 || n > RXR_MAX_N) return -4;
    if (lda < m) return -5;
    if (Q == nullptr) return -6;
    if (ldq < m) return -7;
    if (R == nullptr) return -8;
    if (ldr < n) return -9;
    if (out == nullptr) return -10;
    DeviceGuard g(h->device);
    const int blocks = (int)std::min<int64_t>(cdiv(m, 256), 4 * h->sms);
    if (grow((void **)&h->eval_buf, &h->eval_bytes, ((size_t)blocks * 2 + 8) * 8)) return RXR_ERR_NOMEM;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t smem = (n * (n + 1) / 2 <= 16384) ? (size_t)(n * (n + 1) / 2) * 8 : 0;
    k_resid_partial<<<blocks, 256, smem, st>>>(A, lda, Q, ldq, R, ldr, m, (int)n, h->eval_buf);
    if (launch_ok()) return RXR_ERR_CUDA;
    double *res = h->eval_buf + (size_t)blocks * 2;
    k_resid_final<<<1, 32, 0, st>>>(h->eval_buf, blocks, res);
    if (launch_ok()) return RXR_ERR_CUDA;
    if (cudaMemcpyAsync(out, res, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_CUDA;
    }
    return 0;
}

int rxr_fp64_peak(double *tflops, void *stream)
{
    if (tflops == nullptr) return -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RXR_ERR_CUDA;
    const int sms = device_sms(dev);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    double *buf = nullptr;
    if (cudaMalloc(&buf, (size_t)blocks * threads * 8) != cudaSuccess) {
        (void)cudaGetLastError();
        return RXR_ERR_NOMEM;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int rc = 0;
    for (int rep = 0; rep < 4 && rc == 0; ++rep) {
        cudaEventRecord(e0, st);
        k_fp64_peak<<<blocks, threads, 0, st>>>(buf, iters, 0.999, 1e-3);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = RXR_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    if (rc) {
        (void)cudaGetLastError();
        return rc;
    }
    *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
    return 0;
}

int rxr_last_kernel_ms(rxr_handle h, int kernel, float *ms)
{
    if (h == nullptr || ms == nullptr) return -1;
    if (kernel < 0 || kernel >= kTimers) return -1;
    *ms = h->last_ms[kernel];
    return 0;
}

int rxr_set_kernel_timing(rxr_handle h, int enable)
{
    if (h == nullptr) return -1;
    h->timing = enable != 0;
    return 0;
}

}  // extern "C"
