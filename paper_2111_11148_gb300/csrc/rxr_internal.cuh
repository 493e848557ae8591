// rxr_internal.cuh -- device helpers shared by the librxr CUDA translation units.
// Randomized XR-preconditioned CholeskyQR (Fan, Guo & Lin), GB300 (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rxr.h"

#define RXR_THREADS 256

// ---------------------------------------------------------------------------
// Device status word {code, pass, column, flags}.  Kernels set the first
// failure with atomicCAS on code so that the earliest failure in stream order
// wins; every streaming kernel returns immediately when code != 0.
// ---------------------------------------------------------------------------
struct RxrStatus {
    int code;
    int pass;
    int column;
    int flags;
};

__device__ __forceinline__ void rxr_fail(RxrStatus *st, int code, int pass, int column)
{
    if (atomicCAS(&st->code, 0, code) == 0) {
        st->pass = pass;
        st->column = column;
    }
}

__device__ __forceinline__ bool rxr_failed(const RxrStatus *st)
{
    return *((volatile const int *)&st->code) != 0;
}

// The same check taken once for the whole CTA (every thread must call it):
// another CTA may set the status word at any moment, and threads that read it
// at different times and decided differently would leave the others waiting
// at the CTA's next barrier.
__device__ __forceinline__ bool rxr_failed_block(const RxrStatus *st)
{
    return __syncthreads_or(threadIdx.x == 0 && rxr_failed(st)) != 0;
}

// Test hook (rxr_set_test_hook, RXR_HOOK_STALL): when the host sets this bit in
// the status word's flags, the kernels that stream A by TMA skip the first copy
// of their first CTA, so that CTA's bounded wait runs out on an mbarrier that
// nothing arrives at (no copy is in flight) and the call reports
// RXR_ERR_TIMEOUT through the ordinary error path.
constexpr int kFlagStall = 1;
__device__ __forceinline__ bool rxr_stall_requested(const RxrStatus *st)
{
    return (*((volatile const int *)&st->flags) & kFlagStall) != 0;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of
//   (c0,c1,c2,c3) -> (hi(Mb*c2)^c1^k0, lo(Mb*c2), hi(Ma*c0)^c3^k1, lo(Ma*c0))
// with the key bumped by the golden-ratio Weyl increments between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                              uint32_t k1)
{
    constexpr uint32_t Ma = 0xD2511F53u, Mb = 0xCD9E8D57u;
    constexpr uint32_t Wa = 0x9E3779B9u, Wb = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(Ma, c0), loA = Ma * c0;
        const uint32_t hiB = __umulhi(Mb, c2), loB = Mb * c2;
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += Wa;
        k1 += Wb;
    }
}

// ---------------------------------------------------------------------------
// Single-precision log on (0,1] from log x = 2 atanh((x-1)/(x+1)), with
// u = 2^e x, x in [1/sqrt2, sqrt2]; odd series in t = (x-1)/(x+1) through
// t^13, then e*ln2 added in two pieces.  Only explicitly rounded intrinsics, so
// the bits are fixed by IEEE single precision.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rxr_logf(float u)
{
    const uint32_t b = __float_as_uint(u);
    const uint32_t xb = (b & 0x007FFFFFu) | 0x3F800000u;
    const bool big = xb > 0x3FB504F3u;  // above sqrt(2): halve (exact; the exponent field drops by one)
    const int e = (int)((b >> 23) & 0xFFu) - 127 + (big ? 1 : 0);
    const float x = __uint_as_float(big ? xb - 0x00800000u : xb);
    const float t = __fdiv_rn(__fsub_rn(x, 1.0f), __fadd_rn(x, 1.0f));
    const float t2 = __fmul_rn(t, t);
    float p = (float)(2.0 / 13.0);
    p = __fmaf_rn(p, t2, (float)(2.0 / 11.0));
    p = __fmaf_rn(p, t2, (float)(2.0 / 9.0));
    p = __fmaf_rn(p, t2, (float)(2.0 / 7.0));
    p = __fmaf_rn(p, t2, (float)(2.0 / 5.0));
    p = __fmaf_rn(p, t2, (float)(2.0 / 3.0));
    const float lx = __fmaf_rn(__fmul_rn(t, t2), p, __fadd_rn(t, t));
    constexpr double kLn2 = 0.6931471805599453094172321214581766;
    constexpr float kLn2Hi = (float)kLn2;
    constexpr float kLn2Lo = (float)(kLn2 - (double)kLn2Hi);
    const float fe = __int2float_rn(e);
    return __fmaf_rn(fe, kLn2Hi, __fmaf_rn(fe, kLn2Lo, lx));
}

// sin and cos of 2 pi u with u = n 2^-24: the quadrant q = round(4u) is taken in
// integers, the remainder f = 4u - q in [-1/2, 1/2) is exact, and
// sin(pi f / 2), cos(pi f / 2) come from their Maclaurin series in f.
__device__ __forceinline__ void rxr_sincos2pi(uint32_t n, float &s_out, float &c_out)
{
    constexpr double h = 1.5707963267948966192313216916397514;  // pi / 2
    constexpr double h2 = h * h;
    constexpr float s1 = (float)h, s3 = (float)(-h * h2 / 6.0), s5 = (float)(h * h2 * h2 / 120.0);
    constexpr float s7 = (float)(-h * h2 * h2 * h2 / 5040.0), s9 = (float)(h * h2 * h2 * h2 * h2 / 362880.0);
    constexpr float c0 = 1.0f, c2 = (float)(-h2 / 2.0), c4 = (float)(h2 * h2 / 24.0);
    constexpr float c6 = (float)(-h2 * h2 * h2 / 720.0), c8 = (float)(h2 * h2 * h2 * h2 / 40320.0);
    constexpr float c10 = (float)(-h2 * h2 * h2 * h2 * h2 / 3628800.0);
    const int q = (int)((n + (1u << 21)) >> 22);
    const int r = (int)n - q * (1 << 22);
    const float f = __fmul_rn(__int2float_rn(r), 0x1p-22f);
    const float f2 = __fmul_rn(f, f);
    float sp = s9;
    sp = __fmaf_rn(sp, f2, s7);
    sp = __fmaf_rn(sp, f2, s5);
    sp = __fmaf_rn(sp, f2, s3);
    const float sn = __fmaf_rn(__fmul_rn(f, f2), sp, __fmul_rn(s1, f));
    float cp = c10;
    cp = __fmaf_rn(cp, f2, c8);
    cp = __fmaf_rn(cp, f2, c6);
    cp = __fmaf_rn(cp, f2, c4);
    cp = __fmaf_rn(cp, f2, c2);
    const float cs = __fmaf_rn(cp, f2, c0);
    // quadrant q: (sin, cos) = (sn, cs), (cs, -sn), (-sn, -cs), (-cs, sn), by selects
    const float a = (q & 1) ? cs : sn, b = (q & 1) ? sn : cs;
    s_out = (q & 2) ? -a : a;
    c_out = ((q + 1) & 2) ? -b : b;
}

// Four N(0,1) values for sketch rows 4k..4k+3 of column i (row i of A):
// Philox counter (i_lo, i_hi, k, stream), key (seed_lo, seed_hi); uniforms
// u = ((x >> 8) + 1) 2^-24 in (0,1]; Box-Muller pairs (x0,x1) and (x2,x3).
__device__ __forceinline__ void rxr_normal4(uint64_t seed, uint64_t i, uint32_t k, uint32_t stream, float z[4])
{
    uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(i >> 32), c2 = k, c3 = stream;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t xs[4] = {c0, c1, c2, c3};
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const uint32_t na = (xs[2 * hh] >> 8) + 1u, nb = (xs[2 * hh + 1] >> 8) + 1u;
        const float ua = __fmul_rn(__uint2float_rn(na), 0x1p-24f);
        const float rad = __fsqrt_rn(__fmul_rn(-2.0f, rxr_logf(ua)));
        float sn, cs;
        rxr_sincos2pi(nb, sn, cs);
        z[2 * hh] = __fmul_rn(rad, cs);
        z[2 * hh + 1] = __fmul_rn(rad, sn);
    }
}

// Exact float -> double by bit manipulation on the integer pipes (the FP64
// pipe of this part is scarce).  Valid for zero and normal floats, which is
// all the Box-Muller outputs can be.
__device__ __forceinline__ double rxr_f2d_exact(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t sign = b & 0x80000000u;
    const uint32_t mag = b & 0x7FFFFFFFu;
    const uint32_t e = (mag >> 23) + (1023u - 127u);
    const uint32_t mant = mag & 0x007FFFFFu;
    const uint32_t hi = (mag == 0u) ? sign : (sign | (e << 20) | (mant >> 3));  // a select, not a branch
    const uint32_t lo = mant << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// Non-finite test on the integer pipes: exponent field all ones.
__device__ __forceinline__ bool rxr_nonfinite(double v)
{
    return (((uint32_t)__double2hiint(v)) & 0x7FF00000u) == 0x7FF00000u;
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (cp.async.bulk.tensor) helpers.  Every wait is bounded: a
// waiter polls with try_wait (its own suspend limit, the fastest wake-up on
// this part) and gives up after kSpinLimit polls or kWaitLimitNs of the global
// timer, whichever comes first, recording RXR_ERR_TIMEOUT.  The timer is read
// once per kPollsPerCheck polls, outside the tight polling loop (any code in
// that loop slowed the tensor-core Gram's producer/consumer hand-offs).
constexpr uint32_t kSpinLimit = 1u << 20;
constexpr uint32_t kPollsPerCheck = 4096;
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false (and records a timeout) if the phase never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, RxrStatus *st)
{
    uint64_t t0 = 0;
    for (uint32_t outer = 0; outer < kSpinLimit / kPollsPerCheck; ++outer) {
        for (uint32_t it = 0; it < kPollsPerCheck; ++it)
            if (mbar_try_wait(bar, phase)) return true;
        const uint64_t t = globaltimer_ns();
        if (outer == 0)
            t0 = t;
        else if (t - t0 > kWaitLimitNs)
            break;
    }
    rxr_fail(st, RXR_ERR_TIMEOUT, -1, -1);
    return false;
}

// 2-D tiled TMA load of a box at element coordinates (x = row, y = column)
// into shared memory, completing on `bar`.  x * 8 must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(smem_dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 1-D bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load_1d(void *smem_dst, const void *gsrc, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(smem_dst)),
                 "l"((uint64_t)gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 2-D tiled TMA store of a shared-memory box to element coordinates (x = row,
// y = column); rows past the tensor's extent are not written.  Completion is
// tracked by the issuing thread's bulk async-group.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *smem_src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(smem_u32(smem_src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of every committed store have been read
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// every committed store has completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Block-wide helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

namespace rxr {
// Per-problem arguments of the batched launches (one entry per problem).
struct SketchJob {
    const double *A;
    int64_t lda, m;
    int n, s;
    uint64_t seed;
    int64_t panels_total, panels_per_cta;
    int box_cols, gx;
    double *Ypart;
    RxrStatus *st;
};
struct ReduceJob {
    const double *parts;
    int nparts;
    int64_t stride;
    int rows, cols;
    double scale;
    int symmetric;
    double *out;
    int64_t ldo;
    RxrStatus *st;
};
struct SubstJob {
    const double *src;
    int64_t lds, m;
    int n;
    const double *R;
    int64_t ldr;
    int unit_r;
    double *dst;
    int64_t ldd;
    int do_gram;
    double *Gpart;
    int64_t panels_total, panels_per_cta;
    int check_finite;
    RxrStatus *st;
};
struct XrJob {
    const double *Y;
    int s, n;
    int64_t ldy;
    int variant;
    double *W, *Rs, *Racc;
    RxrStatus *st;
};
struct FactorJob {
    const double *G;
    int n;
    double *Rp, *Racc, *C;
    RxrStatus *st;
};
struct FinishJob {
    const double *Racc;
    int n;
    double *R;
    int64_t ldr;
    const RxrStatus *st;
    int *status_out;
};

// Launch geometry and workspace offsets of one factorisation.
struct Plan {
    int64_t m, n, s;
    int64_t row0;  // global index of A's first row: Omega's columns follow it (row shards)
    int prec;
    int sms;
    // sketch
    int sk_gx, sk_gy;
    int64_t sk_panels, sk_ppc;
    int64_t yslots;  // partial sums the sketch buffer holds (>= sk_gx; the split sketch may use more)
    // substitution + Gram
    int sg_gx;
    int64_t sg_panels, sg_ppc;
    size_t sg_smem;
    int sg_maxt;
    // wide panels (n > 128): column-blocked substitution + tiled Gram
    int wide;
    int gt_gx, gt_gy;
    int64_t gt_ppc;
    // workspace pieces
    char *base;
    RxrStatus *status;
    double *Ypart, *Y, *W, *Gpart, *G, *Rs, *Rp, *Racc, *C;
    char *split;  // split-precision scratch
    size_t bytes;
};
}  // namespace rxr

namespace rxr {
// Row chunks of the split sketch's CTA partition: the sketch of a matrix that
// arrives from the host in this many row chunks starts on each chunk as it
// lands, with the partition (and so the result) of a single launch.
constexpr int kSketchChunks = 8;
// From this many partial sums on, k_reduce_parts gives each output a warp
// (launch it with 32 threads per output).
constexpr int kReduceWarpParts = 256;
int64_t balanced_chunks(int64_t gy, int64_t slots, int64_t max_gx);
// split-precision contractions (split_kernels.cu)
int split_sketch_enqueue(Plan &p, const double *A, int64_t lda, uint64_t seed, cudaStream_t st);
void split_sketch_grid(const Plan &p, int64_t *gx, int64_t *spc);
int split_sketch_part_enqueue(Plan &p, const double *A, int64_t lda, uint64_t seed, int64_t cta_begin, int64_t cta_end,
                              cudaStream_t st);
int split_sketch_reduce_enqueue(Plan &p, cudaStream_t st);
int split_gram_enqueue(Plan &p, const double *X, int64_t ldx, cudaStream_t st);
// colexp_ready: the column exponents of X (n <= 64) are already in
// split_colexp(p), written by the substitution that produced X
int ozaki_gram_enqueue(Plan &p, const double *X, int64_t ldx, cudaStream_t st, bool colexp_ready = false);
int *split_colexp(const Plan &p);
int ozaki_apply_enqueue(Plan &p, double *X, int64_t ldx, const double *R, cudaStream_t st);
int ozaki_apply_prepare(Plan &p, const double *R, cudaStream_t st);
int ozaki_apply_rows(Plan &p, double *X, int64_t ldx, int64_t r0, int64_t rows, cudaStream_t st);
int blocked_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                          int64_t ldx, cudaStream_t st);
int fused_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                        int64_t ldx, int *colexp_out, cudaStream_t st, const int *sel = nullptr);
int middle_pass_enqueue(Plan &p, double *X, int64_t ldx, const double *R, int *colexp_out, int *sel,
                        cudaStream_t st);
int *split_select_flag(const Plan &p);
// sel (nullable): a device flag; nonzero makes the substitution return at once
// colexp_out (nullable, zeroed by the caller): X's largest exponent per column
// is max-ed into it (for the FP64-grade Gram that follows)
int fused128_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                           int64_t ldx, cudaStream_t st, const int *sel = nullptr, int *colexp_out = nullptr);
// 64 < n <= 128: X <- X R^{-1}, the FP32 correction X + X (R^{-1} - I) when
// |R^{-1} - I| <= 2^-38 (chosen on the device), else the fused substitution
int delta128_apply_enqueue(Plan &p, double *X, int64_t ldx, const double *R, cudaStream_t st);
// 2-D tensor map of a column-major FP64 matrix (api.cu); false where TMA's
// alignment rules are not met.  swizzle128: 128-byte swizzle (box_rows <= 16;
// in shared memory, 16-byte chunk c of box column j sits at chunk c ^ (j mod 8))
bool encode_tile_map(CUtensorMap *map, const void *ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                     int box_cols, bool swizzle128 = false);
size_t split_workspace_bytes(int64_t m, int64_t n, int64_t s, int sms);
// dynamic shared memory of the one-CTA factorisations (small_kernels.cu)
size_t xr_smem_bytes(int64_t s, int64_t n);
size_t factor_smem_bytes(int64_t n);
cudaError_t set_small_smem();
// blocked multi-CTA rQR of the sketch (small_kernels.cu)
int blocked_qr_enqueue(const double *Y, int s, int n, int64_t ldy, double *W, double *Rs, int64_t ldrs,
                       double *scratch, RxrStatus *status, cudaStream_t st);
size_t blocked_qr_scratch_doubles(int64_t s, int64_t n);
// blocked multi-CTA Cholesky R_p = chol(G) (+ R_acc <- R_p R_acc) for n > 64
int blocked_factor_enqueue(const double *G, int n, int64_t ldg, double *Rp, double *Racc, double *C, int pass,
                           int update_racc, RxrStatus *status, cudaStream_t st);
// randomized SVD (rsvd_kernels.cu): sparse products, the k x k SVD and the
// finishing products; every launcher returns 0 or RXR_ERR_CUDA
int rsvd_transpose_enqueue(const double *X, int64_t ldx, int64_t rows, int k, double *Xr, cudaStream_t st);
int rsvd_spmm_enqueue(const int64_t *ptr, const int32_t *idx, const double *val, int64_t nnz, int64_t rows,
                      int64_t cols, const double *Xr, int k, double *Y, int64_t ldy, RxrStatus *acc, cudaStream_t st);
// max_sweeps outside 1..40 takes the default bound of 40 sweeps
int rsvd_jacobi_enqueue(const double *R, int64_t ldr, int k, double *Ur, double *Vr, double *S, double *Vg,
                        RxrStatus *acc, int max_sweeps, cudaStream_t st);
int rsvd_right_mult_enqueue(const double *X, int64_t ldx, int64_t rows, int k, const double *T, double *Y,
                            int64_t ldy, const RxrStatus *acc, cudaStream_t st);
int rsvd_status_keep_enqueue(const RxrStatus *cur, RxrStatus *acc, int call, cudaStream_t st);
cudaError_t set_rsvd_smem();
}  // namespace rxr
