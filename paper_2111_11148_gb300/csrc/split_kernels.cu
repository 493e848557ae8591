// split_kernels.cu -- the two contractions that only shape the preconditioner,
// computed on the 5th-generation tensor cores (tcgen05, BF16 operands in shared
// memory, FP32 accumulators in tensor memory) instead of the scarce FP64 pipe.
//
// k_sketch_split: Y' = Omega' A (Section 2.3, Gaussian ensemble) with
//   Omega' = rint(4096 z) / 4096 / sqrt(s), the same Philox draws on the 2^-12
//   grid, so every entry is two 8-bit integers: 4096 z' = 256 zeta0 + zeta1.
//   A is cut into 512-row windows; in each window column j is written in fixed
//   point relative to 2^(e_j+1) (e_j = the largest exponent of the column in the
//   window) as a 55-bit integer, cut into seven 8-bit digits alpha_0..alpha_6
//   (balanced, |alpha| <= 128).  Every product
//   zeta_p * alpha_q is an integer below 2^14, the pairs with equal weight
//   p + q = d share one tensor-memory accumulator (at most two pairs), and a
//   window of 512 rows keeps every accumulated sum below 2^24: the FP32
//   accumulation is exact.  Once per window the seven accumulators are combined
//   (weights 2^-8d) and added to FP64 registers.  The result equals Omega' A up
//   to the dropped digit products (weight <= 2^-53 relative to the column) and
//   the FP64 sums: an FP64-grade sketch of A for any conditioning.
// k_gram_split: G = X^T X (the first CholeskyQR pass's Gram, Algorithm 1 step 1)
//   with each entry of X cut into three BF16 pieces (the top three 8-bit chunks
//   of its significand) and the six piece products of combined weight >= 2^-16
//   accumulated in FP32 in tensor memory, drained to FP64 every 64 rows (the
//   tensor core's FP32 accumulation truncates, so its error grows with the
//   number of accumulations: 24 per drain, <= 24 * 2^-23 of the partial sums).
//   Relative accuracy ~2^-19: enough because X = A R_s^{-1} is well conditioned
//   (Theorem 3.4) and the error of G only perturbs R_1, which the second, FP64
//   CholeskyQR pass corrects (Algorithm 2).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "rxr_internal.cuh"

namespace rxr {

// ---------------------------------------------------------------------------
// tcgen05 helpers
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, K-major, no swizzle: core matrices of 8
// rows x 16 bytes stored contiguously; lbo = byte step between core matrices
// along K, sbo = byte step between 8-row groups along M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;
}

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with FP16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[t]);
}

// Byte offset of element (row, k) in a K-major, no-swizzle operand tile with
// K = 64 (8 core matrices of 128 bytes along K per 8-row group).
__device__ __forceinline__ int kmaj_off(int row, int k)
{
    return (row & 7) * 16 + (row >> 3) * 1024 + (k & 7) * 2 + (k >> 3) * 128;
}

__device__ __forceinline__ void st_bf16(unsigned char *base, int off, float v)
{
    *reinterpret_cast<unsigned short *>(base + off) = __bfloat16_as_ushort(__float2bfloat16_rn(v));
}

// Wait for the tensor-core work committed to `bar` (phase `phase`), bounded;
// the decision is made block-uniform.
__device__ __forceinline__ bool mma_wait(uint64_t *bar, uint32_t phase, RxrStatus *st)
{
    const bool ok = mbar_wait_bounded(bar, phase, st);
    return __syncthreads_or(ok ? 0 : 1) == 0;
}

// ---------------------------------------------------------------------------
// Split sketch
// ---------------------------------------------------------------------------
constexpr int kSpWin = 512;  // rows per exact-accumulation window
constexpr int kSpSub = 64;   // rows per operand tile (MMA K extent 4 x 16)
constexpr int kSpM = 128;    // sketch rows per tile (MMA M)
constexpr int kSpN = 64;     // columns per tile (MMA N)
constexpr int kSpDigits = 7; // balanced 8-bit digits of A
constexpr int kSpZ = 2;      // 8-bit pieces of 4096 z'
constexpr int kSpB = kSpN * kSpSub * 2;  // bytes of one B tile (8 KB)
constexpr int kSpA = kSpM * kSpSub * 2;  // bytes of one A tile (16 KB)


// ---------------------------------------------------------------------------
// Split Gram
// ---------------------------------------------------------------------------
constexpr int kGsWin = 64;   // drain after every tile: the tensor core truncates FP32 sums
constexpr int kGsSub = 64;
constexpr int kGsM = 128;               // n <= 128, rows >= n of the tiles are zero
constexpr int kGsPieces = 3;
constexpr int kGsTile = kGsM * kGsSub * 2;  // 16 KB
constexpr size_t kGsSmem = (size_t)kGsPieces * kGsTile;

// The j-th BF16 piece (j = 0, 1, 2) of x: the 8-bit chunk of its significand
// starting at bit 7 + 8j below the leading one, with x's sign and weight.
__device__ __forceinline__ float piece_of(unsigned long long bits, int j)
{
    const int ea = (int)((bits >> 52) & 0x7FF);
    if (ea == 0 || ea == 0x7FF) return 0.0f;
    const int e = ea - 1023 - 7 - 8 * j;  // weight of the chunk's lowest bit
    if (e < -120 || e > 120) return 0.0f;
    const unsigned long long m53 = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const unsigned c = (unsigned)((m53 >> (45 - 8 * j)) & 255u);
    const float w = __uint_as_float((uint32_t)(e + 127) << 23);
    const float v = __fmul_rn(__uint2float_rn(c), w);
    return (bits >> 63) ? -v : v;
}

__global__ void __launch_bounds__(256, 1)
    k_gram_split(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int64_t win_total, int64_t win_per_cta,
                 double *__restrict__ Gpart, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = (n + 15) & ~15;

    for (int e = tid; e < (int)(kGsSmem / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(&mma_bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(kGsM, N);

    const int q4 = warp & 3, half = warp >> 2;
    const int my_row = 32 * q4 + lane;  // row j of G
    double acc[64];
#pragma unroll
    for (int t = 0; t < 64; ++t) acc[t] = 0.0;

    uint32_t phase = 0;
    bool pending = false, ok = true;
    const int64_t w_begin = blockIdx.x * win_per_cta;
    const int64_t w_end = min(win_total, w_begin + win_per_cta);
    for (int64_t w = w_begin; w < w_end && ok; ++w) {
        for (int sp = 0; sp < kGsWin / kGsSub; ++sp) {
            const int64_t r0 = w * kGsWin + sp * kGsSub;
            if (pending) {
                ok = mma_wait(&mma_bar, phase, st);
                if (!ok) break;
                phase ^= 1u;
                pending = false;
            }
            // up to 32 elements per thread (n <= 128), in two batches of 16
            // loads in flight
#pragma unroll
            for (int hb = 0; hb < 2; ++hb) {
                unsigned long long vbits[16];
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int e = tid + 256 * (16 * hb + t);
                    const int k = e & (kGsSub - 1), j = e >> 6;
                    const int64_t gr = r0 + k;
                    vbits[t] = (j < n && gr < m) ? (unsigned long long)__double_as_longlong(X[gr + (int64_t)j * ldx])
                                                 : 0ull;
                }
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int e = tid + 256 * (16 * hb + t);
                    const int k = e & (kGsSub - 1), j = e >> 6;
                    if (j < n) {
                        const int off = kmaj_off(j, k);
#pragma unroll
                        for (int pc = 0; pc < kGsPieces; ++pc)
                            st_bf16(smem + pc * kGsTile, off, piece_of(vbits[t], pc));
                    }
                }
            }
            fence_proxy_async_shared();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t b0 = smem_u32(smem);
#pragma unroll
                for (int kk = 0; kk < kGsSub / 16; ++kk) {
                    int first = 1;
#pragma unroll
                    for (int p = 0; p < kGsPieces; ++p)
#pragma unroll
                        for (int q = 0; p + q < kGsPieces; ++q) {
                            const uint32_t acc_on = (sp > 0 || kk > 0 || !first) ? 1u : 0u;
                            first = 0;
                            tc_mma(tmem, smem_desc(b0 + p * kGsTile + kk * 256, 128, 1024),
                                   smem_desc(b0 + q * kGsTile + kk * 256, 128, 1024), idesc, acc_on);
                        }
                }
                tc_commit(&mma_bar);
            }
            pending = true;
        }
        if (!ok) break;
        ok = mma_wait(&mma_bar, phase, st);
        if (!ok) break;
        phase ^= 1u;
        pending = false;
        tc_fence_after();
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
            const int col0 = half * 64 + c16 * 16;
            if (col0 < N) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + col0, v);
#pragma unroll
                for (int t = 0; t < 16; ++t) acc[c16 * 16 + t] += rxr_f2d_exact(v[t]);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (pending) {
        mma_wait(&mma_bar, phase, st);
        tc_fence_after();
    }
    if (ok && my_row < n) {
        double *out = Gpart + (int64_t)blockIdx.x * n * n;
#pragma unroll
        for (int t = 0; t < 64; ++t) {
            const int c = half * 64 + t;
            if (c < n && my_row <= c) out[my_row + (int64_t)c * n] = acc[t];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// FP64-grade Gram on the tensor cores (Ozaki-style exact splitting): for each
// 128-row window, column j of X is written in fixed point relative to 2^(e_j+1)
// as seven 8-bit digits (the same digits as the split sketch's A).  The
// ordered digit pairs (p, q), p + q <= 6, accumulate into seven tensor-memory
// groups d = p + q; a group holds at most seven pairs of products below 2^14
// over 128 rows, so every sum stays below 2^24 and the FP32 accumulation is
// exact.  Per window the groups are combined (weights 2^-8d) and added in FP64
// with the scale 2^(e_j + e_l).  The result is X^T X to about 2^-53 of
// |X|^T |X| column-normwise: it serves the CholeskyQR passes that must be
// FP64-accurate (the second pass's Gram).  n <= 128; grid.y = 64-column
// blocks of G.
// ---------------------------------------------------------------------------
constexpr int kOzWin = 128;
constexpr int kOzSub = 64;
constexpr int kOzM = 128;
constexpr int kOzN = 64;
constexpr int kOzDigits = 7;
constexpr int kOzTile = kOzM * kOzSub * 2;   // 16 KB per digit (A operand)
constexpr int kOzBTile = kOzN * kOzSub * 2;  // 8 KB per digit (separate B operand)
constexpr size_t kOzSmem = (size_t)kOzDigits * (kOzTile + kOzBTile);

// Seven digits of a 55-bit fixed-point value of x relative to 2^(emax+1),
// emax = biased exponent of the largest entry of its group: six balanced
// digits in [-128, 127] from the bottom, the rest (in [-128, 128]) on top.
// Digit q has weight 2^(emax - 1029 - 8q).
// The 55-bit fixed-point integer T of an FP64 value relative to 2^(emax + 1)
// (rounded to nearest; zero for zeros, subnormals and non-finite values),
// returned in offset form U = T + 0x808080808080: because T = sum_q alpha_q
// 256^(6-q) with balanced digits alpha_1..6 in [-128, 127], byte k of U is
// alpha_(6-k) + 128 (k = 0..5) and U >> 48 (arithmetic) is alpha_0: the
// carries of the offset do the balancing.
// Without branches: with x = 4 m53 (< 2^55) and sh = emax - ea >= 0, T = x / 2^sh
// rounded to nearest (halves away from zero, on the magnitude) is
// (x + 2^(sh-1)) >> sh, which is exact for sh <= 2 and zero from sh = 56 on.
__device__ __forceinline__ unsigned long long digits_offset(unsigned long long bits, int emax)
{
    const int ea = (int)((bits >> 52) & 0x7FF);
    const int sh = emax - ea;
    const unsigned long long x = ((bits & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 2;
    const int s = min(max(sh, 0), 63);
    unsigned long long t = (x + ((1ull << s) >> 1)) >> s;
    if (sh < 0) t = x << min(-sh, 8);  // only if emax is not the largest exponent
    long long T = (bits >> 63) ? -(long long)t : (long long)t;
    T = (ea > 0 && ea < 0x7FF) ? T : 0;
    return (unsigned long long)(T + 0x808080808080ll);
}

// FP32 bit pattern of digit q of offset form U (an integer in [-128, 128]:
// exact, and its upper 16 bits are its BF16 encoding).
__device__ __forceinline__ uint32_t digit_bits(unsigned long long U, int q)
{
    const uint32_t b = (q == 0) ? (uint32_t)((int)((long long)U >> 48) + 128)
                                : (uint32_t)(U >> (8 * (6 - q))) & 0xFFu;
    return __float_as_uint(__fadd_rn(__uint_as_float(0x4B000000u | b), -8388736.0f));  // 2^23 + b - (2^23 + 128)
}

// Seven balanced 8-bit digits alpha_0..alpha_6 of the value (alpha_0 may be
// +-128), as floats.
__device__ __forceinline__ void digits7(unsigned long long bits, int emax, float dg[kOzDigits])
{
    const unsigned long long U = digits_offset(bits, emax);
#pragma unroll
    for (int q = 0; q < kOzDigits; ++q) dg[q] = __uint_as_float(digit_bits(U, q));
}

// f * 2^(be - 1023) as a double, built on the integer pipes (exact: f is
// normal and the result's exponent stays in range; results below the normal
// range are flushed to zero, above it they become infinite).
__device__ __forceinline__ double f2d_pow2(float f, int be)
{
    const uint32_t u = __float_as_uint(f);
    const int e8 = (int)((u >> 23) & 0xFFu);
    const int e = e8 - 127 + be;
    const uint32_t sign = u & 0x80000000u;
    const bool zero = (e8 == 0) | (e <= 0), inf = e >= 2047;  // selects, not branches
    const uint32_t hi = zero ? 0u : inf ? (sign | 0x7FF00000u) : (sign | ((uint32_t)e << 20) | ((u & 0x7FFFFFu) >> 3));
    const uint32_t lo = (zero | inf) ? 0u : (u << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// (hi + lo) * 2^(be - 1023) as one double, on the integer pipes: the FP32 pair of
// a tensor-memory drain (hi, lo zero or normal, in any order) is renormalised by
// an exact two-sum (s + e = hi + lo, |e| <= ulp(s) / 2), e's bits are aligned
// below s's 24 in a 53-bit integer (those below 2^-29 ulp(s) are truncated: a
// relative error below 2^-52), and the double is assembled from it; flush and
// overflow as f2d_pow2.  One FP64 operation fewer than converting hi and lo
// and adding them.
__device__ __forceinline__ double pair2d_pow2(float hi, float lo, int be)
{
    const float s = __fadd_rn(hi, lo);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(lo, bb));
    const uint32_t us = __float_as_uint(s), ue = __float_as_uint(e);
    const int es = (int)((us >> 23) & 0xFFu), ee = (int)((ue >> 23) & 0xFFu);
    const uint32_t ms = (us & 0x7FFFFFu) | 0x800000u;
    const uint32_t me = (ee == 0) ? 0u : ((ue & 0x7FFFFFu) | 0x800000u);
    const int g = es - ee;  // at least 24 when e is not zero
    const uint32_t eu = (g <= 29) ? (me << (29 - g)) : (me >> min(g - 29, 31));
    long long M = ((long long)ms << 29) + ((((us ^ ue) >> 31) != 0u) ? -(long long)eu : (long long)eu);
    const bool low = M < (1ll << 52);  // M lies in [2^51, 2^53)
    M = low ? (M << 1) : M;
    const int E = es - 127 + be - (low ? 1 : 0);
    const uint32_t sign = us & 0x80000000u;
    const bool zero = (es == 0) | (E <= 0), inf = E >= 2047;  // selects, not branches
    const uint32_t h32 =
        zero ? 0u : inf ? (sign | 0x7FF00000u) : (sign | ((uint32_t)E << 20) | ((uint32_t)(M >> 32) & 0xFFFFFu));
    const uint32_t l32 = (zero | inf) ? 0u : (uint32_t)M;
    return __hiloint2double((int)h32, (int)l32);
}

// Digit q of two offset forms as one packed FP16 pair (value a in the low
// half): 0x6400 | (digit + 128) encodes the FP16 number 1024 + digit + 128
// (exact: at most 9 bits over 2^10), so one packed subtraction of 1152 leaves
// the digits themselves, exact in FP16.
__device__ __forceinline__ uint32_t digit_pair_f16(unsigned long long Ua, unsigned long long Ub, int q)
{
    uint32_t w;
    if (q == 0) {
        const uint32_t ta = (uint32_t)((int)((long long)Ua >> 48) + 128);
        const uint32_t tb = (uint32_t)((int)((long long)Ub >> 48) + 128);
        w = ta | (tb << 16) | 0x64006400u;
    } else {
        const int k = 6 - q, kb = k & 3;  // byte k of U: digit q + 128
        const uint32_t wa = (k < 4) ? (uint32_t)Ua : (uint32_t)(Ua >> 32);
        const uint32_t wb = (k < 4) ? (uint32_t)Ub : (uint32_t)(Ub >> 32);
        w = (__byte_perm(wa, wb, (uint32_t)(kb | ((4 + kb) << 8))) & 0x00FF00FFu) | 0x64006400u;
    }
    const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&w), __half2half2(__ushort_as_half((unsigned short)0x6480u)));
    return *reinterpret_cast<const uint32_t *>(&r);
}

// Digit plane q of eight consecutive K elements (offset forms U[0..7]) as one
// 16-byte FP16 store.
__device__ __forceinline__ uint4 pack_plane_f16(const unsigned long long U[8], int q)
{
    uint4 w;
    w.x = digit_pair_f16(U[0], U[1], q);
    w.y = digit_pair_f16(U[2], U[3], q);
    w.z = digit_pair_f16(U[4], U[5], q);
    w.w = digit_pair_f16(U[6], U[7], q);
    return w;
}

// Four small integers t[i] + 128 in [0, 256] (i = 0..3) as FP16 t[i].
__device__ __forceinline__ uint2 pack_int4x_f16(const uint32_t t[4])
{
    uint32_t w[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint32_t v = t[2 * i] | (t[2 * i + 1] << 16) | 0x64006400u;
        const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&v), __half2half2(__ushort_as_half((unsigned short)0x6480u)));
        w[i] = *reinterpret_cast<const uint32_t *>(&r);
    }
    return make_uint2(w[0], w[1]);
}

// Eight small integers t[i] + 128 in [0, 256] (i = 0..7) as FP16 t[i].
__device__ __forceinline__ uint4 pack_int8x_f16(const uint32_t t[8])
{
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t v = t[2 * i] | (t[2 * i + 1] << 16) | 0x64006400u;
        const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&v), __half2half2(__ushort_as_half((unsigned short)0x6480u)));
        w[i] = *reinterpret_cast<const uint32_t *>(&r);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Largest exponent of columns [c0, c0 + ncol) of X over the window rows, one
// warp per column, into ex[0..ncol).
__device__ __forceinline__ void window_colexp(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int64_t wr0,
                                              int c0, int ncol, int *ex)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int col = warp; col < ncol; col += 8) {
        unsigned e = 0;
        if (c0 + col < n) {
            unsigned hv[kOzWin / 32];
#pragma unroll
            for (int t = 0; t < kOzWin / 32; ++t) {
                const int64_t gr = wr0 + lane + 32 * t;
                hv[t] = (gr < m) ? (unsigned)__double2hiint(X[gr + (int64_t)(c0 + col) * ldx]) : 0u;
            }
#pragma unroll
            for (int t = 0; t < kOzWin / 32; ++t) e = max(e, (hv[t] >> 20) & 0x7FFu);
        }
        e = __reduce_max_sync(0xFFFFFFFFu, e);
        if (lane == 0) ex[col] = (int)e;
    }
}

// Digits of columns [c0, c0 + ncol) of a 64-row tile into `ncol`-row operand
// tiles (one per digit, `tile_bytes` apart), 16 loads in flight per thread.
__device__ __forceinline__ void tile_digits(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int64_t r0, int c0,
                                            int ncol, const int *ex, unsigned char *dst, int tile_bytes)
{
    const int tid = threadIdx.x;
    const int iters = (kOzSub * ncol + 255) / 256;
    for (int base = 0; base < iters; base += 16) {
        unsigned long long vb[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * (base + t);
            const int k = e & (kOzSub - 1), j = e >> 6;
            const int64_t gr = r0 + k;
            vb[t] = (base + t < iters && j < ncol && c0 + j < n && gr < m)
                        ? (unsigned long long)__double_as_longlong(X[gr + (int64_t)(c0 + j) * ldx])
                        : 0ull;
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * (base + t);
            const int k = e & (kOzSub - 1), j = e >> 6;
            if (base + t < iters && j < ncol) {
                float dg[kOzDigits];
                digits7(vb[t], ex[j], dg);
                const int off = kmaj_off(j, k);
#pragma unroll
                for (int q = 0; q < kOzDigits; ++q) st_bf16(dst + q * tile_bytes, off, dg[q]);
            }
        }
    }
}

// Output block list: block b covers rows [128 I, 128 I + 128) and columns
// [64 J, 64 J + 64) of G, for the pairs that meet the upper triangle.
__host__ __device__ inline int ozaki_blocks(int n)
{
    const int nI = (n + kOzM - 1) / kOzM, nJ = (n + kOzN - 1) / kOzN;
    int cnt = 0;
    for (int I = 0; I < nI; ++I)
        for (int J = 0; J < nJ; ++J)
            if (kOzN * J + kOzN - 1 >= kOzM * I) ++cnt;
    return cnt;
}

__device__ __forceinline__ void ozaki_block(int n, int b, int &I, int &J)
{
    const int nI = (n + kOzM - 1) / kOzM, nJ = (n + kOzN - 1) / kOzN;
    for (I = 0; I < nI; ++I)
        for (J = 0; J < nJ; ++J)
            if (kOzN * J + kOzN - 1 >= kOzM * I && b-- == 0) return;
}

// ---------------------------------------------------------------------------
// FP64-grade Gram on the tensor cores (Ozaki-style exact splitting): for each
// 128-row window, column j of X is written in fixed point relative to 2^(e_j+1)
// as seven 8-bit digits (the same digits as the split sketch's A).  The
// ordered digit pairs (p, q), p + q <= 6, accumulate into seven tensor-memory
// groups d = p + q; a group holds at most seven pairs of products below 2^14
// over 128 rows, so every sum stays below 2^24 and the FP32 accumulation is
// exact.  Per window the groups are combined (weights 2^-8d) and added in FP64
// with the scale 2^(e_j + e_l).  The result is X^T X to about 2^-53 of
// |X|^T |X| column-normwise: it serves the CholeskyQR passes that must be
// FP64-accurate.  grid.y = output blocks of 128 rows x 64 columns of G meeting
// the upper triangle; the B operand is a view into the A digits when its
// columns lie inside the block's rows, else digits of its own.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1)
    k_gram_ozaki(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int64_t win_total, int64_t win_per_cta,
                 double *__restrict__ Gpart, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *aop = smem;
    unsigned char *bsep = smem + kOzDigits * kOzTile;
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int exA[kOzM];
    __shared__ int exB[kOzN];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int bI, bJ;
    ozaki_block(n, blockIdx.y, bI, bJ);
    const int a0c = bI * kOzM, b0c = bJ * kOzN;
    const bool b_inside = (b0c >= a0c) && (b0c + kOzN <= a0c + kOzM);

    for (int e = tid; e < (int)(kOzSmem / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(&mma_bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16(kOzM, kOzN);
    const int q4 = warp & 3, half = warp >> 2;
    const int my_row = 32 * q4 + lane;  // row a0c + my_row of G
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;

    uint32_t phase = 0;
    bool pending = false, ok = true;
    const int64_t w_begin = blockIdx.x * win_per_cta;
    const int64_t w_end = min(win_total, w_begin + win_per_cta);
    for (int64_t w = w_begin; w < w_end && ok; ++w) {
        const int64_t wr0 = w * kOzWin;
        window_colexp(X, ldx, m, n, wr0, a0c, kOzM, exA);
        if (!b_inside) window_colexp(X, ldx, m, n, wr0, b0c, kOzN, exB);
        __syncthreads();
        for (int sp = 0; sp < kOzWin / kOzSub; ++sp) {
            const int64_t r0 = wr0 + sp * kOzSub;
            if (pending) {
                ok = mma_wait(&mma_bar, phase, st);
                if (!ok) break;
                phase ^= 1u;
                pending = false;
            }
            tile_digits(X, ldx, m, n, r0, a0c, kOzM, exA, aop, kOzTile);
            if (!b_inside) tile_digits(X, ldx, m, n, r0, b0c, kOzN, exB, bsep, kOzBTile);
            fence_proxy_async_shared();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = smem_u32(aop);
                const uint32_t bb = b_inside ? a0 + ((b0c - a0c) / 8) * 1024 : smem_u32(bsep);
                const uint32_t bstride = b_inside ? kOzTile : kOzBTile;
#pragma unroll
                for (int kk = 0; kk < kOzSub / 16; ++kk)
#pragma unroll
                    for (int p = 0; p < kOzDigits; ++p)
#pragma unroll
                        for (int q = 0; p + q < kOzDigits; ++q) {
                            const uint32_t acc_on = (sp > 0 || kk > 0 || p > 0) ? 1u : 0u;
                            tc_mma(tmem + (uint32_t)((p + q) * kOzN), smem_desc(a0 + p * kOzTile + kk * 256, 128, 1024),
                                   smem_desc(bb + q * bstride + kk * 256, 128, 1024), idesc, acc_on);
                        }
                tc_commit(&mma_bar);
            }
            pending = true;
        }
        if (!ok) break;
        ok = mma_wait(&mma_bar, phase, st);
        if (!ok) break;
        phase ^= 1u;
        pending = false;
        tc_fence_after();
        const int ej = exA[my_row];
#pragma unroll
        for (int c16 = 0; c16 < 2; ++c16) {
            const int col0 = half * 32 + c16 * 16;
            float hi[16], lo[16], v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + col0, hi);
#pragma unroll
            for (int t = 0; t < 16; ++t) lo[t] = 0.0f;
#pragma unroll
            for (int d = 1; d < kOzDigits; ++d) {
                tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + d * kOzN + col0, v);
                const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float x = __fmul_rn(v[t], w8);
                    const float sum = __fadd_rn(hi[t], x);
                    const float bb = __fsub_rn(sum, hi[t]);
                    const float err = __fadd_rn(__fsub_rn(hi[t], __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                    hi[t] = sum;
                    lo[t] = __fadd_rn(lo[t], err);
                }
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int lc = col0 + t;  // column b0c + lc of G
                const int el = b_inside ? exA[b0c - a0c + lc] : exB[lc];
                const int be = ej + el - 1035;  // biased exponent of 2^(e_j + e_l - 2058)
                if (ej > 0 && el > 0 && be > 0 && be < 2047) acc[c16 * 16 + t] += pair2d_pow2(hi[t], lo[t], be);
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (pending) {
        mma_wait(&mma_bar, phase, st);
        tc_fence_after();
    }
    const int gr = a0c + my_row;
    if (ok && gr < n) {
        double *out = Gpart + (int64_t)blockIdx.x * n * n;
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int c = b0c + half * 32 + t;
            if (c < n && gr <= c) out[gr + (int64_t)c * n] = acc[t];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// operand tiles of the blocked substitution's trailing update (k_update_ozaki)
constexpr int kApM = 128, kApK = 64, kApN = 64, kApDigits = 7;
constexpr int kApATile = kApM * kApK * 2;  // 16 KB per digit
constexpr int kApBTile = kApN * kApK * 2;  // 8 KB per digit
constexpr size_t kApSmem = (size_t)kApDigits * (kApATile + kApBTile);


// ---------------------------------------------------------------------------
// Trailing update of the blocked substitution, on the tensor cores at FP64
// grade:  C[:, tc0 : tc0 + N) = B[:, tc0 : tc0 + N) - X[:, xc0 : xc0 + K) R[xc0 : xc0 + K, tc0 : tc0 + N)
// (B = nullptr: C = + X R-block).  X rows are split relative to their own
// largest exponent over the K entries, R's block columns relative to theirs,
// seven 8-bit digits each; K <= 64 keeps every group's integer sum below 2^24
// (exact).  grid.x = 128-row tiles, grid.y = 64-column tiles of the trailing
// block.  X's columns are disjoint from C's, so C may alias B and X's matrix.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1)
    k_update_ozaki(const double *X, int64_t ldx, int xc0, int K, const double *__restrict__ R, int64_t ldr, int tc0,
                   int N, const double *B, int64_t ldb, double *C, int64_t ldc, int64_t m, int64_t tiles_total,
                   int64_t tiles_per_cta, const int *__restrict__ sel, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (sel != nullptr && *sel != 1) return;  // the substitution was chosen instead
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *aop = smem;
    unsigned char *bop = smem + kApDigits * kApATile;
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int rowexp[kApM];
    __shared__ int colexp_t[kApN];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.y * kApN;             // this CTA's columns [tc0 + n0, tc0 + n0 + nw)
    const int nw = min(kApN, N - n0);
    const int ksteps = (K + 15) / 16;

    for (int e = tid; e < (int)(kApSmem / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        mbar_init(&mma_bar, 1);
        fence_barrier_init();
    }
    // digits of the R block: B tile element (l, k) = R[xc0 + k][tc0 + n0 + l]
    if (tid < kApN) {
        unsigned ex = 0;
        if (tid < nw)
            for (int k = 0; k < K; ++k)
                ex = max(ex, ((unsigned)__double2hiint(R[(xc0 + k) + (int64_t)(tc0 + n0 + tid) * ldr]) >> 20) & 0x7FFu);
        colexp_t[tid] = (int)ex;
    }
    __syncthreads();
    for (int e = tid; e < K * nw; e += blockDim.x) {
        const int k = e % K, l = e / K;
        const unsigned long long bits =
            (unsigned long long)__double_as_longlong(R[(xc0 + k) + (int64_t)(tc0 + n0 + l) * ldr]);
        float dg[kApDigits];
        digits7(bits, colexp_t[l], dg);
        const int off = kmaj_off(l, k);
#pragma unroll
        for (int q = 0; q < kApDigits; ++q) st_bf16(bop + q * kApBTile, off, dg[q]);
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_bf16(kApM, kApN);
    const int q4 = warp & 3, half = warp >> 2;
    const int my_row = 32 * q4 + lane;

    uint32_t phase = 0;
    bool pending = false, ok = true;
    const int64_t t_begin = blockIdx.x * tiles_per_cta;
    const int64_t t_end = min(tiles_total, t_begin + tiles_per_cta);
    for (int64_t tile = t_begin; tile < t_end && ok; ++tile) {
        const int64_t r0 = tile * kApM;
        if (tid < kApM) {
            unsigned ex = 0;
            const int64_t gr = r0 + tid;
            if (gr < m)
                for (int k = 0; k < K; ++k)
                    ex = max(ex, ((unsigned)__double2hiint(X[gr + (int64_t)(xc0 + k) * ldx]) >> 20) & 0x7FFu);
            rowexp[tid] = (int)ex;
        }
        __syncthreads();
        const int iters = (kApM * K + 255) / 256;
        for (int base = 0; base < iters; base += 16) {
            unsigned long long vb[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int e = tid + 256 * (base + t);
                const int i = e & (kApM - 1), k = e >> 7;
                const int64_t gr = r0 + i;
                vb[t] = (base + t < iters && k < K && gr < m)
                            ? (unsigned long long)__double_as_longlong(X[gr + (int64_t)(xc0 + k) * ldx])
                            : 0ull;
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int e = tid + 256 * (base + t);
                const int i = e & (kApM - 1), k = e >> 7;
                if (base + t < iters && k < K) {
                    float dg[kApDigits];
                    digits7(vb[t], rowexp[i], dg);
                    const int off = kmaj_off(i, k);
#pragma unroll
                    for (int q = 0; q < kApDigits; ++q) st_bf16(aop + q * kApATile, off, dg[q]);
                }
            }
        }
        fence_proxy_async_shared();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(aop), b0 = smem_u32(bop);
            for (int kk = 0; kk < ksteps; ++kk)
#pragma unroll
                for (int p = 0; p < kApDigits; ++p)
#pragma unroll
                    for (int q = 0; p + q < kApDigits; ++q) {
                        const uint32_t acc_on = (kk > 0 || p > 0) ? 1u : 0u;
                        tc_mma(tmem + (uint32_t)((p + q) * kApN), smem_desc(a0 + p * kApATile + kk * 256, 128, 1024),
                               smem_desc(b0 + q * kApBTile + kk * 256, 128, 1024), idesc, acc_on);
                    }
            tc_commit(&mma_bar);
        }
        pending = true;
        ok = mma_wait(&mma_bar, phase, st);
        if (!ok) break;
        phase ^= 1u;
        pending = false;
        tc_fence_after();
        const int ei = rowexp[my_row];
        const int64_t gr = r0 + my_row;
#pragma unroll
        for (int c16 = 0; c16 < 2; ++c16) {
            const int col0 = half * 32 + c16 * 16;
            if (col0 >= nw) continue;  // warp-uniform
            // B's 16 values, all in flight before the first store (C may alias B,
            // so a store between them would order each load after it)
            double bv[16];
#pragma unroll
            for (int t = 0; t < 16; ++t)
                bv[t] = (B != nullptr && col0 + t < nw && gr < m) ? B[gr + (int64_t)(tc0 + n0 + col0 + t) * ldb] : 0.0;
            float hi[16], lo[16], v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + col0, hi);
#pragma unroll
            for (int t = 0; t < 16; ++t) lo[t] = 0.0f;
#pragma unroll
            for (int d = 1; d < kApDigits; ++d) {
                tmem_ld16(tmem + ((uint32_t)(32 * q4) << 16) + d * kApN + col0, v);
                const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float x = __fmul_rn(v[t], w8);
                    const float sum = __fadd_rn(hi[t], x);
                    const float bb = __fsub_rn(sum, hi[t]);
                    const float err = __fadd_rn(__fsub_rn(hi[t], __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                    hi[t] = sum;
                    lo[t] = __fadd_rn(lo[t], err);
                }
            }
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int l = col0 + t;
                if (l < nw && gr < m) {
                    const int el = colexp_t[l];
                    const int be = ei + el - 1035;
                    const double prod = (ei > 0 && el > 0 && be > 0 && be < 2047) ? pair2d_pow2(hi[t], lo[t], be) : 0.0;
                    const int64_t cc = tc0 + n0 + l;
                    C[gr + cc * ldc] = B ? bv[t] - prod : prod;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    if (pending) {
        mma_wait(&mma_bar, phase, st);
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// Diagonal block of the blocked substitution, FP64:
//   X[:, c0 : c0 + b) = B[:, c0 : c0 + b) R[c0 : c0 + b, c0 : c0 + b)^{-1}
// 256-row tiles, one thread per row, the tile's b columns in shared memory
// (column-major), the block of R packed and 1 / R_jj in shared memory.  X may
// alias B.
constexpr int kSbRows = 256;

__global__ void __launch_bounds__(256)
    k_solve_block(const double *B, int64_t ldb, double *X, int64_t ldx, const double *__restrict__ R, int64_t ldr,
                  int c0, int b, int64_t m, int64_t tiles_total, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *xs = reinterpret_cast<double *>(smem_raw);  // [b][kSbRows]
    double *rb = xs + (int64_t)b * kSbRows;              // packed upper block of R
    double *dv = rb + b * (b + 1) / 2;
    const int t = threadIdx.x;
    for (int j = 0; j < b; ++j)
        for (int k = t; k <= j; k += blockDim.x) rb[j * (j + 1) / 2 + k] = R[(c0 + k) + (int64_t)(c0 + j) * ldr];
    for (int j = t; j < b; j += blockDim.x) dv[j] = 1.0 / R[(c0 + j) + (int64_t)(c0 + j) * ldr];
    for (int64_t tile = blockIdx.x; tile < tiles_total; tile += gridDim.x) {
        const int64_t i = tile * kSbRows + t;
        __syncthreads();
        for (int j = 0; j < b; ++j) xs[j * kSbRows + t] = (i < m) ? B[i + (int64_t)(c0 + j) * ldb] : 0.0;
        __syncthreads();
        for (int j = 0; j < b; ++j) {
            const double *rc = rb + j * (j + 1) / 2;
            double acc = xs[j * kSbRows + t];
#pragma unroll 4
            for (int k = 0; k < j; ++k) acc = fma(-xs[k * kSbRows + t], rc[k], acc);
            xs[j * kSbRows + t] = acc * dv[j];
        }
        if (i < m)
            for (int j = 0; j < b; ++j) X[i + (int64_t)(c0 + j) * ldx] = xs[j * kSbRows + t];
    }
}

// ---------------------------------------------------------------------------
// Fused blocked substitution X = B R^{-1} for n <= 64, one pass over B.
// The CTA runs two independent groups of four warps; each group walks its own
// stream of 128-row tiles of B (TMA load into the group's shared-memory tile,
// TMA store back), so that one group's loads, tensor-core waits and epilogues
// overlap the other group's FP64 work and every scheduler holds two warps
// issuing FP64.  A tile is solved in shared memory by column blocks of 16:
//   * the diagonal block by FP64 row substitution, one thread per row,
//     right-looking inside the block (for every column the same FMA sequence
//     as the plain substitution: seeded with b_j, k ascending, times 1/R_jj);
//   * the trailing columns receive -X_blk R_blk from the tensor cores at FP64
//     grade: each row of X_blk is written as seven 8-bit digits relative to its
//     own largest exponent, each column of R_blk relative to its own, and the
//     digit pairs p + q = d accumulate in tensor-memory group d (K = 16:
//     every group sum is an integer below 2^24, exact in FP32); each output
//     combines its seven groups once and is subtracted in FP64.
// The same thread owns a row in the solve and in the epilogue (tensor-memory
// lane = row), so a tile's rows never cross threads.  dst may equal src: a
// tile is read completely before it is written, and only by its own group.
// ---------------------------------------------------------------------------
constexpr int kFuM = 128, kFuBw = 16, kFuMaxN = 64, kFuDigits = 7;
constexpr int kFuATile = kFuM * kFuBw * 2;  // bytes of one digit plane of X_blk (4 KB)
constexpr int kFuChunk = 32;                // trailing columns per tensor-core round
constexpr int kFuGroupTmem = 256;           // tensor-memory columns per warp group (7 x 32 used)

__host__ __device__ inline int fu_blocks(int n) { return (n + kFuBw - 1) / kFuBw; }
// trailing columns after block c, padded to the MMA's N granularity (16)
__host__ __device__ inline int fu_npad(int n, int c)
{
    const int N = n - kFuBw * (c + 1);
    return N > 0 ? (N + 15) & ~15 : 0;
}
// byte offset of block c's R digits, and its first column-exponent slot
__host__ __device__ inline int fu_bdig_off(int n, int c)
{
    int off = 0;
    for (int q = 0; q < c; ++q) off += kFuDigits * fu_npad(n, q) * kFuBw * 2;
    return off;
}
__host__ __device__ inline int fu_cbase(int n, int c)
{
    int off = 0;
    for (int q = 0; q < c; ++q) off += fu_npad(n, q);
    return off;
}
__host__ __device__ inline size_t fu_smem_bytes(int n)
{
    const int nb = fu_blocks(n);
    return 2 * (size_t)kFuM * n * 8 + 2 * (size_t)kFuDigits * kFuATile + (size_t)fu_bdig_off(n, nb) +
           (size_t)nb * (kFuBw * kFuBw + kFuBw) * 8;
}

// Byte offset of element (row, k) in a K-major, no-swizzle operand tile with
// K = 16 (two core matrices of 128 bytes along K per 8-row group).
__device__ __forceinline__ int kmaj16_off(int row, int k)
{
    return (row & 7) * 16 + (row >> 3) * 256 + (k & 7) * 2 + (k >> 3) * 128;
}



// 16 tensor-memory columns into registers without waiting (tcgen05.wait::ld
// must follow before the values are used).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t r[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t r[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Barrier of one 128-thread warp group (named barrier 1 + g), and the same
// barrier returning the OR of a predicate over the group.
__device__ __forceinline__ void group_bar(int g) { asm volatile("bar.sync %0, 128;" ::"r"(g + 1) : "memory"); }
__device__ __forceinline__ bool group_or(int g, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(g + 1)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(256, 1)
    k_subst_fused(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_dst, int use_tma,
                  const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int n,
                  const double *__restrict__ R, int64_t ldr, int64_t tiles_total, int *colexp_out,
                  const int *__restrict__ sel, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (sel != nullptr && *sel != 0) return;  // the explicit-inverse product was chosen instead
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nb = fu_blocks(n);
    const size_t tile_bytes = (size_t)kFuM * n * 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = warp >> 2;        // warp group
    const int row = tid & (kFuM - 1);  // this thread's row of the group's tile (= tensor-memory lane)
    double *xs = reinterpret_cast<double *>(smem + g * tile_bytes);
    unsigned char *adig_all = smem + 2 * tile_bytes;         // [2 groups][7][128 x 16] X_blk digits
    unsigned char *adig = adig_all + g * kFuDigits * kFuATile;
    unsigned char *bdig = adig_all + 2 * kFuDigits * kFuATile;  // R digits per block [7][Npad x 16]
    double *rdg = reinterpret_cast<double *>(bdig + fu_bdig_off(n, nb));  // [nb][16 x 16]: r(k, j) at j*16 + k
    double *dvs = rdg + nb * kFuBw * kFuBw;                                 // 1 / R_jj, zero past n
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int colexp[2 * kFuMaxN];
    __shared__ int out_exp[kFuMaxN];  // largest exponent per column of the tiles written

    // --- per-CTA setup: R's diagonal blocks, 1 / R_jj and the digits of R's
    // off-diagonal blocks (the same for every tile)
    {
        const int zbytes = 2 * kFuDigits * kFuATile + fu_bdig_off(n, nb);
        for (int e = tid; e < zbytes / 16; e += blockDim.x)
            reinterpret_cast<uint4 *>(adig_all)[e] = make_uint4(0, 0, 0, 0);
    }
    for (int e = tid; e < nb * kFuBw * kFuBw; e += blockDim.x) {
        const int c = e / (kFuBw * kFuBw), j = (e / kFuBw) % kFuBw, k = e % kFuBw;
        const int gk = kFuBw * c + k, gj = kFuBw * c + j;
        rdg[e] = (k < j && gj < n) ? R[gk + (int64_t)gj * ldr] : 0.0;
    }
    for (int e = tid; e < nb * kFuBw; e += blockDim.x) dvs[e] = (e < n) ? 1.0 / R[e + (int64_t)e * ldr] : 0.0;
    if (tid < kFuMaxN) out_exp[tid] = 0;
    for (int c = 0; c + 1 < nb; ++c) {
        const int Nc = n - kFuBw * (c + 1);
        for (int l = tid; l < Nc; l += blockDim.x) {
            unsigned ex = 0;
            for (int k = 0; k < kFuBw; ++k)
                ex = max(ex, ((unsigned)__double2hiint(R[(kFuBw * c + k) + (int64_t)(kFuBw * (c + 1) + l) * ldr]) >> 20) &
                                 0x7FFu);
            colexp[fu_cbase(n, c) + l] = (int)ex;
        }
    }
    if (tid == 0) {
        mbar_init(&full_bar[0], 1);
        mbar_init(&full_bar[1], 1);
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    for (int c = 0; c + 1 < nb; ++c) {
        const int Nc = n - kFuBw * (c + 1), Np = fu_npad(n, c);
        unsigned char *bd = bdig + fu_bdig_off(n, c);
        for (int l = tid; l < Nc; l += blockDim.x) {
            const int ex = colexp[fu_cbase(n, c) + l];
            for (int k0 = 0; k0 < kFuBw; k0 += 8) {
                unsigned long long U[8];
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    U[k] = digits_offset((unsigned long long)__double_as_longlong(
                                             R[(kFuBw * c + k0 + k) + (int64_t)(kFuBw * (c + 1) + l) * ldr]),
                                         ex);
#pragma unroll
                for (int q = 0; q < kFuDigits; ++q)
                    *reinterpret_cast<uint4 *>(bd + q * Np * kFuBw * 2 + kmaj16_off(l, k0)) = pack_plane_f16(U, q);
            }
        }
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base + (uint32_t)(g * kFuGroupTmem) + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t tmem_mma = tmem_base + (uint32_t)(g * kFuGroupTmem);
    const bool leader = (row == 0);  // issues this group's TMA copies and MMAs

    // --- this group's tile stream: tiles 2 * blockIdx.x + g, + 2 * gridDim.x, ...
    uint32_t loads = 0, mphase = 0;  // TMA loads consumed; tensor-core commits consumed
    unsigned cmax_lo = 0, cmax_hi = 0;  // largest exponent of columns lane and lane + 32 (colexp_out)
    bool ok = true, load_pending = false, mma_pending = false;
    // the stall test hook: group 0 of the first CTA skips its first copy, so its
    // wait runs out with nothing in flight and the drain below runs
    bool stall = use_tma && blockIdx.x == 0 && g == 0 && rxr_stall_requested(st);
    const int64_t stride = 2 * (int64_t)gridDim.x;
    for (int64_t tile = 2 * (int64_t)blockIdx.x + g; tile < tiles_total && ok; tile += stride) {
        const int64_t r0 = tile * kFuM;
        if (use_tma) {
            if (leader) {
                bulk_wait_read_all();  // the previous tile's store has left shared memory
                if (!stall) {
                    mbar_arrive_expect_tx(&full_bar[g], (uint32_t)tile_bytes);
                    tma_load_2d(xs, &tm_src, (int)r0, 0, &full_bar[g]);
                }
            }
            stall = false;
            load_pending = true;
            const bool got = mbar_wait_bounded(&full_bar[g], loads & 1u, st);
            ok = !group_or(g, !got);
            if (!ok) break;
            load_pending = false;
            ++loads;
        } else {
            for (int e = row; e < kFuM * n; e += kFuM) {
                const int rr = e & (kFuM - 1), col = e >> 7;
                xs[e] = (r0 + rr < m) ? src[r0 + rr + (int64_t)col * lds] : 0.0;
            }
            group_bar(g);
        }
        for (int c = 0; c < nb && ok; ++c) {
            const int c16 = kFuBw * c;
            const int Nc = n - c16 - kFuBw;  // trailing columns after this block
            int ei;
            {
                const double *rb = rdg + c * kFuBw * kFuBw;
                const double *dvb = dvs + c16;
                double v[kFuBw];
#pragma unroll
                for (int j = 0; j < kFuBw; ++j) v[j] = (c16 + j < n) ? xs[(c16 + j) * kFuM + row] : 0.0;
#pragma unroll
                for (int k = 0; k < kFuBw; ++k) {
                    v[k] *= dvb[k];
#pragma unroll
                    for (int j = k + 1; j < kFuBw; ++j) v[j] = fma(-v[k], rb[j * kFuBw + k], v[j]);
                }
                unsigned ex = 0;
#pragma unroll
                for (int j = 0; j < kFuBw; ++j) {
                    if (c16 + j < n) xs[(c16 + j) * kFuM + row] = v[j];
                    const unsigned ej = ((unsigned)__double2hiint(v[j]) >> 20) & 0x7FFu;
                    ex = max(ex, ej);
                    if (colexp_out != nullptr) {
                        // these columns are final: the warp's largest exponent per
                        // column is kept by lane (column mod 32)
                        const unsigned w = __reduce_max_sync(0xFFFFFFFFu, ej);
                        if (((c16 + j) & 31) == lane) {
                            if (c16 + j < 32)
                                cmax_lo = max(cmax_lo, w);
                            else
                                cmax_hi = max(cmax_hi, w);
                        }
                    }
                }
                ei = (int)ex;
                if (Nc > 0) {
#pragma unroll
                    for (int j0 = 0; j0 < kFuBw; j0 += 8) {
                        unsigned long long U[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) U[j] = digits_offset((unsigned long long)__double_as_longlong(v[j0 + j]), ei);
#pragma unroll
                        for (int q = 0; q < kFuDigits; ++q)
                            *reinterpret_cast<uint4 *>(adig + q * kFuATile + kmaj16_off(row, j0)) = pack_plane_f16(U, q);
                    }
                }
            }
            if (Nc <= 0) break;
            const int Np = fu_npad(n, c);
            const int cb = fu_cbase(n, c);
            const unsigned char *bd = bdig + fu_bdig_off(n, c);
            // trailing columns in rounds of at most 32 (7 groups x 32 tensor-memory columns)
            for (int n0 = 0; n0 < Np && ok; n0 += kFuChunk) {
                const int nw = min(kFuChunk, Np - n0);
                fence_proxy_async_shared();
                tc_fence_before();
                group_bar(g);
                if (leader) {
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(adig), b0 = smem_u32(bd) + (uint32_t)(n0 * kFuBw * 2);
                    const uint32_t idesc = idesc_f16(kFuM, nw);
#pragma unroll
                    for (int p = 0; p < kFuDigits; ++p)
#pragma unroll
                        for (int q = 0; p + q < kFuDigits; ++q)
                            tc_mma(tmem_mma + (uint32_t)((p + q) * kFuChunk), smem_desc(a0 + p * kFuATile, 128, 256),
                                   smem_desc(b0 + q * Np * kFuBw * 2, 128, 256), idesc, p > 0 ? 1u : 0u);
                    tc_commit(&mma_bar[g]);
                }
                mma_pending = true;
                const bool got = mbar_wait_bounded(&mma_bar[g], mphase, st);
                ok = !group_or(g, !got);
                if (!ok) break;
                mphase ^= 1u;
                mma_pending = false;
                tc_fence_after();
                // epilogue: this thread's row, 16 columns at a time
                for (int h0 = 0; h0 < nw; h0 += 16) {
                    uint32_t gv[kFuDigits][16];
#pragma unroll
                    for (int d = 0; d < kFuDigits; ++d) tmem_ld16_issue(tmem + d * kFuChunk + h0, gv[d]);
                    tmem_wait_ld();
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        float hi = __uint_as_float(gv[0][t]), lo = 0.0f;
#pragma unroll
                        for (int d = 1; d < kFuDigits; ++d) {
                            const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
                            const float x = __fmul_rn(__uint_as_float(gv[d][t]), w8);
                            const float sum = __fadd_rn(hi, x);
                            const float bb = __fsub_rn(sum, hi);
                            const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                            hi = sum;
                            lo = __fadd_rn(lo, err);
                        }
                        const int l = n0 + h0 + t;
                        if (l < Nc) {
                            const int el = colexp[cb + l];
                            const int be = ei + el - 1035;  // 2^(e_i + e_l - 2058) as a biased exponent
                            if (ei > 0 && el > 0 && be > 0 && be < 2047) {
                                double *xp = xs + (c16 + kFuBw + l) * kFuM + row;
                                *xp = *xp - pair2d_pow2(hi, lo, be);
                            }
                        }
                    }
                }
                tc_fence_before();
            }
        }
        if (!ok) break;
        if (use_tma) {
            fence_proxy_async_shared();
            group_bar(g);
            if (leader) {
                tma_store_2d(&tm_dst, (int)r0, 0, xs);
                bulk_commit();
            }
        } else {
            group_bar(g);
            for (int e = row; e < kFuM * n; e += kFuM) {
                const int rr = e & (kFuM - 1), col = e >> 7;
                if (r0 + rr < m) dst[r0 + rr + (int64_t)col * ldd] = xs[e];
            }
            group_bar(g);
        }
    }
    // drain this group's tensor-core work, TMA load and stores (bounded waits)
    if (mma_pending) {
        mbar_wait_bounded(&mma_bar[g], mphase, st);
        tc_fence_after();
    }
    if (leader && use_tma) {
        if (load_pending) mbar_wait_bounded(&full_bar[g], loads & 1u, st);
        bulk_wait_all();
    }
    if (colexp_out != nullptr) {
        if (cmax_lo > 0) atomicMax(&out_exp[lane], (int)cmax_lo);
        if (cmax_hi > 0) atomicMax(&out_exp[lane + 32], (int)cmax_hi);
    }
    tc_fence_before();
    __syncthreads();
    if (colexp_out != nullptr && tid < n && out_exp[tid] > 0) atomicMax(colexp_out + tid, out_exp[tid]);
    if (warp == 0) tmem_dealloc(tmem_base, 512);
}

// One exact window of k_gram_oz64, read out of tensor memory: lane 32 q4 +
// lane, columns 32 half .. + 31 of the seven accumulator blocks, combined with
// weights 2^-8d into FP32 pairs (TwoSum; hi + lo carries the window's sum to
// about 2^-48 of it).  Eight columns per tensor-memory load keep the register
// footprint small.
__device__ __forceinline__ void gram64_read(uint32_t tmem, int q4, int half, float hi[32], float lo[32])
{
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        uint32_t g[kOzDigits][8];
#pragma unroll
        for (int d = 0; d < kOzDigits; ++d) {
            const uint32_t ta = tmem + ((uint32_t)(32 * q4) << 16) + d * 64 + 32 * half + 8 * c8;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(g[d][0]), "=r"(g[d][1]), "=r"(g[d][2]), "=r"(g[d][3]), "=r"(g[d][4]), "=r"(g[d][5]),
                           "=r"(g[d][6]), "=r"(g[d][7])
                         : "r"(ta)
                         : "memory");
        }
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float h = __uint_as_float(g[0][t]), l = 0.0f;
#pragma unroll
            for (int d = 1; d < kOzDigits; ++d) {
                const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
                const float x = __fmul_rn(__uint_as_float(g[d][t]), w8);
                const float sum = __fadd_rn(h, x);
                const float bb = __fsub_rn(sum, h);
                const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                h = sum;
                l = __fadd_rn(l, err);
            }
            hi[8 * c8 + t] = h;
            lo[8 * c8 + t] = l;
        }
    }
}

__device__ __forceinline__ void gram64_accumulate(const float hi[32], const float lo[32], double acc[32])
{
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] += rxr_f2d_exact(hi[t]) + rxr_f2d_exact(lo[t]);
}

// The same with one FP64 addition per sum (pair2d_pow2: more integer work,
// less FP64; k_gram_oz128 gains from it, k_gram_oz64, whose digit production
// keeps the integer pipes busier, does not).
__device__ __forceinline__ void gram_accumulate_pair(const float hi[32], const float lo[32], double acc[32])
{
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] += pair2d_pow2(hi[t], lo[t], 1023);
}

// ---------------------------------------------------------------------------
// Fused blocked substitution X = B R^{-1} for 64 < n <= 128, one pass over B.
// Same scheme as k_subst_fused (16-column FP64 diagonal solves, FP64-grade
// tensor-core trailing updates, 128-row tiles resident in shared memory), with
// one tile per CTA (a 128 x 128 FP64 tile is 128 KB).  R's per-block data no
// longer fits in shared memory at once: k_rprep128 lays it out in global
// memory, one contiguous record per column block (FP16 digits of the
// off-diagonal block, their column exponents, the diagonal block, 1 / R_jj),
// and the CTA streams the records through two shared-memory slots by 1-D bulk
// copies, one block ahead.  The trailing update runs in rounds of up to 64
// columns (7 groups x 64 tensor-memory columns).
// ---------------------------------------------------------------------------
constexpr int kF2MaxN = 128;
constexpr int kF2Slot = 28672;  // largest record (n = 128, block 0): 7 x 112 x 32 + 112 x 4 + 2048 + 128 bytes

__host__ __device__ inline int f2_rec_bytes(int n, int c)
{
    const int Np = fu_npad(n, c);
    return kFuDigits * Np * kFuBw * 2 + Np * 4 + kFuBw * kFuBw * 8 + kFuBw * 8;
}
__host__ __device__ inline int f2_rec_off(int n, int c)
{
    int off = 0;
    for (int q = 0; q < c; ++q) off += f2_rec_bytes(n, q);
    return off;
}
__host__ __device__ inline size_t f2_smem_bytes(int n)
{
    return (size_t)kFuM * n * 8 + (size_t)kFuDigits * kFuATile + 2 * (size_t)kF2Slot;
}

// One record per column block c (grid.x = blocks): see k_subst_fused128.
__global__ void __launch_bounds__(256) k_rprep128(const double *__restrict__ R, int64_t ldr, int n,
                                                  unsigned char *__restrict__ rec, const int *__restrict__ sel,
                                                  RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (sel != nullptr && *sel != 0) return;  // the FP32-correction apply was chosen instead
    const int c = blockIdx.x, tid = threadIdx.x;
    const int Np = fu_npad(n, c), Nc = n - kFuBw * (c + 1);
    unsigned char *r = rec + f2_rec_off(n, c);
    int *cexp = reinterpret_cast<int *>(r + kFuDigits * Np * kFuBw * 2);
    double *diag = reinterpret_cast<double *>(r + kFuDigits * Np * kFuBw * 2 + Np * 4);
    double *dinv = diag + kFuBw * kFuBw;
    for (int e = tid; e < kFuBw * kFuBw; e += blockDim.x) {
        const int j = e / kFuBw, k = e % kFuBw;
        const int gk = kFuBw * c + k, gj = kFuBw * c + j;
        diag[e] = (k < j && gj < n) ? R[gk + (int64_t)gj * ldr] : 0.0;
    }
    for (int e = tid; e < kFuBw; e += blockDim.x) {
        const int g = kFuBw * c + e;
        dinv[e] = (g < n) ? 1.0 / R[g + (int64_t)g * ldr] : 0.0;
    }
    for (int l = tid; l < Np; l += blockDim.x) {
        unsigned ex = 0;
        if (l < Nc)
            for (int k = 0; k < kFuBw; ++k)
                ex = max(ex, ((unsigned)__double2hiint(R[(kFuBw * c + k) + (int64_t)(kFuBw * (c + 1) + l) * ldr]) >> 20) &
                                 0x7FFu);
        cexp[l] = (int)ex;
        for (int k0 = 0; k0 < kFuBw; k0 += 8) {
            unsigned long long U[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                U[k] = (l < Nc) ? digits_offset((unsigned long long)__double_as_longlong(
                                                    R[(kFuBw * c + k0 + k) + (int64_t)(kFuBw * (c + 1) + l) * ldr]),
                                                (int)ex)
                                : 0x808080808080ull;  // the offset form of zero
#pragma unroll
            for (int q = 0; q < kFuDigits; ++q)
                *reinterpret_cast<uint4 *>(r + q * Np * kFuBw * 2 + kmaj16_off(l, k0)) = pack_plane_f16(U, q);
        }
    }
}

// Columns [lo, hi) (16-column chunks) of one update round of k_subst_fused128
// applied to this thread's row of the tile: the seven tensor-memory groups
// of each output combined in FP32 pairs and subtracted in FP64.  lane0 is the
// thread's tensor-memory lane base (32 x its warp's lane quarter).
__device__ __forceinline__ void f2_apply(uint32_t tmem, int q4, int lane, int ei, int lo, int hi, int n0,
                                         const int *cexp, int cexp_base, double *xs, int col0, int Nc)
{
    const int erow = 32 * q4 + lane;
    for (int h0 = lo; h0 < hi; h0 += 16) {
        uint32_t gv[kFuDigits][16];
#pragma unroll
        for (int d = 0; d < kFuDigits; ++d) tmem_ld16_issue(tmem + ((uint32_t)(32 * q4) << 16) + d * 64 + h0, gv[d]);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            float fhi = __uint_as_float(gv[0][t]), flo = 0.0f;
#pragma unroll
            for (int d = 1; d < kFuDigits; ++d) {
                const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
                const float x = __fmul_rn(__uint_as_float(gv[d][t]), w8);
                const float sum = __fadd_rn(fhi, x);
                const float bb = __fsub_rn(sum, fhi);
                const float err = __fadd_rn(__fsub_rn(fhi, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                fhi = sum;
                flo = __fadd_rn(flo, err);
            }
            const int l = n0 + h0 + t;  // trailing column of the block
            if (l < Nc) {
                const int el = cexp[l - cexp_base];
                if (ei > 0 && el > 0) {
                    const int be = ei + el - 1035;  // 2^(e_i + e_l - 2058) as a biased exponent
                    double *xp = xs + (col0 + l) * kFuM + erow;
                    *xp = *xp - pair2d_pow2(fhi, flo, be);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256, 1)
    k_subst_fused128(const __grid_constant__ CUtensorMap tm_src, const __grid_constant__ CUtensorMap tm_dst,
                     int use_tma, const double *src, int64_t lds, double *dst, int64_t ldd, int64_t m, int n,
                     const unsigned char *__restrict__ rec, int64_t tiles_total, const int *__restrict__ sel,
                     int *colexp_out, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (sel != nullptr && *sel != 0) return;  // the FP32-correction apply was chosen instead
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nb = fu_blocks(n);
    const size_t tile_bytes = (size_t)kFuM * n * 8;
    double *xs = reinterpret_cast<double *>(smem);
    unsigned char *adig = smem + tile_bytes;                      // X_blk digits [7][128 x 16]
    unsigned char *slots = adig + kFuDigits * kFuATile;           // two record slots
    __shared__ __align__(8) uint64_t full_bar, mma_bar;
    __shared__ __align__(8) uint64_t rbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int rowexp[2][kFuM];   // by block parity (the deferred epilogue reads the previous block's)
    __shared__ int defexp[kF2MaxN];   // column exponents of the deferred columns
    __shared__ int out_exp[kF2MaxN];  // largest exponent per column of X (colexp_out)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid < kF2MaxN) out_exp[tid] = 0;

    if (tid == 0) {
        mbar_init(&full_bar, 1);
        mbar_init(&mma_bar, 1);
        mbar_init(&rbar[0], 1);
        mbar_init(&rbar[1], 1);
        fence_barrier_init();
    }
    for (int e = tid; e < kFuDigits * kFuATile / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(adig)[e] = make_uint4(0, 0, 0, 0);
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int64_t first = blockIdx.x;
    // record sequence: rs = (tile iteration) * nb + c, slot rs & 1
    auto issue_record = [&](int64_t rs) {
        const int c = (int)(rs % nb);
        const uint32_t bytes = (uint32_t)f2_rec_bytes(n, c);
        mbar_arrive_expect_tx(&rbar[rs & 1], bytes);
        bulk_load_1d(slots + (rs & 1) * kF2Slot, rec + f2_rec_off(n, c), bytes, &rbar[rs & 1]);
    };
    if (tid == 0 && first < tiles_total) {
        issue_record(0);
        if (use_tma) {
            mbar_arrive_expect_tx(&full_bar, (uint32_t)tile_bytes);
            tma_load_2d(xs, &tm_src, (int)(first * kFuM), 0, &full_bar);
        }
    }
    // Waits are per thread and bounded; one that gives up records a timeout and
    // the thread carries on (the loops are bounded), so no thread is left at a
    // barrier; the status then flags the result.
    uint32_t mphase = 0;
    int64_t rs = 0;
    int it = 0;
    // Lookahead: the last update round of block c holds block c + 1's columns
    // first; all warps apply those, and warps 4-7 apply the round's other
    // columns while warps 0-3 solve block c + 1 (disjoint columns of the tile),
    // so that two warps per scheduler issue FP64.  Rounds further right go
    // first and are applied by all warps.
    bool has_def = false;
    int def_nw = 0, def_col0 = 0, def_Nc = 0, def_par = 0;
    const int64_t ntiles = (first < tiles_total) ? (tiles_total - 1 - first) / gridDim.x + 1 : 0;
    for (int64_t tile = first; tile < tiles_total; tile += gridDim.x, ++it) {
        const int64_t r0 = tile * kFuM;
        if (use_tma) {
            mbar_wait_bounded(&full_bar, it & 1, st);
        } else {
            for (int e = tid; e < kFuM * n; e += blockDim.x) {
                const int row = e & (kFuM - 1), col = e >> 7;
                xs[e] = (r0 + row < m) ? src[r0 + row + (int64_t)col * lds] : 0.0;
            }
            __syncthreads();
        }
        for (int c = 0; c < nb; ++c, ++rs) {
            const int c16 = kFuBw * c;
            const int Nc = n - c16 - kFuBw, Np = fu_npad(n, c);
            // the next record goes into the other slot (its last readers finished
            // at the previous block's closing barrier)
            if (tid == 0 && rs + 1 < ntiles * nb) issue_record(rs + 1);
            mbar_wait_bounded(&rbar[rs & 1], (uint32_t)((rs >> 1) & 1), st);
            const unsigned char *slot = slots + (rs & 1) * kF2Slot;
            const int *cexp = reinterpret_cast<const int *>(slot + kFuDigits * Np * kFuBw * 2);
            const double *rb = reinterpret_cast<const double *>(slot + kFuDigits * Np * kFuBw * 2 + Np * 4);
            const double *dvb = rb + kFuBw * kFuBw;
            if (tid >= kFuM && has_def) {
                // deferred columns [16, def_nw) of the previous block's first round
                const int q4 = warp & 3;
                f2_apply(tmem, q4, lane, rowexp[def_par][32 * q4 + lane], 16, def_nw, 0, defexp, 16, xs, def_col0,
                         def_Nc);
                tc_fence_before();
            }
            has_def = false;
            if (tid < kFuM) {
                const int row = tid;
                double v[kFuBw];
#pragma unroll
                for (int j = 0; j < kFuBw; ++j) v[j] = (c16 + j < n) ? xs[(c16 + j) * kFuM + row] : 0.0;
#pragma unroll
                for (int k = 0; k < kFuBw; ++k) {
                    v[k] *= dvb[k];
#pragma unroll
                    for (int j = k + 1; j < kFuBw; ++j) v[j] = fma(-v[k], rb[j * kFuBw + k], v[j]);
                }
                unsigned ex = 0;
#pragma unroll
                for (int j = 0; j < kFuBw; ++j) {
                    if (c16 + j < n) xs[(c16 + j) * kFuM + row] = v[j];
                    ex = max(ex, ((unsigned)__double2hiint(v[j]) >> 20) & 0x7FFu);
                }
                rowexp[c & 1][row] = (int)ex;
                if (Nc > 0) {
#pragma unroll
                    for (int j0 = 0; j0 < kFuBw; j0 += 8) {
                        unsigned long long U[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            U[j] = digits_offset((unsigned long long)__double_as_longlong(v[j0 + j]), (int)ex);
#pragma unroll
                        for (int q = 0; q < kFuDigits; ++q)
                            *reinterpret_cast<uint4 *>(adig + q * kFuATile + kmaj16_off(row, j0)) = pack_plane_f16(U, q);
                    }
                }
            }
            // trailing columns in rounds of at most 64, the rightmost first
            const int nrounds = (Np + 63) / 64;
            for (int r = nrounds - 1; r >= 0; --r) {
                const int n0 = 64 * r, nw = min(64, Np - n0);
                fence_proxy_async_shared();
                tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint64_t da = smem_desc(smem_u32(adig), 128, 256);
                    const uint64_t db = smem_desc(smem_u32(slot) + (uint32_t)(n0 * kFuBw * 2), 128, 256);
                    const uint32_t idesc = idesc_f16(kFuM, nw);
#pragma unroll
                    for (int p = 0; p < kFuDigits; ++p)
#pragma unroll
                        for (int q = 0; p + q < kFuDigits; ++q)
                            tc_mma(tmem + (uint32_t)((p + q) * 64), da + (uint64_t)((p * kFuATile) >> 4),
                                   db + (uint64_t)((q * Np * kFuBw * 2) >> 4), idesc, p > 0 ? 1u : 0u);
                    tc_commit(&mma_bar);
                }
                mbar_wait_bounded(&mma_bar, mphase, st);
                mphase ^= 1u;
                tc_fence_after();
                const int q4 = warp & 3, hf = warp >> 2;
                const int ei = rowexp[c & 1][32 * q4 + lane];
                if (r > 0) {
                    // two warps per lane quarter, 32 columns each
                    f2_apply(tmem, q4, lane, ei, 32 * hf, min(32 * hf + 32, nw), n0, cexp, 0, xs, c16 + kFuBw, Nc);
                } else {
                    // block c + 1's columns now; the rest of the round is deferred
                    if (hf == 0) f2_apply(tmem, q4, lane, ei, 0, 16, 0, cexp, 0, xs, c16 + kFuBw, Nc);
                    if (nw > 16) {
                        for (int e = tid; e < nw - 16; e += blockDim.x) defexp[e] = cexp[16 + e];
                        has_def = true;
                        def_nw = nw;
                        def_col0 = c16 + kFuBw;
                        def_Nc = Nc;
                        def_par = c & 1;
                    }
                }
                tc_fence_before();
            }
            __syncthreads();
        }
        if (colexp_out != nullptr) {
            // the tile's largest exponent per column of X (for the FP64-grade
            // Gram that follows): warp w scans columns 16 w .. 16 w + 15
            for (int c = 16 * warp; c < min(n, 16 * warp + 16); ++c) {
                unsigned ex = 0;
#pragma unroll
                for (int i = 0; i < kFuM / 32; ++i)
                    ex = max(ex, ((unsigned)__double2hiint(xs[c * kFuM + lane + 32 * i]) >> 20) & 0x7FFu);
                ex = __reduce_max_sync(0xFFFFFFFFu, ex);
                if (lane == 0) out_exp[c] = max(out_exp[c], (int)ex);
            }
        }
        // tile done: store it and fetch the next one into the same buffer once
        // the store has read it out
        if (use_tma) {
            fence_proxy_async_shared();
            __syncthreads();
            if (tid == 0) {
                tma_store_2d(&tm_dst, (int)r0, 0, xs);
                bulk_commit();
                if (tile + gridDim.x < tiles_total) {
                    bulk_wait_read_all();
                    mbar_arrive_expect_tx(&full_bar, (uint32_t)tile_bytes);
                    tma_load_2d(xs, &tm_src, (int)((tile + gridDim.x) * kFuM), 0, &full_bar);
                }
            }
        } else {
            for (int e = tid; e < kFuM * n; e += blockDim.x) {
                const int row = e & (kFuM - 1), col = e >> 7;
                if (r0 + row < m) dst[r0 + row + (int64_t)col * ldd] = xs[e];
            }
            __syncthreads();
        }
    }
    if (tid == 0 && use_tma) bulk_wait_all();
    tc_fence_before();
    __syncthreads();
    if (colexp_out != nullptr && tid < n && out_exp[tid] > 0) atomicMax(colexp_out + tid, out_exp[tid]);
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// FP64-grade Gram G = X^T X for n <= 64 on the tensor cores.  Column j of X is
// written as seven 8-bit digits relative to 2^(e_j + 1), e_j the largest
// exponent of the column over all m rows (so the scale of every product is
// fixed and tensor-memory sums stay integers across row blocks).  The digit
// planes X_0 .. X_6 (64 columns x 64 rows each, K-major) are followed by a zero
// plane X_7, so that a 128-row A operand starting at plane p is the stack
// [X_p; X_{p+1}]: one MMA with B = X_q forms the digit products (p, q) in
// tensor-memory lanes 0-63 and (p + 1, q) in lanes 64-127.  Sixteen stacks
// (p even) cover all 28 products with p + q <= 6; accumulator block d = p + q
// holds weight group d in its upper lanes and group d + 1 in its lower lanes.
// Every accumulator sums at most four products below 2^14 per row, so a
// window of 256 rows keeps it an integer below 2^24 (exact in FP32); after
// each window the groups are combined (weights 2^-8d) and added in FP64, and
// the fixed scale 2^(e_i + e_j - 2058) is applied once at the end.  Operand
// buffers of 64 rows alternate so that the digits of one are written while
// the tensor core reads the other.
// ---------------------------------------------------------------------------
constexpr int kG6Rows = 64;                     // rows of X per operand buffer (K = 4 x 16)
constexpr int kG6Window = 4;                    // buffers per exact accumulation window (256 rows)
constexpr int kG6Plane = 64 * kG6Rows * 2;      // one digit plane, 8 KB
constexpr int kG6Planes = 8;                    // X_0 .. X_6 and the zero plane
constexpr int kG6Buf = kG6Planes * kG6Plane;    // 64 KB per buffer
constexpr int kG6Stage = kG6Rows * 64 * 8;      // 32 KB: X's 64 rows x 64 columns, four swizzled TMA boxes
constexpr size_t kG6Smem = 2 * (size_t)kG6Buf + 2 * (size_t)kG6Stage;  // 192 KB

// Largest exponent field of each column over all rows: atomicMax into
// colexp[0 .. n) (zeroed by the caller).  grid.y = column.
__global__ void k_colexp(const double *__restrict__ X, int64_t ldx, int64_t m, int *colexp, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    const int col = blockIdx.y;
    unsigned e = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += (int64_t)gridDim.x * blockDim.x)
        e = max(e, ((unsigned)__double2hiint(X[r + (int64_t)col * ldx]) >> 20) & 0x7FFu);
    e = __reduce_max_sync(0xFFFFFFFFu, e);
    if ((threadIdx.x & 31) == 0 && e > 0) atomicMax(colexp + col, (int)e);
}

// All eight warps load rows and write digits; six of them drain tensor memory
// (two quarters have nothing on or above the diagonal), and lane 0 of warp 3,
// one that never drains, also issues the MMAs.
constexpr int kG6Producers = 256;
constexpr int kG6MmaWarp = 3;

__global__ void __launch_bounds__(kG6Producers, 1)
    k_gram_oz64(const __grid_constant__ CUtensorMap tm_x, int use_tma, const double *__restrict__ X, int64_t ldx,
                int64_t m, int n, const int *__restrict__ colexp_g, int64_t bufs_total, int64_t bufs_per_cta,
                double *__restrict__ Gpart, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t ready[2];  // producers -> MMA thread: digits of a buffer written (256 arrivals)
    __shared__ __align__(8) uint64_t done[2];   // MMA thread -> producers: a buffer's MMAs completed (commit)
    __shared__ __align__(8) uint64_t tfree;     // producers -> MMA thread: a window's accumulators read (256)
    __shared__ __align__(8) uint64_t full[2];   // TMA -> producers: a staging slot holds its 64 rows of X
    __shared__ uint32_t tmem_base;
    __shared__ int cex[64];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool producer = true;
    const bool mma_thread = (warp == kG6MmaWarp && lane == 0);

    for (int e = tid; e < (int)(kG6Smem / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    if (tid < 64) {
        cex[tid] = (tid < n) ? colexp_g[tid] : 0;
        if (cex[tid] == 0x7FF) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);  // NaN or Inf in X
    }
    if (tid == 0) {
        mbar_init(&ready[0], kG6Producers);
        mbar_init(&ready[1], kG6Producers);
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        mbar_init(&tfree, kG6Producers);
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int64_t b_begin = blockIdx.x * bufs_per_cta;
    const int64_t b_end = min(bufs_total, b_begin + bufs_per_cta);
    const int nbufs = (b_end > b_begin) ? (int)(b_end - b_begin) : 0;
    // Waits are per thread and bounded; one that gives up records a timeout in
    // the status and the thread carries on (every arrival still happens), so
    // no thread is left waiting and the sums are not published.
    bool ok = true;

    // epilogue role: tensor-memory lane quarter q4 (rows of G: lanes 0-63 the
    // upper halves of the stacks, 64-127 the lower), 32 columns of G per half;
    // the quarter of rows 32-63 has nothing on or above the diagonal in the
    // first 32 columns
    const int q4 = warp & 3, half = (warp >> 2) & 1;
    const bool skip_epi = (q4 & 1) && half == 0;
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;

    if (producer) {
        // column of X and 16-row quarter of each buffer this thread converts; the
        // eight lanes of each quarter-warp take eight consecutive columns, so
        // their 16-byte digit stores (and swizzled staging reads) fall in
        // distinct banks
        const int j = 8 * warp + (lane & 7), rq = lane >> 3;
        const int ej = cex[j];
        const bool has_col = j < n;
        const double *xcol = X + (int64_t)j * ldx;
        const uint64_t desc0 = smem_desc(smem_u32(smem), 128, 1024);
        constexpr uint32_t idesc = idesc_f16(128, 64);
        constexpr int kP[16] = {0, 2, 4, 6, 0, 2, 4, 0, 2, 4, 0, 2, 0, 2, 0, 0};
        constexpr int kQ[16] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 4, 4, 5, 6};
        unsigned char *stage = smem + 2 * kG6Buf;  // [2 slots][4 boxes of 16 rows x 64 columns]
        // X's rows of buffer it: four 16-row x 64-column boxes (128-byte swizzle)
        auto issue_load = [&](int it_load) {
            unsigned char *slot = stage + (it_load & 1) * kG6Stage;
            mbar_arrive_expect_tx(&full[it_load & 1], (uint32_t)kG6Stage);
            const int r0 = (int)((b_begin + it_load) * kG6Rows);
#pragma unroll
            for (int q = 0; q < 4; ++q) tma_load_2d(slot + q * (kG6Stage / 4), &tm_x, r0 + 16 * q, 0, &full[it_load & 1]);
        };
        if (use_tma && mma_thread) {
            if (nbufs > 0) issue_load(0);
            if (nbufs > 1) issue_load(1);
        }
        for (int it = 0; it < nbufs; ++it) {
            const int64_t b = b_begin + it;
            const int buf = it & 1;
            unsigned char *base = smem + buf * kG6Buf;
            if (use_tma) ok &= mbar_wait_bounded(&full[buf], (it >> 1) & 1, st);
            // the MMAs issued two buffers ago read this digit buffer
            if (it >= 2) ok &= mbar_wait_bounded(&done[buf], ((it - 2) >> 1) & 1, st);
            if (has_col) {
                const unsigned char *box = stage + buf * kG6Stage + rq * (kG6Stage / 4) + j * 128;
#pragma unroll
                for (int g8 = 0; g8 < 2; ++g8) {
                    // eight rows of column j: swizzled 16-byte chunks 4 g8 .. 4 g8 + 3 of the box
                    double v[8];
                    if (use_tma) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const double2 w = *reinterpret_cast<const double2 *>(box + (((4 * g8 + c) ^ (j & 7)) << 4));
                            v[2 * c] = w.x;
                            v[2 * c + 1] = w.y;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int64_t r = b * kG6Rows + 16 * rq + 8 * g8 + i;
                            v[i] = (r < m) ? xcol[r] : 0.0;
                        }
                    }
                    unsigned long long U[8];
#pragma unroll
                    for (int r = 0; r < 8; ++r) U[r] = digits_offset((unsigned long long)__double_as_longlong(v[r]), ej);
#pragma unroll
                    for (int q = 0; q < kOzDigits; ++q)
                        *reinterpret_cast<uint4 *>(base + q * kG6Plane + kmaj_off(j, 16 * rq + 8 * g8)) =
                            pack_plane_f16(U, q);
                }
            }
            fence_proxy_async_shared();
            mbar_arrive(&ready[buf]);
            if ((it % kG6Window) == 0 && it > 0) {
                // the previous window is complete once its last buffer's MMAs
                // are: read its sums into FP32 pairs, release tensor memory,
                // then add them in FP64
                ok &= mbar_wait_bounded(&done[buf ^ 1], ((it - 1) >> 1) & 1, st);
                tc_fence_after();
                float hi[32], lo[32];
                if (!skip_epi) gram64_read(tmem, q4, half, hi, lo);
                tc_fence_before();
                mbar_arrive(&tfree);
                if (!skip_epi) gram64_accumulate(hi, lo, acc);
            }
            if (mma_thread) {
                // every producer's digits of this buffer (and, at a window start,
                // every read of the last window's sums) are in: issue its MMAs
                const bool first_of_window = (it % kG6Window) == 0;
                ok &= mbar_wait_bounded(&ready[buf], (it >> 1) & 1, st);
                // every producer has read staging slot `buf`: refill it
                if (use_tma && it + 2 < nbufs) issue_load(it + 2);
                if (first_of_window && it > 0) ok &= mbar_wait_bounded(&tfree, ((it / kG6Window) - 1) & 1, st);
                tc_fence_after();
                const uint64_t dbuf = desc0 + (uint64_t)(buf * (kG6Buf >> 4));
#pragma unroll
                for (int kk = 0; kk < kG6Rows / 16; ++kk)
#pragma unroll
                    for (int x = 0; x < 16; ++x) {
                        // the first MMA into each block (x < 7 lists blocks 0, 2, 4, 6, 1, 3, 5) starts the window
                        const uint32_t acc_on = (!first_of_window || kk > 0 || x >= 7) ? 1u : 0u;
                        tc_mma(tmem + (uint32_t)((kP[x] + kQ[x]) * 64),
                               dbuf + (uint64_t)((kP[x] * kG6Plane + kk * 256) >> 4),
                               dbuf + (uint64_t)((kQ[x] * kG6Plane + kk * 256) >> 4), idesc, acc_on);
                    }
                tc_commit(&done[buf]);
            }
        }
        // last window
        if (nbufs > 0) {
            ok &= mbar_wait_bounded(&done[(nbufs - 1) & 1], ((nbufs - 1) >> 1) & 1, st);
            tc_fence_after();
            float hi[32], lo[32];
            if (!skip_epi) {
                gram64_read(tmem, q4, half, hi, lo);
                gram64_accumulate(hi, lo, acc);
            }
        }
    }
    ok = __syncthreads_and(ok) != 0;
    tc_fence_before();
    // G[i][j] = 2^(e_i + e_j - 2058) (upper-lane sum + 2^-8 lower-lane sum):
    // the lower lanes hand their sums over through shared memory
    double *low = reinterpret_cast<double *>(smem);  // [64][64], i + 64 j
    const int gi = 32 * (q4 & 1) + lane;
    if (producer && q4 >= 2 && !skip_epi) {
#pragma unroll
        for (int t = 0; t < 32; ++t) low[gi + 64 * (32 * half + t)] = acc[t];
    }
    __syncthreads();
    if (ok && producer && q4 < 2 && !skip_epi && gi < n) {
        double *out = Gpart + (int64_t)blockIdx.x * n * n;
        const int ei = cex[gi];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int gj = 32 * half + t;
            if (gj < n && gi <= gj) {
                const int e = ei + cex[gj] - 2058;
                const double v = acc[t] + ldexp(low[gi + 64 * gj], -8);
                out[gi + (int64_t)gj * n] = (ei > 0 && cex[gj] > 0) ? ldexp(v, e) : 0.0;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// FP64-grade Gram G = X^T X for 64 < n <= 128 on the tensor cores, pipelined
// like k_gram_oz64.  Column j of X is cut into seven 8-bit digits relative to
// 2^(e_j + 1), e_j its largest exponent over all m rows.  Two kinds of CTA
// share the grid (tensor memory holds seven accumulator groups d = p + q of 64
// columns, so one CTA forms one 128 x 64 block):
//   J = 1 (the first g1 CTAs): the digit planes X_0 .. X_6 of a 32-row buffer
//     hold all n columns (the A operand, M = 128, rows >= n zero) and columns
//     64 .. n - 1 of the same planes are the B operand (N = 64): the blocks
//     G[0:64, 64:n] and G[64:n, 64:n];
//   J = 0 (the other g0 CTAs): only columns 0 .. 63 are cut (A rows 64 .. 127
//     stay zero) for G[0:64, 0:64], half the digit work per row (the row
//     split between the two kinds: oz128_grid).
// Each group sums at most seven products below 2^14 a row, so a window of
// four buffers (128 rows) keeps it an integer below 2^24 (exact in FP32);
// after each window the groups are combined (weights 2^-8d) and added in
// FP64, and the fixed scale 2^(e_i + e_j - 2058) is applied once at the end.
// Rows of X arrive by TMA as two 16-row x n-column boxes (128-byte swizzle)
// into two staging slots; eight producer warps write 16-byte digit stores into
// two operand buffers and signal an mbarrier; lane 0 of a ninth warp waits for
// it, refills the staging slot and issues the buffer's 56 MMAs (so no producer
// waits while the MMAs are issued).
// ---------------------------------------------------------------------------
constexpr int kG8Rows = 32;                       // rows of X per operand buffer (K = 2 x 16)
constexpr int kG8Window = 4;                      // buffers per exact accumulation window (128 rows)
constexpr int kG8Plane = 128 * kG8Rows * 2;       // one digit plane, 8 KB
constexpr int kG8Buf = kOzDigits * kG8Plane;      // 56 KB per buffer
constexpr int kG8Box = 16 * 128 * 8;              // one 16-row x 128-column staging box, 16 KB
constexpr int kG8Stage = 2 * kG8Box;              // 32 KB: the buffer's 32 rows
constexpr size_t kG8Smem = 2 * (size_t)kG8Buf + 2 * (size_t)kG8Stage;  // 176 KB
constexpr int kG8Producers = 256;                 // warps 0-7; warp 8 issues the copies and MMAs
constexpr int kG8Threads = kG8Producers + 32;     // nine warps: 168 registers a thread (an SMSP holds three)

// Byte offset of element (row, k) in a K-major, no-swizzle operand tile with
// K = 32 (4 core matrices of 128 bytes along K per 8-row group).
__device__ __forceinline__ int kmaj32_off(int row, int k)
{
    return (row & 7) * 16 + (row >> 3) * 512 + (k & 7) * 2 + (k >> 3) * 128;
}

__global__ void __launch_bounds__(kG8Threads, 1)
    k_gram_oz128(const __grid_constant__ CUtensorMap tm_x, const __grid_constant__ CUtensorMap tm_h, int use_tma,
                 const double *__restrict__ X, int64_t ldx, int64_t m, int n, const int *__restrict__ colexp_g,
                 int64_t bufs_total, int g1, int64_t bpc1, int g0, int64_t bpc0, double *__restrict__ Gpart,
                 RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t ready[2];  // producers -> MMA thread: digits of a buffer written (256 arrivals)
    __shared__ __align__(8) uint64_t done[2];   // MMA thread -> producers: a buffer's MMAs completed (commit)
    __shared__ __align__(8) uint64_t tfree;     // producers -> MMA thread: a window's accumulators read (256)
    __shared__ __align__(8) uint64_t full[2];   // TMA -> producers: a staging slot holds its 32 rows of X
    __shared__ uint32_t tmem_base;
    __shared__ int cex[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int J = ((int)blockIdx.x < g1) ? 1 : 0;
    const int slot = J ? (int)blockIdx.x : (int)blockIdx.x - g1;  // partial-sum slot and row chunk
    const int ncut = J ? n : 64;                                  // columns cut into digits
    const bool producer = tid < kG8Producers;
    const bool mma_thread = tid == kG8Producers;

    // digit buffers zeroed once (rows >= n stay zero); the staging slots are
    // written by TMA only
    for (int e = tid; e < (int)(2 * kG8Buf / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    fence_proxy_async_shared();
    if (tid < 128) {
        cex[tid] = (tid < n) ? colexp_g[tid] : 0;
        if (cex[tid] == 0x7FF) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);  // NaN or Inf in X
    }
    if (tid == 0) {
        mbar_init(&ready[0], 256);
        mbar_init(&ready[1], 256);
        mbar_init(&done[0], 1);
        mbar_init(&done[1], 1);
        mbar_init(&tfree, 256);
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int64_t bpc = J ? bpc1 : bpc0;
    const int64_t b_begin = slot * bpc;
    const int64_t b_end = min(bufs_total, b_begin + bpc);
    const int nbufs = (b_end > b_begin) ? (int)(b_end - b_begin) : 0;
    // Waits are per thread and bounded; one that gives up records a timeout in
    // the status and the thread carries on (every arrival still happens), so
    // no thread is left waiting and the sums are not published.
    bool ok = true;

    // epilogue role: tensor-memory lane quarter q4 (rows 32 q4 .. of G), 32
    // columns of the block per half; quarters with nothing on or above the
    // diagonal skip the reads
    const int q4 = warp & 3, half = (warp >> 2) & 1;
    const bool skip_epi =
        !producer || ((J == 0) ? (q4 >= 2 || (q4 == 1 && half == 0)) : (q4 == 3 && half == 0));
    double acc[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) acc[t] = 0.0;

    // this thread's column of X and its rows of each buffer: J = 1, 16-row half
    // hq (both 8-row groups); J = 0, the 8-row group g8 of half hq.  The eight
    // lanes of each quarter-warp take eight consecutive columns, so their
    // 16-byte digit stores (and swizzled staging reads) fall in distinct banks
    const int j = J ? (16 * warp + (lane & 15)) : (8 * warp + (lane & 7));
    const int hq = J ? (lane >> 4) : ((lane >> 3) & 1);
    const int g8_lo = J ? 0 : (lane >> 4), g8_hi = J ? 2 : (lane >> 4) + 1;
    const bool has_col = producer && j < ncut;
    const int ej = has_col ? cex[j] : 0;
    const double *xcol = X + (int64_t)j * ldx;
    const uint64_t desc0 = smem_desc(smem_u32(smem), 128, 512);
    constexpr uint32_t idesc = idesc_f16(128, 64);
    unsigned char *stage = smem + 2 * kG8Buf;  // [2 slots][2 boxes of 16 rows x n columns]
    const uint32_t box_bytes = (uint32_t)(16 * ncut * 8);
    const CUtensorMap *tmap = J ? &tm_x : &tm_h;
    auto issue_load = [&](int it_load) {
        unsigned char *sl = stage + (it_load & 1) * kG8Stage;
        mbar_arrive_expect_tx(&full[it_load & 1], 2 * box_bytes);
        const int r0 = (int)((b_begin + it_load) * kG8Rows);
#pragma unroll
        for (int q = 0; q < 2; ++q) tma_load_2d(sl + q * kG8Box, tmap, r0 + 16 * q, 0, &full[it_load & 1]);
    };
    if (use_tma && mma_thread) {
        if (nbufs > 0) issue_load(0);
        if (nbufs > 1) issue_load(1);
    }
    for (int it = 0; producer && it < nbufs; ++it) {
        const int64_t b = b_begin + it;
        const int buf = it & 1;
        unsigned char *base = smem + buf * kG8Buf;
        if (use_tma) ok &= mbar_wait_bounded(&full[buf], (it >> 1) & 1, st);
        // the MMAs issued two buffers ago read this digit buffer
        if (it >= 2) ok &= mbar_wait_bounded(&done[buf], ((it - 2) >> 1) & 1, st);
        if (has_col) {
            const unsigned char *box = stage + buf * kG8Stage + hq * kG8Box + j * 128;
            for (int g8 = g8_lo; g8 < g8_hi; ++g8) {
                // eight rows of column j: swizzled 16-byte chunks 4 g8 .. 4 g8 + 3 of the box
                double v[8];
                if (use_tma) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double2 w = *reinterpret_cast<const double2 *>(box + (((4 * g8 + c) ^ (j & 7)) << 4));
                        v[2 * c] = w.x;
                        v[2 * c + 1] = w.y;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int64_t r = b * kG8Rows + 16 * hq + 8 * g8 + i;
                        v[i] = (r < m) ? xcol[r] : 0.0;
                    }
                }
                unsigned long long U[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) U[r] = digits_offset((unsigned long long)__double_as_longlong(v[r]), ej);
#pragma unroll
                for (int q = 0; q < kOzDigits; ++q)
                    *reinterpret_cast<uint4 *>(base + q * kG8Plane + kmaj32_off(j, 16 * hq + 8 * g8)) =
                        pack_plane_f16(U, q);
            }
        }
        fence_proxy_async_shared();
        mbar_arrive(&ready[buf]);
        if ((it % kG8Window) == 0 && it > 0) {
            // the previous window is complete once its last buffer's MMAs
            // are: read its sums into FP32 pairs, release tensor memory,
            // then add them in FP64
            ok &= mbar_wait_bounded(&done[buf ^ 1], ((it - 1) >> 1) & 1, st);
            tc_fence_after();
            float hi[32], lo[32];
            if (!skip_epi) gram64_read(tmem, q4, half, hi, lo);
            tc_fence_before();
            mbar_arrive(&tfree);
            if (!skip_epi) gram_accumulate_pair(hi, lo, acc);
        }
    }
    for (int it = 0; mma_thread && it < nbufs; ++it) {
        const int buf = it & 1;
        // every producer's digits of this buffer (and, at a window start,
        // every read of the last window's sums) are in: issue its MMAs
        const bool first_of_window = (it % kG8Window) == 0;
        ok &= mbar_wait_bounded(&ready[buf], (it >> 1) & 1, st);
        // every producer has read staging slot `buf`: refill it
        if (use_tma && it + 2 < nbufs) issue_load(it + 2);
        if (first_of_window && it > 0) ok &= mbar_wait_bounded(&tfree, ((it / kG8Window) - 1) & 1, st);
        tc_fence_after();
        const uint64_t dbuf = desc0 + (uint64_t)(buf * (kG8Buf >> 4));
#pragma unroll
        for (int kk = 0; kk < kG8Rows / 16; ++kk)
#pragma unroll
            for (int p = 0; p < kOzDigits; ++p)
#pragma unroll
                for (int q = 0; p + q < kOzDigits; ++q) {
                    // p = 0 lists every group first: it starts the window's sums
                    const uint32_t acc_on = (!first_of_window || kk > 0 || p > 0) ? 1u : 0u;
                    tc_mma(tmem + (uint32_t)((p + q) * 64), dbuf + (uint64_t)((p * kG8Plane + kk * 256) >> 4),
                           dbuf + (uint64_t)((q * kG8Plane + J * 4096 + kk * 256) >> 4), idesc, acc_on);
                }
        tc_commit(&done[buf]);
    }
    // last window
    if (producer && nbufs > 0) {
        ok &= mbar_wait_bounded(&done[(nbufs - 1) & 1], ((nbufs - 1) >> 1) & 1, st);
        tc_fence_after();
        float hi[32], lo[32];
        if (!skip_epi) {
            gram64_read(tmem, q4, half, hi, lo);
            gram_accumulate_pair(hi, lo, acc);
        }
    }
    ok = __syncthreads_and(ok) != 0;
    tc_fence_before();
    const int gi = 32 * q4 + lane;
    if (ok && J == 1 && slot >= g0) {
        // no J = 0 CTA has this slot: its block G[0:64, 0:64] adds zero
        double *out = Gpart + (int64_t)slot * n * n;
        for (int e = tid; e < 64 * 64; e += blockDim.x) out[(e & 63) + (int64_t)(e >> 6) * n] = 0.0;
    }
    if (ok && !skip_epi && gi < n) {
        double *out = Gpart + (int64_t)slot * n * n;
        const int ei = cex[gi];
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int gj = 64 * J + 32 * half + t;
            if (gj < n && gi <= gj) {
                const int e = ei + cex[gj] - 2058;
                out[gi + (int64_t)gj * n] = (ei > 0 && cex[gj] > 0) ? ldexp(acc[t], e) : 0.0;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// FP64-grade product Q = X T on the tensor cores for n <= 64 (the last
// CholeskyQR pass's apply, T = R_P^{-1}), in place.  A CTA walks 128-row
// tiles of X: one TMA load per tile into shared memory (the next tile's load
// is issued as soon as the current tile's digits are all written), each row
// of X written as seven 8-bit digits relative to its own largest exponent,
// each column of T relative to its own (digits of T built once per CTA).  The
// digit products p + q = d accumulate in tensor-memory group d over K = n
// (at most seven pairs of products below 2^14 per row: exact in FP32); the
// X digits are produced one 16-column K-step at a time into two alternating
// buffers, so the tensor core works on one K-step while the next is written.
// The epilogue combines the seven groups of each output and writes Q with one
// FP64 addition.
// ---------------------------------------------------------------------------
constexpr int kAqM = 128;
constexpr int kAqPlane = kAqM * 16 * 2;  // one X digit plane of a K-step (4 KB)
constexpr int kAqTPlane = 64 * 64 * 2;   // one T digit plane (8 KB), K-major, K = 64
__host__ __device__ inline size_t aq_smem_bytes(int n)
{
    return (size_t)kAqM * n * 8 + 2 * (size_t)kOzDigits * kAqPlane + (size_t)kOzDigits * kAqTPlane;
}

// ACC: the product is added into D (a column block of X other than the one
// read) instead of overwriting the columns read; a template parameter, so that
// the overwriting form carries none of the adding form's registers.
template <bool ACC>
__global__ void __launch_bounds__(256, 1)
    k_apply_oz64(const __grid_constant__ CUtensorMap tm_x, int use_tma, double *X, int64_t ldx, int64_t m, int n,
                 const double *__restrict__ T, int64_t ldt, int64_t tiles_total, const int *__restrict__ sel,
                 int want, int *colexp_out, int nout, int full, double *D, int64_t ldd, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (sel != nullptr && *sel != want) return;  // the other form was chosen
    extern __shared__ __align__(1024) unsigned char smem[];
    const size_t tile_bytes = (size_t)kAqM * n * 8;
    double *xs = reinterpret_cast<double *>(smem);            // [n][128]
    unsigned char *adig = smem + tile_bytes;                  // [2][7][128 x 16]
    unsigned char *tdig = adig + 2 * kOzDigits * kAqPlane;    // [7][64 x 64]
    __shared__ __align__(8) uint64_t full_bar;
    __shared__ __align__(8) uint64_t abar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int colexp_t[64];
    __shared__ int pexp[2][kAqM];
    __shared__ int out_exp[64];  // largest exponent per column of Q (colexp_out)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & (kAqM - 1), h = tid >> 7;  // digit role: row of the tile, 8-column half of a K-step

    for (int e = tid; e < (int)((2 * kOzDigits * kAqPlane + kOzDigits * kAqTPlane) / 16); e += blockDim.x)
        reinterpret_cast<uint4 *>(adig)[e] = make_uint4(0, 0, 0, 0);
    if (tid < 64) out_exp[tid] = 0;
    if (tid < 64) {
        unsigned ex = 0;
        if (tid < nout)
            for (int k = 0; k < (full ? n : tid + 1); ++k)
                ex = max(ex, ((unsigned)__double2hiint(T[k + (int64_t)tid * ldt]) >> 20) & 0x7FFu);
        colexp_t[tid] = (int)ex;
    }
    if (tid == 0) {
        mbar_init(&full_bar, 1);
        mbar_init(&abar[0], 1);
        mbar_init(&abar[1], 1);
        fence_barrier_init();
    }
    __syncthreads();
    // digits of T: B operand element (l, k) = T[k][l] (zero below the diagonal
    // unless the block is full)
    for (int e = tid; e < nout * 8; e += blockDim.x) {
        const int l = e >> 3, k0 = 8 * (e & 7);
        unsigned long long U[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int k = k0 + r;
            const unsigned long long bits =
                ((full || k <= l) && k < n) ? (unsigned long long)__double_as_longlong(T[k + (int64_t)l * ldt]) : 0ull;
            U[r] = digits_offset(bits, colexp_t[l]);
        }
#pragma unroll
        for (int q = 0; q < kOzDigits; ++q) {
            const uint4 w = pack_plane_f16(U, q);
            *reinterpret_cast<uint4 *>(tdig + q * kAqTPlane + kmaj_off(l, k0)) = w;
        }
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint64_t da0 = smem_desc(smem_u32(adig), 128, 256);   // X digits, K = 16 per plane
    const uint64_t dt0 = smem_desc(smem_u32(tdig), 128, 1024);  // T digits, K = 64
    constexpr uint32_t idesc = idesc_f16(kAqM, 64);
    const int nk = (n + 15) / 16;

    if (use_tma && tid == 0 && (int64_t)blockIdx.x < tiles_total) {
        mbar_arrive_expect_tx(&full_bar, (uint32_t)tile_bytes);
        tma_load_2d(xs, &tm_x, (int)(blockIdx.x * kAqM), 0, &full_bar);
    }
    // Waits are per thread and bounded; one that gives up records a timeout and
    // the loop runs to its end without further effect on the result's status.
    bool ok = true;
    uint32_t loads = 0, ksteps = 0;
    for (int64_t tile = blockIdx.x; tile < tiles_total; tile += gridDim.x) {
        const int64_t r0 = tile * kAqM;
        if (use_tma) {
            ok &= mbar_wait_bounded(&full_bar, loads & 1u, st);
            ++loads;
        } else {
            for (int e = tid; e < kAqM * n; e += blockDim.x) {
                const int rr = e & (kAqM - 1), col = e >> 7;
                xs[e] = (r0 + rr < m) ? X[r0 + rr + (int64_t)col * ldx] : 0.0;
            }
            __syncthreads();
        }
        // largest exponent of each row (two threads per row, 32 columns each)
        {
            unsigned ex = 0;
            for (int c = 32 * h; c < min(n, 32 * h + 32); ++c)
                ex = max(ex, ((unsigned)__double2hiint(xs[c * kAqM + row]) >> 20) & 0x7FFu);
            pexp[h][row] = (int)ex;
        }
        __syncthreads();
        const int ei = max(pexp[0][row], pexp[1][row]);
        for (int kk = 0; kk < nk; ++kk, ++ksteps) {
            const int buf = ksteps & 1;
            // the MMAs of two K-steps ago read this buffer
            if (ksteps >= 2) ok &= mbar_wait_bounded(&abar[buf], ((ksteps - 2) >> 1) & 1, st);
            {
                unsigned long long U[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const int c = 16 * kk + 8 * h + r;
                    U[r] = digits_offset(c < n ? (unsigned long long)__double_as_longlong(xs[c * kAqM + row]) : 0ull, ei);
                }
                unsigned char *plane = adig + buf * kOzDigits * kAqPlane;
#pragma unroll
                for (int q = 0; q < kOzDigits; ++q) {
                    const uint4 w = pack_plane_f16(U, q);
                    *reinterpret_cast<uint4 *>(plane + q * kAqPlane + kmaj16_off(row, 8 * h)) = w;
                }
            }
            fence_proxy_async_shared();
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                // every read of this tile's X is done: fetch the next tile
                if (kk == nk - 1 && use_tma && tile + gridDim.x < tiles_total) {
                    mbar_arrive_expect_tx(&full_bar, (uint32_t)tile_bytes);
                    tma_load_2d(xs, &tm_x, (int)((tile + gridDim.x) * kAqM), 0, &full_bar);
                }
                const uint64_t da = da0 + (uint64_t)((buf * kOzDigits * kAqPlane) >> 4);
#pragma unroll
                for (int p = 0; p < kOzDigits; ++p)
#pragma unroll
                    for (int q = 0; p + q < kOzDigits; ++q)
                        tc_mma(tmem + (uint32_t)((p + q) * 64), da + (uint64_t)((p * kAqPlane) >> 4),
                               dt0 + (uint64_t)((q * kAqTPlane + kk * 256) >> 4), idesc, (kk > 0 || p > 0) ? 1u : 0u);
                tc_commit(&abar[buf]);
            }
        }
        // the tile's last K-step completes after all earlier ones
        ok &= mbar_wait_bounded(&abar[(ksteps - 1) & 1], ((ksteps - 1) >> 1) & 1, st);
        tc_fence_after();
        {
            const int q4 = warp & 3, half = warp >> 2;
            const int erow = 32 * q4 + lane;
            const int er = max(pexp[0][erow], pexp[1][erow]);
            const int64_t gr = r0 + erow;
#pragma unroll
            for (int c16 = 0; c16 < 2; ++c16) {
                const int col0 = 32 * half + 16 * c16;
                if (col0 >= nout) continue;  // warp-uniform
                // the accumulated destination's 16 values, all in flight before
                // the tensor-memory reads (none waits for another)
                double dv[16];
                if (ACC) {
#pragma unroll
                    for (int t = 0; t < 16; ++t)
                        dv[t] = (col0 + t < nout && gr < m) ? __ldcs(D + gr + (int64_t)(col0 + t) * ldd) : 0.0;
                }
                uint32_t g[kOzDigits][16];
#pragma unroll
                for (int d = 0; d < kOzDigits; ++d)
                    tmem_ld16_issue(tmem + ((uint32_t)(32 * q4) << 16) + d * 64 + col0, g[d]);
                tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    float hi = __uint_as_float(g[0][t]), lo = 0.0f;
#pragma unroll
                    for (int d = 1; d < kOzDigits; ++d) {
                        const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
                        const float x = __fmul_rn(__uint_as_float(g[d][t]), w8);
                        const float sum = __fadd_rn(hi, x);
                        const float bb = __fsub_rn(sum, hi);
                        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                        hi = sum;
                        lo = __fadd_rn(lo, err);
                    }
                    const int l = col0 + t;
                    double qv = 0.0;
                    if (l < nout && gr < m) {
                        const int el = colexp_t[l];
                        const int be = er + el - 1035;  // 2^(e_i + e_l - 2058) as a biased exponent
                        qv = (er > 0 && el > 0) ? pair2d_pow2(hi, lo, be) : 0.0;
                        if (ACC) {
                            qv = dv[t] + qv;
                            __stcs(D + gr + (int64_t)l * ldd, qv);
                        } else {
                            X[gr + (int64_t)l * ldx] = qv;
                        }
                    }
                    if (colexp_out != nullptr) {
                        const unsigned e = __reduce_max_sync(0xFFFFFFFFu, ((unsigned)__double2hiint(qv) >> 20) & 0x7FFu);
                        if (lane == 0 && e > 0 && l < nout) atomicMax(&out_exp[l], (int)e);
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    // drain: a load still in flight after a timeout (bounded)
    if (tid == 0 && use_tma && !ok) mbar_wait_bounded(&full_bar, loads & 1u, st);
    tc_fence_before();
    __syncthreads();
    if (colexp_out != nullptr && tid < nout && out_exp[tid] > 0) atomicMax(colexp_out + tid, out_exp[tid]);
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// T = R^{-1} for upper-triangular R, n <= 64: CTA c (one warp) solves
// R t = e_c by column-oriented back substitution.  Lane l holds rows l and
// l + 32 of t; for k = c, c - 1, ..., 0 the owner of row k forms
// t_k = s_k / R_kk (times the precomputed reciprocal), one shuffle broadcasts
// it, and every lane updates its rows i < k: s_i -= R_ik t_k (k descending, a
// fixed order).  R's leading c + 1 columns are staged in shared memory.  One
// warp per SM keeps the FP64 pipe free of contention: the chain of
// dependent operations, not FP64 throughput, sets the time.
__global__ void __launch_bounds__(32) k_tri_inverse64(const double *__restrict__ R, int n, int64_t ldr,
                                                       double *__restrict__ T, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double rs[64 * 64];  // R[i][k] at k * 64 + i
    const int c = blockIdx.x, lane = threadIdx.x;
    for (int k = 0; k <= c; ++k) {
        rs[k * 64 + lane] = (lane <= k) ? R[lane + (int64_t)k * ldr] : 0.0;
        if (lane + 32 < n) rs[k * 64 + lane + 32] = (lane + 32 <= k) ? R[lane + 32 + (int64_t)k * ldr] : 0.0;
    }
    const double d0 = (lane < n) ? 1.0 / R[lane + (int64_t)lane * ldr] : 0.0;
    const double d1 = (lane + 32 < n) ? 1.0 / R[(lane + 32) + (int64_t)(lane + 32) * ldr] : 0.0;
    __syncwarp();
    double s0 = (lane == c) ? 1.0 : 0.0, s1 = (lane + 32 == c) ? 1.0 : 0.0;
    for (int k = c; k >= 0; --k) {
        const double own = (k < 32) ? s0 * d0 : s1 * d1;  // right only in the owner lane
        const double tk = __shfl_sync(0xFFFFFFFFu, own, k & 31);
        if (k < 32) {
            if (lane == k) s0 = tk;
        } else if (lane == k - 32) {
            s1 = tk;
        }
        if (lane < k) s0 = fma(-rs[k * 64 + lane], tk, s0);
        if (lane + 32 < k) s1 = fma(-rs[k * 64 + lane + 32], tk, s1);
    }
    if (lane < n) T[lane + (int64_t)c * n] = (lane <= c) ? s0 : 0.0;
    if (lane + 32 < n) T[lane + 32 + (int64_t)c * n] = (lane + 32 <= c) ? s1 : 0.0;
}

// The same column-oriented back substitution for 64 < n <= 128: lane owns
// rows lane + 32 q (q < 4) of column c of T; R's leading c + 1 columns are
// staged in dynamic shared memory (column k at k * 128), (c + 1) * 1 KB.
__global__ void __launch_bounds__(32) k_tri_inverse128(const double *__restrict__ R, int n, int64_t ldr,
                                                        double *__restrict__ T, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ double rs128[];  // R[i][k] at k * 128 + i
    const int c = blockIdx.x, lane = threadIdx.x;
    for (int k = 0; k <= c; ++k)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            rs128[k * 128 + i] = (i <= k) ? R[i + (int64_t)k * ldr] : 0.0;
        }
    double d[4], sv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        d[q] = (i < n) ? 1.0 / R[i + (int64_t)i * ldr] : 0.0;
        sv[q] = (i == c) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int k = c; k >= 0; --k) {
        const int qk = k >> 5;
        // right only in the owner lane (k & 31) of row k
        const double own = (qk == 0) ? sv[0] * d[0] : (qk == 1) ? sv[1] * d[1] : (qk == 2) ? sv[2] * d[2] : sv[3] * d[3];
        const double tk = __shfl_sync(0xFFFFFFFFu, own, k & 31);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = lane + 32 * q;
            if (i == k) sv[q] = tk;
            if (i < k) sv[q] = fma(-rs128[k * 128 + i], tk, sv[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        if (i < n) T[i + (int64_t)c * n] = (i <= c) ? sv[q] : 0.0;
    }
}

// One exact window of the split sketch folded into this thread's FP64
// accumulators (tensor-memory lane 32 q4 + lane, columns col0 .. + 15):
// weights 2^-8d combined in FP32 pairs, added in FP64 without the column
// scale.
__device__ __forceinline__ void sketch_drain(uint32_t tmem, int q4, int col0, double acc[16])
{
#pragma unroll
    for (int c8 = 0; c8 < 2; ++c8) {
        uint32_t g[kSpDigits][8];
#pragma unroll
        for (int d = 0; d < kSpDigits; ++d)
            tmem_ld8_issue(tmem + ((uint32_t)(32 * q4) << 16) + d * kSpN + col0 + 8 * c8, g[d]);
        tmem_wait_ld();
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float hi = __uint_as_float(g[0][t]), lo = 0.0f;
#pragma unroll
            for (int d = 1; d < kSpDigits; ++d) {
                const float w8 = __uint_as_float((uint32_t)(127 - 8 * d) << 23);
                const float x = __fmul_rn(__uint_as_float(g[d][t]), w8);
                const float sum = __fadd_rn(hi, x);
                const float bb = __fsub_rn(sum, hi);
                const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(sum, bb)), __fsub_rn(x, bb));
                hi = sum;
                lo = __fadd_rn(lo, err);
            }
            acc[8 * c8 + t] += pair2d_pow2(hi, lo, 1023);
        }
    }
}

// ---------------------------------------------------------------------------
// Split sketch Y' = Omega' A (see the file header; Omega's columns follow the
// global row index row0 + i, so a row shard's sketch is its share of the
// whole one).  grid.y = (s-tile,
// n-tile) output tiles of 128 x 64; grid.x = row chunks (CTA cta0 + blockIdx.x
// of the whole sketch: a caller may launch the chunks of a matrix that is
// still arriving one group at a time, with the same result).  Column j of A is
// cut into seven digits relative to 2^(e_j + 1), e_j its largest exponent over
// the CTA's rows (found in a first pass over them), so the scale of every
// product in the CTA is fixed.  Operand tiles of 64 rows alternate between two
// buffers: the Omega' pieces and A digits of one are written while the tensor
// core reads the other.  Sixteen warps (at most 128 registers a thread) in two
// roles that run side by side: warps 0-7 generate and quantise Omega' (the
// generator's long dependent chains), warps 8-15 cut A into digits and issue
// the MMAs; all sixteen drain the window sums.  Every 512 rows the seven
// tensor-memory groups (each an exact integer below 2^24: at most two pairs of
// products below 2^14 per row) are combined in FP32 pairs and added in FP64;
// the fixed scale 2^(e_j - 1033) is applied once at the end.
// ---------------------------------------------------------------------------
constexpr int kSpBuf = kSpDigits * kSpB + kSpZ * kSpA;  // 88 KB per buffer
constexpr size_t kSpSmem2 = 2 * (size_t)kSpBuf;

__global__ void __launch_bounds__(512, 1)
    k_sketch_split(const double *__restrict__ A, int64_t lda, int64_t m, int n, int s, uint64_t seed, int64_t cta0,
                   int64_t subs_total, int64_t subs_per_cta, double *__restrict__ Ypart, RxrStatus *st, int64_t row0)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int cex[kSpN];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_tiles = (n + kSpN - 1) / kSpN;
    const int si = blockIdx.y / n_tiles, ni = blockIdx.y % n_tiles;
    const int s0 = si * kSpM, c0 = ni * kSpN;
    const int sw = min(kSpM, s - s0), nw = min(kSpN, n - c0);

    const int64_t cta = cta0 + blockIdx.x;
    const int64_t b_begin = cta * subs_per_cta;
    const int64_t b_end = min(subs_total, b_begin + subs_per_cta);
    for (int e = tid; e < (int)(kSpSmem2 / 16); e += blockDim.x) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0, 0, 0, 0);
    // largest exponent of each column over this CTA's rows: warp w scans
    // columns w, w + 16, ... (four at a time, coalesced down the rows)
    {
        const int64_t ra = b_begin * kSpSub, rb = min(m, b_end * kSpSub);
        for (int cl = warp; cl < kSpN; cl += 16) {
            unsigned ex = 0;
            if (cl < nw) {
                const double *col = A + (int64_t)(c0 + cl) * lda;
                int64_t r = ra + lane;
                for (; r + 96 < rb; r += 128) {
                    const double a0 = col[r], a1 = col[r + 32], a2 = col[r + 64], a3 = col[r + 96];
                    ex = max(ex, max(max(((unsigned)__double2hiint(a0) >> 20) & 0x7FFu, ((unsigned)__double2hiint(a1) >> 20) & 0x7FFu),
                                     max(((unsigned)__double2hiint(a2) >> 20) & 0x7FFu, ((unsigned)__double2hiint(a3) >> 20) & 0x7FFu)));
                }
                for (; r < rb; r += 32) ex = max(ex, ((unsigned)__double2hiint(col[r]) >> 20) & 0x7FFu);
            }
            ex = __reduce_max_sync(0xFFFFFFFFu, ex);
            if (lane == 0) {
                cex[cl] = (int)ex;
                if (ex == 0x7FFu) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);
            }
        }
    }
    if (tid == 0) {
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_f16(kSpM, kSpN);
    const uint64_t desc0 = smem_desc(smem_u32(smem), 128, 1024);

    // roles: warps 0-7 Omega' -> sketch rows 4 kq .. + 3, data rows 8 warp .. + 7;
    // warps 8-15 A digits -> column j, rows 16 rq .. + 15 of each 64-row tile
    // (the eight lanes of a quarter-warp take eight consecutive columns: their
    // 16-byte digit stores fall in distinct banks)
    const bool gauss = warp < 8;
    const int j = gauss ? 0 : 8 * (warp - 8) + (lane & 7), rq = lane >> 3;
    const int kq = lane;
    const bool has_col = !gauss && j < nw;
    const int ej = cex[j];
    const double *acol = A + (int64_t)(c0 + j) * lda;
    // epilogue: tensor-memory lane quarter (sketch rows), 16-column quarter
    const int q4 = warp & 3, cq = warp >> 2;
    double acc[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t] = 0.0;

    // Waits are per thread and bounded; one that gives up records a timeout
    // and the loop runs to its end without publishing the sums.
    bool ok = true;
    int it = 0;
    constexpr int kWinSubs = kSpWin / kSpSub;
    for (int64_t b = b_begin; b < b_end; ++b, ++it) {
        const int buf = it & 1;
        unsigned char *bop = smem + buf * kSpBuf;  // A digits: kSpDigits planes, N x K
        unsigned char *aop = bop + kSpDigits * kSpB;  // Omega' pieces: kSpZ planes, M x K
        const int64_t r0 = b * kSpSub;
        // A's rows for the digit warps (their phase is shorter than the
        // generator's, so the load latency stays off the critical path)
        double v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int64_t r = r0 + 16 * rq + i;
            v[i] = (has_col && r < m) ? acol[r] : 0.0;
        }
        if (it >= 2) ok &= mbar_wait_bounded(&mma_bar[buf], ((it - 2) >> 1) & 1, st);
        // Omega' on the 2^-12 grid: 4096 z' = 256 zeta0 + zeta1 (round to nearest
        // even by the 1.5 * 2^23 addition, as rint), both pieces exact in FP16
        if (gauss && 4 * kq < sw) {
            float z[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                rxr_normal4(seed, (uint64_t)(row0 + r0 + 8 * warp + i), (uint32_t)(s0 / 4 + kq), 0u, z[i]);
#pragma unroll
            for (int t4 = 0; t4 < 4; ++t4) {
                uint32_t p0[8], p1[8];  // zeta + 128, in [0, 256]
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int q = (int)(__float_as_uint(__fadd_rn(__fmul_rn(z[i][t4], 4096.0f), 12582912.0f)) & 0x7FFFFFu) -
                                  0x400000;
                    const int z0 = (q + 128) >> 8;
                    const int z1 = q - (z0 << 8);
                    p0[i] = (uint32_t)(z0 + 128);
                    p1[i] = (uint32_t)(z1 + 128);
                }
                const int r = 4 * kq + t4;
                if (r < sw) {
                    *reinterpret_cast<uint4 *>(aop + kmaj_off(r, 8 * warp)) = pack_int8x_f16(p0);
                    *reinterpret_cast<uint4 *>(aop + kSpA + kmaj_off(r, 8 * warp)) = pack_int8x_f16(p1);
                }
            }
        }
        // digits of A: element (row k, column j) -> B tile (j, k)
        if (has_col) {
#pragma unroll
            for (int g8 = 0; g8 < 2; ++g8) {
                unsigned long long U[8];
#pragma unroll
                for (int r = 0; r < 8; ++r)
                    U[r] = digits_offset((unsigned long long)__double_as_longlong(v[8 * g8 + r]), ej);
#pragma unroll
                for (int q = 0; q < kSpDigits; ++q) {
                    const uint4 w = pack_plane_f16(U, q);
                    *reinterpret_cast<uint4 *>(bop + q * kSpB + kmaj_off(j, 16 * rq + 8 * g8)) = w;
                }
            }
        }
        const bool first_of_window = (it % kWinSubs) == 0;
        if (first_of_window && it > 0) {
            ok &= mbar_wait_bounded(&mma_bar[buf ^ 1], ((it - 1) >> 1) & 1, st);
            tc_fence_after();
            sketch_drain(tmem, q4, 16 * cq, acc);
        }
        fence_proxy_async_shared();
        tc_fence_before();
        __syncthreads();
        if (tid == 256) {
            tc_fence_after();
            const uint64_t db = desc0 + (uint64_t)((buf * kSpBuf) >> 4);
            const uint64_t da = db + (uint64_t)((kSpDigits * kSpB) >> 4);
#pragma unroll
            for (int kk = 0; kk < kSpSub / 16; ++kk)
#pragma unroll
                for (int p = 0; p < kSpZ; ++p)
#pragma unroll
                    for (int q = 0; q + p < kSpDigits; ++q) {
                        const uint32_t acc_on = (!first_of_window || kk > 0 || p > 0) ? 1u : 0u;
                        tc_mma(tmem + (uint32_t)((p + q) * kSpN), da + (uint64_t)((p * kSpA + kk * 256) >> 4),
                               db + (uint64_t)((q * kSpB + kk * 256) >> 4), idesc, acc_on);
                    }
            tc_commit(&mma_bar[buf]);
        }
    }
    if (it > 0) {
        ok &= mbar_wait_bounded(&mma_bar[(it - 1) & 1], ((it - 1) >> 1) & 1, st);
        tc_fence_after();
        sketch_drain(tmem, q4, 16 * cq, acc);
    }
    ok = __syncthreads_and(ok) != 0;
    if (ok) {
        double *out = Ypart + cta * s * n;
        const int my_row = 32 * q4 + lane;
        const int r = s0 + my_row;
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int cl = 16 * cq + t;
            if (my_row < sw && cl < nw) {
                const int ce = cex[cl];
                out[r + (int64_t)(c0 + cl) * s] = (ce > 0) ? ldexp(acc[t], ce - 1033) : 0.0;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}


__global__ void k_reduce_parts(const double *, int, int64_t, int, int, double, int, double *, int64_t, RxrStatus *);

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static inline int64_t cdiv64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Extra workspace of the split path: the per-CTA partial sums of the split
// Gram and of the FP64-grade tensor-core Gram (the split sketch reuses the FP64
// sketch's partial buffer, which is larger).
static int64_t ozaki_chunks(int64_t m, int64_t n, int sms)
{
    return balanced_chunks(ozaki_blocks((int)n), sms, cdiv64(m, kOzWin));
}

// Row chunks of k_gram_oz128, one CTA per SM: g1 chunks for the J = 1 CTAs and
// g0 for the J = 0 ones.  kG8HalfCost is a J = 0 CTA's time per buffer relative
// to a J = 1 CTA's, which sets their share of the rows; 1 (equal chunks) measured
// fastest: the J = 0 CTAs cut half the columns, but the MMAs and drains are the
// same, and equal chunks let the two blocks' CTAs share their rows of X in L2.
constexpr double kG8HalfCost = 1.0;
struct Oz128Grid {
    int g1, g0;
    int64_t bpc1, bpc0;
};
static Oz128Grid oz128_grid(int64_t m, int sms)
{
    const int64_t total = cdiv64(m, kG8Rows);
    int64_t g1 = std::max<int64_t>(1, (int64_t)(sms / (1.0 + kG8HalfCost) + 0.5));
    int64_t g0 = std::max<int64_t>(1, sms - g1);
    g1 = std::min(g1, total);
    g0 = std::min(g0, total);
    Oz128Grid g;
    g.bpc1 = cdiv64(total, g1);
    g.g1 = (int)cdiv64(total, g.bpc1);
    g.bpc0 = cdiv64(total, std::min<int64_t>(g0, g.g1));  // every J = 0 slot has a J = 1 CTA
    g.g0 = (int)cdiv64(total, g.bpc0);
    return g;
}
static int64_t oz128_chunks(int64_t m, int sms)
{
    return oz128_grid(m, sms).g1;
}

static size_t split_partial_bytes(int64_t m, int64_t n, int sms)
{
    int64_t gx = std::max<int64_t>(std::min<int64_t>(sms, cdiv64(m, kGsWin)), ozaki_chunks(m, n, sms));
    if (n > 64 && n <= 128) gx = std::max<int64_t>(gx, oz128_chunks(m, sms));
    return ((size_t)gx * n * n * sizeof(double) + 255) & ~(size_t)255;
}

// records of R for the 64 < n <= 128 fused substitution
static size_t split_rec_bytes(int64_t n)
{
    return (n > kFuMaxN && n <= kF2MaxN) ? ((size_t)f2_rec_off((int)n, fu_blocks((int)n)) + 255) & ~(size_t)255 : 0;
}

// partial sums, a column-exponent array (int[512]: the split sketch's columns
// of A, later the n <= 64 Gram's columns of X), then the records of R
size_t split_workspace_bytes(int64_t m, int64_t n, int64_t, int sms)
{
    return split_partial_bytes(m, n, sms) + RXR_MAX_N * sizeof(int) + split_rec_bytes(n) + 256 + 128 * 128 * 4;
}

// E = R^{-1} - I of the last pass in FP32 (64 x 64), after the selection flags
static float *split_delta(const Plan &p)
{
    return reinterpret_cast<float *>(reinterpret_cast<char *>(split_select_flag(p)) + 256);
}

int *split_select_flag(const Plan &p)
{
    return reinterpret_cast<int *>(p.split + split_partial_bytes(p.m, p.n, p.sms) + RXR_MAX_N * sizeof(int) +
                                   split_rec_bytes(p.n));
}

int *split_colexp(const Plan &p)
{
    return reinterpret_cast<int *>(p.split + split_partial_bytes(p.m, p.n, p.sms));
}

static unsigned char *split_records(const Plan &p)
{
    return reinterpret_cast<unsigned char *>(p.split + split_partial_bytes(p.m, p.n, p.sms) + RXR_MAX_N * sizeof(int));
}

// X <- X R^{-1} on the tensor cores through the explicit inverse (n <= 64);
// T is held in the XR scratch (s x n >= n x n).
// ---------------------------------------------------------------------------
// The last pass's Q = X R_P^{-1} when R_P is within rounding of I: with
// T = R_P^{-1} = I + E, Q = X + X E, and X E is a tiny correction (|E| <= 2^-38
// checked on the device), so single precision is plenty for it: its error is
// below n 2^-24 |E| |X| <= 2^-56 |X| for n <= 64.  k_delta_select forms E in FP32
// and the flag; k_apply_delta computes the correction as an FP32 product over
// 128-row tiles and adds it to X in FP64 (one addition per entry).
// ---------------------------------------------------------------------------
constexpr double kDeltaMax = 0x1p-38;

// E = T - I (n <= ld, ld = 64 or 128) as FP32, row-major and zero padded to
// ld x ld (Ef[k * ld + j] = E(k, j)), and the selection flag: 1 when every
// |E(k, j)| <= 2^-38 and T is finite, else 0.
__global__ void __launch_bounds__(256) k_delta_select(const double *__restrict__ T, int n, int ld,
                                                      float *__restrict__ Ef, int *sel, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double red[8];
    const int tid = threadIdx.x;
    double mx = 0.0;
    bool bad = false;
    for (int e = tid; e < ld * ld; e += blockDim.x) {
        const int k = e / ld, j = e % ld;
        double d = 0.0;
        if (k < n && j < n) {
            d = T[k + (int64_t)j * n] - (k == j ? 1.0 : 0.0);
            bad |= rxr_nonfinite(d);
            mx = fmax(mx, fabs(d));
        }
        Ef[e] = (float)d;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    bad = __syncthreads_or(bad);
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v = fmax(v, red[w]);
        *sel = (!bad && v <= kDeltaMax) ? 1 : 0;
    }
}

// X <- X + X E over 128-row tiles (three CTAs per SM, grid-stride, so that
// their loads, FP32 products and FP64 additions overlap).  Warp w
// owns columns 8w .. 8w + 7, lane l rows l, l + 32, l + 64, l + 96 of a tile
// (coalesced for any leading dimension).  The FP64 pipe (two operations per
// clock per SM) does only the final addition: X enters FP32 scaled by its
// row's largest power of two (x 2^(1023 - e_r), e_r the row's largest biased
// exponent) by integer operations on its bits (mantissa truncated: relative
// error 2^-23; entries below 2^-126 of the row's largest flush to zero), and
// the FP32 correction leaves scaled back by f2d_pow2.  The tile's scaled X is
// shared in FP32 (xf[k * 128 + r], conflict-free for the column stores and the
// row reads; a register pair (x, x) makes it the packed FP32 FMA's row
// operand) and E's row k as two broadcast 16-byte loads (its column pairs).
// The FP64 entries are read again for the addition (an L2 hit: the tile was
// read moments before), which keeps a thread within 80 registers.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// x 2^(1023 - er) in FP32 with the mantissa truncated; zero when x is zero,
// subnormal or below 2^-126 of 2^(er - 1023)
__device__ __forceinline__ float d2f_pow2(double x, int er)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const int ed = (int)((hi >> 20) & 0x7FFu);
    const int ef = ed - er + 127;
    const uint32_t mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
    return (ed == 0 || ef <= 0) ? 0.0f : __uint_as_float((hi & 0x80000000u) | ((uint32_t)min(ef, 254) << 23) | mant);
}

// NW warps per CTA own 8 columns each: n <= 8 NW (64 with 8 warps, three CTAs
// per SM; 128 with 16 warps, one CTA per SM); E's rows are 8 NW floats apart.
__host__ __device__ constexpr size_t delta_smem_bytes(int n, int nw)
{
    return (size_t)n * 8 * nw * 4 + (size_t)n * 128 * 4;
}

template <int NW>
__global__ void __launch_bounds__(32 * NW, NW == 8 ? 3 : 1)
    k_apply_delta(double *X, int64_t ldx, int64_t m, int n, const float *__restrict__ Ef, int64_t tiles_total,
                  const int *__restrict__ sel, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    if (*sel != 1) return;  // the FP64-grade product was chosen instead
    constexpr int ES = 8 * NW;
    extern __shared__ __align__(16) float dsm_delta[];
    float *es = dsm_delta;  // n x ES
    float *xf = es + n * ES;  // n x 128
    __shared__ int rowe[2][128];  // the rows' largest biased exponents (double buffered)
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int e = tid; e < n * ES; e += blockDim.x) es[e] = Ef[e];
    for (int e = tid; e < 256; e += blockDim.x) rowe[e >> 7][e & 127] = 0;
    __syncthreads();
    const int j0 = 8 * w;
    const int nb = max(0, min(8, n - j0));
    for (int64_t tile = blockIdx.x, buf = 0; tile < tiles_total; tile += gridDim.x, buf ^= 1) {
        const int64_t r0 = tile * 128;
        double x[4][8];
#pragma unroll
        for (int b = 0; b < 8; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t gr = r0 + lane + 32 * a;
                x[a][b] = (b < nb && gr < m) ? X[gr + (int64_t)(j0 + b) * ldx] : 0.0;
            }
        if (nb > 0) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                int e = 0;
#pragma unroll
                for (int b = 0; b < 8; ++b) e = max(e, (int)(((uint32_t)__double2hiint(x[a][b]) >> 20) & 0x7FFu));
                atomicMax(&rowe[buf][lane + 32 * a], e);
            }
        }
        __syncthreads();  // the row exponents are complete; the previous tile's reads of xf are done
        if (nb > 0) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int er = rowe[buf][lane + 32 * a];
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    if (b < nb) {
                        xf[(j0 + b) * 128 + lane + 32 * a] = d2f_pow2(x[a][b], er);
                    }
            }
        }
        if (tid < 128) rowe[buf ^ 1][tid] = 0;  // read last in the previous tile, before the barrier above
        __syncthreads();
        if (nb == 0) continue;
        unsigned long long acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][c] = 0ull;
#pragma unroll 4
        for (int k = 0; k < n; ++k) {
            const ulonglong2 e01 = *reinterpret_cast<const ulonglong2 *>(es + k * ES + j0);
            const ulonglong2 e23 = *reinterpret_cast<const ulonglong2 *>(es + k * ES + j0 + 4);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const uint32_t xv = __float_as_uint(xf[k * 128 + lane + 32 * a]);
                const unsigned long long xa = ((unsigned long long)xv << 32) | xv;
                acc[a][0] = ffma2(xa, e01.x, acc[a][0]);
                acc[a][1] = ffma2(xa, e01.y, acc[a][1]);
                acc[a][2] = ffma2(xa, e23.x, acc[a][2]);
                acc[a][3] = ffma2(xa, e23.y, acc[a][3]);
            }
        }
        if constexpr (NW == 8) {
            // X again (from L2), value by value (within 80 registers)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t gr = r0 + lane + 32 * a;
                const int er = rowe[buf][lane + 32 * a];
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    if (b < nb && gr < m) {
                        double *xp = X + gr + (int64_t)(j0 + b) * ldx;
                        const uint32_t cb = (uint32_t)(acc[a][b >> 1] >> (32 * (b & 1)));
                        __stcs(xp, __ldcs(xp) + f2d_pow2(__uint_as_float(cb), er));
                    }
            }
        } else {
            // X again (from L2), in groups of two rows whose 16 loads are all in
            // flight before the group's first store (a store between them would
            // order each load after it)
#pragma unroll
            for (int a0 = 0; a0 < 4; a0 += 2) {
                double xo[2][8];
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 8; ++b) {
                        const int64_t gr = r0 + lane + 32 * (a0 + a);
                        xo[a][b] = (b < nb && gr < m) ? __ldcs(X + gr + (int64_t)(j0 + b) * ldx) : 0.0;
                    }
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int64_t gr = r0 + lane + 32 * (a0 + a);
                    const int er = rowe[buf][lane + 32 * (a0 + a)];
#pragma unroll
                    for (int b = 0; b < 8; ++b)
                        if (b < nb && gr < m) {
                            const uint32_t cb = (uint32_t)(acc[a0 + a][b >> 1] >> (32 * (b & 1)));
                            __stcs(X + gr + (int64_t)(j0 + b) * ldx, xo[a][b] + f2d_pow2(__uint_as_float(cb), er));
                        }
                }
            }
        }
    }
}

static void delta_launch(int sms, double *X, int64_t ldx, int64_t m, int n, const float *Ef, int64_t tiles,
                         const int *sel, RxrStatus *status, cudaStream_t st)
{
    if (n <= 64)
        k_apply_delta<8><<<(unsigned)std::min<int64_t>(3 * (int64_t)sms, tiles), 256, delta_smem_bytes(n, 8), st>>>(
            X, ldx, m, n, Ef, tiles, sel, status);
    else
        k_apply_delta<16><<<(unsigned)std::min<int64_t>(sms, tiles), 512, delta_smem_bytes(n, 16), st>>>(
            X, ldx, m, n, Ef, tiles, sel, status);
}

// Estimate of cond_2(R) = ||R||_2 ||R^{-1}||_2 (n <= 128, one CTA): twelve power
// iterations on R^T R and on T^T T (T = R^{-1}) from the all-ones vector, in a
// fixed order (deterministic).  *sel = 1 when the estimate is at most kExplicitCond,
// else 0: the middle CholeskyQR pass then multiplies by T on the tensor cores
// instead of substituting.
constexpr double kExplicitCond = 16.0;

// NM = 64 or 128 (n <= NM), 4 NM threads (four a row), the matrix in
// NM (NM + 1) doubles of dynamic shared memory.
template <int NM>
__global__ void __launch_bounds__(4 * NM) k_cond_select(const double *__restrict__ R, const double *__restrict__ T,
                                                        int n, int *sel, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    constexpr int LD = NM + 1, NW = NM / 8;  // padded stride; warps
    extern __shared__ double Ms[];  // the matrix, column-major with a padded stride (zero below the diagonal)
    __shared__ double v[NM], w[NM], red[NW];
    const int tid = threadIdx.x, row = tid >> 2, q = tid & 3, lane = tid & 31, warp = tid >> 5;
    double est[2];
    for (int which = 0; which < 2; ++which) {
        const double *M = which == 0 ? R : T;  // upper triangular, ld n
        for (int e = tid; e < NM * NM; e += blockDim.x) {
            const int i = e % NM, k = e / NM;
            Ms[i + k * LD] = (i <= k && k < n) ? M[i + (int64_t)k * n] : 0.0;
        }
        if (q == 0) v[row] = (row < n) ? 1.0 : 0.0;
        __syncthreads();
        double nrm = 0.0;
        for (int itn = 0; itn < 12; ++itn) {
            // w = M v: four threads per row, terms k = q, q + 4, ...
            double a = 0.0;
#pragma unroll
            for (int k = q; k < NM; k += 4) a = fma(Ms[row + k * LD], v[k], a);
            a += __shfl_xor_sync(0xFFFFFFFFu, a, 1);
            a += __shfl_xor_sync(0xFFFFFFFFu, a, 2);
            if (q == 0) w[row] = a;
            __syncthreads();
            // v = M^T w
            double b = 0.0;
#pragma unroll
            for (int k = q; k < NM; k += 4) b = fma(Ms[k + row * LD], w[k], b);
            b += __shfl_xor_sync(0xFFFFFFFFu, b, 1);
            b += __shfl_xor_sync(0xFFFFFFFFu, b, 2);
            double t = (q == 0) ? b * b : 0.0;
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
            if (lane == 0) red[warp] = t;
            __syncthreads();
            double ss = 0.0;
#pragma unroll
            for (int k = 0; k < NW; ++k) ss += red[k];  // every thread, same order
            nrm = sqrt(sqrt(ss));  // ||M^T M v||^(1/2) with ||v|| = 1 before: an estimate of ||M||_2
            const double inv = (ss > 0.0) ? 1.0 / sqrt(ss) : 0.0;
            if (q == 0) v[row] = b * inv;
            __syncthreads();
        }
        est[which] = nrm;
    }
    if (tid == 0) {
        const double c = est[0] * est[1];
        *sel = (c > 0.0 && c <= kExplicitCond && !rxr_nonfinite(c)) ? 1 : 0;
    }
}

// The middle CholeskyQR pass for n <= 64: X <- X R^{-1} by the tensor-core
// product with T = R^{-1} when R is well conditioned (estimate <= 16), else by
// the fused substitution; both kernels are launched and the one not selected
// returns at once (no host synchronisation).  X's column exponents go to
// colexp_out for the Gram that follows.
// 64 < n <= 128: X <- X T with T = R^{-1} in 64-column blocks, when the
// estimate of cond_2(R) is at most 16 (else the fused substitution):
//   X_b <- X_b T_11,  X_b <- X_b + X_a T_01,  X_a <- X_a T_00,
// X_a = columns 0..63, X_b = 64..n-1; each step an FP64-grade tensor-core
// product (the second one adds into X_b), in this order so that each reads
// columns not yet overwritten.  colexp_out (nullable, zeroed by the caller):
// the columns' largest exponents of the result, from whichever form runs.
static int middle_pass128_enqueue(Plan &p, double *X, int64_t ldx, const double *R, int *colexp_out, int *sel,
                                  cudaStream_t st)
{
    const int n = (int)p.n, nb = n - 64;
    double *T = p.W;
    k_tri_inverse128<<<(unsigned)n, 32, (size_t)n * 128 * sizeof(double), st>>>(R, n, p.n, T, p.status);
    k_cond_select<128><<<1, 512, 128 * 129 * sizeof(double), st>>>(R, T, n, sel, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    const int64_t tiles = cdiv64(p.m, kAqM);
    const int gx = (int)std::min<int64_t>(p.sms, tiles);
    double *Xb = X + 64 * ldx;
    CUtensorMap mb, ma;
    const int tma_b = encode_tile_map(&mb, Xb, p.m, nb, ldx, kAqM, nb) ? 1 : 0;
    const int tma_a = encode_tile_map(&ma, X, p.m, 64, ldx, kAqM, 64) ? 1 : 0;
    k_apply_oz64<false><<<gx, 256, aq_smem_bytes(nb), st>>>(mb, tma_b, Xb, ldx, p.m, nb, T + 64 + 64 * p.n, p.n, tiles, sel,
                                                     1, nullptr, nb, 0, nullptr, 0, p.status);
    // X_b += X_a T_01 (the full 64 x nb block)
    k_apply_oz64<true><<<gx, 256, aq_smem_bytes(64), st>>>(ma, tma_a, X, ldx, p.m, 64, T + 64 * p.n, p.n, tiles, sel, 1,
                                                     colexp_out ? colexp_out + 64 : nullptr, nb, 1, Xb, ldx,
                                                     p.status);
    k_apply_oz64<false><<<gx, 256, aq_smem_bytes(64), st>>>(ma, tma_a, X, ldx, p.m, 64, T, p.n, tiles, sel, 1, colexp_out,
                                                     64, 0, nullptr, 0, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    return fused128_subst_enqueue(p, X, ldx, R, p.n, X, ldx, st, sel, colexp_out);
}

int middle_pass_enqueue(Plan &p, double *X, int64_t ldx, const double *R, int *colexp_out, int *sel,
                        cudaStream_t st)
{
    if (p.n > 128) return RXR_ERR_UNSUPPORTED;
    double *T = p.W;
    if (p.n > 64) return middle_pass128_enqueue(p, X, ldx, R, colexp_out, sel, st);
    k_tri_inverse64<<<(unsigned)p.n, 32, 0, st>>>(R, (int)p.n, p.n, T, p.status);
    k_cond_select<64><<<1, 256, 64 * 65 * sizeof(double), st>>>(R, T, (int)p.n, sel, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    const int n = (int)p.n;
    CUtensorMap mx;
    const int use_tma = encode_tile_map(&mx, X, p.m, n, ldx, kAqM, n) ? 1 : 0;
    const int64_t tiles = cdiv64(p.m, kAqM);
    const int gx = (int)std::min<int64_t>(p.sms, tiles);
    k_apply_oz64<false><<<gx, 256, aq_smem_bytes(n), st>>>(mx, use_tma, X, ldx, p.m, n, T, p.n, tiles, sel, 1, colexp_out,
                                                    n, 0, nullptr, 0, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    return fused_subst_enqueue(p, X, ldx, R, p.n, X, ldx, colexp_out, st, sel);
}

// X <- X R^{-1} for the last pass (n <= 64): T = R^{-1}; when |T - I| <= 2^-38
// (R within rounding of I) the FP32 correction Q = X + X (T - I), else the
// FP64-grade tensor-core product; both launched, the one not selected returns
// at once.  T lives in the XR scratch W (s x n doubles >= n^2).
int ozaki_apply_prepare(Plan &p, const double *R, cudaStream_t st)
{
    if (p.n > 128) return RXR_ERR_UNSUPPORTED;
    if (p.n <= 64) {
        k_tri_inverse64<<<(unsigned)p.n, 32, 0, st>>>(R, (int)p.n, p.n, p.W, p.status);
        k_delta_select<<<1, 256, 0, st>>>(p.W, (int)p.n, 64, split_delta(p), split_select_flag(p) + 1, p.status);
    } else {
        k_tri_inverse128<<<(unsigned)p.n, 32, (size_t)p.n * 128 * sizeof(double), st>>>(R, (int)p.n, p.n, p.W,
                                                                                       p.status);
        k_delta_select<<<1, 256, 0, st>>>(p.W, (int)p.n, 128, split_delta(p), split_select_flag(p) + 1, p.status);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

// 64 < n <= 128: X <- X R^{-1} by the FP32 correction when R^{-1} - I is
// within 2^-38 (the last pass after a repeated one), else by the fused
// substitution; both launched after the selection, the one not chosen returns
// at once.
int delta128_apply_enqueue(Plan &p, double *X, int64_t ldx, const double *R, cudaStream_t st)
{
    if (p.n <= 64 || p.n > 128) return RXR_ERR_UNSUPPORTED;
    if (int e = ozaki_apply_prepare(p, R, st)) return e;
    const int *sel = split_select_flag(p) + 1;
    delta_launch(p.sms, X, ldx, p.m, (int)p.n, split_delta(p), cdiv64(p.m, 128), sel, p.status, st);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    return fused128_subst_enqueue(p, X, ldx, R, p.n, X, ldx, st, sel);
}

// Rows [r0, r0 + rows) of X (r0 a multiple of 128): both product forms, the
// one not selected returns at once.
int ozaki_apply_rows(Plan &p, double *X, int64_t ldx, int64_t r0, int64_t rows, cudaStream_t st)
{
    if (rows <= 0) return 0;
    const int n = (int)p.n;
    double *Xr = X + r0;
    const int *sel = split_select_flag(p) + 1;
    const int64_t tiles = cdiv64(rows, kAqM);
    CUtensorMap mx;
    const int use_tma = encode_tile_map(&mx, Xr, rows, n, ldx, kAqM, n) ? 1 : 0;
    delta_launch(p.sms, Xr, ldx, rows, n, split_delta(p), tiles, sel, p.status, st);
    const int gx = (int)std::min<int64_t>(p.sms, tiles);
    k_apply_oz64<false><<<gx, 256, aq_smem_bytes(n), st>>>(mx, use_tma, Xr, ldx, rows, n, p.W, p.n, tiles, sel, 0, nullptr,
                                                    n, 0, nullptr, 0, p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

int ozaki_apply_enqueue(Plan &p, double *X, int64_t ldx, const double *R, cudaStream_t st)
{
    if (int e = ozaki_apply_prepare(p, R, st)) return e;
    return ozaki_apply_rows(p, X, ldx, 0, p.m, st);
}

// X = B R^{-1} by right-looking column blocks of width bw: FP64 substitution of
// each diagonal block, trailing updates on the tensor cores (FP64 grade).
int blocked_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                          int64_t ldx, cudaStream_t st)
{
    const int n = (int)p.n;
    const int bw = (n <= 64) ? 16 : (n <= 128 ? 32 : 64);
    const int64_t tiles = cdiv64(p.m, kApM);
    const int64_t stiles = cdiv64(p.m, kSbRows);
    for (int c0 = 0; c0 < n; c0 += bw) {
        const int b = std::min(bw, n - c0);
        const double *src = (c0 == 0) ? Bsrc : X;
        const int64_t lds = (c0 == 0) ? ldb : ldx;
        const size_t smem = ((size_t)b * kSbRows + b * (b + 1) / 2 + b) * sizeof(double);
        const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / smem));
        const int sblocks = (int)std::min<int64_t>(stiles, (int64_t)p.sms * per_sm);
        k_solve_block<<<sblocks, 256, smem, st>>>(src, lds, X, ldx, R, ldr, c0, b, p.m, stiles, p.status);
        if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
        const int tc0 = c0 + b, N = n - tc0;
        if (N <= 0) break;
        const int gy = (int)cdiv64(N, kApN);
        int64_t gx = balanced_chunks(gy, p.sms, tiles);
        const int64_t tpc = cdiv64(tiles, gx);
        gx = cdiv64(tiles, tpc);
        // the first trailing update reads B (= A) and writes X; later ones work in X
        k_update_ozaki<<<dim3((unsigned)gx, (unsigned)gy), 256, kApSmem, st>>>(
            X, ldx, c0, b, R, ldr, tc0, N, (c0 == 0) ? Bsrc : X, (c0 == 0) ? ldb : ldx, X, ldx, p.m, tiles, tpc,
            nullptr, p.status);
        if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    }
    return 0;
}

// X = B R^{-1} for n <= 64 in one pass over B (k_subst_fused); X may equal B.
int fused_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                        int64_t ldx, int *colexp_out, cudaStream_t st, const int *sel)
{
    if (p.n > kFuMaxN) return RXR_ERR_UNSUPPORTED;
    const int n = (int)p.n;
    CUtensorMap ms, md;
    const int use_tma =
        (encode_tile_map(&ms, Bsrc, p.m, n, ldb, kFuM, n) && encode_tile_map(&md, X, p.m, n, ldx, kFuM, n)) ? 1 : 0;
    const int64_t tiles = cdiv64(p.m, kFuM);
    const int gx = (int)std::min<int64_t>(p.sms, cdiv64(tiles, 2));  // two tile streams per CTA
    k_subst_fused<<<gx, 256, fu_smem_bytes(n), st>>>(ms, md, use_tma, Bsrc, ldb, X, ldx, p.m, n, R, ldr, tiles,
                                                      colexp_out, sel, p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

// X = B R^{-1} for 64 < n <= 128 in one pass over B (k_rprep128 + k_subst_fused128).
int fused128_subst_enqueue(Plan &p, const double *Bsrc, int64_t ldb, const double *R, int64_t ldr, double *X,
                           int64_t ldx, cudaStream_t st, const int *sel, int *colexp_out)
{
    if (p.n <= kFuMaxN || p.n > kF2MaxN) return RXR_ERR_UNSUPPORTED;
    const int n = (int)p.n, nb = fu_blocks(n);
    unsigned char *rec = split_records(p);
    k_rprep128<<<nb, 256, 0, st>>>(R, ldr, n, rec, sel, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    CUtensorMap ms, md;
    const int use_tma =
        (encode_tile_map(&ms, Bsrc, p.m, n, ldb, kFuM, n) && encode_tile_map(&md, X, p.m, n, ldx, kFuM, n)) ? 1 : 0;
    const int64_t tiles = cdiv64(p.m, kFuM);
    const int gx = (int)std::min<int64_t>(p.sms, tiles);
    k_subst_fused128<<<gx, 256, f2_smem_bytes(n), st>>>(ms, md, use_tma, Bsrc, ldb, X, ldx, p.m, n, rec, tiles,
                                                         sel, colexp_out, p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

int ozaki_gram_enqueue(Plan &p, const double *X, int64_t ldx, cudaStream_t st, bool colexp_ready)
{
    if (p.n > RXR_MAX_N) return RXR_ERR_UNSUPPORTED;
    if (p.n <= 64) {
        int *cx = split_colexp(p);
        if (!colexp_ready) {
            if (cudaMemsetAsync(cx, 0, 64 * sizeof(int), st) != cudaSuccess) return RXR_ERR_CUDA;
            const int bx = (int)std::min<int64_t>(64, cdiv64(p.m, 256));
            k_colexp<<<dim3((unsigned)bx, (unsigned)p.n), 256, 0, st>>>(X, ldx, p.m, cx, p.status);
            if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
        }
        const int64_t total = cdiv64(p.m, kG6Rows);
        int64_t gx = std::min<int64_t>(p.sms, total);
        const int64_t bpc = cdiv64(total, gx);
        gx = cdiv64(total, bpc);
        double *parts = reinterpret_cast<double *>(p.split);
        CUtensorMap mx;
        const int use_tma = encode_tile_map(&mx, X, p.m, p.n, ldx, 16, 64, true) ? 1 : 0;
        k_gram_oz64<<<(unsigned)gx, kG6Producers, kG6Smem, st>>>(mx, use_tma, X, ldx, p.m, (int)p.n, cx, total, bpc,
                                                                 parts, p.status);
        if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
        const int64_t nn = p.n * p.n;
        k_reduce_parts<<<(int)cdiv64(nn, 256), 256, 0, st>>>(parts, (int)gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G,
                                                             p.n, p.status);
        return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
    }
    if (p.n <= 128) {
        // 64 < n <= 128: the pipelined Gram over the columns' global exponents
        // (recorded by the substitution that produced X, or found here)
        int *cx = split_colexp(p);
        if (!colexp_ready) {
            if (cudaMemsetAsync(cx, 0, p.n * sizeof(int), st) != cudaSuccess) return RXR_ERR_CUDA;
            const int bx = (int)std::min<int64_t>(64, cdiv64(p.m, 256));
            k_colexp<<<dim3((unsigned)bx, (unsigned)p.n), 256, 0, st>>>(X, ldx, p.m, cx, p.status);
            if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
        }
        const int64_t total = cdiv64(p.m, kG8Rows);
        const Oz128Grid gg = oz128_grid(p.m, p.sms);
        const int64_t gx = gg.g1;  // partial-sum slots
        double *parts = reinterpret_cast<double *>(p.split);
        CUtensorMap mx, mh;
        const int use_tma = (encode_tile_map(&mx, X, p.m, p.n, ldx, 16, (int)p.n, true) &&
                             encode_tile_map(&mh, X, p.m, p.n, ldx, 16, 64, true))
                                ? 1
                                : 0;
        k_gram_oz128<<<(unsigned)(gg.g1 + gg.g0), kG8Threads, kG8Smem, st>>>(mx, mh, use_tma, X, ldx, p.m, (int)p.n, cx,
                                                                       total, gg.g1, gg.bpc1, gg.g0, gg.bpc0, parts,
                                                                       p.status);
        if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
        const int64_t nn = p.n * p.n;
        k_reduce_parts<<<(int)cdiv64(nn, 256), 256, 0, st>>>(parts, (int)gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G,
                                                             p.n, p.status);
        return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
    }
    const int64_t win_total = cdiv64(p.m, kOzWin);
    int64_t gx = ozaki_chunks(p.m, p.n, p.sms);
    const int64_t wpc = cdiv64(win_total, gx);
    gx = cdiv64(win_total, wpc);
    const int gy = ozaki_blocks((int)p.n);
    double *parts = reinterpret_cast<double *>(p.split);
    k_gram_ozaki<<<dim3((unsigned)gx, gy), 256, kOzSmem, st>>>(X, ldx, p.m, (int)p.n, win_total, wpc, parts, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    const int64_t nn = p.n * p.n;
    k_reduce_parts<<<(int)cdiv64(nn, 256), 256, 0, st>>>(parts, (int)gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G, p.n,
                                                         p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

cudaError_t set_split_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_sketch_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpSmem2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGsSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_update_ozaki, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kApSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_solve_block, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_subst_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fu_smem_bytes(kFuMaxN));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_oz64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kG6Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_oz128, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kG8Smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_subst_fused128, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)f2_smem_bytes(kF2MaxN));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_oz64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)aq_smem_bytes(64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_oz64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)aq_smem_bytes(64));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_delta<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)delta_smem_bytes(64, 8));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_apply_delta<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)delta_smem_bytes(128, 16));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tri_inverse128, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 128 * 128 * (int)sizeof(double));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cond_select<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 128 * 129 * (int)sizeof(double));
    return e;
}

// Row partition of the split sketch: gx CTAs of spc 64-row sub-tiles each.
// Where every CTA still gets a 512-row window, kSketchChunks times the
// balanced CTA count, so that each of kSketchChunks row chunks spreads over
// the whole GPU.
void split_sketch_grid(const Plan &p, int64_t *gx_out, int64_t *spc_out)
{
    const int64_t gy = cdiv64(p.s, kSpM) * cdiv64(p.n, kSpN);
    const int64_t subs_total = cdiv64(p.m, kSpSub);
    int64_t gx = balanced_chunks(gy, p.sms, cdiv64(p.m, kSpWin));
    if (subs_total >= (int64_t)kSketchChunks * gx * (kSpWin / kSpSub)) gx *= kSketchChunks;
    const int64_t spc = cdiv64(subs_total, gx);
    *gx_out = cdiv64(subs_total, spc);
    *spc_out = spc;
}

// CTAs [cta_begin, cta_end) of the split sketch (rows [cta_begin * spc * 64,
// cta_end * spc * 64) of A): their partial sums only.
int split_sketch_part_enqueue(Plan &p, const double *A, int64_t lda, uint64_t seed, int64_t cta_begin, int64_t cta_end,
                              cudaStream_t st)
{
    int64_t gx, spc;
    split_sketch_grid(p, &gx, &spc);
    if (gx > p.yslots) return RXR_ERR_NOMEM;  // partial buffer of the plan
    cta_end = std::min(cta_end, gx);
    if (cta_end <= cta_begin) return 0;
    const int64_t gy = cdiv64(p.s, kSpM) * cdiv64(p.n, kSpN);
    k_sketch_split<<<dim3((unsigned)(cta_end - cta_begin), (unsigned)gy), 512, kSpSmem2, st>>>(
        A, lda, p.m, (int)p.n, (int)p.s, seed, cta_begin, cdiv64(p.m, kSpSub), spc, p.Ypart, p.status, p.row0);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

// Y = Omega' A / sqrt(s) from the partial sums of all CTAs.
int split_sketch_reduce_enqueue(Plan &p, cudaStream_t st)
{
    int64_t gx, spc;
    split_sketch_grid(p, &gx, &spc);
    const int64_t sn = p.s * p.n;
    const int64_t threads = (gx >= kReduceWarpParts) ? 32 * sn : sn;
    k_reduce_parts<<<(int)cdiv64(threads, 256), 256, 0, st>>>(p.Ypart, (int)gx, sn, (int)p.s, (int)p.n,
                                                         1.0 / sqrt((double)p.s), 0, p.Y, p.s, p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

int split_sketch_enqueue(Plan &p, const double *A, int64_t lda, uint64_t seed, cudaStream_t st)
{
    int64_t gx, spc;
    split_sketch_grid(p, &gx, &spc);
    if (int e = split_sketch_part_enqueue(p, A, lda, seed, 0, gx, st)) return e;
    return split_sketch_reduce_enqueue(p, st);
}

int split_gram_enqueue(Plan &p, const double *X, int64_t ldx, cudaStream_t st)
{
    if (p.n > kGsM) return RXR_ERR_UNSUPPORTED;
    const int64_t win_total = cdiv64(p.m, kGsWin);
    int64_t gx = std::min<int64_t>(p.sms, win_total);
    const int64_t wpc = cdiv64(win_total, gx);
    gx = cdiv64(win_total, wpc);
    if ((size_t)gx * p.n * p.n * sizeof(double) > split_workspace_bytes(p.m, p.n, p.s, p.sms)) return RXR_ERR_NOMEM;
    double *parts = reinterpret_cast<double *>(p.split);
    k_gram_split<<<(unsigned)gx, 256, kGsSmem, st>>>(X, ldx, p.m, (int)p.n, win_total, wpc, parts, p.status);
    if (cudaGetLastError() != cudaSuccess) return RXR_ERR_CUDA;
    const int64_t nn = p.n * p.n;
    k_reduce_parts<<<(int)cdiv64(nn, 256), 256, 0, st>>>(parts, (int)gx, nn, (int)p.n, (int)p.n, 1.0, 1, p.G, p.n,
                                                         p.status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

}  // namespace rxr
