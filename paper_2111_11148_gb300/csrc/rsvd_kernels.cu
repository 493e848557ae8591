// rsvd_kernels.cu -- the kernels of the randomized SVD with power iteration
// (Algorithm 7, Section 5.1) around the library's CholeskyQR:
//   * k_rm_transpose: an m x k column-major block to row-major (row i's k
//                     values contiguous), so that a sparse product gathers
//                     whole rows with one coalesced load per nonzero;
//   * k_csr_spmm    : Y = A X for A in compressed sparse row form, a warp per
//                     row (lanes over the k columns), 32 rows per CTA written
//                     back column-major through shared memory; row pointers
//                     and column indices are range-checked;
//   * k_jacobi_svd  : R = U_r diag(S) V_r^T of the final k x k triangular
//                     factor by one-sided (Hestenes) Jacobi in one CTA, pairs
//                     of columns in round-robin order, one warp per pair;
//   * k_right_mult  : Y = X T for X (rows x k) and a k x k T held in shared
//                     memory (the finishing products U = Q V_r, V = Q_z U_r);
//   * k_status_keep : keeps the first failure over the sequence of
//                     factorisations.
#include <algorithm>

#include "rxr_internal.cuh"

namespace rxr {

namespace {

constexpr int kSpRows = 32;         // rows of one sparse-product CTA
constexpr int kSvdMaxK = 128;       // widest block of the randomized SVD
constexpr int kJacobiThreads = 512;
constexpr int kJacobiSweeps = 40;   // bound on the sweeps; convergence is quadratic
constexpr int kJacobiVSmemK = 112;  // V_r in shared memory next to W up to here (200 KB)
constexpr int kRmRows = 64;         // rows of one k_right_mult CTA

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

__global__ void k_rm_transpose(const double *__restrict__ X, int64_t ldx, int64_t rows, int k, double *__restrict__ Xr)
{
    __shared__ double t[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += 8) {
        const int64_t r = r0 + tx;
        const int c = c0 + j;
        if (r < rows && c < k) t[j][tx] = X[r + (int64_t)c * ldx];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int64_t r = r0 + j;
        const int c = c0 + tx;
        if (r < rows && c < k) Xr[r * k + c] = t[tx][j];
    }
}

// Y(rows x k, column-major, ldy) = A X with A given by (ptr, idx, val) and X
// row-major (cols x k).  Each row's products are summed in the order of its
// nonzeros.  A row pointer outside [0, nnz], a decreasing pair or a column
// index outside [0, cols) sets RXR_ERR_BAD_SPARSE and the entry is skipped.
__global__ void __launch_bounds__(256) k_csr_spmm(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                                                  const double *__restrict__ val, int64_t nnz, int64_t rows,
                                                  int64_t cols, const double *__restrict__ Xr, int k,
                                                  double *__restrict__ Y, int64_t ldy, RxrStatus *acc)
{
    __shared__ double tile[kSvdMaxK][kSpRows + 1];
    if (rxr_failed_block(acc)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kSpRows;
    bool bad = false;
    for (int rr = warp; rr < kSpRows; rr += 8) {
        const int64_t row = r0 + rr;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        if (row < rows) {
            const int64_t beg = ptr[row], end = ptr[row + 1];
            if (beg < 0 || end < beg || end > nnz) {
                bad = true;
            } else {
                for (int64_t e0 = beg; e0 < end; e0 += 32) {
                    const int64_t e = e0 + lane;
                    int c = 0;
                    double v = 0.0;
                    if (e < end) {
                        c = idx[e];
                        v = val[e];
                        if (c < 0 || (int64_t)c >= cols) {
                            bad = true;
                            c = 0;
                            v = 0.0;
                        }
                    }
                    const int cnt = (end - e0 < 32) ? (int)(end - e0) : 32;
                    for (int t = 0; t < cnt; ++t) {
                        const int cc = __shfl_sync(0xffffffffu, c, t);
                        const double vv = __shfl_sync(0xffffffffu, v, t);
                        const double *xr = Xr + (int64_t)cc * k;
                        if (lane < k) a0 = fma(vv, xr[lane], a0);
                        if (lane + 32 < k) a1 = fma(vv, xr[lane + 32], a1);
                        if (lane + 64 < k) a2 = fma(vv, xr[lane + 64], a2);
                        if (lane + 96 < k) a3 = fma(vv, xr[lane + 96], a3);
                    }
                }
            }
        }
        if (lane < k) tile[lane][rr] = a0;
        if (lane + 32 < k) tile[lane + 32][rr] = a1;
        if (lane + 64 < k) tile[lane + 64][rr] = a2;
        if (lane + 96 < k) tile[lane + 96][rr] = a3;
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) rxr_fail(acc, RXR_ERR_BAD_SPARSE, -1, (r0 < INT32_MAX) ? (int)r0 : INT32_MAX);
        return;
    }
    const int r = threadIdx.x & 31;
    if (r0 + r < rows)
        for (int j = threadIdx.x >> 5; j < k; j += 8) Y[r0 + r + (int64_t)j * ldy] = tile[j][r];
}

// R (k x k, ldr) = U_r diag(S) V_r^T: one-sided Jacobi on W = R (columns
// rotated in pairs until every pair's cosine is below sqrt(k) eps, LAPACK's
// threshold when singular vectors are wanted; sweeps end once none rotates a
// pair by more than 2^-27), V_r the product of the rotations, S the column norms of W and
// U_r = W diag(S)^{-1}; columns sorted by decreasing S.  Outputs k x k
// column-major with leading dimension k.  Vg: k x k global scratch used for
// V_r when k > 112.  One CTA of 512 threads; at most max_sweeps sweeps, and
// RXR_ERR_NO_CONVERGENCE in acc when the last one still rotated a pair by more
// than 2^-27.
__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_svd(const double *__restrict__ R, int64_t ldr, int k,
                                                              double *__restrict__ Ur, double *__restrict__ Vr,
                                                              double *__restrict__ S, double *__restrict__ Vg,
                                                              RxrStatus *acc, int max_sweeps)
{
    extern __shared__ double sm[];
    __shared__ double sig[kSvdMaxK];
    __shared__ int rank[kSvdMaxK];
    if (rxr_failed_block(acc)) return;
    double *W = sm;
    double *V = (k <= kJacobiVSmemK) ? sm + k * k : Vg;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    for (int i = tid; i < k * k; i += blockDim.x) {
        const int r = i % k, c = i / k;
        W[i] = R[r + (int64_t)c * ldr];
        V[i] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int kk = k + (k & 1);  // an odd k adds a dummy column that sits out one pair per round
    const double tol = sqrt((double)k) * 0x1p-52;
    bool converged = false;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        // convergence is quadratic: once no rotation of a sweep had a cosine above
        // 2^-27, the cosines it leaves are at rounding level and the next sweep
        // would rotate noise only
        bool large = false;
        for (int round = 0; round < kk - 1; ++round) {
            // circle method: position kk-1 fixed, the others turn one step per round
            for (int pr = warp; pr < kk / 2; pr += nwarps) {
                int p, q;
                if (pr == 0) {
                    p = kk - 1;
                    q = round;
                } else {
                    p = (round + pr) % (kk - 1);
                    q = (round - pr + (kk - 1)) % (kk - 1);
                }
                if (p >= k || q >= k) continue;
                double *wp = W + p * k, *wq = W + q * k;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < k; r += 32) {
                    const double x = wp[r], y = wq[r];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                const double nrm = sqrt(al) * sqrt(be);
                if (!(fabs(ga) > tol * nrm)) continue;  // also for NaN
                // rotation that makes columns p, q orthogonal: t the smaller root of
                // t^2 + 2 zeta t - 1 = 0, zeta = (be - al) / (2 ga)
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (fabs(zeta) > 1e150) ? 0.5 / zeta
                                                      : copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int r = lane; r < k; r += 32) {
                    const double x = wp[r], y = wq[r];
                    wp[r] = c * x - s * y;
                    wq[r] = s * x + c * y;
                }
                double *vp = V + p * k, *vq = V + q * k;
                for (int r = lane; r < k; r += 32) {
                    const double x = vp[r], y = vq[r];
                    vp[r] = c * x - s * y;
                    vq[r] = s * x + c * y;
                }
                large |= fabs(ga) > 0x1p-27 * nrm;
            }
            __syncthreads();
        }
        if (!__syncthreads_or(large)) {
            converged = true;
            break;
        }
    }
    // the sweep limit reached with a rotation above 2^-27 in the last sweep:
    // the columns may not be orthogonal yet, reported (column = the limit)
    if (!converged && tid == 0) rxr_fail(acc, RXR_ERR_NO_CONVERGENCE, -1, max_sweeps);
    for (int j = tid; j < k; j += blockDim.x) {
        double s2 = 0.0;
        for (int r = 0; r < k; ++r) s2 = fma(W[j * k + r], W[j * k + r], s2);
        sig[j] = sqrt(s2);
    }
    __syncthreads();
    for (int j = tid; j < k; j += blockDim.x) {
        int rk = 0;
        for (int i = 0; i < k; ++i) rk += (sig[i] > sig[j]) || (sig[i] == sig[j] && i < j);
        rank[j] = min(rk, k - 1);
    }
    __syncthreads();
    for (int i = tid; i < k * k; i += blockDim.x) {
        const int r = i % k, j = i / k, d = rank[j];
        const double sj = sig[j];
        Ur[r + d * k] = (sj > 0.0) ? W[i] / sj : 0.0;
        Vr[r + d * k] = V[i];
    }
    for (int j = tid; j < k; j += blockDim.x) S[rank[j]] = sig[j];
}

// Y (rows x k, ldy) = X (rows x k, ldx) T (k x k, column-major, ld k); Y and X
// must not overlap.  A CTA takes 64 rows; thread (r, g) sums columns g, g+4,
// ..., g + 4(NC-1) below k, NC >= k/4 (a multiple of 2 or 8, so that the
// warp-uniform column guards skip at most 3/8 of the FP64 issue).
template <int NC>
__global__ void __launch_bounds__(256) k_right_mult(const double *__restrict__ X, int64_t ldx, int64_t rows, int k,
                                                    const double *__restrict__ T, double *__restrict__ Y, int64_t ldy,
                                                    const RxrStatus *acc)
{
    extern __shared__ double Ts[];
    if (rxr_failed_block(acc)) return;
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Ts[i] = T[i];
    __syncthreads();
    const int r = threadIdx.x & (kRmRows - 1), g = threadIdx.x / kRmRows;
    const int64_t row = (int64_t)blockIdx.x * kRmRows + r;
    if (row >= rows) return;
    double a[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) a[i] = 0.0;
    for (int l = 0; l < k; ++l) {
        const double x = X[row + (int64_t)l * ldx];
        const double *tl = Ts + l;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const int c = g + 4 * i;
            if (c < k) a[i] = fma(x, tl[c * k], a[i]);
        }
    }
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        const int c = g + 4 * i;
        if (c < k) Y[row + (int64_t)c * ldy] = a[i];
    }
}

__global__ void k_status_keep(const RxrStatus *cur, RxrStatus *acc, int call)
{
    if (threadIdx.x == 0 && acc->code == 0 && cur->code != 0) {
        acc->code = cur->code;
        acc->pass = cur->pass;
        acc->column = cur->column;
        acc->flags = call;
    }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static int rsvd_launch_ok()
{
    return (cudaGetLastError() == cudaSuccess) ? 0 : RXR_ERR_CUDA;
}

int rsvd_transpose_enqueue(const double *X, int64_t ldx, int64_t rows, int k, double *Xr, cudaStream_t st)
{
    if (rows < 1) return 0;
    const dim3 grid((unsigned)cdiv(rows, 32), (unsigned)cdiv(k, 32));
    k_rm_transpose<<<grid, dim3(32, 8), 0, st>>>(X, ldx, rows, k, Xr);
    return rsvd_launch_ok();
}

int rsvd_spmm_enqueue(const int64_t *ptr, const int32_t *idx, const double *val, int64_t nnz, int64_t rows,
                      int64_t cols, const double *Xr, int k, double *Y, int64_t ldy, RxrStatus *acc, cudaStream_t st)
{
    if (rows < 1) return 0;
    k_csr_spmm<<<(unsigned)cdiv(rows, kSpRows), 256, 0, st>>>(ptr, idx, val, nnz, rows, cols, Xr, k, Y, ldy, acc);
    return rsvd_launch_ok();
}

size_t rsvd_jacobi_smem(int k)
{
    return (size_t)((k <= kJacobiVSmemK) ? 2 : 1) * k * k * sizeof(double);
}

int rsvd_jacobi_enqueue(const double *R, int64_t ldr, int k, double *Ur, double *Vr, double *S, double *Vg,
                        RxrStatus *acc, int max_sweeps, cudaStream_t st)
{
    if (max_sweeps < 1 || max_sweeps > kJacobiSweeps) max_sweeps = kJacobiSweeps;
    k_jacobi_svd<<<1, kJacobiThreads, rsvd_jacobi_smem(k), st>>>(R, ldr, k, Ur, Vr, S, Vg, acc, max_sweeps);
    return rsvd_launch_ok();
}

int rsvd_right_mult_enqueue(const double *X, int64_t ldx, int64_t rows, int k, const double *T, double *Y,
                            int64_t ldy, const RxrStatus *acc, cudaStream_t st)
{
    if (rows < 1) return 0;
    const unsigned grid = (unsigned)cdiv(rows, kRmRows);
    const size_t smem = (size_t)k * k * sizeof(double);
    if (k <= 8)
        k_right_mult<2><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    else if (k <= 16)
        k_right_mult<4><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    else if (k <= 32)
        k_right_mult<8><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    else if (k <= 64)
        k_right_mult<16><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    else if (k <= 96)
        k_right_mult<24><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    else
        k_right_mult<32><<<grid, 256, smem, st>>>(X, ldx, rows, k, T, Y, ldy, acc);
    return rsvd_launch_ok();
}

int rsvd_status_keep_enqueue(const RxrStatus *cur, RxrStatus *acc, int call, cudaStream_t st)
{
    k_status_keep<<<1, 32, 0, st>>>(cur, acc, call);
    return rsvd_launch_ok();
}

cudaError_t set_rsvd_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_jacobi_svd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max(rsvd_jacobi_smem(kJacobiVSmemK), rsvd_jacobi_smem(kSvdMaxK)));
    const int rm = (int)(kSvdMaxK * kSvdMaxK * sizeof(double));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_right_mult<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, rm);
    return e;
}

}  // namespace rxr
