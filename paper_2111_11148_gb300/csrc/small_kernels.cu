// small_kernels.cu -- the O(s n^2) and O(n^3) steps that run on one CTA between
// the streaming passes, plus the accuracy evaluators and the FP64 calibration.
//   * k_xr_factor : R_s = R factor of the sketch Y (s x n) by Householder QR
//                   (Algorithm 5 step 2) or LU with partial pivoting (Algorithm
//                   4 step 2), rows scaled so that diag(R_s) > 0, singularity
//                   test |R_kk| <= n u max|R_jj| (Section 2.2: a degenerate R_1
//                   from bad sampling or a rank-deficient A);
//   * k_factor    : R_p = chol(G_p) (Algorithm 1 step 2; breakdown reported as
//                   in Section 2.1) and R_acc <- R_p R_acc (R = R_2 R_1 R_s,
//                   Algorithms 2/4/5 last steps);
//   * k_copy_upper: R to the caller's layout with zeros below the diagonal;
//   * k_orth_* / k_resid_*: ||Q^T Q - I||_F and ||A - QR||_F / ||A||_F of
//                   Section 4.2 with Dot2 compensated dot products (Ogita, Rump
//                   & Oishi 2005);
//   * k_fp64_peak : independent DFMA chains on every SM.
#include <algorithm>

#include "rxr_internal.cuh"

namespace rxr {

constexpr int kSmallThreads = 512;
constexpr int64_t kXrSmemDoubles = 26624;  // 208 KB: the sketch's working copy in shared memory up to here
constexpr int kFactorSmemN = 64;           // C, R_p, R_acc in shared memory (96 KB) up to here

__device__ __forceinline__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------------------
// Step 2.  W (workspace, ld s) receives a copy of Y and is factorised in place.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void xr_body(const double *__restrict__ Y, int s, int n, int64_t ldy, int variant,
                                        double *__restrict__ W, double *__restrict__ Rs, int64_t ldrs, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double red[33];
    __shared__ double sh_beta, sh_v0, sh_piv;
    __shared__ int sh_idx[32];
    __shared__ double sh_val[32];
    __shared__ int sh_p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    for (int64_t e = tid; e < (int64_t)s * n; e += blockDim.x) {
        const int i = (int)(e % s), j = (int)(e / s);
        W[e] = Y[i + j * ldy];
    }
    __syncthreads();

    if (variant == RXR_QR) {
        for (int k = 0; k < n; ++k) {
            double part = 0.0;
            for (int i = k + tid; i < s; i += blockDim.x) part = fma(W[i + (int64_t)k * s], W[i + (int64_t)k * s], part);
            const double ss = block_sum(part, red);
            if (tid == 0) {
                const double alpha = sqrt(ss);
                const double x0 = W[k + (int64_t)k * s];
                const double sg = (x0 < 0.0) ? -1.0 : 1.0;
                sh_v0 = x0 + sg * alpha;
                // beta = 2 / v^T v with v^T v = 2 alpha (alpha + |x0|)
                sh_beta = (alpha > 0.0) ? 1.0 / (alpha * (alpha + fabs(x0))) : 0.0;
                W[k + (int64_t)k * s] = -sg * alpha;
            }
            __syncthreads();
            const double beta = sh_beta, v0 = sh_v0;
            // apply H_k to columns j > k, one warp per column
            for (int j = k + 1 + warp; j < n; j += nwarps) {
                double w = 0.0;
                for (int i = k + 1 + lane; i < s; i += 32) w = fma(W[i + (int64_t)k * s], W[i + (int64_t)j * s], w);
                w = warp_sum(w);
                w = fma(v0, W[k + (int64_t)j * s], w);
                const double f = beta * w;
                if (lane == 0) W[k + (int64_t)j * s] = fma(-f, v0, W[k + (int64_t)j * s]);
                for (int i = k + 1 + lane; i < s; i += 32)
                    W[i + (int64_t)j * s] = fma(-f, W[i + (int64_t)k * s], W[i + (int64_t)j * s]);
            }
            __syncthreads();
        }
    } else {
        for (int k = 0; k < n; ++k) {
            // pivot: largest |W(i,k)|, i >= k, lowest index on ties
            double bv = -1.0;
            int bi = s;
            for (int i = k + tid; i < s; i += blockDim.x) {
                const double a = fabs(W[i + (int64_t)k * s]);
                if (a > bv) {
                    bv = a;
                    bi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xFFFFFFFFu, bv, o);
                const int oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                sh_val[warp] = bv;
                sh_idx[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double v = sh_val[0];
                int idx = sh_idx[0];
                for (int w = 1; w < nwarps; ++w)
                    if (sh_val[w] > v || (sh_val[w] == v && sh_idx[w] < idx)) {
                        v = sh_val[w];
                        idx = sh_idx[w];
                    }
                sh_p = (idx < s) ? idx : k;
            }
            __syncthreads();
            const int p = sh_p;
            if (p != k)
                for (int j = tid; j < n; j += blockDim.x) {
                    const double t = W[k + (int64_t)j * s];
                    W[k + (int64_t)j * s] = W[p + (int64_t)j * s];
                    W[p + (int64_t)j * s] = t;
                }
            __syncthreads();
            if (tid == 0) sh_piv = W[k + (int64_t)k * s];
            __syncthreads();
            const double d = sh_piv;
            if (d != 0.0) {
                const double dinv = 1.0 / d;
                // rows i > k: multiplier and trailing update, one thread per row
                for (int i = k + 1 + tid; i < s; i += blockDim.x) {
                    const double l = W[i + (int64_t)k * s] * dinv;
                    W[i + (int64_t)k * s] = l;
                    for (int j = k + 1; j < n; ++j)
                        W[i + (int64_t)j * s] = fma(-l, W[k + (int64_t)j * s], W[i + (int64_t)j * s]);
                }
            }
            __syncthreads();
        }
    }

    // sign normalisation and singularity test
    __shared__ int sh_bad;
    if (tid == 0) {
        double mx = 0.0;
        int bad = 0;
        for (int k = 0; k < n; ++k) {
            const double d = fabs(W[k + (int64_t)k * s]);
            if (rxr_nonfinite(d)) bad = 1;
            mx = fmax(mx, d);
        }
        const double tol = (double)n * 0x1p-53 * mx;
        for (int k = 0; k < n; ++k)
            if (!(fabs(W[k + (int64_t)k * s]) > tol)) bad = 1;
        sh_bad = bad;
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double v = 0.0;
        if (i <= j) {
            v = W[i + (int64_t)j * s];
            if (W[i + (int64_t)i * s] < 0.0) v = -v;
        }
        Rs[i + j * ldrs] = v;
    }
    if (tid == 0 && sh_bad) rxr_fail(st, RXR_ERR_SKETCH_SINGULAR, 0, -1);
}

// The working copy of Y lives in shared memory when it fits (dynamic size
// s * n * 8 bytes, launched by xr_smem_bytes), else in the global scratch W.
__global__ void __launch_bounds__(kSmallThreads)
    k_xr_factor(const double *__restrict__ Y, int s, int n, int64_t ldy, int variant, double *__restrict__ W,
                double *__restrict__ Rs, int64_t ldrs, RxrStatus *st)
{
    extern __shared__ double xr_smem[];
    const bool in_smem = (int64_t)s * n <= kXrSmemDoubles;
    xr_body(Y, s, n, ldy, variant, in_smem ? xr_smem : W, Rs, ldrs, st);
}

size_t xr_smem_bytes(int64_t s, int64_t n)
{
    return (s * n <= kXrSmemDoubles) ? (size_t)(s * n) * sizeof(double) : 0;
}

// ---------------------------------------------------------------------------
// R_p = chol(G) (upper, from G's upper triangle), then R_acc <- R_p R_acc.
// C is n x n workspace.  Right-looking: for column j, R_jj = sqrt(C_jj),
// R_jl = C_jl / R_jj, then C_kl -= R_jk R_jl for j < k <= l.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void factor_body(const double *__restrict__ G, int n, int64_t ldg, double *__restrict__ Rp,
                                            double *__restrict__ Racc, double *__restrict__ C, int pass,
                                            int update_racc, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ int sh_bad;
    __shared__ double sh_rjj;
    const int tid = threadIdx.x;
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        C[e] = (i <= j) ? G[i + j * ldg] : 0.0;
        Rp[e] = 0.0;
    }
    if (tid == 0) sh_bad = -1;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (tid == 0) {
            const double d = C[j + (int64_t)j * n];
            if (!(d > 0.0) || rxr_nonfinite(d)) {
                sh_bad = j;
            } else {
                sh_rjj = sqrt(d);
            }
        }
        __syncthreads();
        if (sh_bad >= 0) break;
        const double rjj = sh_rjj, inv = 1.0 / rjj;
        for (int l = j + tid; l < n; l += blockDim.x)
            Rp[j + (int64_t)l * n] = (l == j) ? rjj : C[j + (int64_t)l * n] * inv;
        __syncthreads();
        const int w = n - j - 1;
        const int64_t pairs = (int64_t)w * w;
        for (int64_t e = tid; e < pairs; e += blockDim.x) {
            const int k = j + 1 + (int)(e % w), l = j + 1 + (int)(e / w);
            if (k <= l) C[k + (int64_t)l * n] = fma(-Rp[j + (int64_t)k * n], Rp[j + (int64_t)l * n], C[k + (int64_t)l * n]);
        }
        __syncthreads();
    }
    if (sh_bad >= 0) {
        if (tid == 0) rxr_fail(st, RXR_ERR_CHOL_BREAKDOWN, pass, sh_bad);
        return;
    }
    if (!update_racc) return;
    // C <- R_p R_acc (upper x upper), then R_acc <- C
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double acc = 0.0;
        if (i <= j)
            for (int k = i; k <= j; ++k) acc = fma(Rp[i + (int64_t)k * n], Racc[k + (int64_t)j * n], acc);
        C[e] = acc;
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) Racc[e] = C[e];
}

// n <= 64: C, R_p and R_acc are worked on in shared memory (3 n^2 doubles,
// launched by factor_smem_bytes) and R_p, R_acc written back at the end.
__global__ void __launch_bounds__(kSmallThreads)
    k_factor(const double *__restrict__ G, int n, int64_t ldg, double *__restrict__ Rp, double *__restrict__ Racc,
             double *__restrict__ C, int pass, int update_racc, RxrStatus *st)
{
    if (n > kFactorSmemN) {
        factor_body(G, n, ldg, Rp, Racc, C, pass, update_racc, st);
        return;
    }
    if (rxr_failed_block(st)) return;
    extern __shared__ double fac_smem[];
    const int nn = n * n;
    double *Cs = fac_smem, *Rps = fac_smem + nn, *Ras = fac_smem + 2 * nn;
    if (update_racc)
        for (int e = threadIdx.x; e < nn; e += blockDim.x) Ras[e] = Racc[e];
    __syncthreads();
    factor_body(G, n, ldg, Rps, Ras, Cs, pass, update_racc, st);
    __syncthreads();
    if (rxr_failed_block(st)) return;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        Rp[e] = Rps[e];
        if (update_racc) Racc[e] = Ras[e];
    }
}

size_t factor_smem_bytes(int64_t n)
{
    return (n <= kFactorSmemN) ? (size_t)(3 * n * n) * sizeof(double) : 0;
}

// Batched forms of the one-CTA steps: block k serves problem k.  The XR step
// also seeds R_acc = R_s (R_s = I without preconditioner).
__global__ void __launch_bounds__(kSmallThreads) k_xr_factor_batched(const XrJob *__restrict__ jobs)
{
    const XrJob j = jobs[blockIdx.x];
    if (j.variant == RXR_NONE) {
        if (rxr_failed(j.st)) return;
        for (int64_t e = threadIdx.x; e < (int64_t)j.n * j.n; e += blockDim.x) {
            const double v = ((e % j.n) == (e / j.n)) ? 1.0 : 0.0;
            j.Rs[e] = v;
            j.Racc[e] = v;
        }
        return;
    }
    xr_body(j.Y, j.s, j.n, j.s, j.variant, j.W, j.Rs, j.n, j.st);
    __syncthreads();
    if (rxr_failed(j.st)) return;
    for (int64_t e = threadIdx.x; e < (int64_t)j.n * j.n; e += blockDim.x) j.Racc[e] = j.Rs[e];
}

__global__ void __launch_bounds__(kSmallThreads) k_factor_batched(const FactorJob *__restrict__ jobs, int pass)
{
    const FactorJob j = jobs[blockIdx.x];
    factor_body(j.G, j.n, j.n, j.Rp, j.Racc, j.C, pass, 1, j.st);
}

// R to the caller's layout and the status to the caller's array.
__global__ void k_finish_batched(const FinishJob *__restrict__ jobs)
{
    const FinishJob j = jobs[blockIdx.x];
    const bool failed = rxr_failed(j.st);
    if (!failed && j.R != nullptr)
        for (int64_t e = threadIdx.x; e < (int64_t)j.n * j.n; e += blockDim.x) {
            const int i = (int)(e % j.n), c = (int)(e / j.n);
            j.R[i + c * j.ldr] = (i <= c) ? j.Racc[e] : 0.0;
        }
    if (threadIdx.x == 0) {
        j.status_out[0] = j.st->code;
        j.status_out[1] = j.st->pass;
        j.status_out[2] = j.st->column;
        j.status_out[3] = 0;
    }
}

// R (n x n, ld n) -> out (ld ldo), zeros strictly below the diagonal.
__global__ void k_copy_upper(const double *__restrict__ R, int n, double *__restrict__ out, int64_t ldo,
                             const RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        out[i + j * ldo] = (i <= j) ? R[e] : 0.0;
    }
}

// Identity into an n x n (ld n) matrix.
// Shifted CholeskyQR's first Gram (Section 2.1, sCholeskyQR3): G += eps I with
// eps = coef lambda_max(G), lambda_max(G) = ||A||_2^2 estimated by 40 power
// iterations from the all-ones vector in a fixed order (G is symmetric
// positive semidefinite, so ||G v|| / ||v|| rises towards lambda_max).  One
// CTA of 256 threads, n <= 512, G column-major with leading dimension ldg.
__global__ void __launch_bounds__(256) k_shift_gram(double *__restrict__ G, int n, int64_t ldg, double coef,
                                                    RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double v[512], w[512], red[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += blockDim.x) v[i] = 1.0;
    __syncthreads();
    double lam = 0.0;
    for (int it = 0; it < 40; ++it) {
        double t = 0.0;
        for (int i = tid; i < n; i += blockDim.x) {
            double a = 0.0;
            for (int k = 0; k < n; ++k) a = fma(G[i + (int64_t)k * ldg], v[k], a);
            w[i] = a;
            t = fma(a, a, t);
        }
        double u = 0.0;  // ||v||^2
        for (int i = tid; i < n; i += blockDim.x) u = fma(v[i], v[i], u);
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
            u += __shfl_xor_sync(0xFFFFFFFFu, u, o);
        }
        __syncthreads();  // every thread's reads of v are done
        if (lane == 0) red[warp] = t;
        __syncthreads();
        double ss = 0.0;
        for (int k = 0; k < 8; ++k) ss += red[k];  // ||G v||^2, same order in every thread
        __syncthreads();
        if (lane == 0) red[warp] = u;
        __syncthreads();
        double vv = 0.0;
        for (int k = 0; k < 8; ++k) vv += red[k];
        if (!(ss > 0.0) || !(vv > 0.0)) break;  // G = 0 (or not finite): no shift
        lam = sqrt(ss / vv);
        const double inv = 1.0 / sqrt(ss);
        for (int i = tid; i < n; i += blockDim.x) v[i] = w[i] * inv;
        __syncthreads();
    }
    if (!rxr_nonfinite(lam))
        for (int i = tid; i < n; i += blockDim.x) G[i + (int64_t)i * ldg] += coef * lam;
}

// Least squares (Section 5.2), c = B^T b over one CTA's rows: warp w takes the
// (column j, right-hand side r) pairs w, w + 8, ..., its lanes the rows (a
// fixed order, then a shuffle tree); partial sums to parts[cta][j + n r].
// A NaN or Inf in b is reported.
__global__ void __launch_bounds__(256) k_ls_btb(const double *__restrict__ B, int64_t ldb, int64_t m, int n,
                                                const double *__restrict__ b, int64_t ldbb, int k, int64_t rows_per_cta,
                                                double *__restrict__ parts, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r0 = blockIdx.x * rows_per_cta, r1 = min(m, r0 + rows_per_cta);
    bool bad = false;
    for (int q = warp; q < n * k; q += 8) {
        const int j = q % n, r = q / n;
        const double *bc = B + (int64_t)j * ldb, *rc = b + (int64_t)r * ldbb;
        double a = 0.0;
        for (int64_t i = r0 + lane; i < r1; i += 32) {
            const double bv = rc[i];
            bad |= (j == 0) && rxr_nonfinite(bv);
            a = fma(bc[i], bv, a);
        }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
        if (lane == 0) parts[(int64_t)blockIdx.x * n * k + q] = a;
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);
}

// Least squares (Section 5.2), the small solves: R_G^T z = c, R_G y = z,
// R_s x = y for the k right-hand sides (c: n x k packed, R_G and R_s upper n x
// n packed), in place in x (n x k, ldx).  Column-oriented substitution: step
// j fixes entry j of every right-hand side, then all threads update the
// remaining entries (one CTA, one barrier per step; global writes are visible
// to the CTA after the barrier).
__global__ void __launch_bounds__(512) k_ls_solve(const double *__restrict__ RG, const double *__restrict__ Rs, int n,
                                                  int k, const double *__restrict__ c, double *x, int64_t ldx,
                                                  RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < n * k; e += nt) x[e % n + (int64_t)(e / n) * ldx] = c[e];
    __syncthreads();
    // forward: R_G^T z = c  (z_j = v_j / R_jj, then v_l -= R_jl z_j for l > j)
    for (int j = 0; j < n; ++j) {
        for (int r = tid; r < k; r += nt) x[j + r * ldx] /= RG[j + (int64_t)j * n];
        __syncthreads();
        for (int e = tid; e < (n - j - 1) * k; e += nt) {
            const int l = j + 1 + e % (n - j - 1), r = e / (n - j - 1);
            x[l + r * ldx] = fma(-RG[j + (int64_t)l * n], x[j + r * ldx], x[l + r * ldx]);
        }
        __syncthreads();
    }
    // backward twice: R_G y = z, then R_s x = y  (y_j = v_j / R_jj, v_l -= R_lj y_j for l < j)
    for (int pass = 0; pass < 2; ++pass) {
        const double *R = pass == 0 ? RG : Rs;
        for (int j = n - 1; j >= 0; --j) {
            for (int r = tid; r < k; r += nt) x[j + r * ldx] /= R[j + (int64_t)j * n];
            __syncthreads();
            for (int e = tid; e < j * k; e += nt) {
                const int l = e % j, r = e / j;
                x[l + r * ldx] = fma(-R[l + (int64_t)j * n], x[j + r * ldx], x[l + r * ldx]);
            }
            __syncthreads();
        }
    }
}

__global__ void k_identity(double *__restrict__ R, int n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x)
        R[e] = ((e % n) == (e / n)) ? 1.0 : 0.0;
}

// Copy the device status into a caller-owned int[4].
__global__ void k_status_out(const RxrStatus *st, int *out)
{
    if (threadIdx.x == 0) {
        out[0] = st->code;
        out[1] = st->pass;
        out[2] = st->column;
        out[3] = 0;
    }
}

// ---------------------------------------------------------------------------
// Dot2 accumulator: (p, s) with p + s the compensated value.
// ---------------------------------------------------------------------------
struct Dot2 {
    double p, s;
};
__device__ __forceinline__ void dot2_add(Dot2 &d, double x, double y)
{
    const double h = x * y;
    const double r = fma(x, y, -h);
    const double p = d.p + h;
    const double z = p - d.p;
    const double q = (d.p - (p - z)) + (h - z);
    d.p = p;
    d.s += q + r;
}

// Orthogonality: per (pair, row chunk) partial Dot2 sums of Q^T Q.  grid.x =
// row chunks, grid.y = pair blocks of blockDim.x pairs (j <= l).
__global__ void __launch_bounds__(256)
    k_orth_partial(const double *__restrict__ Q, int64_t m, int n, int64_t ldq, int64_t rows_per_chunk, int kEvP,
                   double *__restrict__ parts)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *qp = reinterpret_cast<double *>(smem_raw);  // [n][kEvP]
    const int npairs = n * (n + 1) / 2;
    const int pair = blockIdx.y * blockDim.x + threadIdx.x;
    int j = -1, l = -1;
    if (pair < npairs) {
        int rem = pair;
        j = 0;
        while (rem >= n - j) {
            rem -= n - j;
            ++j;
        }
        l = j + rem;
    }
    Dot2 d = {0.0, 0.0};
    const int64_t r_begin = blockIdx.x * rows_per_chunk;
    const int64_t r_end = min(m, r_begin + rows_per_chunk);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kEvP) {
        for (int e = threadIdx.x; e < kEvP * n; e += blockDim.x) {
            const int row = e % kEvP, col = e / kEvP;
            const int64_t gr = r0 + row;
            qp[e] = (gr < r_end) ? Q[gr + (int64_t)col * ldq] : 0.0;
        }
        __syncthreads();
        if (j >= 0)
            for (int r = 0; r < kEvP; ++r) dot2_add(d, qp[j * kEvP + r], qp[l * kEvP + r]);
        __syncthreads();
    }
    if (pair < npairs) {
        parts[((int64_t)blockIdx.x * npairs + pair) * 2 + 0] = d.p;
        parts[((int64_t)blockIdx.x * npairs + pair) * 2 + 1] = d.s;
    }
}

// Combine the chunks per pair (error-free sums of the p parts plus the s
// parts), subtract the identity, and sum squares (off-diagonal pairs twice).
__global__ void k_orth_final(const double *__restrict__ parts, int nchunks, int n, double *out)
{
    __shared__ double red[33];
    const int npairs = n * (n + 1) / 2;
    double acc = 0.0;
    for (int pair = threadIdx.x; pair < npairs; pair += blockDim.x) {
        int rem = pair, j = 0;
        while (rem >= n - j) {
            rem -= n - j;
            ++j;
        }
        const int l = j + rem;
        Dot2 d = {0.0, 0.0};
        if (j == l) dot2_add(d, -1.0, 1.0);
        for (int c = 0; c < nchunks; ++c) {
            dot2_add(d, parts[((int64_t)c * npairs + pair) * 2 + 0], 1.0);
            d.s += parts[((int64_t)c * npairs + pair) * 2 + 1];
        }
        const double e = d.p + d.s;
        acc += (j == l ? 1.0 : 2.0) * e * e;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[0] = sqrt(acc);
}

// Residual: one thread per row; for every column j the entry A_ij - sum_k
// Q_ik R_kj as one Dot2 sum; per-CTA partial sums of squares of the residual
// and of A.
__global__ void __launch_bounds__(256)
    k_resid_partial(const double *__restrict__ A, int64_t lda, const double *__restrict__ Q, int64_t ldq,
                    const double *__restrict__ R, int64_t ldr, int64_t m, int n, double *__restrict__ parts)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *rs = reinterpret_cast<double *>(smem_raw);  // packed upper R (when it fits)
    __shared__ double red[33];
    const bool r_smem = (int64_t)n * (n + 1) / 2 <= 16384;
    if (r_smem)
        for (int j = 0; j < n; ++j)
            for (int k = threadIdx.x; k <= j; k += blockDim.x) rs[j * (j + 1) / 2 + k] = R[k + (int64_t)j * ldr];
    __syncthreads();
    double num = 0.0, den = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        for (int j = 0; j < n; ++j) {
            Dot2 d = {0.0, 0.0};
            const double a = A[i + (int64_t)j * lda];
            dot2_add(d, a, 1.0);
            if (r_smem) {
                const double *rc = rs + j * (j + 1) / 2;
                for (int k = 0; k <= j; ++k) dot2_add(d, -Q[i + (int64_t)k * ldq], rc[k]);
            } else {
                for (int k = 0; k <= j; ++k) dot2_add(d, -Q[i + (int64_t)k * ldq], R[k + (int64_t)j * ldr]);
            }
            const double e = d.p + d.s;
            num = fma(e, e, num);
            den = fma(a, a, den);
        }
    }
    num = block_sum(num, red);
    den = block_sum(den, red);
    if (threadIdx.x == 0) {
        parts[2 * blockIdx.x] = num;
        parts[2 * blockIdx.x + 1] = den;
    }
}

__global__ void k_resid_final(const double *__restrict__ parts, int nparts, double *out)
{
    if (threadIdx.x == 0) {
        double num = 0.0, den = 0.0;
        for (int c = 0; c < nparts; ++c) {
            num += parts[2 * c];
            den += parts[2 * c + 1];
        }
        out[0] = sqrt(num) / sqrt(den);
    }
}

// ---------------------------------------------------------------------------
// FP64 calibration: 8 independent FMA chains per thread.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fp64_peak(double *out, int iters, double a, double b)
{
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = fma(acc[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// Blocked Householder QR of the sketch (rQR, Algorithm 5 step 2) spread over
// the GPU: for each panel of kQrB columns one CTA factors the panel with
// reflectors H_k = I - tau_k v_k v_k^T (v_k(k) = 1, stored below the
// diagonal; R on and above it) and forms the compact-WY factor T with
// H_1 ... H_b = I - V T V^T; the trailing columns C then receive
// C <- (I - V T^T V^T) C on many CTAs: partial V^T C over 128-row chunks, a
// fixed-order sum of the chunks, W = T^T (V^T C), C -= V W.  Mathematically the
// same Householder QR as the one-CTA form; the rounding order differs.
// ---------------------------------------------------------------------------
constexpr int kQrB = 32;       // panel width
constexpr int kQrCols = 8;     // trailing columns per CTA of the update
constexpr int kQrRows = 128;   // rows per chunk of the update

__device__ __forceinline__ double qr_v(const double *W, int s, int kc, int i)  // V(i, column kc of W)
{
    return (i == kc) ? 1.0 : (i > kc ? W[i + (int64_t)kc * s] : 0.0);
}

__global__ void __launch_bounds__(kSmallThreads) k_qr_panel(double *__restrict__ W, int s, int n, int k0,
                                                            double *__restrict__ T, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double red[33];
    __shared__ double sh_tau[kQrB];
    __shared__ double sh_S[kQrB * kQrB];   // V^T V, (q, k) at k * kQrB + q
    __shared__ double sh_T[kQrB * kQrB];   // T, (q, k) at k * kQrB + q
    __shared__ double sh_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int bw = min(kQrB, n - k0);
    for (int kk = 0; kk < bw; ++kk) {
        const int k = k0 + kk;
        double part = 0.0;
        for (int i = k + 1 + tid; i < s; i += blockDim.x) part = fma(W[i + (int64_t)k * s], W[i + (int64_t)k * s], part);
        const double xn2 = block_sum(part, red);
        if (tid == 0) {
            const double alpha = W[k + (int64_t)k * s];
            double tau = 0.0, scale = 0.0, beta = alpha;
            if (xn2 > 0.0) {
                beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
                tau = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            W[k + (int64_t)k * s] = beta;
            sh_tau[kk] = tau;
            sh_scale = scale;
        }
        __syncthreads();
        const double scale = sh_scale, tau = sh_tau[kk];
        for (int i = k + 1 + tid; i < s; i += blockDim.x) W[i + (int64_t)k * s] *= scale;
        __syncthreads();
        // H_k on the panel's later columns, one warp per column
        for (int j = k + 1 + warp; j < k0 + bw; j += nwarps) {
            double w = 0.0;
            for (int i = k + 1 + lane; i < s; i += 32) w = fma(W[i + (int64_t)k * s], W[i + (int64_t)j * s], w);
            w = warp_sum(w) + W[k + (int64_t)j * s];
            const double f = tau * w;
            if (lane == 0) W[k + (int64_t)j * s] -= f;
            for (int i = k + 1 + lane; i < s; i += 32) W[i + (int64_t)j * s] = fma(-f, W[i + (int64_t)k * s], W[i + (int64_t)j * s]);
        }
        __syncthreads();
    }
    // S = V^T V (q < k), one warp per pair
    for (int pr = warp; pr < bw * bw; pr += nwarps) {
        const int q = pr % bw, k = pr / bw;
        if (q >= k) continue;
        double d = 0.0;
        for (int i = k0 + k + lane; i < s; i += 32) d = fma(qr_v(W, s, k0 + q, i), qr_v(W, s, k0 + k, i), d);
        d = warp_sum(d);
        if (lane == 0) sh_S[k * kQrB + q] = d;
    }
    __syncthreads();
    // T(k, k) = tau_k, T(0:k, k) = -tau_k T(0:k, 0:k) S(0:k, k), column by column
    for (int k = 0; k < bw; ++k) {
        if (tid < k) {
            double acc = 0.0;
            for (int q = tid; q < k; ++q) acc = fma(sh_T[q * kQrB + tid], sh_S[k * kQrB + q], acc);
            sh_T[k * kQrB + tid] = -sh_tau[k] * acc;
        } else if (tid == k) {
            sh_T[k * kQrB + k] = sh_tau[k];
        }
        __syncthreads();
    }
    for (int e = tid; e < kQrB * kQrB; e += blockDim.x) {
        const int q = e % kQrB, k = e / kQrB;
        T[e] = (q < bw && k < bw && q <= k) ? sh_T[e] : 0.0;
    }
}

// P[(chunk * nc + c) * kQrB + k] = sum over the chunk's rows of V(i, k) C(i, c).
__global__ void __launch_bounds__(256) k_qr_vtc(const double *__restrict__ W, int s, int n, int k0,
                                                double *__restrict__ P, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double sv[kQrRows * kQrB];
    __shared__ double sc[kQrRows * kQrCols];
    const int bw = min(kQrB, n - k0), nc = n - k0 - bw;
    const int c0 = blockIdx.x * kQrCols, i0 = k0 + blockIdx.y * kQrRows;
    const int rows = min(kQrRows, s - i0);
    const int tid = threadIdx.x;
    for (int e = tid; e < kQrRows * kQrB; e += blockDim.x) {
        const int r = e % kQrRows, k = e / kQrRows;
        sv[e] = (r < rows && k < bw) ? qr_v(W, s, k0 + k, i0 + r) : 0.0;
    }
    for (int e = tid; e < kQrRows * kQrCols; e += blockDim.x) {
        const int r = e % kQrRows, c = e / kQrRows;
        sc[e] = (r < rows && c0 + c < nc) ? W[(i0 + r) + (int64_t)(k0 + bw + c0 + c) * s] : 0.0;
    }
    __syncthreads();
    const int k = tid >> 3, c = tid & 7;
    double acc = 0.0;
    for (int r = 0; r < rows; ++r) acc = fma(sv[k * kQrRows + r], sc[c * kQrRows + r], acc);
    if (k < bw && c0 + c < nc) P[((int64_t)blockIdx.y * nc + c0 + c) * kQrB + k] = acc;
}

// C -= V (T^T (sum_chunks P)) for the CTA's kQrCols columns and kQrRows rows.
__global__ void __launch_bounds__(256) k_qr_apply(double *__restrict__ W, int s, int n, int k0,
                                                  const double *__restrict__ P, int nchunks,
                                                  const double *__restrict__ T, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double w1[kQrB * kQrCols], w2[kQrB * kQrCols];
    const int bw = min(kQrB, n - k0), nc = n - k0 - bw;
    const int c0 = blockIdx.x * kQrCols, i0 = k0 + blockIdx.y * kQrRows;
    const int rows = min(kQrRows, s - i0);
    const int tid = threadIdx.x;
    {
        const int k = tid >> 3, c = tid & 7;
        double acc = 0.0;
        if (k < bw && c0 + c < nc)
            for (int ch = 0; ch < nchunks; ++ch) acc += P[((int64_t)ch * nc + c0 + c) * kQrB + k];
        w1[c * kQrB + k] = acc;
    }
    __syncthreads();
    {
        const int k = tid >> 3, c = tid & 7;
        double acc = 0.0;
        for (int q = 0; q <= k && q < bw; ++q) acc = fma(T[k * kQrB + q], w1[c * kQrB + q], acc);
        w2[c * kQrB + k] = (k < bw) ? acc : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < kQrRows * kQrCols; e += blockDim.x) {
        const int r = e % kQrRows, c = e / kQrRows;
        if (r >= rows || c0 + c >= nc) continue;
        const int i = i0 + r;
        double *cp = W + i + (int64_t)(k0 + bw + c0 + c) * s;
        double acc = *cp;
        for (int k = 0; k < bw; ++k) acc = fma(-qr_v(W, s, k0 + k, i), w2[c * kQrB + k], acc);
        *cp = acc;
    }
}

// Sign normalisation (rows of R scaled so diag > 0) and singularity test of
// the factored W (R in its leading n x n upper triangle), R_s written out.
__global__ void __launch_bounds__(kSmallThreads) k_xr_finish(const double *__restrict__ W, int s, int n,
                                                             double *__restrict__ Rs, int64_t ldrs, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ int sh_bad;
    const int tid = threadIdx.x;
    if (tid == 0) {
        double mx = 0.0;
        int bad = 0;
        for (int k = 0; k < n; ++k) {
            const double d = fabs(W[k + (int64_t)k * s]);
            if (rxr_nonfinite(d)) bad = 1;
            mx = fmax(mx, d);
        }
        const double tol = (double)n * 0x1p-53 * mx;
        for (int k = 0; k < n; ++k)
            if (!(fabs(W[k + (int64_t)k * s]) > tol)) bad = 1;
        sh_bad = bad;
    }
    __syncthreads();
    for (int64_t e = tid; e < (int64_t)n * n; e += blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double v = 0.0;
        if (i <= j) {
            v = W[i + (int64_t)j * s];
            if (W[i + (int64_t)i * s] < 0.0) v = -v;
        }
        Rs[i + j * ldrs] = v;
    }
    if (tid == 0 && sh_bad) rxr_fail(st, RXR_ERR_SKETCH_SINGULAR, 0, -1);
}

// The rQR factorisation of Y (s x n, ld ldy) into R_s: Y copied to W (ld s),
// then the panels.  Scratch: T (kQrB^2 doubles) and P (ceil(s / kQrRows) x n
// x kQrB doubles) from `scratch`.
int blocked_qr_enqueue(const double *Y, int s, int n, int64_t ldy, double *W, double *Rs, int64_t ldrs,
                       double *scratch, RxrStatus *status, cudaStream_t st)
{
    if (cudaMemcpy2DAsync(W, (size_t)s * 8, Y, (size_t)ldy * 8, (size_t)s * 8, n, cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
        return RXR_ERR_CUDA;
    double *T = scratch, *P = scratch + kQrB * kQrB;
    for (int k0 = 0; k0 < n; k0 += kQrB) {
        k_qr_panel<<<1, kSmallThreads, 0, st>>>(W, s, n, k0, T, status);
        const int bw = std::min(kQrB, n - k0), nc = n - k0 - bw;
        if (nc <= 0) continue;
        const dim3 grid((unsigned)((nc + kQrCols - 1) / kQrCols), (unsigned)((s - k0 + kQrRows - 1) / kQrRows));
        k_qr_vtc<<<grid, 256, 0, st>>>(W, s, n, k0, P, status);
        k_qr_apply<<<grid, 256, 0, st>>>(W, s, n, k0, P, (int)grid.y, T, status);
    }
    k_xr_finish<<<1, kSmallThreads, 0, st>>>(W, s, n, Rs, ldrs, status);
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

size_t blocked_qr_scratch_doubles(int64_t s, int64_t n)
{
    return (size_t)kQrB * kQrB + (size_t)((s + kQrRows - 1) / kQrRows) * n * kQrB;
}

// ---------------------------------------------------------------------------
// Blocked Cholesky R_p = chol(G) (upper) and R_acc <- R_p R_acc for n > 64,
// spread over the GPU: per panel of kChB columns one CTA factors the diagonal
// block, a column-parallel kernel forms the panel's rows of R_p, and an
// upper-triangle update of the trailing block runs over kChB x kChB tiles.
// Every entry sees exactly the FMA sequence of the one-CTA form (updates in
// ascending panel order, R_jl = C_jl * (1 / R_jj)), so the result is the same
// to the bit.  C (n x n scratch, ld n) holds the working copy.
// ---------------------------------------------------------------------------
constexpr int kChB = 32;

__global__ void __launch_bounds__(256) k_chol_init(const double *__restrict__ G, int n, int64_t ldg,
                                                   double *__restrict__ C, double *__restrict__ Rp, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        C[e] = (i <= j) ? G[i + j * ldg] : 0.0;
        Rp[e] = 0.0;
    }
}

// Diagonal block [k0, k0 + b): unblocked Cholesky of the updated block; the
// block's rows of R_p (its own columns) are written.
__global__ void __launch_bounds__(256) k_chol_diag(double *__restrict__ C, double *__restrict__ Rp, int n, int k0,
                                                   int pass, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double cs[kChB * kChB], rs[kChB * kChB];
    __shared__ double sh_rjj;
    __shared__ int sh_bad;
    const int b = min(kChB, n - k0), tid = threadIdx.x;
    for (int e = tid; e < kChB * kChB; e += blockDim.x) {
        const int i = e % kChB, j = e / kChB;
        cs[e] = (i < b && j < b) ? C[(k0 + i) + (int64_t)(k0 + j) * n] : 0.0;
        rs[e] = 0.0;
    }
    if (tid == 0) sh_bad = -1;
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (tid == 0) {
            const double d = cs[j + j * kChB];
            if (!(d > 0.0) || rxr_nonfinite(d)) sh_bad = j;
            else sh_rjj = sqrt(d);
        }
        __syncthreads();
        if (sh_bad >= 0) break;
        const double rjj = sh_rjj, inv = 1.0 / rjj;
        for (int l = j + tid; l < b; l += blockDim.x) rs[j + l * kChB] = (l == j) ? rjj : cs[j + l * kChB] * inv;
        __syncthreads();
        const int w = b - j - 1;
        for (int e = tid; e < w * w; e += blockDim.x) {
            const int k = j + 1 + e % w, l = j + 1 + e / w;
            if (k <= l) cs[k + l * kChB] = fma(-rs[j + k * kChB], rs[j + l * kChB], cs[k + l * kChB]);
        }
        __syncthreads();
    }
    if (sh_bad >= 0) {
        if (tid == 0) rxr_fail(st, RXR_ERR_CHOL_BREAKDOWN, pass, k0 + sh_bad);
        return;
    }
    for (int e = tid; e < kChB * kChB; e += blockDim.x) {
        const int i = e % kChB, j = e / kChB;
        if (i < b && j < b) Rp[(k0 + i) + (int64_t)(k0 + j) * n] = rs[e];
    }
}

// Panel rows of R_p right of the diagonal block: column l (one thread each)
// runs the one-CTA form's sequence for rows j of the block: C_jl receives the
// block's earlier rows' updates, then R_jl = C_jl * (1 / R_jj).
__global__ void __launch_bounds__(256) k_chol_panel(const double *__restrict__ C, double *__restrict__ Rp, int n,
                                                    int k0, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double rk[kChB * kChB];
    __shared__ double inv[kChB];
    const int b = min(kChB, n - k0), tid = threadIdx.x;
    for (int e = tid; e < kChB * kChB; e += blockDim.x) {
        const int i = e % kChB, j = e / kChB;
        rk[e] = (i < b && j < b) ? Rp[(k0 + i) + (int64_t)(k0 + j) * n] : 0.0;
    }
    __syncthreads();
    if (tid < b) inv[tid] = 1.0 / rk[tid + tid * kChB];
    __syncthreads();
    const int l = k0 + b + blockIdx.x * blockDim.x + tid;
    if (l >= n) return;
    double x[kChB];
#pragma unroll
    for (int j = 0; j < kChB; ++j) x[j] = (j < b) ? C[(k0 + j) + (int64_t)l * n] : 0.0;
#pragma unroll
    for (int j = 0; j < kChB; ++j) {
        if (j < b) {
            x[j] = x[j] * inv[j];
#pragma unroll
            for (int k = j + 1; k < kChB; ++k)
                if (k < b) x[k] = fma(-rk[j + k * kChB], x[j], x[k]);
        }
    }
#pragma unroll
    for (int j = 0; j < kChB; ++j)
        if (j < b) Rp[(k0 + j) + (int64_t)l * n] = x[j];
}

// Trailing update C_kl -= sum_{j in panel} R_jk R_jl for k0 + b <= k <= l < n,
// one kChB x kChB tile (I <= J) per CTA.
__global__ void __launch_bounds__(256) k_chol_syrk(double *__restrict__ C, const double *__restrict__ Rp, int n,
                                                   int k0, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    __shared__ double ri[kChB * kChB], rj[kChB * kChB];  // panel rows x tile columns
    const int b = min(kChB, n - k0), t0 = k0 + b;
    const int nt = (n - t0 + kChB - 1) / kChB;
    int I = 0, rem = blockIdx.x;
    while (rem >= nt - I) {
        rem -= nt - I;
        ++I;
    }
    const int J = I + rem;
    const int ci = t0 + I * kChB, cj = t0 + J * kChB, tid = threadIdx.x;
    for (int e = tid; e < kChB * kChB; e += blockDim.x) {
        const int q = e % kChB, c = e / kChB;
        ri[e] = (q < b && ci + c < n) ? Rp[(k0 + q) + (int64_t)(ci + c) * n] : 0.0;
        rj[e] = (q < b && cj + c < n) ? Rp[(k0 + q) + (int64_t)(cj + c) * n] : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < kChB * kChB; e += blockDim.x) {
        const int a = e % kChB, c = e / kChB;
        const int k = ci + a, l = cj + c;
        if (k >= n || l >= n || k > l) continue;
        double acc = C[k + (int64_t)l * n];
        for (int q = 0; q < b; ++q) acc = fma(-ri[q + a * kChB], rj[q + c * kChB], acc);
        C[k + (int64_t)l * n] = acc;
    }
}

// out_ij = sum_{k = i..j} Rp_ik Racc_kj (upper x upper), then copied to Racc.
__global__ void __launch_bounds__(256) k_trmm_upper(const double *__restrict__ Rp, const double *__restrict__ Racc,
                                                    double *__restrict__ out, int n, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        double acc = 0.0;
        if (i <= j)
            for (int k = i; k <= j; ++k) acc = fma(Rp[i + (int64_t)k * n], Racc[k + (int64_t)j * n], acc);
        out[e] = acc;
    }
}

int blocked_factor_enqueue(const double *G, int n, int64_t ldg, double *Rp, double *Racc, double *C, int pass,
                           int update_racc, RxrStatus *status, cudaStream_t st)
{
    const int64_t nn = (int64_t)n * n;
    const int g = (int)std::min<int64_t>(1024, (nn + 255) / 256);
    k_chol_init<<<g, 256, 0, st>>>(G, n, ldg, C, Rp, status);
    for (int k0 = 0; k0 < n; k0 += kChB) {
        k_chol_diag<<<1, 256, 0, st>>>(C, Rp, n, k0, pass, status);
        const int b = std::min(kChB, n - k0), rest = n - k0 - b;
        if (rest <= 0) continue;
        k_chol_panel<<<(rest + 255) / 256, 256, 0, st>>>(C, Rp, n, k0, status);
        const int nt = (rest + kChB - 1) / kChB;
        k_chol_syrk<<<nt * (nt + 1) / 2, 256, 0, st>>>(C, Rp, n, k0, status);
    }
    if (update_racc) {
        k_trmm_upper<<<g, 256, 0, st>>>(Rp, Racc, C, n, status);
        if (cudaMemcpyAsync(Racc, C, (size_t)nn * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            return RXR_ERR_CUDA;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : RXR_ERR_CUDA;
}

cudaError_t set_small_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_xr_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(kXrSmemDoubles * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_factor, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * kFactorSmemN * kFactorSmemN * sizeof(double)));
    return e;
}

}  // namespace rxr
