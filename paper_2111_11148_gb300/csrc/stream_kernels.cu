// stream_kernels.cu -- the passes that stream A (m x n, m >> n) through HBM:
//   * k_omega        : the z values of the Gaussian sketch (test hook);
//   * k_sketch_fp64  : Y = Omega A with Omega generated in-kernel (Section 2.3);
//   * k_subst_gram   : X = B R^{-1} by row-wise substitution, optionally written
//                      out, fused with G = X^T X (Algorithm 1 steps 1 and 3 and
//                      steps 3 of Algorithms 4/5);
//   * k_reduce_parts : fixed-order sum of the per-CTA partial sums (the
//                      paper's MPI reduce of local Grams, Section 2.4).
//
// On GB300 the FP64 pipe issues about 2 FMAs per clock per SM (64 times fewer
// than FP32), so these kernels are bound by FP64 arithmetic, not by HBM: they
// are written to issue nothing but useful DFMAs on the FP64 pipe; the random
// numbers, conversions, finiteness checks and address arithmetic all run on
// the FP32/integer pipes alongside.
#include "rxr_internal.cuh"

namespace rxr {

// ---------------------------------------------------------------------------
// Omega test hook: d_z[(i - row0) * s + r]
// ---------------------------------------------------------------------------
__global__ void k_omega(uint64_t seed, int64_t s, int64_t row0, int64_t rows, float *__restrict__ z)
{
    const int64_t calls_per_row = (s + 3) / 4;
    const int64_t total = rows * calls_per_row;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < total;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c / calls_per_row;
        const uint32_t k = (uint32_t)(c % calls_per_row);
        float v[4];
        rxr_normal4(seed, (uint64_t)(row0 + i), k, 0u, v);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int64_t r = 4 * (int64_t)k + t;
            if (r < s) z[i * s + r] = v[t];
        }
    }
}

// ---------------------------------------------------------------------------
// Panel staging: rows [r0, r0 + P) x columns [c0, c0 + nc) of a column-major
// matrix into shared memory, column-major with leading dimension P.  With a
// valid tensor map one thread issues a 2-D TMA box load (rows past m arrive as
// zeros); otherwise all threads copy with coalesced loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool load_panel(double *dst, const CUtensorMap *map, bool use_tma, uint64_t *bar,
                                           uint32_t &phase, const double *__restrict__ src, int64_t ld, int64_t m,
                                           int64_t r0, int c0, int P, int nc, int ncols_total, RxrStatus *st,
                                           bool skip_copy = false)
{
    if (use_tma) {
        // skip_copy (the stall test hook): nothing arrives, the wait runs out
        if (threadIdx.x == 0 && !skip_copy) {
            mbar_arrive_expect_tx(bar, (uint32_t)(P * nc * 8));
            tma_load_2d(dst, map, (int)r0, c0, bar);
        }
        const bool ok = mbar_wait_bounded(bar, phase, st);
        phase ^= 1u;
        // every thread leaves with the same decision (no thread left at a barrier)
        return __syncthreads_or(ok ? 0 : 1) == 0;
    }
    const int total = P * nc;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int row = e % P, col = e / P;
        const int64_t gr = r0 + row;
        dst[e] = (gr < m && c0 + col < ncols_total) ? src[gr + (int64_t)(c0 + col) * ld] : 0.0;
    }
    // the panel is read by other threads than those that loaded it (element e
    // comes from thread e mod blockDim.x): every load lands before any use
    __syncthreads();
    return true;
}

// Row-wise substitution x R = b in shared memory with two lanes per row (lane
// parity h takes the columns k = h mod 2): for each column j both lanes form
// their partial sums, the pair exchanges them by one shuffle, and the lane
// that owns column j (j mod 2 = h) writes x_j = (b_j - sum) / R_jj.  Only the
// owner ever reads x_j again.  x is column-major with leading dimension xs;
// R is packed by columns (packed = true: column j at j (j + 1) / 2) or square
// with leading dimension 64.  Every lane of the block must call this.
__device__ __forceinline__ void pair_substitute(double *x, int xs, const double *r, const double *dinv, int n, int row,
                                                int h, bool packed)
{
    for (int j = 0; j < n; ++j) {
        const double *rc = packed ? r + j * (j + 1) / 2 : r + j * 64;
        const bool owner = (j & 1) == h;
        double acc = owner ? x[j * xs + row] : 0.0;
#pragma unroll 4
        for (int k = h; k < j; k += 2) acc = fma(-x[k * xs + row], rc[k], acc);
        const double other = __shfl_xor_sync(0xFFFFFFFFu, acc, 1);
        if (owner) x[j * xs + row] = (acc + other) * dinv[j];
    }
}

// ---------------------------------------------------------------------------
// Sketch Y = Omega A in FP64.  grid.x = row chunks (contiguous runs of P-row
// panels), grid.y = (s-tile, n-tile) output tiles of at most 128 x 64.  Each
// thread owns an 8 x 4 register block of the tile; when the tile is small the
// CTA splits into `ngroups` row groups that walk interleaved rows and are
// summed in a fixed order at the end.  Omega's column for each row of A is
// generated into shared memory once per panel; the unscaled sum
// Ypart = sum_i z_i a_i^T is written per chunk (the scale 1/sqrt(s) is
// applied by the reduction).
// ---------------------------------------------------------------------------
constexpr int kSkP = 64;      // rows per panel
constexpr int kSkSTile = 128; // max sketch rows per tile
constexpr int kSkNTile = 64;  // max columns per tile

// row0: the global index of A's first row (Omega's columns follow the global
// rows, so a row shard's partial sketch is its share of the whole one)
__device__ __forceinline__ void sketch_body(const CUtensorMap *tmapA, int use_tma, const double *__restrict__ A,
                                            int64_t lda, int64_t m, int n, int s, uint64_t seed, int64_t panels_total,
                                            int64_t panels_per_cta, int box_cols, double *__restrict__ Ypart,
                                            RxrStatus *st, int bx, int by, int64_t row0 = 0)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *ap = reinterpret_cast<double *>(smem_raw);  // [kSkNTile][kSkP]
    double *zp = ap + kSkNTile * kSkP;                   // [kSkP][kSkSTile]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int bad_flag;

    const int n_tiles = (n + kSkNTile - 1) / kSkNTile;
    const int si = by / n_tiles, ni = by % n_tiles;
    const int s0 = si * kSkSTile, c0 = ni * kSkNTile;
    const int sw = min(kSkSTile, s - s0), nw = min(kSkNTile, n - c0);
    const int ts = (sw + 7) / 8, tn = (nw + 3) / 4;
    const int tg = ts * tn;
    const int ngroups = RXR_THREADS / tg;
    const int g = threadIdx.x / tg, lt = threadIdx.x % tg;
    const bool active = g < ngroups;
    const int sb = lt / tn, nb = lt % tn;
    const int k0 = s0 / 4, kcount = (sw + 3) / 4;  // Philox calls per row for this tile

    if (threadIdx.x == 0) {
        bad_flag = 0;
        if (use_tma) {
            mbar_init(&bar, 1);
            fence_barrier_init();
        }
    }
    // zero the padding columns once (TMA writes only the first nw columns)
    for (int e = threadIdx.x; e < kSkNTile * kSkP; e += blockDim.x) ap[e] = 0.0;
    __syncthreads();
    uint32_t phase = 0;

    double acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

    const int64_t p_begin = bx * panels_per_cta;
    const int64_t p_end = min(panels_total, p_begin + panels_per_cta);
    const bool stall = use_tma && bx == 0 && by == 0 && rxr_stall_requested(st);
    for (int64_t p = p_begin; p < p_end; ++p) {
        const int64_t r0 = p * kSkP;
        if (!load_panel(ap, tmapA, use_tma, &bar, phase, A, lda, m, r0, c0, kSkP, box_cols, n, st,
                        stall && p == p_begin))
            return;
        // Omega columns for the panel's rows: zp[row][r - s0]
        for (int c = threadIdx.x; c < kSkP * kcount; c += blockDim.x) {
            const int row = c / kcount, kk = c % kcount;
            float v[4];
            rxr_normal4(seed, (uint64_t)(row0 + r0 + row), (uint32_t)(k0 + kk), 0u, v);
            double *zr = zp + row * kSkSTile + 4 * kk;
#pragma unroll
            for (int t = 0; t < 4; ++t) zr[t] = rxr_f2d_exact(v[t]);
        }
        // non-finite entries of A (integer test on the loaded panel)
        {
            bool bad = false;
            for (int e = threadIdx.x; e < kSkP * nw; e += blockDim.x) bad |= rxr_nonfinite(ap[e]);
            if (bad) bad_flag = 1;
        }
        __syncthreads();
        if (active) {
            // rows g, g + ngroups, ... of the panel, visited in an order rotated
            // by nb so that threads of a warp read different shared-memory banks
            const int cnt = (kSkP - g + ngroups - 1) / ngroups;
            for (int i = 0; i < cnt; ++i) {
                int ii = i + nb;
                ii = (ii >= cnt) ? ii - cnt * (ii / cnt) : ii;
                const int row = g + ii * ngroups;
                const double *zr = zp + row * kSkSTile + sb * 8;
                double zv[8], av[4];
#pragma unroll
                for (int a = 0; a < 8; ++a) zv[a] = zr[a];
#pragma unroll
                for (int b = 0; b < 4; ++b) av[b] = ap[(nb * 4 + b) * kSkP + row];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(zv[a], av[b], acc[a][b]);
            }
        }
        __syncthreads();
    }
    if (bad_flag) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);

    // combine the row groups in a fixed order (group 0 first)
    double *out = Ypart + (int64_t)bx * s * n;
    if (ngroups == 1) {
        // threads past the one group (tg < 256) hold no sums: only the group writes
        if (active)
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int r = s0 + sb * 8 + a, c = c0 + nb * 4 + b;
                    if (r < s && c < n) out[r + (int64_t)c * s] = acc[a][b];
                }
        return;
    }
    double *red = reinterpret_cast<double *>(smem_raw);  // [ngroups][tg][32]
    if (active) {
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) red[((int64_t)g * tg + lt) * 32 + a * 4 + b] = acc[a][b];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tg * 32; e += blockDim.x) {
        const int l = e / 32, ab = e % 32;
        const int r = s0 + (l / tn) * 8 + ab / 4, c = c0 + (l % tn) * 4 + ab % 4;
        double v = red[e];
        for (int gg = 1; gg < ngroups; ++gg) v += red[(int64_t)gg * tg * 32 + e];
        if (r < s && c < n) out[r + (int64_t)c * s] = v;
    }
}

__global__ void __launch_bounds__(RXR_THREADS, 2)
    k_sketch_fp64(const __grid_constant__ CUtensorMap tmapA, int use_tma, const double *__restrict__ A, int64_t lda,
                  int64_t m, int n, int s, uint64_t seed, int64_t panels_total, int64_t panels_per_cta,
                  int box_cols, double *__restrict__ Ypart, RxrStatus *st, int64_t row0)
{
    sketch_body(&tmapA, use_tma, A, lda, m, n, s, seed, panels_total, panels_per_cta, box_cols, Ypart, st,
                blockIdx.x, blockIdx.y, row0);
}

// ---------------------------------------------------------------------------
// out[r + c*ldo] = scale * sum_{x < nparts} parts[x*stride + r + c*rows], in
// the order x = 0, 1, ...  (deterministic).  With `symmetric`, only entries
// r <= c are summed and mirrored (Gram matrices).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void reduce_body(const double *__restrict__ parts, int nparts, int64_t stride, int rows,
                                            int cols, double scale, int symmetric, double *__restrict__ out,
                                            int64_t ldo, RxrStatus *st, int bx, int nbx)
{
    if (rxr_failed_block(st)) return;
    const int64_t total = (int64_t)rows * cols;
    if (nparts >= kReduceWarpParts) {
        // many partial sums: one warp per output, lane l adding partials l,
        // l + 32, ..., then a fixed shuffle tree (lane 0's order is fixed)
        const int lane = threadIdx.x & 31;
        const int64_t w0 = (bx * (int64_t)blockDim.x + threadIdx.x) >> 5, nw = ((int64_t)nbx * blockDim.x) >> 5;
        for (int64_t e = w0; e < total; e += nw) {
            const int r = (int)(e % rows), c = (int)(e / rows);
            if (symmetric && r > c) continue;
            double v = 0.0;
            for (int x = lane; x < nparts; x += 32) v += parts[x * stride + e];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            if (lane == 0) {
                v *= scale;
                out[r + c * ldo] = v;
                if (symmetric && r != c) out[c + r * ldo] = v;
            }
        }
        return;
    }
    for (int64_t e = bx * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)nbx * blockDim.x) {
        const int r = (int)(e % rows), c = (int)(e / rows);
        if (symmetric && r > c) continue;
        double v = 0.0;
        for (int x = 0; x < nparts; ++x) v += parts[x * stride + e];
        v *= scale;
        out[r + c * ldo] = v;
        if (symmetric && r != c) out[c + r * ldo] = v;
    }
}

// ---------------------------------------------------------------------------
// Row extraction (Section 2.3; Theorem 3.2's equal-probability case): row k
// of Y is row idx_k of A, idx_k = floor(u_k m / 2^64) with u_k = out0 +
// 2^32 out1 of Philox4x32-10 at counter (k_lo, k_hi, 0, 3), key (seed_lo,
// seed_hi) -- independent draws, each row with probability 1/m.  One warp per
// drawn row, lanes across the columns.
// ---------------------------------------------------------------------------
__global__ void k_sketch_rows(const double *__restrict__ A, int64_t lda, int64_t m, int n, int64_t l, uint64_t seed,
                              double *__restrict__ Y, int64_t ldy, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    const int lane = threadIdx.x & 31;
    const int64_t k = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= l) return;
    uint32_t c0 = (uint32_t)k, c1 = (uint32_t)((uint64_t)k >> 32), c2 = 0u, c3 = 3u;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t u = (uint64_t)c0 | ((uint64_t)c1 << 32);
    const int64_t i = (int64_t)__umul64hi(u, (uint64_t)m);
    bool bad = false;
    for (int j = lane; j < n; j += 32) {
        const double v = A[i + (int64_t)j * lda];
        bad |= rxr_nonfinite(v);
        Y[k + (int64_t)j * ldy] = v;
    }
    if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);
}

// NaN or Inf anywhere in A (m x n, lda) -> RXR_ERR_NONFINITE (grid-stride).
__global__ void k_check_finite(const double *__restrict__ A, int64_t lda, int64_t m, int n, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    bool bad = false;
    const int64_t total = m * (int64_t)n, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride)
        bad |= rxr_nonfinite(A[e % m + (e / m) * lda]);
    if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);
}

__global__ void k_reduce_parts(const double *__restrict__ parts, int nparts, int64_t stride, int rows, int cols,
                               double scale, int symmetric, double *__restrict__ out, int64_t ldo, RxrStatus *st)
{
    reduce_body(parts, nparts, stride, rows, cols, scale, symmetric, out, ldo, st, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// X = B R^{-1} (row-wise forward substitution, x R = b) fused with the Gram
// G += X^T X.  B is read from `src` (A or the previous pass's X), X optionally
// written to `dst` (may equal src: each panel is read completely before it is
// written).  R (n x n upper, global) is packed into shared memory column by
// column and read as a broadcast; 1/R_jj is precomputed.  Panel = P rows,
// one thread per row for the substitution; for the Gram each thread owns up
// to MAXT 4 x 4 tiles of the upper triangle.  unit_r skips the substitution
// (R = I, plain CholeskyQR).
// ---------------------------------------------------------------------------
constexpr int kSgP = 128;

template <int MAXT>
__device__ __forceinline__ void subst_gram_body(const CUtensorMap *tmapB, int use_tma, const double *__restrict__ src,
                                                int64_t lds, int64_t m, int n, const double *__restrict__ R,
                                                int64_t ldr, int unit_r, double *dst, int64_t ldd, int do_gram,
                                                double *__restrict__ Gpart, int64_t panels_total,
                                                int64_t panels_per_cta, int check_finite, RxrStatus *st, int bx)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int n4 = (n + 3) & ~3;
    double *xp = reinterpret_cast<double *>(smem_raw);  // [n4][kSgP]
    double *rp = xp + (int64_t)n4 * kSgP;                // packed upper R: column j at j(j+1)/2
    double *dinv = rp + (int64_t)n * (n + 1) / 2;        // [n]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int bad_flag;

    if (threadIdx.x == 0) {
        bad_flag = 0;
        if (use_tma) {
            mbar_init(&bar, 1);
            fence_barrier_init();
        }
    }
    for (int e = threadIdx.x; e < n4 * kSgP; e += blockDim.x) xp[e] = 0.0;
    if (!unit_r) {
        for (int j = 0; j < n; ++j)
            for (int k = threadIdx.x; k <= j; k += blockDim.x) rp[j * (j + 1) / 2 + k] = R[k + j * ldr];
        for (int j = threadIdx.x; j < n; j += blockDim.x) dinv[j] = 1.0 / R[j + j * ldr];
    }
    __syncthreads();
    uint32_t phase = 0;

    // Gram tiles owned by this thread.  The upper triangle is cut into 4 x 4
    // tiles; the NT(NT-1)/2 off-diagonal tiles are numbered first and the NT
    // diagonal tiles start at the next multiple of 32, so that no warp mixes
    // the two kinds (a diagonal tile needs 10 FMAs per row, an off-diagonal
    // one 16; a mixed warp would issue both sequences).  Thread t owns entries
    // t, t + 256, ... of that list.
    const int NT = n4 / 4;
    const int n_off = NT * (NT - 1) / 2;
    const int d0 = (n_off + 31) & ~31;
    int tbj[MAXT], tbl[MAXT];
    double acc[MAXT][16];
#pragma unroll
    for (int q = 0; q < MAXT; ++q) {
        const int e = threadIdx.x + q * RXR_THREADS;
        int bj = -1, bl = -1;
        if (do_gram) {
            if (e < n_off) {
                int rem = e;
                bj = 0;
                while (rem >= NT - 1 - bj) {
                    rem -= NT - 1 - bj;
                    ++bj;
                }
                bl = bj + 1 + rem;
            } else if (e >= d0 && e - d0 < NT) {
                bj = bl = e - d0;
            }
        }
        tbj[q] = bj;
        tbl[q] = bl;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc[q][k] = 0.0;
    }

    const int64_t p_begin = bx * panels_per_cta;
    const int64_t p_end = min(panels_total, p_begin + panels_per_cta);
    for (int64_t p = p_begin; p < p_end; ++p) {
        const int64_t r0 = p * kSgP;
        if (!load_panel(xp, tmapB, use_tma, &bar, phase, src, lds, m, r0, 0, kSgP, n, n, st)) return;
        if (check_finite) {
            bool bad = false;
            for (int e = threadIdx.x; e < kSgP * n; e += blockDim.x) bad |= rxr_nonfinite(xp[e]);
            if (bad) bad_flag = 1;
        }
        // substitution, one thread per row: x_j = (b_j - sum_{k<j} x_k R_kj) / R_jj
        // as one FMA chain seeded with b_j (no FP64 operation beyond the
        // n(n-1)/2 FMAs and n multiplications by 1/R_jj)
        if (!unit_r) {
            if (n <= 64) {
                // narrow rows run two CTAs per SM: one thread per row, one chain
                if (threadIdx.x < kSgP) {
                    const int t = threadIdx.x;
                    for (int j = 0; j < n; ++j) {
                        const double *rc = rp + j * (j + 1) / 2;
                        double accj = xp[j * kSgP + t];
#pragma unroll 4
                        for (int k = 0; k < j; ++k) accj = fma(-xp[k * kSgP + t], rc[k], accj);
                        xp[j * kSgP + t] = accj * dinv[j];
                    }
                }
            } else {
                // wide rows fit one CTA per SM; two lanes per row keep two warps
                // per scheduler busy (ncu: one working warp per scheduler left
                // the FP64 pipe 27 % idle)
                pair_substitute(xp, kSgP, rp, dinv, n, threadIdx.x >> 1, threadIdx.x & 1, true);
            }
        }
        __syncthreads();
        if (dst != nullptr) {
            for (int e = threadIdx.x; e < kSgP * n; e += blockDim.x) {
                const int row = e % kSgP, col = e / kSgP;
                const int64_t gr = r0 + row;
                if (gr < m) dst[gr + (int64_t)col * ldd] = xp[e];
            }
        }
        if (do_gram) {
#pragma unroll
            for (int q = 0; q < MAXT; ++q) {
                const int bj = tbj[q], bl = tbl[q];
                if (bj < 0) continue;
                const double *cj = xp + (bj * 4) * kSgP;
                const double *cl = xp + (bl * 4) * kSgP;
                // rows visited from a per-tile offset so that the threads of a
                // warp (different tiles, same step) hit different banks
                const int rot = threadIdx.x & 31;
                if (bj == bl) {
                    for (int i = 0; i < kSgP; ++i) {
                        const int r = (i + rot) & (kSgP - 1);
                        const double x0 = cj[r], x1 = cj[kSgP + r], x2 = cj[2 * kSgP + r], x3 = cj[3 * kSgP + r];
                        acc[q][0] = fma(x0, x0, acc[q][0]);
                        acc[q][1] = fma(x0, x1, acc[q][1]);
                        acc[q][2] = fma(x0, x2, acc[q][2]);
                        acc[q][3] = fma(x0, x3, acc[q][3]);
                        acc[q][5] = fma(x1, x1, acc[q][5]);
                        acc[q][6] = fma(x1, x2, acc[q][6]);
                        acc[q][7] = fma(x1, x3, acc[q][7]);
                        acc[q][10] = fma(x2, x2, acc[q][10]);
                        acc[q][11] = fma(x2, x3, acc[q][11]);
                        acc[q][15] = fma(x3, x3, acc[q][15]);
                    }
                } else {
                    for (int i = 0; i < kSgP; ++i) {
                        const int r = (i + rot) & (kSgP - 1);
                        double u[4], v[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            u[a] = cj[a * kSgP + r];
                            v[a] = cl[a * kSgP + r];
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[q][a * 4 + b] = fma(u[a], v[b], acc[q][a * 4 + b]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (bad_flag) rxr_fail(st, RXR_ERR_NONFINITE, 0, -1);
    if (do_gram) {
        double *out = Gpart + (int64_t)bx * n * n;
#pragma unroll
        for (int q = 0; q < MAXT; ++q) {
            const int bj = tbj[q], bl = tbl[q];
            if (bj < 0) continue;
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int r = bj * 4 + a, c = bl * 4 + b;
                    if (r < n && c < n && r <= c) out[r + (int64_t)c * n] = acc[q][a * 4 + b];
                }
        }
    }
}

template <int MAXT>
__global__ void __launch_bounds__(RXR_THREADS)
    k_subst_gram(const __grid_constant__ CUtensorMap tmapB, int use_tma, const double *__restrict__ src, int64_t lds,
                 int64_t m, int n, const double *__restrict__ R, int64_t ldr, int unit_r, double *dst, int64_t ldd,
                 int do_gram, double *__restrict__ Gpart, int64_t panels_total, int64_t panels_per_cta,
                 int check_finite, RxrStatus *st)
{
    subst_gram_body<MAXT>(&tmapB, use_tma, src, lds, m, n, R, ldr, unit_r, dst, ldd, do_gram, Gpart, panels_total,
                          panels_per_cta, check_finite, st, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Batched forms: one launch per stage serves every problem of a batch.  Work
// item b (a row chunk or a reduction block of one problem) belongs to the
// problem k with start[k] <= b < start[k+1] (binary search over the per-stage
// item offsets); the problem's own block index is b - start[k].  Panels are
// staged with plain coalesced loads (no per-problem tensor maps).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_job(const int *__restrict__ start, int count, int b)
{
    int lo = 0, hi = count;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= b)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Persistent forms: gridDim.x CTAs pull work items b = 0 .. total - 1 (a
// problem's row chunk, or its reduction block) from the device counter
// *next (zeroed before the launch) until the queue is empty; item b belongs
// to the problem k with start[k] <= b < start[k+1].
__device__ __forceinline__ int next_item(int *next)
{
    __shared__ int item;
    __syncthreads();  // every thread has read the previous item (and the CTA's shared memory is free)
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    return item;
}

__global__ void __launch_bounds__(RXR_THREADS, 2)
    k_sketch_fp64_batched(const SketchJob *__restrict__ jobs, const int *__restrict__ start, int count, int total,
                          int *next)
{
    for (int b = next_item(next); b < total; b = next_item(next)) {
        const int k = find_job(start, count, b);
        const SketchJob j = jobs[k];
        const int local = b - start[k];
        sketch_body(nullptr, 0, j.A, j.lda, j.m, j.n, j.s, j.seed, j.panels_total, j.panels_per_cta, j.box_cols,
                    j.Ypart, j.st, local % j.gx, local / j.gx);
    }
}

__global__ void k_reduce_parts_batched(const ReduceJob *__restrict__ jobs, const int *__restrict__ start, int count,
                                       int total, int *next)
{
    for (int b = next_item(next); b < total; b = next_item(next)) {
        const int k = find_job(start, count, b);
        const ReduceJob j = jobs[k];
        reduce_body(j.parts, j.nparts, j.stride, j.rows, j.cols, j.scale, j.symmetric, j.out, j.ldo, j.st,
                    b - start[k], start[k + 1] - start[k]);
    }
}

// do_gram < 0 keeps each job's own flag; 0 or 1 overrides it for all jobs
__global__ void __launch_bounds__(RXR_THREADS)
    k_subst_gram_batched(const SubstJob *__restrict__ jobs, const int *__restrict__ start, int count, int do_gram,
                         int total, int *next)
{
    for (int b = next_item(next); b < total; b = next_item(next)) {
        const int k = find_job(start, count, b);
        const SubstJob j = jobs[k];
        subst_gram_body<3>(nullptr, 0, j.src, j.lds, j.m, j.n, j.R, j.ldr, j.unit_r, j.dst, j.ldd,
                           do_gram < 0 ? j.do_gram : do_gram, j.Gpart, j.panels_total, j.panels_per_cta,
                           j.check_finite, j.st, b - start[k]);
    }
}

// ---------------------------------------------------------------------------
// Wide panels (n > 128): R no longer fits in shared memory next to a panel.
// k_subst_wide: X = B R^{-1} by 64-column blocks, per panel of 128 rows:
//   X_J = (B_J - sum_{I<J} X_I R_IJ) R_JJ^{-1}.
// The sum is a register-tiled FP64 product (each thread owns 4 rows x 8
// columns of the block) with X_I (already written to dst by this CTA) and R_IJ
// staged through shared memory; the diagonal block is solved by row-wise
// substitution.  dst may equal src (block J of B is read before X_J is written).
// k_gram_tiles: G_IJ = X_I^T X_J for the 64 x 64 blocks I <= J of the upper
// triangle (grid.y = block pair), per row chunk, fixed-order partials.
// ---------------------------------------------------------------------------
constexpr int kWP = 128;  // rows per panel
constexpr int kWB = 64;   // column block

// A 128-row x 64-column block of a column-major matrix into shared memory
// (column-major, leading dimension 128), zeros outside rows < m and columns <
// ncols; 256 threads, 16 loads in flight per thread.
__device__ __forceinline__ void load_block_128x64(double *dst, const double *__restrict__ src, int64_t ld, int64_t m,
                                                  int64_t r0, int c0, int ncols)
{
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        double v[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = threadIdx.x + 256 * (16 * b + t);
            const int row = e & 127, col = e >> 7;
            const int64_t gr = r0 + row;
            v[t] = (gr < m && c0 + col < ncols) ? src[gr + (int64_t)(c0 + col) * ld] : 0.0;
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) dst[threadIdx.x + 256 * (16 * b + t)] = v[t];
    }
}


__global__ void __launch_bounds__(RXR_THREADS, 1)
    k_subst_wide(const double *__restrict__ src, int64_t lds, int64_t m, int n, const double *__restrict__ R,
                 int64_t ldr, double *dst, int64_t ldd, int64_t panels_total, int64_t panels_per_cta, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *ut = reinterpret_cast<double *>(smem_raw);  // [kWB][kWP] block being solved
    double *xi = ut + kWB * kWP;                          // [kWB][kWP] an earlier block of X
    double *rb = xi + kWB * kWP;                          // [kWB cols][kWB rows] block of R
    double *dv = rb + kWB * kWB;                          // [kWB] 1 / R_jj
    const int tid = threadIdx.x;
    const int tr = tid & 31, tc = tid >> 5;  // thread tile: rows 4 tr..4 tr+3, columns 8 tc..8 tc+7
    const int nb = (n + kWB - 1) / kWB;
    const int64_t p_begin = blockIdx.x * panels_per_cta;
    const int64_t p_end = min(panels_total, p_begin + panels_per_cta);
    for (int64_t p = p_begin; p < p_end; ++p) {
        const int64_t r0 = p * kWP;
        for (int J = 0; J < nb; ++J) {
            const int cJ = J * kWB, wJ = min(kWB, n - cJ);
            double acc[4][8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const int64_t gr = r0 + 4 * tr + a;
                    const int c = 8 * tc + b;
                    acc[a][b] = (gr < m && c < wJ) ? src[gr + (int64_t)(cJ + c) * lds] : 0.0;
                }
            for (int I = 0; I < J; ++I) {
                const int cI = I * kWB;
                __syncthreads();
                load_block_128x64(xi, dst, ldd, m, r0, cI, n);
                for (int e = tid; e < kWB * kWB; e += blockDim.x) {
                    const int k = e % kWB, c = e / kWB;
                    rb[e] = (c < wJ) ? R[(cI + k) + (int64_t)(cJ + c) * ldr] : 0.0;
                }
                __syncthreads();
#pragma unroll 2
                for (int k = 0; k < kWB; ++k) {
                    double xv[4], rv[8];
#pragma unroll
                    for (int a = 0; a < 4; ++a) xv[a] = xi[k * kWP + 4 * tr + a];
#pragma unroll
                    for (int b = 0; b < 8; ++b) rv[b] = rb[(8 * tc + b) * kWB + k];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 8; ++b) acc[a][b] = fma(-xv[a], rv[b], acc[a][b]);
                }
            }
            __syncthreads();
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) ut[(8 * tc + b) * kWP + 4 * tr + a] = acc[a][b];
            for (int e = tid; e < kWB * kWB; e += blockDim.x) {
                const int k = e % kWB, c = e / kWB;
                rb[e] = (c < wJ && k < wJ) ? R[(cJ + k) + (int64_t)(cJ + c) * ldr] : 0.0;
            }
            if (tid < kWB) dv[tid] = (tid < wJ) ? 1.0 / R[(cJ + tid) + (int64_t)(cJ + tid) * ldr] : 0.0;
            __syncthreads();
            pair_substitute(ut, kWP, rb, dv, wJ, tid >> 1, tid & 1, false);
            __syncthreads();
            for (int e = tid; e < kWB * kWP; e += blockDim.x) {
                const int row = e % kWP, col = e / kWP;
                const int64_t gr = r0 + row;
                if (gr < m && col < wJ) dst[gr + (int64_t)(cJ + col) * ldd] = ut[e];
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(RXR_THREADS)
    k_gram_tiles(const double *__restrict__ X, int64_t ldx, int64_t m, int n, int64_t panels_total,
                 int64_t panels_per_cta, double *__restrict__ Gpart, RxrStatus *st)
{
    if (rxr_failed_block(st)) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    double *xa = reinterpret_cast<double *>(smem_raw);  // [kWB][kWP]
    double *xb = xa + kWB * kWP;
    const int nb = (n + kWB - 1) / kWB;
    // block pair (I, J), I <= J, from blockIdx.y
    int I = 0, rem = blockIdx.y;
    while (rem >= nb - I) {
        rem -= nb - I;
        ++I;
    }
    const int J = I + rem;
    const int cI = I * kWB, cJ = J * kWB;
    const int tid = threadIdx.x, ti = tid & 15, tj = tid >> 4;  // 4 x 4 outputs per thread
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    const int64_t p_begin = blockIdx.x * panels_per_cta;
    const int64_t p_end = min(panels_total, p_begin + panels_per_cta);
    for (int64_t p = p_begin; p < p_end; ++p) {
        const int64_t r0 = p * kWP;
        __syncthreads();
        load_block_128x64(xa, X, ldx, m, r0, cI, n);
        if (J != I) load_block_128x64(xb, X, ldx, m, r0, cJ, n);
        __syncthreads();
        const int rot = tid & 31;
        for (int i = 0; i < kWP; ++i) {
            const int r = (i + rot) & (kWP - 1);
            double u[4], v[4];
            const double *xv = (J != I) ? xb : xa;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                u[a] = xa[(4 * ti + a) * kWP + r];
                v[a] = xv[(4 * tj + a) * kWP + r];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fma(u[a], v[b], acc[a][b]);
        }
    }
    double *out = Gpart + (int64_t)blockIdx.x * n * n;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = cI + 4 * ti + a, c = cJ + 4 * tj + b;
            if (r < n && c < n && r <= c) out[r + (int64_t)c * n] = acc[a][b];
        }
}

cudaError_t set_wide_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_subst_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((2 * kWB * kWP + kWB * kWB + kWB) * sizeof(double)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_gram_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * kWB * kWP * sizeof(double)));
    return e;
}

// Host-side dispatch over the tile count (template kernels stay in this unit).
cudaError_t launch_subst_gram(int maxt, dim3 grid, size_t smem, cudaStream_t st, const CUtensorMap &map, int use_tma,
                              const double *src, int64_t lds, int64_t m, int n, const double *R, int64_t ldr,
                              int unit_r, double *dst, int64_t ldd, int do_gram, double *Gpart, int64_t panels_total,
                              int64_t panels_per_cta, int check_finite, RxrStatus *status)
{
    switch (maxt) {
    case 1:
        k_subst_gram<1><<<grid, RXR_THREADS, smem, st>>>(map, use_tma, src, lds, m, n, R, ldr, unit_r, dst, ldd,
                                                         do_gram, Gpart, panels_total, panels_per_cta, check_finite,
                                                         status);
        break;
    case 2:
        k_subst_gram<2><<<grid, RXR_THREADS, smem, st>>>(map, use_tma, src, lds, m, n, R, ldr, unit_r, dst, ldd,
                                                         do_gram, Gpart, panels_total, panels_per_cta, check_finite,
                                                         status);
        break;
    default:
        k_subst_gram<3><<<grid, RXR_THREADS, smem, st>>>(map, use_tma, src, lds, m, n, R, ldr, unit_r, dst, ldd,
                                                         do_gram, Gpart, panels_total, panels_per_cta, check_finite,
                                                         status);
        break;
    }
    return cudaGetLastError();
}

cudaError_t set_batched_smem(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_sketch_fp64_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subst_gram_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

cudaError_t set_subst_gram_smem(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_subst_gram<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subst_gram<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_subst_gram<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

}  // namespace rxr
