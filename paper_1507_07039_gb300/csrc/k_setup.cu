// One-time kernels of panda_create / panda_set_state: input validation, the
// Z-score of each network (Section II-A, NormalizeNetwork) with FP64
// statistics, stripping the diagonals of P and C into FP64 vectors, the
// transposed copy of W and the initial squared norms.
//
// Every reduction here runs with a fixed grid and a fixed summation order, so
// results are identical from run to run.
#include "panda_internal.cuh"

namespace panda {

namespace {

constexpr int RED_BLOCKS = 1024;
constexpr int RED_THREADS = 256;

// flags[0] |= 1 on a non-finite entry (rows x cols, row stride ld): block b
// reads rows b, b + gridDim.x, ... along the row.
__global__ void k_check_finite(const float *__restrict__ X, int rows, int cols, int ld, int *flags)
{
    int bad = 0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x)
        for (int c = threadIdx.x; c < cols; c += blockDim.x)
            bad |= !isfinite(X[(size_t)r * ld + c]);
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(&flags[0], 1);
}

// A square n x n matrix as 32 x 32 blocks: each pair of mirror blocks (bi, bj)
// and (bj, bi), bi <= bj, is read once, along rows, into shared memory, so the
// whole matrix is read once and coalesced.  flags[0] |= 1 on a non-finite
// entry, flags[1] |= 1 when X[i][j] != X[j][i].  Pairs are numbered column by
// column of the upper triangle: pair t has bj = the largest j with
// j(j+1)/2 <= t and bi = t - bj(bj+1)/2.  256 threads.
__global__ void k_check_finite_sym(const float *__restrict__ X, int n, int ld, int npairs, int *flags)
{
    __shared__ float a[32][33], b[32][33];
    __shared__ int pij[2];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    int bad = 0, asym = 0;
    for (int t = blockIdx.x; t < npairs; t += gridDim.x) {
        if (threadIdx.x == 0) {
            // 8t + 1 < 2^24 for n <= 46000, so the FP32 square root is close; the loops correct it
            int j = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
            while (j > 0 && (long long)j * (j + 1) / 2 > t)
                --j;
            while ((long long)(j + 1) * (j + 2) / 2 <= t)
                ++j;
            pij[0] = t - (int)((long long)j * (j + 1) / 2);
            pij[1] = j;
        }
        __syncthreads();
        const int i0 = pij[0] * 32, j0 = pij[1] * 32;
#pragma unroll
        for (int k = ty; k < 32; k += 8) {
            const int ra = i0 + k, ca = j0 + tx, rb = j0 + k, cb = i0 + tx;
            a[k][tx] = (ra < n && ca < n) ? X[(size_t)ra * ld + ca] : 0.0f;
            b[k][tx] = (rb < n && cb < n) ? X[(size_t)rb * ld + cb] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = ty; k < 32; k += 8) {
            // a[k][tx] = X[i0 + k][j0 + tx], its mirror X[j0 + tx][i0 + k] = b[tx][k]
            const float v = a[k][tx];
            bad |= !isfinite(v) | !isfinite(b[k][tx]);
            asym |= (i0 + k < n && j0 + tx < n && v != b[tx][k]);
        }
        __syncthreads();
    }
    bad = __syncthreads_or(bad);
    asym = __syncthreads_or(asym);
    if (threadIdx.x == 0) {
        if (bad)
            atomicOr(&flags[0], 1);
        if (asym)
            atomicOr(&flags[1], 1);
    }
}

__device__ double block_sum_fixed(double v, double *sh)
{
    // fixed-shape tree: the result does not depend on scheduling
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// The FP32 pairs the element kernels use, stored after the FP64 statistics:
// stats[0] = mean, stats[1] = population std, then as floats (16-byte
// aligned) mean = mh + ml and 1 / std = rh + rl, each to about 2^-48.
__device__ __forceinline__ float4 *stats_pairs(double *stats) { return reinterpret_cast<float4 *>(stats + 2); }
__device__ __forceinline__ float4 stats_pairs(const double *stats)
{
    return *reinterpret_cast<const float4 *>(stats + 2);
}

// x - (mh + ml) = s + t: s = fl(x - mh) and t its rounding error minus ml
__device__ __forceinline__ void centre(float x, float mh, float ml, float &s, float &t)
{
    float e;
    two_sum(x, -mh, s, e);
    t = __fsub_rn(e, ml);
}

// Adds the terms of one element to a compensated pair: mode 0 adds x; mode 1
// adds (x - mean)^2 = (s + t)^2 = p + (pe + 2 s t + t^2), with s^2 = p + pe
// exact.
template <int MODE>
__device__ __forceinline__ void stats_term(float x, float mh, float ml, float &acc, float &cmp)
{
    if (MODE == 0) {
        two_sum_add(acc, cmp, x);
    } else {
        float s, t, p, pe;
        centre(x, mh, ml, s, t);
        two_prod(s, s, p, pe);
        two_sum_add(acc, cmp, p);
        cmp = __fadd_rn(cmp, __fmaf_rn(t, t, __fmaf_rn(__fmul_rn(2.0f, s), t, pe)));
    }
}

// Partial sums for the Z-score in a fixed order.  Block b takes rows b,
// b + gridDim.x, ...; thread x takes the 4-wide column groups x, x + 256, ...
// of each (rows start 16-byte aligned), then the ragged columns.  A thread's
// terms within one row go into a compensated FP32 pair (TwoSum), the pair
// into the thread's FP64 total at the row's end, and the block's totals
// through a fixed tree.  Mode 0: sum of x.  Mode 1: sum of (x - mean)^2,
// mean from stats (the difference kept as an FP32 pair, its square from
// two_prod).  About as accurate as FP64 sums of the FP32 entries, on the FP32
// pipe.
template <int MODE>
__global__ void k_stats_partial(const float *__restrict__ X, int rows, int cols, int ld, const double *stats,
                                double *partials)
{
    __shared__ double sh[RED_THREADS];
    float mh = 0.0f, ml = 0.0f;
    if (MODE == 1) {
        const float4 q = stats_pairs(stats);
        mh = q.x;
        ml = q.y;
    }
    const int c4n = cols >> 2;
    double tot = 0.0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float *x = X + (size_t)r * ld;
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        float acc = 0.0f, cmp = 0.0f;
#pragma unroll 2
        for (int c = threadIdx.x; c < c4n; c += RED_THREADS) {
            const float4 v = __ldcs(x4 + c);
            stats_term<MODE>(v.x, mh, ml, acc, cmp);
            stats_term<MODE>(v.y, mh, ml, acc, cmp);
            stats_term<MODE>(v.z, mh, ml, acc, cmp);
            stats_term<MODE>(v.w, mh, ml, acc, cmp);
        }
        for (int c = (c4n << 2) + threadIdx.x; c < cols; c += RED_THREADS)
            stats_term<MODE>(x[c], mh, ml, acc, cmp);
        tot += (double)acc + (double)cmp;
    }
    double s = block_sum_fixed(tot, sh);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = s;
}

// Mode 0: stats[0] = mean and its FP32 pair.  Mode 1: stats[1] = population
// std and the FP32 pair of its reciprocal (zero when std is not positive).
__global__ void k_stats_final(const double *partials, int n, double count, int mode, double *stats)
{
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc += partials[i];
    double s = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) {
        float4 *q = stats_pairs(stats);
        if (mode == 0) {
            const double m = s / count;
            stats[0] = m;
            const float mh = (float)m;
            q->x = mh;
            q->y = (float)(m - (double)mh);
        } else {
            const double sd = sqrt(s / count);
            stats[1] = sd;
            const double r = sd > 0.0 ? 1.0 / sd : 0.0;
            const float rh = (float)r;
            q->z = rh;
            q->w = (float)(r - (double)rh);
        }
    }
}

// z = (x - mean) / std (Section II-A, NormalizeNetwork) from the FP32 pairs:
// (s + t) (rh + rl) = s rh + (its exact rounding error + s rl + t rh), the
// terms left out being below 2^-44 of z; the final FP32 addition rounds that
// sum once.  The FP32 result therefore equals the correctly rounded quotient
// except when that lies within about 2^-44 relative of a rounding midpoint.
__device__ __forceinline__ float zscore_one(float x, float4 q)
{
    float s, t, p, pe;
    centre(x, q.x, q.y, s, t);
    two_prod(s, q.z, p, pe);
    return __fadd_rn(p, __fmaf_rn(t, q.z, __fmaf_rn(s, q.w, pe)));
}

// Block b takes rows b, b + gridDim.x, ...; 4-wide column groups, then the
// ragged columns.
__global__ void k_apply_zscore(float *X, int rows, int cols, int ld, const double *stats)
{
    if (!(stats[1] > 0.0))
        return;
    const float4 q = stats_pairs(stats);
    const int c4n = cols >> 2;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        float *x = X + (size_t)r * ld;
        float4 *x4 = reinterpret_cast<float4 *>(x);
#pragma unroll 2
        for (int c = threadIdx.x; c < c4n; c += blockDim.x) {
            float4 v = x4[c];
            v.x = zscore_one(v.x, q);
            v.y = zscore_one(v.y, q);
            v.z = zscore_one(v.z, q);
            v.w = zscore_one(v.w, q);
            x4[c] = v;
        }
        for (int c = (c4n << 2) + threadIdx.x; c < cols; c += blockDim.x)
            x[c] = zscore_one(x[c], q);
    }
}

__global__ void k_split_diag(float *X, int n, int ld, double *d, float *df)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    size_t o = (size_t)i * ld + i;
    double v = (double)X[o];
    d[i] = v;
    df[i] = (float)v;
    X[o] = 0.0f;
}

__global__ void k_diag_to_float(const double *d, float *df, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        df[i] = (float)d[i];
}

// Y (cols_p x rows_p) = X^T (X is rows_p x cols_p); both multiples of 32.
__global__ void k_transpose(const float *__restrict__ X, int rows_p, int cols_p, float *__restrict__ Y)
{
    __shared__ float tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = ty; k < 32; k += 8)
        tile[k][tx] = X[(size_t)(by + k) * cols_p + bx + tx];
    __syncthreads();
    for (int k = ty; k < 32; k += 8)
        Y[(size_t)(bx + k) * rows_p + by + tx] = tile[tx][k];
}

// x^2 into a compensated FP32 pair: x^2 = p + pe exactly, p through TwoSum
__device__ __forceinline__ void sq_add(float x, float &acc, float &cmp)
{
    float p, pe;
    two_prod(x, x, p, pe);
    two_sum_add(acc, cmp, p);
    cmp = __fadd_rn(cmp, pe);
}

// out[i] = sum_j X[i][j]^2 (+ diag[i]^2): one warp per row, lane l taking the
// 4-wide column groups l, l + 32, ... (rows start 16-byte aligned), then the
// ragged columns.  Compensated FP32 pairs folded into an FP64 total every 16
// groups, FP64 across the warp: a fixed order.
__global__ void k_row_norms(const float *__restrict__ X, int rows, int cols, int ld,
                            const double *diag, float *out)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= rows)
        return;
    const float *x = X + (size_t)warp * ld;
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const int c4n = cols >> 2;
    double tot = 0.0;
    for (int c0 = 0; c0 < c4n; c0 += 16 * 32) {
        float acc = 0.0f, cmp = 0.0f;
        const int ce = min(c4n, c0 + 16 * 32);
#pragma unroll 4
        for (int c = c0 + lane; c < ce; c += 32) {
            const float4 v = x4[c];
            sq_add(v.x, acc, cmp);
            sq_add(v.y, acc, cmp);
            sq_add(v.z, acc, cmp);
            sq_add(v.w, acc, cmp);
        }
        tot += (double)acc + (double)cmp;
    }
    {
        float acc = 0.0f, cmp = 0.0f;
        for (int c = (c4n << 2) + lane; c < cols; c += 32)
            sq_add(x[c], acc, cmp);
        tot += (double)acc + (double)cmp;
    }
    for (int o = 16; o > 0; o >>= 1)
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) {
        if (diag)
            tot += diag[warp] * diag[warp];
        out[warp] = (float)tot;
    }
}

// out[j] = sum_i X[i][j]^2 over the first `rows` rows: the squared column
// norms of a row-major matrix without its transpose.  Thread j walks column
// j down the rows (a warp's loads are 32 consecutive columns of one row),
// compensated FP32 pairs folded into an FP64 total every 256 rows.
__global__ void k_col_norms(const float *__restrict__ X, int rows, int cols, int ld, float *out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols)
        return;
    double tot = 0.0;
    for (int r0 = 0; r0 < rows; r0 += 256) {
        float acc = 0.0f, cmp = 0.0f;
        const int re = min(rows, r0 + 256);
#pragma unroll 4
        for (int r = r0; r < re; ++r)
            sq_add(X[(size_t)r * ld + j], acc, cmp);
        tot += (double)acc + (double)cmp;
    }
    out[j] = (float)tot;
}

__global__ void k_scan_nonfinite(const float *__restrict__ X, long long n, int *flag)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    int bad = 0;
    for (; i < n; i += stride)
        bad |= !isfinite(X[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(flag, 1);
}

// Lower triangle from the upper one: X[r][c] = X[c][r] for r > c (32 x 32
// blocks through shared memory, so both sides are read and written along rows).
__global__ void k_symmetrize(float *X, int n, int ld)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;  // destination block (row by, column bx)
    if (by < bx)
        return;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int k = ty; k < 32; k += 8) {  // source block (row bx, column by)
        const int r = bx * 32 + k, c = by * 32 + tx;
        tile[k][tx] = (r < n && c < n) ? X[(size_t)r * ld + c] : 0.0f;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int r = by * 32 + k, c = bx * 32 + tx;  // destination (r, c) = source (c, r)
        if (r < n && c < n && r > c)
            X[(size_t)r * ld + c] = tile[tx][k];
    }
}

}  // namespace

namespace {

// Pearson initialisation (Sec. II-A), first step: row g of the expression
// matrix X (G x N, row-major) becomes z_g = (x_g - m_g) / |x_g - m_g|, so that
// z_g . z_h is the correlation of genes g and h.  One warp per row; mean and
// centred norm in FP64 (two passes, fixed lane order); z stored as a BF16
// split (hi = bf16(z), lo = bf16(z - hi)) in Zh, Zl ([G][Kp], the padding left
// zero by the caller).  flags[0] |= 1 on a non-finite sample, |= 2 on a row of
// zero variance.
__global__ void k_standardize_rows(const float *__restrict__ X, int G, int N, __nv_bfloat16 *__restrict__ Zh,
                                   __nv_bfloat16 *__restrict__ Zl, int Kp, int *flags)
{
    const int g = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (g >= G)
        return;
    const float *x = X + (size_t)g * N;
    double s = 0.0;
    bool finite = true;
    for (int k = lane; k < N; k += 32) {
        finite = finite && isfinite(x[k]);
        s += (double)x[k];
    }
    for (int off = 16; off >= 1; off >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, off);
    const double m = s / (double)N;
    double q = 0.0;
    for (int k = lane; k < N; k += 32) {
        const double d = (double)x[k] - m;
        q += d * d;
    }
    for (int off = 16; off >= 1; off >>= 1)
        q += __shfl_xor_sync(0xffffffffu, q, off);
    const unsigned bad = __ballot_sync(0xffffffffu, !finite);
    if (lane == 0 && (bad || !(q > 0.0)))
        atomicOr(flags, (bad ? 1 : 0) | (q > 0.0 ? 0 : 2));
    if (bad || !(q > 0.0))
        return;
    const double inv = 1.0 / sqrt(q);
    for (int k = lane; k < N; k += 32) {
        const float z = (float)(((double)x[k] - m) * inv);
        const __nv_bfloat16 hi = __float2bfloat16_rn(z);
        Zh[(size_t)g * Kp + k] = hi;
        Zl[(size_t)g * Kp + k] = __float2bfloat16_rn(z - __bfloat162float(hi));
    }
}

// out[r][c] = hi[r][c] + lo[r][c] for r <= c < n: the upper triangle of a
// matrix held as a BF16 split pair (the sum is exact in FP32: lo's last bit is
// no finer than the last bit of the FP32 value the pair was split from).
__global__ void k_unsplit_upper(const __nv_bfloat16 *__restrict__ H, const __nv_bfloat16 *__restrict__ L, int n,
                                int ldi, float *__restrict__ out, int ldo)
{
    const int r = blockIdx.y;
    for (int c = r + blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const size_t i = (size_t)r * ldi + c;
        out[(size_t)r * ldo + c] = __bfloat162float(H[i]) + __bfloat162float(L[i]);
    }
}

// X_ii = 1 for i < n (a correlation matrix's diagonal)
__global__ void k_unit_diag(float *X, int n, int ld)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        X[(size_t)i * ld + i] = 1.0f;
}

}  // namespace

cudaError_t launch_standardize_rows(const float *X, int G, int N, __nv_bfloat16 *Zh, __nv_bfloat16 *Zl, int Kp,
                                    int *flags, cudaStream_t s)
{
    k_standardize_rows<<<ceil_div(G, 8), 256, 0, s>>>(X, G, N, Zh, Zl, Kp, flags);
    return cudaGetLastError();
}

cudaError_t launch_unit_diag(float *X, int n, int ld, cudaStream_t s)
{
    k_unit_diag<<<ceil_div(n, 256), 256, 0, s>>>(X, n, ld);
    return cudaGetLastError();
}

cudaError_t launch_unsplit_sym(const __nv_bfloat16 *H, const __nv_bfloat16 *L, int n, int ldi, float *out, int ldo,
                              cudaStream_t s)
{
    if (n <= 0)
        return cudaSuccess;
    k_unsplit_upper<<<dim3(ceil_div(n, 1024) < 8 ? ceil_div(n, 1024) : 8, n), 256, 0, s>>>(H, L, n, ldi, out, ldo);
    cudaError_t e = cudaGetLastError();
    return e ? e : launch_symmetrize(out, n, ldo, s);
}

cudaError_t launch_symmetrize(float *X, int n, int ld, cudaStream_t s)
{
    dim3 grid(ceil_div(n, 32), ceil_div(n, 32)), block(32, 8);
    k_symmetrize<<<grid, block, 0, s>>>(X, n, ld);
    return cudaGetLastError();
}

// The element kernels read rows as float4: the row stride and base must
// keep every row 16-byte aligned.
static bool rows_aligned(const void *X, int ld) { return (ld & 3) == 0 && ((uintptr_t)X & 15) == 0; }

cudaError_t launch_check_finite_sym(const float *X, int rows, int cols, int ld, bool sym,
                                    int *flags, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0)
        return cudaSuccess;
    if (sym) {
        if (rows != cols)
            return cudaErrorInvalidValue;
        const int nb = ceil_div(rows, 32);
        const int npairs = (int)((long long)nb * (nb + 1) / 2);
        k_check_finite_sym<<<npairs < 152 * 8 ? npairs : 152 * 8, 256, 0, s>>>(X, rows, ld, npairs, flags);
    } else {
        k_check_finite<<<rows < RED_BLOCKS ? rows : RED_BLOCKS, 256, 0, s>>>(X, rows, cols, ld, flags);
    }
    return cudaGetLastError();
}

cudaError_t launch_zscore(float *X, int rows, int cols, int ld, double *stats, double *partials,
                          cudaStream_t s)
{
    if (!rows_aligned(X, ld) || ((uintptr_t)stats & 15))
        return cudaErrorInvalidValue;
    double count = (double)rows * (double)cols;
    k_stats_partial<0><<<RED_BLOCKS, RED_THREADS, 0, s>>>(X, rows, cols, ld, stats, partials);
    k_stats_final<<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, count, 0, stats);
    k_stats_partial<1><<<RED_BLOCKS, RED_THREADS, 0, s>>>(X, rows, cols, ld, stats, partials);
    k_stats_final<<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, count, 1, stats);
    k_apply_zscore<<<rows < 152 * 8 ? rows : 152 * 8, 256, 0, s>>>(X, rows, cols, ld, stats);
    return cudaGetLastError();
}

cudaError_t launch_split_diag(float *X, int n, int ld, double *d, float *df, cudaStream_t s)
{
    k_split_diag<<<ceil_div(n, 256), 256, 0, s>>>(X, n, ld, d, df);
    return cudaGetLastError();
}

cudaError_t launch_diag_to_float(const double *d, float *df, int n, cudaStream_t s)
{
    k_diag_to_float<<<ceil_div(n, 256), 256, 0, s>>>(d, df, n);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float *X, int rows_p, int cols_p, float *Y, cudaStream_t s)
{
    dim3 grid(cols_p / 32, rows_p / 32), block(32, 8);
    k_transpose<<<grid, block, 0, s>>>(X, rows_p, cols_p, Y);
    return cudaGetLastError();
}

cudaError_t launch_row_norms(const float *X, int rows, int cols, int ld, const double *diag,
                             float *out, cudaStream_t s)
{
    if (!rows_aligned(X, ld))
        return cudaErrorInvalidValue;
    k_row_norms<<<ceil_div(rows * 32, 256), 256, 0, s>>>(X, rows, cols, ld, diag, out);
    return cudaGetLastError();
}

cudaError_t launch_col_norms(const float *X, int rows, int cols, int ld, float *out, cudaStream_t s)
{
    k_col_norms<<<ceil_div(cols, 256), 256, 0, s>>>(X, rows, cols, ld, out);
    return cudaGetLastError();
}

cudaError_t launch_scan_nonfinite(const float *X, long long n, int *flag, cudaStream_t s)
{
    k_scan_nonfinite<<<1024, 256, 0, s>>>(X, n, flag);
    return cudaGetLastError();
}

}  // namespace panda
