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

// flags[0] |= 1 on a non-finite entry; flags[1] |= 1 when X[i][j] != X[j][i].
__global__ void k_check_finite_sym(const float *__restrict__ X, int rows, int cols, int ld,
                                   int sym, int *flags)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols)
        return;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        float v = X[(size_t)r * ld + c];
        if (!isfinite(v))
            atomicOr(&flags[0], 1);
        if (sym && c > r && v != X[(size_t)c * ld + r])
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

// mode 0: sum of x; mode 1: sum of (x - mean)^2 with mean = stats[0]
__global__ void k_stats_partial(const float *__restrict__ X, int rows, int cols, int ld, int mode,
                                const double *stats, double *partials)
{
    __shared__ double sh[RED_THREADS];
    double mean = mode ? stats[0] : 0.0;
    double acc = 0.0;
    for (int r = blockIdx.x; r < rows; r += gridDim.x)
        for (int c = threadIdx.x; c < cols; c += blockDim.x) {
            double v = (double)X[(size_t)r * ld + c];
            if (mode) {
                double d = v - mean;
                acc += d * d;
            } else {
                acc += v;
            }
        }
    double s = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0)
        partials[blockIdx.x] = s;
}

// stats[0] = mean (mode 0) or stats[1] = population std (mode 1)
__global__ void k_stats_final(const double *partials, int n, double count, int mode, double *stats)
{
    __shared__ double sh[RED_THREADS];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        acc += partials[i];
    double s = block_sum_fixed(acc, sh);
    if (threadIdx.x == 0) {
        if (mode == 0)
            stats[0] = s / count;
        else
            stats[1] = sqrt(s / count);
    }
}

__global__ void k_apply_zscore(float *X, int rows, int cols, int ld, const double *stats)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    double sd = stats[1];
    if (c >= cols || !(sd > 0.0))
        return;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        size_t o = (size_t)r * ld + c;
        X[o] = (float)(((double)X[o] - stats[0]) / sd);
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

// out[i] = sum_j X[i][j]^2 (+ diag[i]^2): one warp per row, FP64, fixed order.
__global__ void k_row_norms(const float *__restrict__ X, int rows, int cols, int ld,
                            const double *diag, float *out)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= rows)
        return;
    const float *x = X + (size_t)warp * ld;
    double acc = 0.0;
    for (int c = lane; c < cols; c += 32) {
        double v = (double)x[c];
        acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        if (diag)
            acc += diag[warp] * diag[warp];
        out[warp] = (float)acc;
    }
}

// out[j] = sum_i X[i][j]^2: one thread per column, FP64, rows in order.
__global__ void k_col_norms(const float *__restrict__ X, int rows, int cols, int ld, float *out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols)
        return;
    double acc = 0.0;
    for (int i = 0; i < rows; ++i) {
        double v = (double)X[(size_t)i * ld + j];
        acc += v * v;
    }
    out[j] = (float)acc;
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

cudaError_t launch_symmetrize(float *X, int n, int ld, cudaStream_t s)
{
    dim3 grid(ceil_div(n, 32), ceil_div(n, 32)), block(32, 8);
    k_symmetrize<<<grid, block, 0, s>>>(X, n, ld);
    return cudaGetLastError();
}

cudaError_t launch_check_finite_sym(const float *X, int rows, int cols, int ld, bool sym,
                                    int *flags, cudaStream_t s)
{
    dim3 grid(ceil_div(cols, 256), rows < 65535 ? rows : 65535);
    k_check_finite_sym<<<grid, 256, 0, s>>>(X, rows, cols, ld, sym ? 1 : 0, flags);
    return cudaGetLastError();
}

cudaError_t launch_zscore(float *X, int rows, int cols, int ld, double *stats, double *partials,
                          cudaStream_t s)
{
    double count = (double)rows * (double)cols;
    k_stats_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(X, rows, cols, ld, 0, stats, partials);
    k_stats_final<<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, count, 0, stats);
    k_stats_partial<<<RED_BLOCKS, RED_THREADS, 0, s>>>(X, rows, cols, ld, 1, stats, partials);
    k_stats_final<<<1, RED_THREADS, 0, s>>>(partials, RED_BLOCKS, count, 1, stats);
    dim3 grid(ceil_div(cols, 256), rows < 65535 ? rows : 65535);
    k_apply_zscore<<<grid, 256, 0, s>>>(X, rows, cols, ld, stats);
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
