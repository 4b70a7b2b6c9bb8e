// FP32 SIMT path of one PANDA iteration, plus the tail shared by every path.
//
// Per iteration (Section II-B), with cur the buffer holding W^(t-1):
//   k_rn        Rn    = P_off . W                           (numerator of Eq. 3, off-diagonal part)
//   k_phase1    An    = W . C_off, then per edge (i, j):
//               R = Tan(Rn + p_i W_ij), A = Tan(An + W_ij c_j)   (Eqs. 3, 4)
//               W' = (1-a) W + a/2 (R + A)                       (Eq. 2)
//               partial sums of |W' - W| (Eq. 7), |W'_i.|^2 and |W'_.j|^2
//   k_reduce_wnorms  FP64 sums of those partials
//   k_phase2    upper-triangle tiles of W'.W'^T and W'^T.W' with the damped
//               off-diagonal update of Eq. 5, a mirrored store, and per-row
//               partial sums for the standard deviations of Eq. 6
//   k_fin       diagonals (Eq. 6) and the squared norms of P' and C'
//   k_tail      h (Eq. 7), the iteration counter and the stop test
//
// The products are one SIMT tile routine: out(m, n) = sum_k X[k][m] Y[k][n]
// over 128 x 128 tiles, each thread owning an 8 x 8 block of outputs.  The
// operands it needs are all "k-rows" of a stored matrix:
//   P_off . W      X = P_off (symmetric, so its rows are its columns), Y = W
//   W . C_off      X = W^T,  Y = C_off
//   W' . W'^T      X = Y = W'^T
//   W'^T . W'      X = Y = W'
// Every reduction has a fixed order, so an iteration is deterministic.
#include "panda_internal.cuh"

namespace panda {

namespace {

constexpr int BM = 128, BK = 8, NT = 256;

struct __align__(16) SmemGemm {
    float a[2][BK][BM];
    float b[2][BK][BM];
};

// acc[i][j] += sum_{k < K} X[k][m0 + row(i)] * Y[k][n0 + col(j)]
// row(i) = (i < 4 ? 0 : 64) + ty*4 + (i & 3), col(j) likewise with tx.
__device__ __forceinline__ void simt_tile(const float *__restrict__ X, int ldx,
                                          const float *__restrict__ Y, int ldy, int m0, int n0,
                                          int K, float (&acc)[8][8], SmemGemm &sm)
{
    const int tid = threadIdx.x;
    const int lk = tid >> 5;         // k row this thread loads
    const int lm = (tid & 31) << 2;  // 4 consecutive m (or n) it loads
    const int ty = tid >> 4, tx = tid & 15;
    const float *xp = X + (size_t)lk * ldx + m0 + lm;
    const float *yp = Y + (size_t)lk * ldy + n0 + lm;

    float4 xa = *reinterpret_cast<const float4 *>(xp);
    float4 yb = *reinterpret_cast<const float4 *>(yp);
    *reinterpret_cast<float4 *>(&sm.a[0][lk][lm]) = xa;
    *reinterpret_cast<float4 *>(&sm.b[0][lk][lm]) = yb;
    __syncthreads();

    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) {
            xa = *reinterpret_cast<const float4 *>(xp + (size_t)(k0 + BK) * ldx);
            yb = *reinterpret_cast<const float4 *>(yp + (size_t)(k0 + BK) * ldy);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float4 a0 = *reinterpret_cast<const float4 *>(&sm.a[buf][kk][ty * 4]);
            float4 a1 = *reinterpret_cast<const float4 *>(&sm.a[buf][kk][64 + ty * 4]);
            float4 b0 = *reinterpret_cast<const float4 *>(&sm.b[buf][kk][tx * 4]);
            float4 b1 = *reinterpret_cast<const float4 *>(&sm.b[buf][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            *reinterpret_cast<float4 *>(&sm.a[buf ^ 1][lk][lm]) = xa;
            *reinterpret_cast<float4 *>(&sm.b[buf ^ 1][lk][lm]) = yb;
        }
        __syncthreads();
        buf ^= 1;
    }
}

__device__ __forceinline__ int tile_row(int i) { return ((i & 4) << 4) + (threadIdx.x >> 4) * 4 + (i & 3); }
__device__ __forceinline__ int tile_col(int j) { return ((j & 4) << 4) + (threadIdx.x & 15) * 4 + (j & 3); }

// ---------------------------------------------------------------------------
// Rn = P_off . W   (grid: x = T block, y = G block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT, 2) k_rn(Dev d, int cur)
{
    if (!d.ctl->active)
        return;
    __shared__ SmemGemm sm;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BM;
    float acc[8][8] = {};
    simt_tile(d.Poff, d.Tp, d.W[cur], d.Gp, m0, n0, d.Tp, acc, sm);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float *o = d.Rn + (size_t)(m0 + tile_row(i)) * d.Gp + n0;
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<float4 *>(o + h * 64 + (threadIdx.x & 15) * 4) =
                make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
    }
}

// ---------------------------------------------------------------------------
// Phase 1: An = W . C_off and the fused W update   (grid: x = T block, y = G block)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT, 2) k_phase1(Dev d, int cur)
{
    const Ctl *ctl = d.ctl;
    if (!ctl->active)
        return;
    __shared__ SmemGemm sm;
    __shared__ double hred[NT];
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BM;
    float acc[8][8] = {};
    simt_tile(d.Wt[cur], d.Tp, d.Coff, d.Gp, m0, n0, d.Gp, acc, sm);

    const float a = ctl->alpha;
    const float keep = 1.0f - a, half = 0.5f * a;
    const float *W = d.W[cur];
    float *Wn = d.W[cur ^ 1], *Wtn = d.Wt[cur ^ 1];
    float rowp[8], colp[8];
    float hsum = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        colp[j] = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        rowp[i] = 0.0f;
        const int gi = m0 + tile_row(i);
        const bool ri = gi < d.T;
        const float pdi = ri ? d.pdf[gi] : 0.0f, rsp = ri ? d.rsqP[gi] : 0.0f,
                    rsw = ri ? d.rsqW[gi] : 0.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int gj0 = n0 + h * 64 + (threadIdx.x & 15) * 4;
            const size_t o = (size_t)gi * d.Gp + gj0;
            float4 w4 = *reinterpret_cast<const float4 *>(W + o);
            float4 r4 = *reinterpret_cast<const float4 *>(d.Rn + o);
            float w[4] = {w4.x, w4.y, w4.z, w4.w}, rn[4] = {r4.x, r4.y, r4.z, r4.w}, out[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gj = gj0 + q;
                out[q] = 0.0f;
                if (ri && gj < d.G) {
                    const float rnum = rn[q] + pdi * w[q];                    // P_i. . W_.j
                    const float anum = acc[i][4 * h + q] + w[q] * d.cdf[gj];  // W_i. . C_.j
                    const float R = tanimoto_f(rnum, rsp, d.csqW[gj]);
                    const float A = tanimoto_f(anum, rsw, d.csqC[gj]);
                    const float wn = keep * w[q] + half * (A + R);
                    out[q] = wn;
                    hsum += fabsf(wn - w[q]);
                    rowp[i] += wn * wn;
                    colp[4 * h + q] += wn * wn;
                }
            }
            *reinterpret_cast<float4 *>(Wn + o) = make_float4(out[0], out[1], out[2], out[3]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[i][4 * h + q] = out[q];  // keep W' for the transposed store
        }
    }
    // transposed store: thread owns rows ty*4..+3 (and +64) of column j
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int gj = n0 + tile_col(j);
        float *o = Wtn + (size_t)gj * d.Tp + m0;
#pragma unroll
        for (int h = 0; h < 2; ++h)
            *reinterpret_cast<float4 *>(o + h * 64 + (threadIdx.x >> 4) * 4) =
                make_float4(acc[4 * h][j], acc[4 * h + 1][j], acc[4 * h + 2][j], acc[4 * h + 3][j]);
    }

    // tile partials: rows over the 16 column-threads, columns over the 16 row-threads
    __syncthreads();
    float(*red)[BM] = reinterpret_cast<float(*)[BM]>(&sm);  // [16][128]
#pragma unroll
    for (int i = 0; i < 8; ++i)
        red[threadIdx.x & 15][tile_row(i)] = rowp[i];
    __syncthreads();
    if (threadIdx.x < BM) {
        float s = 0.0f;
        for (int q = 0; q < 16; ++q)
            s += red[q][threadIdx.x];
        d.wrow_part[(size_t)blockIdx.y * d.Tp + m0 + threadIdx.x] = s;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j)
        red[threadIdx.x >> 4][tile_col(j)] = colp[j];
    __syncthreads();
    if (threadIdx.x < BM) {
        float s = 0.0f;
        for (int q = 0; q < 16; ++q)
            s += red[q][threadIdx.x];
        d.wcol_part[(size_t)blockIdx.x * d.Gp + n0 + threadIdx.x] = s;
    }
    hred[threadIdx.x] = (double)hsum;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            hred[threadIdx.x] += hred[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        d.hpart[(size_t)blockIdx.y * d.nbT + blockIdx.x] = hred[0];
}

// Slot sums for 32 consecutive rows per block, 8 threads per row: thread
// (g, x) adds slots g, g + 8, g + 16, ... of row x, then the 8 partial sums
// are added in FP64 in group order (a fixed order, so the result is
// deterministic).  The per-thread sums are compensated FP32 (each addition's
// rounding error recovered exactly by Knuth's TwoSum and carried along), about
// as accurate as FP64 additions of the FP32 slots but on the FP32 pipe, which
// on this GPU is far wider than the FP64 one.
constexpr int RS_ROWS = 32, RS_GROUPS = 8;

// This thread's slots g, g + 8, ... inside [lo, hi), in ascending order
template <int NV>
__device__ __forceinline__ void slot_range(const float *const (&src)[NV], int lo, int hi, int ld, int x,
                                           float (&s)[NV], float (&c)[NV])
{
    const int g = threadIdx.x / RS_ROWS;
    int b = lo + (((g - lo) % RS_GROUPS) + RS_GROUPS) % RS_GROUPS;
    // four slots' loads in flight at a time; the additions keep the order
    for (; b + 3 * RS_GROUPS < hi; b += 4 * RS_GROUPS) {
        float t[NV][4];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                t[v][u] = src[v][(size_t)(b + u * RS_GROUPS) * ld + x];
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                two_sum_add(s[v], c[v], t[v][u]);
    }
    for (; b < hi; b += RS_GROUPS)
#pragma unroll
        for (int v = 0; v < NV; ++v)
            two_sum_add(s[v], c[v], src[v][(size_t)b * ld + x]);
}

// Sums over the slots in [lo0, hi0) and [lo1, hi1) (lo1 >= hi0): slots outside
// them hold zeros, whose additions would change nothing.
template <int NV>
__device__ __forceinline__ void slot_sums(const float *const (&src)[NV], int lo0, int hi0, int lo1, int hi1, int ld,
                                          int x, bool ok, double (&out)[NV], double (*sh)[RS_GROUPS][RS_ROWS])
{
    const int lx = threadIdx.x & (RS_ROWS - 1), g = threadIdx.x / RS_ROWS;
    float s[NV], c[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v)
        s[v] = c[v] = 0.0f;
    if (ok) {
        slot_range<NV>(src, lo0, hi0, ld, x, s, c);
        slot_range<NV>(src, lo1, hi1, ld, x, s, c);
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
        sh[v][g][lx] = (double)s[v] + (double)c[v];
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double t = 0.0;
        for (int q = 0; q < RS_GROUPS; ++q)
            t += sh[v][q][lx];
        out[v] = t;
    }
}

// The largest of one warp's values into *slot (float bits of non-negative
// values order like the values, so an unsigned maximum is exact and the
// result does not depend on the order of the warps).
__device__ __forceinline__ void fp8_norm_max(unsigned *slot, float v)
{
    unsigned u = __float_as_uint(fmaxf(v, 0.0f));
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        u = max(u, __shfl_xor_sync(0xffffffffu, u, off));
    if ((threadIdx.x & 31) == 0)
        atomicMax(slot, u);
}

// rsqW[i] = sum_b wrow_part[b][i], csqW[j] = sum_b wcol_part[b][j] (FP64).
// Blocks [0, ceil(T/32)) take rows of W, the rest its columns.
// block b of one network's launch: b < ceil(T/32) rows of W, the rest its columns
__device__ __forceinline__ void reduce_wnorms_block(const Dev &d, int b)
{
    if (!d.ctl->active)
        return;
    __shared__ double sh[1][RS_GROUPS][RS_ROWS];
    const int bT = ceil_div(d.T, RS_ROWS);
    const bool rows = b < bT;
    const int x = ((rows ? b : b - bT) * RS_ROWS) + (threadIdx.x & (RS_ROWS - 1));
    const bool ok = x < (rows ? d.T : d.G);
    const float *const src[1] = {rows ? d.wrow_part : d.wcol_part};
    double out[1];
    slot_sums<1>(src, 0, rows ? d.nbG : d.nbT, 0, 0, rows ? d.Tp : d.Gp, x, ok, out, sh);
    if (threadIdx.x >= RS_ROWS)
        return;
    if (ok)
        (rows ? d.rsqW : d.csqW)[x] = (float)out[0];
    if (d.fp8)
        fp8_norm_max(&d.f8n[rows ? 2 : 3], ok ? (float)out[0] : 0.0f);
}

__global__ void __launch_bounds__(RS_ROWS * RS_GROUPS) k_reduce_wnorms(const __grid_constant__ Dev d)
{
    reduce_wnorms_block(d, blockIdx.x);
}

// a set of networks: blocks[blockIdx.x] = (network, its block)
__global__ void __launch_bounds__(RS_ROWS * RS_GROUPS) k_reduce_wnorms_set(const Dev *devs, const int2 *blocks)
{
    const int2 w = blocks[blockIdx.x];
    reduce_wnorms_block(devs[w.x], w.y);
}

// ---------------------------------------------------------------------------
// Phase 2: upper-triangle tiles of W'.W'^T (P) then W'^T.W' (C)
// ---------------------------------------------------------------------------
// Row-role partials (over this thread's columns) go to slot_row + tile row;
// column-role partials (over its rows) to slot_col + tile column; a diagonal
// tile adds the two for the same index.  Sixteen threads share each row and
// each column; they are summed in a fixed order.
__device__ __forceinline__ void reduce_roles(const float (&rp)[8], const float (&cp)[8],
                                             float (*red)[BM], float *out, size_t slot_row,
                                             size_t slot_col, bool diag_tile)
{
#pragma unroll
    for (int i = 0; i < 8; ++i)
        red[threadIdx.x & 15][tile_row(i)] = rp[i];
    __syncthreads();
    float rs = 0.0f;
    if (threadIdx.x < BM)
        for (int q = 0; q < 16; ++q)
            rs += red[q][threadIdx.x];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j)
        red[threadIdx.x >> 4][tile_col(j)] = cp[j];
    __syncthreads();
    if (threadIdx.x < BM) {
        float cs = 0.0f;
        for (int q = 0; q < 16; ++q)
            cs += red[q][threadIdx.x];
        if (diag_tile) {
            out[slot_row + threadIdx.x] = rs + cs;
        } else {
            out[slot_row + threadIdx.x] = rs;
            out[slot_col + threadIdx.x] = cs;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void tri_decode(int u, int nb, int &bm, int &bn)
{
    int r = 0;
    while (u >= nb - r) {
        u -= nb - r;
        ++r;
    }
    bm = r;
    bn = r + u;
}

template <bool SIM_SIGMA>
__global__ void __launch_bounds__(NT, 2) k_phase2(Dev d, int cur)
{
    const Ctl *ctl = d.ctl;
    if (!ctl->active)
        return;
    __shared__ SmemGemm sm;
    const int nP = d.nbT * (d.nbT + 1) / 2;
    int u = blockIdx.x, bm, bn;
    const bool isP = u < nP;
    // problem description
    const float *X;
    int ldx, K, n, nb;
    const float *nrm;
    float *Xoff, *S1, *S2, *SV;
    if (isP) {
        nb = d.nbT;
        tri_decode(u, nb, bm, bn);
        X = d.Wt[cur];  // W'^T: rows are genes, so X[k][m] = W'[m][k]
        ldx = d.Tp;
        K = d.Gp;
        n = d.T;
        nrm = d.rsqW;
        Xoff = d.Poff;
        S1 = d.ps_sum; S2 = d.ps_sq; SV = d.ps_vsq;
    } else {
        nb = d.nbG;
        tri_decode(u - nP, nb, bm, bn);
        X = d.W[cur];   // W': rows are TFs, so X[k][m] = W'[k][m]
        ldx = d.Gp;
        K = d.Tp;
        n = d.G;
        nrm = d.csqW;
        Xoff = d.Coff;
        S1 = d.cs_sum; S2 = d.cs_sq; SV = d.cs_vsq;
    }
    const int ld = nb * BM;  // Tp or Gp
    const int m0 = bm * BM, n0 = bn * BM;
    float acc[8][8] = {};
    simt_tile(X, ldx, X, ldx, m0, n0, K, acc, sm);

    const float a = ctl->alpha, keep = 1.0f - a;
    // per-thread partials: [0] row role (sums over my columns), [1] column role
    float r1[8], r2[8], rv[8], c1[8], c2[8], cv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        r1[q] = r2[q] = rv[q] = c1[q] = c2[q] = cv[q] = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int k = m0 + tile_row(i);
        const float nk = k < n ? nrm[k] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int jj = n0 + tile_col(j);
            if (k < jj && jj < n) {  // strict upper triangle, inside the network
                const size_t o = (size_t)k * ld + jj;
                const float s = tanimoto_f(acc[i][j], nk, nrm[jj]);
                const float v = keep * Xoff[o] + a * s;
                Xoff[o] = v;
                Xoff[(size_t)jj * ld + k] = v;
                const float x = SIM_SIGMA ? s : v;
                r1[i] += x; r2[i] += x * x; rv[i] += v * v;
                c1[j] += x; c2[j] += x * x; cv[j] += v * v;
            }
        }
    }
    // reduce the six partial vectors over the 16 threads sharing a row / column
    __syncthreads();
    float(*red)[BM] = reinterpret_cast<float(*)[BM]>(&sm);  // [16][128] (8 KB of 16 KB)
    const size_t slot_row = (size_t)bn * ld + m0, slot_col = (size_t)bm * ld + n0;
    reduce_roles(r1, c1, red, S1, slot_row, slot_col, bm == bn);
    reduce_roles(r2, c2, red, S2, slot_row, slot_col, bm == bn);
    reduce_roles(rv, cv, red, SV, slot_row, slot_col, bm == bn);
}

// ---------------------------------------------------------------------------
// Eq. 6 diagonals and the squared norms of P' and C' (32 rows per block, the
// row partial sums added by 8 threads per row).  Blocks [0, ceil(T/32)) take
// rows of P, the rest rows of C.
// ---------------------------------------------------------------------------
// block b of one network's launch: b < ceil(T/32) rows of P, the rest rows of C
__device__ __forceinline__ void fin_block(const Dev &d, int b)
{
    const Ctl *ctl = d.ctl;
    if (!ctl->active)
        return;
    __shared__ double sh[3][RS_GROUPS][RS_ROWS];
    const int bT = ceil_div(d.T, RS_ROWS);
    const bool isP = b < bT;
    const int i = ((isP ? b : b - bT) * RS_ROWS) + (threadIdx.x & (RS_ROWS - 1));
    const int n = isP ? d.T : d.G;       // network size
    const bool ok = i < n;
    const int ld = isP ? d.Tp : d.Gp;
    const float *const src[3] = {isP ? d.ps_sum : d.cs_sum, isP ? d.ps_sq : d.cs_sq, isP ? d.ps_vsq : d.cs_vsq};
    double sums[3];
    if (d.tri_slots) {
        // a row of 256-block b has row-role partials in slots [b, nb) (tiles (b, bn >= b)) and
        // column-role partials in [nb, nb + 2 b + 2) (tiles (bm <= b, b), one per CTA of the pair)
        const int nb = ceil_div(ld, 256), b256 = ((isP ? b : b - bT) * RS_ROWS) >> 8;
        slot_sums<3>(src, b256, nb, nb, nb + 2 * b256 + 2, ld, i, ok, sums, sh);
    } else {
        const int ns = isP ? (d.nsP ? d.nsP : d.nbT) : (d.nsC ? d.nsC : d.nbG);
        slot_sums<3>(src, 0, ns, 0, 0, ld, i, ok, sums, sh);
    }
    if (threadIdx.x >= RS_ROWS)
        return;
    float nrm = 0.0f;  // the row's new squared norm (0 past the network)
    if (ok) {
        const double s1 = sums[0], s2 = sums[1], sv = sums[2];
        const double alpha = (double)ctl->alpha;
        const int t = ctl->iters + 1;
        const double growth = d.e2tab[t < HIST_CAP ? t : HIST_CAP];
        double sigma = 0.0;  // population std of the n - 1 off-diagonal entries (0 for one entry)
        if (n > 2) {
            const double m = s1 / (double)(n - 1);
            const double var = s2 / (double)(n - 1) - m * m;
            sigma = var > 0.0 ? sqrt(var) : 0.0;
        }
        const double gain = d.diag == 1 ? 1.0 : alpha;  // PANDA_DIAG_D0_LITERAL has no alpha
        const double mult = isP ? (double)d.G : (double)d.T;  // N_a with P, N_e with C
        double *dg = isP ? d.pd : d.cd;
        const double nd = (1.0 - alpha) * dg[i] + gain * mult * sigma * growth;
        dg[i] = nd;
        const float ndf = (float)nd;
        nrm = (float)(sv + nd * nd);
        (isP ? d.pdf : d.cdf)[i] = ndf;
        (isP ? d.rsqP : d.csqC)[i] = nrm;
        if (!isfinite(ndf) || !isfinite(nrm))
            atomicOr(&d.ctl->status, ST_NONFINITE);
    }
    if (d.fp8)  // the whole first warp, past the network too
        fp8_norm_max(&d.f8n[isP ? 0 : 1], nrm);
}

__global__ void __launch_bounds__(RS_ROWS * RS_GROUPS) k_fin(const __grid_constant__ Dev d)
{
    fin_block(d, blockIdx.x);
}

__global__ void __launch_bounds__(RS_ROWS * RS_GROUPS) k_fin_set(const Dev *devs, const int2 *blocks)
{
    const int2 w = blocks[blockIdx.x];
    fin_block(devs[w.x], w.y);
}

// h (Eq. 7), the counter and the stop test: one block per network.
__device__ __forceinline__ void tail_block(const Dev &d)
{
    Ctl *ctl = d.ctl;
    if (!ctl->active)
        return;
    __shared__ double sh[256];
    const int n = d.nbT * d.nbG;
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x)
        s += d.hpart[q];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double h = sh[0] / ((double)d.T * (double)d.G);
        const int t = ctl->iters + 1;
        if (t - 1 < HIST_CAP)
            d.hist[t - 1] = h;
        ctl->iters = t;
        ctl->h_last = h;
        ctl->converged = h < ctl->tol;
        if (d.fp8) {  // the new state's norm maxima, and the scale of the next W' (Eq. 2)
            for (int q = 0; q < 4; ++q) {
                d.f8n[4 + q] = d.f8n[q];
                d.f8n[q] = 0u;
            }
            d.f8[3] = e4m3_scale(fp8_bound_w(__uint_as_float(d.f8n[4]), __uint_as_float(d.f8n[5]),
                                             __uint_as_float(d.f8n[6]), __uint_as_float(d.f8n[7])));
        }
        if (!isfinite(h))
            ctl->status |= ST_NONFINITE;
        if (ctl->converged || t >= ctl->stop_at || ctl->status)
            ctl->active = 0;
    }
}

__global__ void k_tail(const __grid_constant__ Dev d) { tail_block(d); }

__global__ void k_tail_set(const Dev *devs) { tail_block(devs[blockIdx.x]); }

}  // namespace

const char *const SIMT_KERNEL_NAMES[SIMT_KERNELS] = {"k_rn", "k_phase1", "k_reduce_wnorms",
                                                     "k_phase2", "k_fin", "k_tail"};

cudaError_t launch_reduce_wnorms(const Dev &d, cudaStream_t s)
{
    k_reduce_wnorms<<<ceil_div(d.T, RS_ROWS) + ceil_div(d.G, RS_ROWS), RS_ROWS * RS_GROUPS, 0, s>>>(d);
    return cudaGetLastError();
}

cudaError_t launch_reduce_wnorms_set(const Dev *devs, const int2 *blocks, int nblocks, cudaStream_t s)
{
    k_reduce_wnorms_set<<<nblocks, RS_ROWS * RS_GROUPS, 0, s>>>(devs, blocks);
    return cudaGetLastError();
}

cudaError_t launch_fin_tail_set(const Dev *devs, const int2 *blocks, int nblocks, int nnets, cudaStream_t s)
{
    k_fin_set<<<nblocks, RS_ROWS * RS_GROUPS, 0, s>>>(devs, blocks);
    k_tail_set<<<nnets, 256, 0, s>>>(devs);
    return cudaGetLastError();
}

int set_norm_blocks(int T, int G) { return ceil_div(T, RS_ROWS) + ceil_div(G, RS_ROWS); }

cudaError_t launch_fin_tail(const Dev &d, cudaStream_t s, KernelEvents &ke)
{
    k_fin<<<ceil_div(d.T, RS_ROWS) + ceil_div(d.G, RS_ROWS), RS_ROWS * RS_GROUPS, 0, s>>>(d);
    ke.mark(s);
    k_tail<<<1, 256, 0, s>>>(d);
    ke.mark(s);
    return cudaGetLastError();
}

cudaError_t launch_iteration_simt(const Dev &d, int cur, cudaStream_t s, KernelEvents &ke)
{
    dim3 g1(d.nbT, d.nbG);
    ke.mark(s);
    k_rn<<<g1, NT, 0, s>>>(d, cur);
    ke.mark(s);
    k_phase1<<<g1, NT, 0, s>>>(d, cur);
    ke.mark(s);
    launch_reduce_wnorms(d, s);
    ke.mark(s);
    const int tiles = d.nbT * (d.nbT + 1) / 2 + d.nbG * (d.nbG + 1) / 2;
    if (d.diag == 2)
        k_phase2<true><<<tiles, NT, 0, s>>>(d, cur ^ 1);
    else
        k_phase2<false><<<tiles, NT, 0, s>>>(d, cur ^ 1);
    ke.mark(s);
    return launch_fin_tail(d, s, ke);
}

}  // namespace panda

// ---- FP32 FFMA throughput of the device (measurement support) -------------
namespace panda {
namespace {

constexpr int FFMA_CHAINS = 8, FFMA_LOOP = 4096, FFMA_THREADS = 512;

// Every thread runs FFMA_CHAINS independent chains x <- x * a + b for
// FFMA_LOOP rounds (a, b are launch arguments, so nothing is folded); the
// store is taken only if a chain lands on `never`, which the host makes
// unreachable, so the loop is not removed.
__global__ void __launch_bounds__(FFMA_THREADS) k_ffma_loop(float a, float b, float never, float *out)
{
    float x[FFMA_CHAINS];
#pragma unroll
    for (int c = 0; c < FFMA_CHAINS; ++c)
        x[c] = (float)(threadIdx.x + c) * 1e-3f;
#pragma unroll 32  // 256 FMAs per trip through the loop: its counter and branch are noise
    for (int it = 0; it < FFMA_LOOP; ++it)
#pragma unroll
        for (int c = 0; c < FFMA_CHAINS; ++c)
            x[c] = fmaf(x[c], a, b);
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < FFMA_CHAINS; ++c)
        s += x[c];
    if (s == never)
        out[blockIdx.x] = s;
}

}  // namespace

cudaError_t measure_ffma_peak(double *tflops)
{
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(&out, sizeof(float) * 4 * nsm)))
        return e;
    const int blocks = 4 * nsm;  // 4 x 16 warps per SM: 16 per scheduler
    double best_ms = 1e30;
    if (!(e = cudaEventCreate(&e0)) && !(e = cudaEventCreate(&e1))) {
        for (int rep = 0; rep < 12 && !e; ++rep) {
            cudaEventRecord(e0);
            k_ffma_loop<<<blocks, FFMA_THREADS>>>(0.999f, 1e-4f, -1.0f, out);
            cudaEventRecord(e1);
            if (!(e = cudaEventSynchronize(e1))) {
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep >= 2 && ms < best_ms)  // the first launches warm up the clocks
                    best_ms = ms;
            }
        }
        if (!e)
            e = cudaGetLastError();
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(out);
    if (e)
        return e;
    const double flop = 2.0 * FFMA_CHAINS * FFMA_LOOP * (double)FFMA_THREADS * blocks;
    *tflops = flop / (best_ms * 1e-3) / 1e12;
    return cudaSuccess;
}

}  // namespace panda
