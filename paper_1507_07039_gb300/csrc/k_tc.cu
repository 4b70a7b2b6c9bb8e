// BF16X3 tensor-core path of one PANDA iteration (sm_103a, tcgen05 + TMA),
// every GEMM tile on a CTA pair (cta_group::2, 256 x 256 outputs).
//
//   k_tc_phase1   per 256 (TFs) x 256 (genes) tile of W': two TMEM accumulators,
//                   R-num = P_off . W   (K = TFs;   A = P_off rows, B = W columns)
//                   A-num = W . C_off   (K = genes; A = W rows,     B = C_off rows)
//                 then the fused epilogue of Eqs. 1-3 and 2: diagonal terms,
//                 Tanimoto, damped W update, h and norm partials, and the
//                 FP32 W' plus its split copy (under FP8MIX also E4M3 copies
//                 of W' and W'^T).
//   k_reduce_wnorms  (shared with the FP32 path)
//   k_tc_phase2   persistent: upper-triangle 256 x 256 tiles of W'.W'^T (P,
//                 K = genes) and W'^T.W' (C, K = TFs; columns of W' as both
//                 operands) from a balanced host-built
//                 schedule, double-buffered TMEM accumulators, and the Eq. 5
//                 epilogue: Tanimoto, damped update, the FP32 upper triangle,
//                 split copies of the upper triangle (of P: both triangles; of
//                 C: both only inside diagonal 256-blocks), row partial sums
//                 for Eq. 6.  (Only the upper triangle of FP32 P and C is ever
//                 read here; panda_get and panda_save mirror it first.)
//   k_fin, k_tail (shared): Eq. 6 diagonals, norms, h, stop test.
//
// P and C are symmetric.  "P_off rows" are read K-major from the full split
// copy.  For "C_off rows" j against genes k, the availability product reads
// C_off[j][k] K-major where k lies at or past the tile's diagonal 256-block
// (upper triangle and diagonal blocks), and as C_off[k][j], rows k of the
// upper triangle loaded MN-major, where k lies before it: the split copy of
// C's lower triangle outside the diagonal blocks is never written or read.
// W is kept in one orientation: where a product needs columns of W (B of
// R-num, both operands of the C tiles) they are rows k of W's split copy,
// loaded as 64 x 64 boxes and fed to the MMAs MN-major.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include <cuda_fp8.h>

#include "panda_internal.cuh"
#include "tc_common.cuh"

namespace panda {

const char *const TC_KERNEL_NAMES[TC_KERNELS] = {"k_tc_phase1", "k_reduce_wnorms", "k_tc_phase2",
                                                 "k_fin", "k_tail"};

namespace {

using namespace tc;


struct TcMaps {  // split copies, K-major, boxes of 64 x 128 (one CTA's half of a 256-row tile)
    CUtensorMap Ph, Pl;              // P_off split   [Tp][Tp]
    CUtensorMap Wh[2], Wl[2];        // W split       [Tp][Gp]
    CUtensorMap Whm[2], Wlm[2];      // the same arrays in boxes of 64 x 64: W^T operands, MN-major
    CUtensorMap Ch, Cl;              // C_off split   [Gp][Gp]
    CUtensorMap Chm, Clm;            // the same arrays in boxes of 64 x 64, for MN-major loads
    CUtensorMap W8[2], Wt8[2], C8;   // FP8MIX: E4M3 copies, boxes of 128 B x 128 rows
};

// A set of networks iterated by one launch per phase (device arrays, one entry per network)
struct SetArgs {
    const Dev *devs;       // the networks' device state
    const TcMaps *maps;    // their tensor maps (64-byte aligned, in global memory)
    const int *parity;     // W buffer of a network = (parity + its iteration count) & 1
    const int4 *items1;    // phase 1: (network, mt, nt, cost) tiles, listed per CTA pair
    const int *p1_off;     // phase 1: per CTA pair, its range of items1
    float *acc;            // phase 1: per CTA, its running-sum slot (128 x 256 floats)
    const int *sched_off;  // phase 2: per CTA pair, its range of sched
    const int *sched;      // phase 2: packed tiles (as for one network)
    const int *sched_net;  // phase 2: the network of each tile
};

__device__ __forceinline__ int set_cur(const SetArgs &a, int net)
{
    return (a.parity[net] + a.devs[net].ctl->iters) & 1;
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p)
{
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16 &hi, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));  // x - hi is exact in FP32
}

// Eq. 1 from the numerator and the two squared norms with the hardware
// reciprocal square root (rsqrtf, within 2 ulp): the tensor-core path's
// epilogues, whose products carry BF16X3 error far above that; 0 when the
// denominator is 0 (both vectors zero).
__device__ __forceinline__ float tanimoto_fast(float num, float nx, float ny)
{
    const float den = (nx + ny) - fabsf(num);
    return den > 0.0f ? num * rsqrtf(den) : 0.0f;
}

// As tanimoto_fast without the branch: the denominator is at least
// (|x|^2 + |y|^2)/2 > 0 unless both vectors are zero, in which case the
// numerator is 0 too and the clamp keeps the result 0.
__device__ __forceinline__ float tanimoto_clamped(float num, float nx, float ny)
{
    return num * rsqrtf(fmaxf((nx + ny) - fabsf(num), 1e-30f));
}

// hi / lo of two values at once, packed as BF16 pairs (first value in the low half)
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&l);
}

// x0, x1 scaled by s and rounded to E4M3 (nearest even, saturating to +-448), x0 in the low byte
__device__ __forceinline__ uint32_t e4m3x2(float x0, float x1, float s)
{
    return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(x0 * s, x1 * s), __NV_SATFINITE, __NV_E4M3);
}

// E4M3 copy of a whole array, scaled by *scale (padding stays zero): four
// values per thread from one 16-byte load, one 4-byte store (all buffers are
// whole allocations, so aligned; a misaligned one takes the scalar loop)
__global__ void k_to_e4m3(const float *__restrict__ X, size_t n, uint8_t *__restrict__ Q, const float *scale)
{
    const float s = scale ? *scale : 1.0f;
    const size_t n4 = (((uintptr_t)X & 15) | ((uintptr_t)Q & 3)) ? 0 : n >> 2;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = t0; q < n4; q += stride) {
        const float4 v = reinterpret_cast<const float4 *>(X)[q];
        reinterpret_cast<uint32_t *>(Q)[q] = e4m3x2(v.x, v.y, s) | (e4m3x2(v.z, v.w, s) << 16);
    }
    for (size_t q = (n4 << 2) + t0; q < n; q += stride)
        Q[q] = (uint8_t)e4m3x2(X[q], 0.0f, s);
}

// hi / lo of a whole array (padding stays zero because x is zero there); L may
// be NULL (hi only).  Four values per thread from one 16-byte load, 8-byte
// stores; a misaligned buffer takes the scalar loop.
__global__ void k_split(const float *__restrict__ X, size_t n, __nv_bfloat16 *__restrict__ H,
                        __nv_bfloat16 *__restrict__ L)
{
    const size_t n4 = (((uintptr_t)X & 15) | ((uintptr_t)H & 7) | ((uintptr_t)L & 7)) ? 0 : n >> 2;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t q = t0; q < n4; q += stride) {
        const float4 v = reinterpret_cast<const float4 *>(X)[q];
        uint32_t h0, l0, h1, l1;
        split_pair(v.x, v.y, h0, l0);
        split_pair(v.z, v.w, h1, l1);
        reinterpret_cast<uint2 *>(H)[q] = make_uint2(h0, h1);
        if (L)
            reinterpret_cast<uint2 *>(L)[q] = make_uint2(l0, l1);
    }
    for (size_t q = (n4 << 2) + t0; q < n; q += stride) {
        __nv_bfloat16 hi, lo;
        split_bf16(X[q], hi, lo);
        H[q] = hi;
        if (L)
            L[q] = lo;
    }
}

// FP8MIX set-up (one block): the state's squared-norm maxima, latched; the
// scales of the state's E4M3 copies (an entry is at most its row's norm) and
// of the next W'.
__global__ void k_fp8_init(Dev d)
{
    __shared__ float red[4][1024];
    const float *v[4] = {d.rsqP, d.csqC, d.rsqW, d.csqW};
    const int n[4] = {d.T, d.G, d.T, d.G};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float m = 0.0f;
        for (int i = threadIdx.x; i < n[q]; i += blockDim.x)
            m = fmaxf(m, v[q][i]);
        red[q][threadIdx.x] = m;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                red[q][threadIdx.x] = fmaxf(red[q][threadIdx.x], red[q][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) {
            d.f8n[q] = 0u;
            d.f8n[4 + q] = __float_as_uint(red[q][0]);
        }
        d.f8[0] = d.f8[1] = e4m3_scale(1.001f * sqrtf(red[2][0]));
        d.f8[2] = e4m3_scale(1.001f * sqrtf(red[1][0]));
        d.f8[3] = e4m3_scale(fp8_bound_w(red[0][0], red[1][0], red[2][0], red[3][0]));
    }
}

__device__ __forceinline__ void ld16(const float *src, float (&v)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = reinterpret_cast<const float4 *>(src)[q];
        v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
}

// four float4 at p, p + 8 ld, p + 16 ld, p + 24 ld (a warp's coalesced 32-row x 16-column block)
__device__ __forceinline__ void ld_rows4(const float *p, int ld, float4 (&v)[4])
{
#pragma unroll
    for (int i = 0; i < 4; ++i)
        v[i] = *reinterpret_cast<const float4 *>(p + (size_t)(8 * i) * ld);
}

// 16 bytes from global memory, asking L2 to fetch the whole aligned 256-byte
// block around them: a phase-2 epilogue thread reads its row's old values 32
// bytes (16 entries) of each half at a time, and the 256-byte block holds the
// rest of its row segment, which the next sub-chunks read
__device__ __forceinline__ uint4 ld16_l2block(const void *p)
{
    uint4 v;
    asm volatile("ld.global.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// For a matrix held as a BF16 split pair: 16 consecutive values hi + lo of one
// row (the sum is exact in FP32), into v[0..3]
__device__ __forceinline__ void ld_row16_split(const __nv_bfloat16 *h, const __nv_bfloat16 *l, float4 (&v)[4])
{
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint4 a = ld16_l2block(h + 8 * i), b = ld16_l2block(l + 8 * i);
        const uint32_t av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
        float f[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 x = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&av[q]));
            const float2 y = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&bv[q]));
            f[2 * q] = x.x + y.x;
            f[2 * q + 1] = x.y + y.y;
        }
        v[2 * i] = make_float4(f[0], f[1], f[2], f[3]);
        v[2 * i + 1] = make_float4(f[4], f[5], f[6], f[7]);
    }
}

// 16 BF16 values held as 8 packed pairs: two 16-byte stores, or the masked entries
__device__ __forceinline__ void st16_packed(__nv_bfloat16 *dst, const uint32_t (&p)[8], uint32_t mask)
{
    if (mask == 0xffffu) {
        reinterpret_cast<uint4 *>(dst)[0] = make_uint4(p[0], p[1], p[2], p[3]);
        reinterpret_cast<uint4 *>(dst)[1] = make_uint4(p[4], p[5], p[6], p[7]);
    } else {
        uint16_t *d16 = reinterpret_cast<uint16_t *>(dst);
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (mask >> q & 1u)
                d16[q] = (uint16_t)(p[q >> 1] >> (16 * (q & 1)));
    }
}

template <int STAGES>
__device__ __forceinline__ void init_sync(Sync<STAGES> &sy)
{
    for (int s = 0; s < STAGES; ++s) {
        mbar_init(&sy.full[s], 1);
        mbar_init(&sy.empty[s], 1);
    }
    mbar_init(&sy.accum, 1);
    sy.abort = 0;
    sy.issued = 0;
    sy.consumed = 0;
    fence_mbar_init();
}

// store 32 consecutive floats (16-byte aligned destination)
__device__ __forceinline__ void st32(float *dst, const float (&v)[32])
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        reinterpret_cast<float4 *>(dst)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// ---------------------------------------------------------------------------
// Self-test: D (Mp x Np) = A . B^T from split operands, one 128 x 128 tile per CTA
// ---------------------------------------------------------------------------
struct GemmMaps {
    CUtensorMap Ah, Al, Bh, Bl;
};

// stall_kb >= 0: the producer arms stage stall_kb but issues none of its loads,
// so that stage's barrier never completes and the bounded waits must end the
// kernel with ST_TIMEOUT (the timeout path's test).
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_selftest(const __grid_constant__ GemmMaps maps, int Kp, int Np, float *D, Ctl *ctl, int stall_kb)
{
    constexpr int BN = 128, STAGES = 3;
    constexpr uint32_t B_BYTES = BN * BK * 2, STAGE = 2 * A_BYTES + 2 * B_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *stages = align1024(smem_raw);
    Sync<STAGES> &sy = *reinterpret_cast<Sync<STAGES> *>(stages + STAGES * STAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN, nk = Kp / BK;
    if (threadIdx.x == 0)
        init_sync(sy);
    if (warp == 1)
        tmem_alloc(&sy.tmem, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        if (lane == 0)
            run_producer<STAGES>(sy, stages, STAGE, nk, ctl, [&](int kb, uint8_t *st, uint64_t *bar) {
                if (kb == stall_kb)
                    return;
                tma_load_2d(st, &maps.Ah, bar, kb * BK, m0);
                tma_load_2d(st + A_BYTES, &maps.Al, bar, kb * BK, m0);
                tma_load_2d(st + 2 * A_BYTES, &maps.Bh, bar, kb * BK, n0);
                tma_load_2d(st + 2 * A_BYTES + B_BYTES, &maps.Bl, bar, kb * BK, n0);
            });
    } else if (warp == 1) {
        if (lane == 0)
            run_mma<STAGES, BN>(sy, stages, STAGE, nk, ctl, [](int) { return 0u; }, [](int kb) { return kb == 0; });
    } else {
        // the issuer commits `accum` on every path (abort included), so this wait
        // also makes sure that arrival has landed before the CTA leaves
        const int wq = warp & 3;
        const bool ok = wait_bounded(&sy.accum, 0, &sy.abort, ctl, true);
        tc_fence_after();
        if (ok && !*(volatile int *)&sy.abort) {
            const int r = m0 + wq * 32 + lane;
            const uint32_t trow = sy.tmem + ((uint32_t)(wq * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                float v[32];
                tmem_ld32(trow + c * 32, v);
                st32(D + (size_t)r * Np + n0 + c * 32, v);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0)
        drain(sy, ctl);
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(sy.tmem, BN);
    }
}

// ---------------------------------------------------------------------------
// D = A . B^T on CTA pairs over 256 x 256 tiles, one pair of CTAs per tile
// (cluster of 2 along x); CTA r loads A rows m0 + 128 r and B rows n0 + 128 r
// and receives D rows m0 + 128 r .. + 127, all 256 columns.  It serves the
// Gram of the standardised expression (Pearson initialisation) and the
// self-tests of the pair pipeline (MN-major B, E4M3 operands).
// ---------------------------------------------------------------------------
constexpr int PAIR_N = 256, PAIR_ST = 3;
constexpr uint32_t PAIR_STAGE = 4 * A_BYTES;  // per CTA: A hi, A lo, B hi, B lo (128 rows each)

struct SyncPair {
    uint64_t full[PAIR_ST], empty[PAIR_ST];
    uint64_t accum;
    uint32_t tmem;
    int abort, issued, consumed;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS, 1)
    k_tc_gemm_pair(const __grid_constant__ GemmMaps maps, int Kp, int Np, float *D, Ctl *ctl, int mn, int fp8)
{
    // mn bit 0: B stored [K][N] and fed MN-major; bit 1: A stored [K][M] and fed MN-major
    extern __shared__ uint8_t smem_raw[];
    uint8_t *stages = align1024(smem_raw);
    SyncPair &sy = *reinterpret_cast<SyncPair *>(stages + PAIR_ST * PAIR_STAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    // a k-block is 128 B of each row: 64 BF16 or 128 E4M3 values
    const int m0 = (blockIdx.x >> 1) * 256, n0 = blockIdx.y * PAIR_N, nk = Kp / (fp8 ? 2 * BK : BK);
    if (threadIdx.x == 0) {
        for (int q = 0; q < PAIR_ST; ++q) {
            mbar_init(&sy.full[q], 1);
            mbar_init(&sy.empty[q], 1);
        }
        mbar_init(&sy.accum, 1);
        sy.abort = 0;
        sy.issued = 0;
        sy.consumed = 0;
        fence_mbar_init();
    }
    if (warp == 1)
        tmem_alloc_pair(&sy.tmem, PAIR_N);
    tc_fence_before();
    cluster_sync();  // barriers of both CTAs initialised before any cross-CTA signal
    tc_fence_after();
    if (warp == 0) {
        if (lane == 0) {  // both CTAs load their halves; completion is counted on the even CTA's barrier
            int kb = 0;
            for (; kb < nk; ++kb) {
                const int s = kb % PAIR_ST;
                const uint32_t ph = (uint32_t)(kb / PAIR_ST) & 1u;
                if (!wait_bounded(&sy.empty[s], ph ^ 1u, &sy.abort, ctl))
                    break;
                const uint32_t fb = mapa_shared(smem_u32(&sy.full[s]), 0);
                if (rank == 0)
                    mbar_arrive_expect_tx(&sy.full[s], fp8 ? 4 * A_BYTES : 2 * PAIR_STAGE);
                uint8_t *st = stages + (size_t)s * PAIR_STAGE;
                if (fp8) {  // E4M3: one A and one B tile of 128 rows x 128 B
                    tma_load_2d_pair(st, &maps.Ah, fb, kb * 2 * BK, m0 + 128 * rank);
                    tma_load_2d_pair(st + A_BYTES, &maps.Bh, fb, kb * 2 * BK, n0 + 128 * rank);
                    continue;
                }
                if (mn & 2) {  // A^T stored [K][M]: two 64 x 64 boxes per CTA half, M contiguous
                    for (int h = 0; h < 2; ++h) {
                        tma_load_2d_pair(st + h * (A_BYTES / 2), &maps.Ah, fb, m0 + 128 * rank + 64 * h, kb * BK);
                        tma_load_2d_pair(st + A_BYTES + h * (A_BYTES / 2), &maps.Al, fb, m0 + 128 * rank + 64 * h,
                                         kb * BK);
                    }
                } else {
                    tma_load_2d_pair(st, &maps.Ah, fb, kb * BK, m0 + 128 * rank);
                    tma_load_2d_pair(st + A_BYTES, &maps.Al, fb, kb * BK, m0 + 128 * rank);
                }
                if (mn & 1) {  // B^T stored [K][N]: two 64 x 64 boxes per CTA half, N contiguous
                    for (int h = 0; h < 2; ++h) {
                        tma_load_2d_pair(st + 2 * A_BYTES + h * (A_BYTES / 2), &maps.Bh, fb,
                                         n0 + 128 * rank + 64 * h, kb * BK);
                        tma_load_2d_pair(st + 3 * A_BYTES + h * (A_BYTES / 2), &maps.Bl, fb,
                                         n0 + 128 * rank + 64 * h, kb * BK);
                    }
                } else {
                    tma_load_2d_pair(st + 2 * A_BYTES, &maps.Bh, fb, kb * BK, n0 + 128 * rank);
                    tma_load_2d_pair(st + 3 * A_BYTES, &maps.Bl, fb, kb * BK, n0 + 128 * rank);
                }
            }
            sy.issued = kb;
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {  // the even CTA issues the pair's MMAs
            const uint32_t idesc =
                idesc_bf16_f32(256, PAIR_N) | ((mn & 1) ? IDESC_B_MN : 0u) | ((mn & 2) ? IDESC_A_MN : 0u);
            int kb = 0;
            for (; kb < nk; ++kb) {
                const int s = kb % PAIR_ST;
                const uint32_t ph = (uint32_t)(kb / PAIR_ST) & 1u;
                if (!wait_bounded(&sy.full[s], ph, &sy.abort, ctl))
                    break;
                tc_fence_after();
                const uint32_t base = smem_u32(stages + (size_t)s * PAIR_STAGE);
                if (fp8) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)  // K = 32 per MMA, 32 B along the swizzled row
                        mma_e4m3_pair(sy.tmem, sdesc_k_sw128(base + kk * 32), sdesc_k_sw128(base + A_BYTES + kk * 32),
                                      idesc_e4m3_f32(256, PAIR_N), (kb == 0 && kk == 0) ? 0u : 1u);
                    mma_commit_pair(&sy.empty[s]);
                    continue;
                }
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint64_t ah = (mn & 2) ? sdesc_mn_sw128(base + kk * 2048, A_BYTES / 2)
                                                 : sdesc_k_sw128(base + off);
                    const uint64_t al = (mn & 2) ? sdesc_mn_sw128(base + A_BYTES + kk * 2048, A_BYTES / 2)
                                                 : sdesc_k_sw128(base + A_BYTES + off);
                    const uint64_t bh = (mn & 1) ? sdesc_mn_sw128(base + 2 * A_BYTES + kk * 2048, A_BYTES / 2)
                                                 : sdesc_k_sw128(base + 2 * A_BYTES + off);
                    const uint64_t bl = (mn & 1) ? sdesc_mn_sw128(base + 3 * A_BYTES + kk * 2048, A_BYTES / 2)
                                                 : sdesc_k_sw128(base + 3 * A_BYTES + off);
                    mma_bf16_pair(sy.tmem, ah, bh, idesc, (kb == 0 && kk == 0) ? 0u : 1u);
                    mma_bf16_pair(sy.tmem, ah, bl, idesc, 1u);
                    mma_bf16_pair(sy.tmem, al, bh, idesc, 1u);
                }
                mma_commit_pair(&sy.empty[s]);
            }
            sy.consumed = kb;
            mma_commit_pair(&sy.accum);
        }
    } else {
        const int wq = warp & 3;
        const bool ok = wait_bounded(&sy.accum, 0, &sy.abort, ctl);
        tc_fence_after();
        if (ok && !*(volatile int *)&sy.abort) {
            const int r = m0 + 128 * rank + wq * 32 + lane;
            const uint32_t trow = sy.tmem + ((uint32_t)(wq * 32) << 16);
#pragma unroll 1
            for (int c = 0; c < PAIR_N / 32; ++c) {
                float v[32];
                tmem_ld32(trow + c * 32, v);
                st32(D + (size_t)r * Np + n0 + c * 32, v);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && rank == 0)  // loads counted here but not consumed (abort only)
        for (int kb = sy.consumed; kb < sy.consumed + PAIR_ST && kb < nk; ++kb)
            if (kb < sy.issued)
                wait_bounded(&sy.full[kb % PAIR_ST], (uint32_t)(kb / PAIR_ST) & 1u, &sy.abort, ctl, true);
    cluster_sync();  // neither CTA leaves while the pair may still signal it
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(sy.tmem, PAIR_N);
    }
}

// ---------------------------------------------------------------------------
// Phase 1 on CTA pairs: one 256 (TFs) x 256 (genes) tile of W' per pair
// (grid x = 2 x T tiles, y = G tiles).  CTA r loads rows 128 r .. + 127 of
// the tile's A blocks (P_off for R, W for A) and of its B blocks (columns of W
// for R, C_off for A); the even CTA issues cta_group::2 MMAs into two TMEM
// buffers of 256 columns: A-num in chunks alternating between them (drained
// by the epilogue warps into a running sum, see P1_CHUNK), then R-num in the
// buffer the last chunk leaves free.  Warps: 0 TMA, 1 MMA (even CTA), 2-9
// epilogue (two per TMEM lane quarter, each taking 128 of the 256 columns in
// 16-column sub-chunks).
// ---------------------------------------------------------------------------
constexpr int ST1 = 3;
constexpr uint32_t STAGE1 = 4 * A_BYTES;   // per CTA: A hi, A lo, B hi, B lo (128 rows each)
constexpr int EPI1 = 8, THREADS1 = 64 + 32 * EPI1;

// The availability numerator W.C_off runs over all genes (K up to 46080).
// The tensor core's FP32 accumulation loses low bits toward zero on every
// MMA, so a long chain of MMAs into one accumulator drifts: measured, for
// sums of positive products, -3.7e-6 relative at K = 1024 and -1.1e-4 at
// K = 17152 (a sequential FP32 sum: -7e-8).  So A-num is summed in chunks of
// P1_CHUNK k-blocks, each into a fresh accumulator; the two TMEM buffers
// alternate between chunks, the epilogue warps (idle during the main loop)
// add each finished chunk into a running FP32 sum in global memory (this
// CTA's own 128 x 256 slot, L2-resident), and R-num, which is short, runs
// last in the buffer the chunks leave free.  32 k-blocks (2048 genes) per
// chunk: 16 halved the drift again but cost phase 1 5% more time (the
// drains' L2 traffic), 32 costs 4%.
constexpr int P1_CHUNK = 32;
// Phase 2's P tiles (K over genes, a few percent of its work) likewise, in
// chunks of P2_CHUNK k-blocks.
constexpr int P2_CHUNK = 64;

// v added into a running-sum entry in L2 without a round trip (the entry's
// earlier chunks were written by this same thread, so the adds of one entry
// happen in chunk order: the sum is deterministic)
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}
constexpr size_t P1_SLOT = 128 * 256;  // floats of one CTA's running-sum slot

// A tile cut between two CTA pairs at a chunk boundary: the pair holding its
// head (chunks 0 .. b - 1) adds them into a running-sum slot of its own for
// that tile and raises one flag per CTA rank once every add has landed; the
// pair holding its tail (chunks b .. , R-num, the epilogue) waits for the flag
// of its rank before its first access to the slot, so each entry's chunks are
// still added in chunk order.  Gives up like wait_bounded.
__device__ __forceinline__ void flag_raise(int *f)
{
    __threadfence();  // the adds of every epilogue thread of this CTA (ordered before by a barrier)
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(f), "r"(1) : "memory");
}
__device__ __forceinline__ bool flag_wait_bounded(int *f, int *abort, Ctl *ctl)
{
    const long long t0 = clock64();
    while (true) {
        int v;
        asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(f) : "memory");
        if (v) {
            *f = 0;  // consumed: the next launch's head raises it again
            return true;
        }
        if (*(volatile int *)abort)
            return false;
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
            atomicExch(abort, 1);
            atomicOr(&ctl->status, ST_TIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
}

struct Sync1 {
    uint64_t full[ST1], empty[ST1];
    uint64_t accum;
    uint64_t chunk_done[2];  // MMA -> epilogue: an A-num chunk in TMEM buffer b is complete
    uint64_t buf_free[2];    // epilogue warps of both CTAs -> MMA issuer: buffer b has been drained
    uint32_t tmem;
    int abort, issued, consumed;
};

constexpr size_t P1_COLVEC = 3 * 256;   // c_j, |W_.j|^2, |C_.j|^2 of the tile's columns
constexpr size_t P1_COLRED = 4 * 256;   // [quarter][column] sums of W'^2
constexpr size_t P1_ROWRED = 2 * 128;   // [half][row] sums of W'^2
constexpr size_t P1_BLK = 32 * 17;      // per epilogue warp: 32 x 16 staging block (padded)

constexpr size_t phase1_smem()
{
    return 1024 + (size_t)ST1 * STAGE1 + ((sizeof(Sync1) + 15) & ~size_t(15)) +
           (P1_COLVEC + P1_COLRED + P1_ROWRED + EPI1 * P1_BLK) * sizeof(float) + EPI1 * sizeof(double);
}

__device__ __forceinline__ Sync1 &phase1_sync()
{
    extern __shared__ uint8_t smem_raw[];
    return *reinterpret_cast<Sync1 *>(align1024(smem_raw) + ST1 * STAGE1);
}

// Set-up of a phase-1 CTA, once per kernel: the pipeline barriers (their
// phases then run on over every tile the CTA computes, counted by the stage
// counter g and the tile counter of phase1_tile) and the pair's 512 TMEM
// columns (a CTA gives up its allocation permit after the first allocation,
// so a persistent CTA keeps them over all its tiles).  Released by
// phase1_tmem_free.
__device__ __forceinline__ void phase1_tmem_alloc()
{
    Sync1 &sy = phase1_sync();
    if (threadIdx.x == 0) {
        for (int q = 0; q < ST1; ++q) {
            mbar_init(&sy.full[q], 1);
            mbar_init(&sy.empty[q], 1);
        }
        mbar_init(&sy.accum, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&sy.chunk_done[b], 1);
            mbar_init(&sy.buf_free[b], 2 * EPI1);
        }
        sy.abort = 0;
        fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 1)
        tmem_alloc_pair(&sy.tmem, 512);
    tc_fence_before();
    cluster_sync();  // both CTAs' barriers and TMEM address are ready before any cross-CTA signal
    tc_fence_after();
}
__device__ __forceinline__ void phase1_tmem_free()
{
    tc_fence_before();
    cluster_sync();  // both CTAs release together (also when a pair had no tile to run)
    if ((threadIdx.x >> 5) == 1) {
        tc_fence_after();
        tmem_dealloc_pair(phase1_sync().tmem, 512);
    }
}

// The body of phase 1 for the A-num chunks c0 .. c1 - 1 of the tile (mt, nt)
// of one network (c1 at or past the chunk count: through the last chunk, then
// R-num and the epilogue): maps and d are that network's (kernel parameters
// for one network, entries of arrays in global memory for a set), cur its
// current W buffer, scr this CTA's slot of 128 x 256 floats for the running
// A-num sum ([column][row]).  A piece that does not start at chunk 0 waits for
// *flag before it touches scr; one that does not end the tile raises *flag
// when its adds have landed (flag NULL: a whole tile).  g counts the pipeline
// stages, tile the pieces and u[b] the drains of TMEM buffer b this CTA has
// run before (barrier phases follow them); all advance here.  Both CTAs of
// the pair run every call together and end it at a cluster barrier, after
// which TMEM is free for the next piece.
__device__ __forceinline__ void phase1_tile(const TcMaps &maps, const Dev &d, int cur, int mt, int nt, int c0,
                                            int c1, int *flag, int &g, int &tile, int (&u)[2], float *scr)
{
    Ctl *ctl = d.ctl;
    if (!ctl->active)  // both CTAs of a pair see the same value and leave together
        return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *stages = align1024(smem_raw);
    Sync1 &sy = phase1_sync();
    float *colvec = reinterpret_cast<float *>(stages + ST1 * STAGE1 + ((sizeof(Sync1) + 15) & ~size_t(15)));
    float *colred = colvec + P1_COLVEC;
    float *rowred = colred + P1_COLRED;
    float *blocks = rowred + P1_ROWRED;
    double *hred = reinterpret_cast<double *>(blocks + EPI1 * P1_BLK);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int m0 = mt * 256 + 128 * (int)rank;  // this CTA's 128 rows (TFs)
    const int n0 = nt * 256;                    // the tile's 256 columns (genes)
    // k-blocks kb: R-num over TFs (kb < nR, 64 BF16 per row) and A-num over genes (kb >= nR, 64 BF16,
    // or 128 E4M3 under FP8MIX).  A-num runs in nc chunks of P1_CHUNK k-blocks (chunk c in TMEM
    // buffer c & 1), R-num after the last chunk (buffer nc & 1).  This piece issues, in the order
    // s = 0 .. nk - 1, the k-blocks of chunks c0 .. c1 - 1 and, if it ends the tile, R-num.
    const int nR = d.Tp / BK, nA = d.Gp / (d.fp8 ? 2 * BK : BK);
    const int nc = (nA + P1_CHUNK - 1) / P1_CHUNK, bR = nc & 1;
    c1 = c1 < nc ? c1 : nc;
    const bool ends = c1 == nc;                              // R-num and the epilogue are this piece's
    const int a0 = c0 * P1_CHUNK, nAp = min(c1 * P1_CHUNK, nA) - a0;  // the piece's A-num k-blocks
    const int nk = nAp + (ends ? nR : 0);
    auto kb_of = [nR, a0, nAp](int s) { return s < nAp ? nR + a0 + s : s - nAp; };
    const int cd = c1 < nc - 1 ? c1 : nc - 1;  // chunks c0 .. cd - 1 are drained into scr

    const int g0 = g;      // stages run by this CTA before this piece
    const uint32_t tpar = (uint32_t)tile & 1u;  // phase of the accumulator barrier for this piece
    const int u0[2] = {u[0], u[1]};  // drains of each buffer before this piece
    g += nk;
    ++tile;
    if (cd > c0) {  // the piece's i-th drain of a buffer is chunk c0 + 2 i or c0 + 1 + 2 i
        u[c0 & 1] += (cd - c0 + 1) / 2;
        u[(c0 & 1) ^ 1] += (cd - c0) / 2;
    }
    if (threadIdx.x == 0) {
        sy.issued = 0;
        sy.consumed = 0;
    }
    __syncthreads();

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer (both CTAs; completion counted on the even CTA) ----
            const int nb0 = n0 + 128 * (int)rank;  // this CTA's half of the B rows
            int s = 0;
            for (; s < nk; ++s) {
                const int kb = kb_of(s), st = (g0 + s) % ST1;
                if (!wait_bounded(&sy.empty[st], ((uint32_t)((g0 + s) / ST1) & 1u) ^ 1u, &sy.abort, ctl))
                    break;
                const uint32_t fb = mapa_shared(smem_u32(&sy.full[st]), 0);
                if (rank == 0)  // both CTAs' tiles: 4 per CTA, 3 without B's lo half, 2 of E4M3
                    mbar_arrive_expect_tx(&sy.full[st], (kb >= nR && d.fp8 ? 4 : (d.split_b ? 8 : 6)) * A_BYTES);
                uint8_t *b = stages + (size_t)st * STAGE1;
                if (kb < nR) {  // responsibility: P_off rows x W columns, K over TFs
                    const int k = kb * BK;
                    tma_load_2d_pair(b, &maps.Ph, fb, k, m0);
                    tma_load_2d_pair(b + A_BYTES, &maps.Pl, fb, k, m0);
                    for (int h = 0; h < 2; ++h) {  // W rows k.. k + 63, this CTA's 128 genes: MN-major
                        tma_load_2d_pair(b + 2 * A_BYTES + h * (A_BYTES / 2), &maps.Whm[cur], fb, nb0 + 64 * h, k);
                        if (d.split_b)
                            tma_load_2d_pair(b + 3 * A_BYTES + h * (A_BYTES / 2), &maps.Wlm[cur], fb, nb0 + 64 * h,
                                             k);
                    }
                } else if (d.fp8) {  // availability on E4M3 copies (C8 holds both triangles)
                    const int k = (kb - nR) * 2 * BK;
                    tma_load_2d_pair(b, &maps.W8[cur], fb, k, m0);
                    tma_load_2d_pair(b + A_BYTES, &maps.C8, fb, k, nb0);
                } else {        // availability: W rows x C_off rows, K over genes
                    const int k = (kb - nR) * BK;
                    tma_load_2d_pair(b, &maps.Wh[cur], fb, k, m0);
                    tma_load_2d_pair(b + A_BYTES, &maps.Wl[cur], fb, k, m0);
                    if (k >= n0) {  // C_off[j][k], k at or past the tile's diagonal block: stored rows
                        tma_load_2d_pair(b + 2 * A_BYTES, &maps.Ch, fb, k, nb0);
                        if (d.split_b)
                            tma_load_2d_pair(b + 3 * A_BYTES, &maps.Cl, fb, k, nb0);
                    } else {        // k < j: C_off[j][k] = C_off[k][j], rows k of the upper triangle
                        for (int h = 0; h < 2; ++h) {
                            tma_load_2d_pair(b + 2 * A_BYTES + h * (A_BYTES / 2), &maps.Chm, fb, nb0 + 64 * h, k);
                            if (d.split_b)
                                tma_load_2d_pair(b + 3 * A_BYTES + h * (A_BYTES / 2), &maps.Clm, fb, nb0 + 64 * h,
                                                 k);
                        }
                    }
                }
            }
            sy.issued = s;
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {  // ---- MMA issuer of the pair ----
            constexpr uint32_t idesc = idesc_bf16_f32(256, 256);
            int s = 0;
            for (; s < nk; ++s) {
                const int kb = kb_of(s), st = (g0 + s) % ST1;
                // this k-block's accumulator: A-num chunk c in buffer c & 1, R-num in buffer bR; a buffer
                // is written again only once the epilogue has drained the chunk it held two chunks before
                const int a = kb - nR, c = a / P1_CHUNK;
                const int buf = kb >= nR ? (c & 1) : bR;
                const bool fresh = kb >= nR ? a % P1_CHUNK == 0 : kb == 0;
                const int prev = kb >= nR ? c - 2 : nc - 2;  // chunk that last used buf (< c0: none here)
                if (fresh && prev >= c0 &&
                    !wait_bounded(&sy.buf_free[buf], (uint32_t)(u0[buf] + ((prev - c0) >> 1)) & 1u, &sy.abort,
                                  ctl))
                    break;
                if (!wait_bounded(&sy.full[st], (uint32_t)((g0 + s) / ST1) & 1u, &sy.abort, ctl))
                    break;
                tc_fence_after();
                const uint32_t base = smem_u32(stages + (size_t)st * STAGE1);
                const uint32_t dacc = sy.tmem + (uint32_t)buf * 256u;
                // a chunk other than the last ends: the epilogue drains it into the running sum
                const bool chunk_end = kb >= nR && c < nc - 1 && (a % P1_CHUNK == P1_CHUNK - 1);
                if (kb >= nR && d.fp8) {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)  // K = 32 per MMA
                        mma_e4m3_pair(dacc, sdesc_k_sw128(base + kk * 32), sdesc_k_sw128(base + A_BYTES + kk * 32),
                                      idesc_e4m3_f32(256, 256), (fresh && kk == 0) ? 0u : 1u);
                    mma_commit_pair(&sy.empty[st]);
                    if (chunk_end)
                        mma_commit_pair(&sy.chunk_done[buf]);
                    continue;
                }
                const bool bmn = kb < nR || (kb - nR) * BK < n0;  // B block loaded MN-major
                const uint32_t id = bmn ? (idesc | IDESC_B_MN) : idesc;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk) {
                    const uint32_t off = kk * 32;
                    const uint64_t ah = sdesc_k_sw128(base + off);
                    const uint64_t al = sdesc_k_sw128(base + A_BYTES + off);
                    const uint64_t bh = bmn ? sdesc_mn_sw128(base + 2 * A_BYTES + kk * 2048, A_BYTES / 2)
                                            : sdesc_k_sw128(base + 2 * A_BYTES + off);
                    const uint64_t bl = bmn ? sdesc_mn_sw128(base + 3 * A_BYTES + kk * 2048, A_BYTES / 2)
                                            : sdesc_k_sw128(base + 3 * A_BYTES + off);
                    mma_bf16_pair(dacc, ah, bh, id, (fresh && kk == 0) ? 0u : 1u);
                    if (d.split_b)
                        mma_bf16_pair(dacc, ah, bl, id, 1u);
                    mma_bf16_pair(dacc, al, bh, id, 1u);
                }
                mma_commit_pair(&sy.empty[st]);
                if (chunk_end)
                    mma_commit_pair(&sy.chunk_done[buf]);
            }
            sy.consumed = s;
            mma_commit_pair(&sy.accum);  // also on abort, so the epilogues can drain
        }
    } else {  // ---- epilogue: warps 2..9 of both CTAs ----
        const int e = warp - 2, wq = warp & 3, half = e >> 2;
        const int r = wq * 32 + lane, i = m0 + r, k0 = m0 + wq * 32;
        const int tt = threadIdx.x - 64;  // 0..255
        float *blk = blocks + (size_t)e * P1_BLK;
        const int nx = cur ^ 1;
        const float *W = d.W[cur];
        float *Wn = d.W[nx];
        __nv_bfloat16 *Wh = d.Wh[nx], *Wl = d.Wl[nx];
        // FP8MIX: the A-num accumulator holds the scaled E4M3 products; W' gets E4M3 copies too
        const bool q8 = d.fp8 != 0;
        const float ainv = q8 ? 1.0f / (d.f8[cur] * d.f8[2]) : 1.0f, s8 = q8 ? d.f8[3] : 1.0f;
        if (q8 && mt == 0 && nt == 0 && rank == 0 && threadIdx.x == 64)
            d.f8[nx] = s8;  // the scale of W8[nx] and Wt8[nx] from here on
        // what does not depend on the accumulators is fetched before waiting for them
        {
            const int j = n0 + tt;
            const bool cj = j < d.G;
            colvec[tt] = cj ? d.cdf[j] : 0.0f;
            colvec[256 + tt] = cj ? d.csqW[j] : 0.0f;
            colvec[512 + tt] = cj ? d.csqC[j] : 0.0f;
        }
        const bool ri = i < d.T;
        const float pdi = ri ? d.pdf[i] : 0.0f, rsp = ri ? d.rsqP[i] : 0.0f, rsw = ri ? d.rsqW[i] : 0.0f;
        const float *wrow = W + (size_t)i * d.Gp + n0 + half * 128;
        float nxt[16];
        ld16(wrow, nxt);
        epi_bar2();
        const uint32_t trow = sy.tmem + ((uint32_t)(wq * 32) << 16);
        // while the MMAs run on: add each finished A-num chunk but the last into the running sum
        // (this thread's row r, its 128 columns; [column][row] so a warp's accesses are contiguous)
        bool live = true;
        if (c0 > 0) {  // the tile's head was added into scr by another pair: wait for its flag
            if (threadIdx.x == 64 && !flag_wait_bounded(flag, &sy.abort, ctl))
                sy.abort = 1;
            epi_bar2();
            live = !*(volatile int *)&sy.abort;
        }
        const uint32_t bfree_even = mapa_shared(smem_u32(&sy.buf_free[0]), 0);
        for (int c = c0; c < cd && live; ++c) {
            const int b = c & 1;
            live = wait_bounded(&sy.chunk_done[b], (uint32_t)(u0[b] + ((c - c0) >> 1)) & 1u, &sy.abort, ctl) &&
                   !*(volatile int *)&sy.abort;
            tc_fence_after();
            if (!live)
                break;
#pragma unroll 1
            for (int j = 0; j < 8; ++j) {
                float v[16];
                tmem_ld16(trow + (uint32_t)b * 256u + half * 128 + j * 16, v);
                float *sp = scr + (size_t)(half * 128 + j * 16) * 128 + r;
                if (c == 0) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        sp[q * 128] = v[q];
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        red_add(sp + q * 128, v[q]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0)  // this warp is done with the buffer: tell the even CTA's MMA issuer
                mbar_arrive_cluster(bfree_even + (uint32_t)b * (uint32_t)sizeof(uint64_t));
        }
        if (!ends) {  // a head piece: its adds are done; the accumulator barrier's phase still completes
            live = live && wait_bounded(&sy.accum, tpar, &sy.abort, ctl) && !*(volatile int *)&sy.abort;
            epi_bar2();
            if (threadIdx.x == 64 && live)
                flag_raise(flag);
        } else {
        // the running sum's first sub-chunk, from L2 (where the adds landed), in flight while the
        // last chunk and R-num finish; each later one is fetched a sub-chunk ahead
        const float *srow = scr + (size_t)(half * 128) * 128 + r;
        float snxt[16];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            snxt[q] = (live && nc > 1) ? __ldcg(srow + (size_t)q * 128) : 0.0f;
        live = live && wait_bounded(&sy.accum, tpar, &sy.abort, ctl) && !*(volatile int *)&sy.abort;
        tc_fence_after();
        const float a = ctl->alpha, keep = 1.0f - a, halfa = 0.5f * a;
        float rowsq = 0.0f, hsum = 0.0f;
#pragma unroll 1
        for (int c = 0; c < 8 && live; ++c) {
            const int cc = half * 128 + c * 16, j0 = n0 + cc;
            float w[16], rr[16], aa[16], wn[16], sa[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                w[q] = nxt[q];
                sa[q] = snxt[q];
            }
            if (c < 7) {
                ld16(wrow + (c + 1) * 16, nxt);  // next sub-chunk's W and running sum, in flight meanwhile
                if (nc > 1) {
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        snxt[q] = __ldcg(srow + (size_t)((c + 1) * 16 + q) * 128);
                }
            }
            tmem_ld16(trow + (uint32_t)bR * 256u + cc, rr);
            tmem_ld16(trow + (uint32_t)(bR ^ 1) * 256u + cc, aa);  // the last A-num chunk
            if (nc > 1) {
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    aa[q] = sa[q] + aa[q];
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                wn[q] = 0.0f;
                if (ri && j0 + q < d.G) {
                    const float rnum = rr[q] + pdi * w[q];               // P_i. . W_.j
                    const float anum = fmaf(aa[q], ainv, w[q] * colvec[cc + q]);  // W_i. . C_.j
                    const float R = tanimoto_fast(rnum, rsp, colvec[256 + cc + q]);
                    const float A = tanimoto_fast(anum, rsw, colvec[512 + cc + q]);
                    wn[q] = keep * w[q] + halfa * (A + R);
                    hsum += fabsf(wn[q] - w[q]);
                    rowsq += wn[q] * wn[q];
                }
                blk[lane * 17 + q] = wn[q];
            }
            __syncwarp();
            // (a) W' and its split copies, row-major and coalesced: lane l takes 4 columns of rows (l >> 2) + 8 i
#pragma unroll
            for (int i2 = 0; i2 < 4; ++i2) {
                const int rr2 = (lane >> 2) + 8 * i2, jj = j0 + 4 * (lane & 3);
                float f[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    f[q] = blk[rr2 * 17 + 4 * (lane & 3) + q];
                uint32_t h2[2], l2[2];
                split_pair(f[0], f[1], h2[0], l2[0]);
                split_pair(f[2], f[3], h2[1], l2[1]);
                const size_t ro = (size_t)(k0 + rr2) * d.Gp + jj;
                *reinterpret_cast<float4 *>(Wn + ro) = make_float4(f[0], f[1], f[2], f[3]);
                *reinterpret_cast<uint2 *>(Wh + ro) = make_uint2(h2[0], h2[1]);
                *reinterpret_cast<uint2 *>(Wl + ro) = make_uint2(l2[0], l2[1]);
                if (q8)
                    *reinterpret_cast<uint32_t *>(d.W8[nx] + ro) = e4m3x2(f[0], f[1], s8) | e4m3x2(f[2], f[3], s8) << 16;
            }
            // (b) the column sums of W'^2 over the warp's 32 rows (lane l: column (l & 15), rows
            //     16 (l >> 4) + 0..15) and, under FP8MIX, the transposed E4M3 copy
            {
                const int col = lane & 15, h16 = 16 * (lane >> 4);
                float g[16];
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    g[m] = blk[(h16 + m) * 17 + col];
                float c2 = 0.0f;
#pragma unroll
                for (int m = 0; m < 16; ++m)
                    c2 += g[m] * g[m];
                c2 += __shfl_xor_sync(0xffffffffu, c2, 16);
                if (lane < 16)
                    colred[wq * 256 + cc + lane] = c2;
                if (q8) {
                    const size_t to = (size_t)(j0 + col) * d.Tp + k0 + h16;
                    uint32_t p8[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        p8[q] = e4m3x2(g[4 * q], g[4 * q + 1], s8) | e4m3x2(g[4 * q + 2], g[4 * q + 3], s8) << 16;
                    *reinterpret_cast<uint4 *>(d.Wt8[nx] + to) = make_uint4(p8[0], p8[1], p8[2], p8[3]);
                }
            }
            __syncwarp();
        }
        rowred[half * 128 + r] = rowsq;
        double hv = (double)hsum;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
            hv += __shfl_xor_sync(0xffffffffu, hv, off);
        if (lane == 0)
            hred[e] = hv;
        epi_bar2();
        if (live) {
            const int slot = m0 / 128;  // this CTA's 128-row block
            if (n0 + tt < d.Gp)
                d.wcol_part[(size_t)slot * d.Gp + n0 + tt] =
                    ((colred[tt] + colred[256 + tt]) + colred[512 + tt]) + colred[768 + tt];
            if (tt < 128)
                d.wrow_part[(size_t)nt * d.Tp + m0 + tt] = rowred[tt] + rowred[128 + tt];
            if (tt == 0) {
                double hs = 0.0;
                for (int q = 0; q < EPI1; ++q)
                    hs += hred[q];
                d.hpart[(size_t)nt * d.nbT + slot] = hs;
            }
        }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && rank == 0)  // loads counted here but not consumed (abort only)
        for (int s = sy.consumed; s < sy.consumed + ST1 && s < sy.issued; ++s)
            wait_bounded(&sy.full[(g0 + s) % ST1], (uint32_t)((g0 + s) / ST1) & 1u, &sy.abort, ctl, true);
    cluster_sync();  // neither CTA goes on while the pair may still signal it
}


// One network: persistent CTA pairs (at most one per SM pair), pair p over
// its host-built list items[off[p] .. off[p + 1]) of pieces (mt, nt, chunks
// c0 | c1 << 16, cut): whole tiles (cut < 0) in rounds of the gene-block-major
// order, and tiles cut between two pairs at a chunk boundary, whose two
// pieces meet in running-sum slot `cut` (see build_p1).
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS1, 1)
    k_tc_phase1(const __grid_constant__ TcMaps maps, const __grid_constant__ Dev d, int cur, const int4 *items,
                const int *off)
{
    if (!d.ctl->active)  // both CTAs of a pair see the same value and leave together
        return;
    phase1_tmem_alloc();
    int g = 0, tile = 0, u[2] = {0, 0};
    const int pair = blockIdx.x >> 1, rank = (int)cluster_ctarank();
    for (int q = off[pair]; q < off[pair + 1]; ++q) {
        const int4 w = items[q];
        const bool cut = w.w >= 0;
        float *scr = cut ? d.p1_fix + (size_t)(2 * w.w + rank) * P1_SLOT : d.p1_acc + (size_t)blockIdx.x * P1_SLOT;
        phase1_tile(maps, d, cur, w.x, w.y, w.z & 0xffff, w.z >> 16, cut ? d.p1_flag + 2 * w.w + rank : nullptr, g,
                    tile, u, scr);
    }
    phase1_tmem_free();
}

// A set of networks: persistent CTA pairs, each over its host-built list of
// (network, mt, nt) tiles; tiles of networks that have stopped are skipped by
// both CTAs alike.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(THREADS1, 1) k_tc_phase1_set(const SetArgs a)
{
    const int pair = blockIdx.x >> 1;
    phase1_tmem_alloc();
    int g = 0, tile = 0, u[2] = {0, 0};
    float *scr = a.acc + (size_t)blockIdx.x * P1_SLOT;
    for (int q = a.p1_off[pair]; q < a.p1_off[pair + 1]; ++q) {
        const int4 w = a.items1[q];  // (network, mt, nt, cost)
        phase1_tile(a.maps[w.x], a.devs[w.x], set_cur(a, w.x), w.y, w.z, 0, 1 << 15, nullptr, g, tile, u, scr);
    }
    phase1_tmem_free();
}

// ---------------------------------------------------------------------------
// Phase 2: persistent CTA pairs over a host-built schedule of upper-triangle
// 256 x 256 tiles of W'.W'^T (P, K = genes) and W'^T.W' (C, K = TFs).  In a
// pair, CTA r loads rows 128 r .. 128 r + 127 of the tile's A and B blocks;
// the even CTA issues cta_group::2 MMAs (M = N = 256) whose result rows
// 128 r .. + 127 land in CTA r's TMEM.  Two accumulators of 256 columns
// alternate, so the epilogue of one tile overlaps the MMAs of the next.
// Warps: 0 TMA, 1 MMA (even CTA), then EPI epilogue warps (EPI / 4 per
// TMEM lane quarter, splitting the 256 columns in 16-column sub-chunks).
//
// Row partial sums for Eq. 6 use separate slot ranges so the two CTAs of a
// pair never exchange data: the row role (a row of the tile, summed over its
// 256 columns) goes to slot bn, the column role (a column of the tile, summed
// over this CTA's 128 rows) to slot nb + 2 bm + r.
// ---------------------------------------------------------------------------
// Epilogue warps: EPI / 4 per TMEM lane quarter, a template parameter of the
// phase-2 kernels.  A C' tile has K = T, so its MMAs take about as long as its
// 256 x 256 outputs take to finish: where the MMAs are the shorter part
// (T up to about 1300 in BF16X3), twelve epilogue warps with two 64 KB
// operand stages ran phase 2 5% faster than eight with three at 1000 x 17000;
// where they are the longer part, the third stage keeps them fed (1600 x
// 30000: 3.0 ms against 3.7 with two).  p2_epi picks one per launch.
constexpr int N2 = 256;                    // tile edge
constexpr uint32_t STAGE2 = 4 * A_BYTES;   // per CTA: A hi, A lo, B hi, B lo (128 rows each)

// named barrier among the phase-2 epilogue warps
template <int EPI>
__device__ __forceinline__ void epi_bar_p2()
{
    asm volatile("bar.sync 2, %0;" ::"n"(32 * EPI) : "memory");
}

// A tile row's sums for Eq. 6 are taken over four fixed column groups of
// sub-chunks, [0, 5), [5, 8), [8, 10) and [10, 16), each added in column
// order by one warp and then the four in group order: both epilogue
// configurations (parts [0, 5), [5, 10), [10, 16) of twelve warps, [0, 8),
// [8, 16) of eight) split along these boundaries, so the sums, and every
// result, are the same to the bit whichever configuration runs.
constexpr int P2_GROUPS = 4;
__host__ __device__ constexpr int p2_group(int c) { return c < 5 ? 0 : c < 8 ? 1 : c < 10 ? 2 : 3; }

template <bool SIM, int EPI>
struct P2Cfg {
    static constexpr int THREADS = 64 + 32 * EPI;      // TMA warp, MMA warp, epilogue warps
    static constexpr int NS = SIM ? 3 : 2;             // sums per row: x, x^2 (and v^2 under D2)
    static constexpr int ST = EPI > 8 || SIM ? 2 : 3;  // pipeline stages that fit beside the epilogue buffers
    static constexpr size_t COLRED = 4 * NS * N2;      // [quarter][sum][column] floats
    static constexpr size_t ROWRED = P2_GROUPS * NS * 128;  // [column group][sum][row] floats
    static constexpr size_t COLNRM = N2;               // the tile's column norms
    static constexpr size_t BLK = 32 * 17;             // per epilogue warp: 32 x 16 staging block (padded)
};

// A scheduled phase-2 item.  A C tile (bit 31 clear: bits 16-30 row block,
// 0-15 column block) is one item over all of its K (TFs).  A P tile's K runs
// over all genes, so, like phase 1's availability product, it is summed in
// chunks of P2_CHUNK k-blocks, each into a fresh accumulator: the tile is
// scheduled as consecutive items on one CTA pair (bit 31 set: bits 24-30 the
// chunk, 16-23 row block, 0-15 column block); the epilogue adds every chunk
// but the last into the CTA's running-sum slot and finishes the tile on the
// last.
struct P2Item {
    bool isP;
    int bm, bn, kb0, kb1, chunk, nchunks;
};
__host__ __device__ inline int p2_chunks(const Dev &d) { return (d.Gp / BK + P2_CHUNK - 1) / P2_CHUNK; }
__device__ __forceinline__ P2Item p2_item(int tile, const Dev &d)
{
    P2Item it;
    it.isP = tile < 0;
    it.bn = tile & 0xffff;
    if (it.isP) {
        it.bm = (tile >> 16) & 0xff;
        it.chunk = (tile >> 24) & 0x7f;
        it.nchunks = p2_chunks(d);
        it.kb0 = it.chunk * P2_CHUNK;
        it.kb1 = min(d.Gp / BK, it.kb0 + P2_CHUNK);
    } else {
        it.bm = (tile >> 16) & 0x7fff;
        it.chunk = 0;
        it.nchunks = 1;
        it.kb0 = 0;
        it.kb1 = d.Tp / (d.fp8 ? 2 * BK : BK);
    }
    return it;
}

template <int ST>
struct Sync2T {
    uint64_t full[ST], empty[ST];
    uint64_t tfull[2], tempty[2];  // accumulator ready / accumulator drained (by both CTAs)
    uint32_t tmem;
    int abort, issued, consumed;
};

template <bool SIM, int EPI>
constexpr size_t phase2_smem()
{
    using C = P2Cfg<SIM, EPI>;
    return 1024 + (size_t)C::ST * STAGE2 + ((sizeof(Sync2T<C::ST>) + 15) & ~size_t(15)) +
           (C::COLRED + C::ROWRED + C::COLNRM + EPI * C::BLK) * sizeof(float);
}

// Where phase 2 finds the network of each scheduled tile: one network given
// by value (its state, maps and W buffer are kernel parameters), or a set.
struct P2One {
    const TcMaps &m;
    const Dev &d;
    int c;
    const int *off, *tiles;
    __device__ float *scratch() const { return d.p1_acc + (size_t)blockIdx.x * P1_SLOT; }
    __device__ int net(int) const { return 0; }
    __device__ const Dev &dev(int) const { return d; }
    __device__ const TcMaps &maps(int) const { return m; }
    __device__ int cur(int) const { return c; }  // the W' buffer (the launch passes it)
    __device__ bool active(int) const { return true; }  // the kernel left at once otherwise
};
struct P2Set {
    const SetArgs &a;
    const int *off, *tiles;
    __device__ float *scratch() const { return a.acc + (size_t)blockIdx.x * P1_SLOT; }
    __device__ int net(int n) const { return a.sched_net[n]; }
    __device__ const Dev &dev(int k) const { return a.devs[k]; }
    __device__ const TcMaps &maps(int k) const { return a.maps[k]; }
    // phase 2 works on W' (the other buffer: the count moves on only in k_tail)
    __device__ int cur(int k) const { return set_cur(a, k) ^ 1; }
    __device__ bool active(int k) const { return a.devs[k].ctl->active != 0; }
};

// The body of phase 2 for one CTA pair's scheduled tiles.  A stopped network's
// tiles are skipped by every role alike (its control block does not change
// during the launch), so the stage and accumulator counters stay in step.
// ctl: where a timed-out wait outside any tile is reported.
template <bool SIM_SIGMA, int EPI, class Src>
__device__ __forceinline__ void phase2_pair(const Src &src, Ctl *ctl)
{
    using Cfg = P2Cfg<SIM_SIGMA, EPI>;
    constexpr int ST2 = Cfg::ST, NS = Cfg::NS;
    using Sync2 = Sync2T<ST2>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *stages = align1024(smem_raw);
    Sync2 &sy = *reinterpret_cast<Sync2 *>(stages + ST2 * STAGE2);
    float *colred = reinterpret_cast<float *>(stages + ST2 * STAGE2 + ((sizeof(Sync2) + 15) & ~size_t(15)));
    float *rowred = colred + Cfg::COLRED;
    float *colnrm = rowred + Cfg::ROWRED;
    float *blocks = colnrm + Cfg::COLNRM;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const int pair = blockIdx.x >> 1;
    const int first = src.off[pair], last = src.off[pair + 1];

    if (threadIdx.x == 0) {
        for (int q = 0; q < ST2; ++q) {
            mbar_init(&sy.full[q], 1);
            mbar_init(&sy.empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&sy.tfull[q], 1);
            mbar_init(&sy.tempty[q], 2 * EPI);
        }
        sy.abort = 0;
        sy.issued = 0;
        sy.consumed = 0;
        fence_mbar_init();
    }
    if (warp == 1)
        tmem_alloc_pair(&sy.tmem, 2 * N2);
    tc_fence_before();
    cluster_sync();  // both CTAs' barriers exist before any cross-CTA signal
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {  // ---- TMA producer (both CTAs; completion counted on the even CTA) ----
            int g = 0;
            bool ok = true;
            for (int n = first; n < last && ok; ++n) {
                const int net = src.net(n);
                if (!src.active(net))
                    continue;
                const Dev &d = src.dev(net);
                const TcMaps &maps = src.maps(net);
                const int cur = src.cur(net);
                const P2Item it = p2_item(src.tiles[n], d);
                const bool isP = it.isP;
                const int m0 = it.bm * N2 + 128 * rank, n0 = it.bn * N2 + 128 * rank;
                const bool q8 = d.fp8 && !isP;  // FP8MIX: C tiles from the E4M3 copy of W'^T, one term
                // P tiles: rows of W' (K over genes, K-major); C tiles: columns of W' (K over TFs),
                // read from the same arrays MN-major
                const CUtensorMap *mh = isP ? &maps.Wh[cur] : &maps.Whm[cur];
                const CUtensorMap *ml = isP ? &maps.Wl[cur] : &maps.Wlm[cur];
                for (int kb = it.kb0; kb < it.kb1; ++kb, ++g) {
                    const int st = g % ST2;
                    if (!wait_bounded(&sy.empty[st], ((uint32_t)(g / ST2) & 1u) ^ 1u, &sy.abort, d.ctl)) {
                        ok = false;
                        break;
                    }
                    const uint32_t fb = mapa_shared(smem_u32(&sy.full[st]), 0);
                    if (rank == 0)  // both CTAs' tiles: 4 per CTA, 3 without B's lo half, 2 of E4M3
                        mbar_arrive_expect_tx(&sy.full[st], (q8 ? 4 : (d.split_b ? 8 : 6)) * A_BYTES);
                    uint8_t *b = stages + (size_t)st * STAGE2;
                    if (q8) {
                        tma_load_2d_pair(b, &maps.Wt8[cur], fb, kb * 2 * BK, m0);
                        tma_load_2d_pair(b + A_BYTES, &maps.Wt8[cur], fb, kb * 2 * BK, n0);
                        continue;
                    }
                    if (isP) {
                        tma_load_2d_pair(b, mh, fb, kb * BK, m0);
                        tma_load_2d_pair(b + A_BYTES, ml, fb, kb * BK, m0);
                        tma_load_2d_pair(b + 2 * A_BYTES, mh, fb, kb * BK, n0);
                        if (d.split_b)
                            tma_load_2d_pair(b + 3 * A_BYTES, ml, fb, kb * BK, n0);
                        continue;
                    }
                    for (int h = 0; h < 2; ++h) {  // two 64 x 64 boxes per 128 genes
                        const uint32_t o = h * (A_BYTES / 2);
                        tma_load_2d_pair(b + o, mh, fb, m0 + 64 * h, kb * BK);
                        tma_load_2d_pair(b + A_BYTES + o, ml, fb, m0 + 64 * h, kb * BK);
                        tma_load_2d_pair(b + 2 * A_BYTES + o, mh, fb, n0 + 64 * h, kb * BK);
                        if (d.split_b)
                            tma_load_2d_pair(b + 3 * A_BYTES + o, ml, fb, n0 + 64 * h, kb * BK);
                    }
                }
            }
            sy.issued = g;
        }
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {  // ---- MMA issuer of the pair ----
            constexpr uint32_t idesc = idesc_bf16_f32(256, N2);
            int g = 0;
            bool ok = true;
            for (int n = first, idx = -1; n < last && ok; ++n) {
                const int net = src.net(n);
                if (!src.active(net))
                    continue;
                ++idx;
                const Dev &d = src.dev(net);
                const int tile = src.tiles[n];
                const P2Item it = p2_item(tile, d);
                const bool q8 = d.fp8 && tile >= 0;
                const int buf = idx & 1;
                if (!wait_bounded(&sy.tempty[buf], ((uint32_t)(idx >> 1) & 1u) ^ 1u, &sy.abort, d.ctl))
                    break;
                tc_fence_after();
                const uint32_t dacc = sy.tmem + buf * N2;
                for (int kb = it.kb0; kb < it.kb1; ++kb, ++g) {
                    const bool first = kb == it.kb0;  // a fresh accumulator for every item
                    const int st = g % ST2;
                    if (!wait_bounded(&sy.full[st], (uint32_t)(g / ST2) & 1u, &sy.abort, d.ctl)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(stages + (size_t)st * STAGE2);
                    if (q8) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)  // K = 32 per MMA
                            mma_e4m3_pair(dacc, sdesc_k_sw128(base + kk * 32),
                                          sdesc_k_sw128(base + A_BYTES + kk * 32), idesc_e4m3_f32(256, N2),
                                          (first && kk == 0) ? 0u : 1u);
                        mma_commit_pair(&sy.empty[st]);
                        continue;
                    }
                    const bool mn = tile >= 0;  // C tiles: both operands MN-major
                    const uint32_t id = mn ? (idesc | IDESC_A_MN | IDESC_B_MN) : idesc;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint32_t off = kk * 32, moff = kk * 2048;
                        const uint64_t ah = mn ? sdesc_mn_sw128(base + moff, A_BYTES / 2) : sdesc_k_sw128(base + off);
                        const uint64_t al = mn ? sdesc_mn_sw128(base + A_BYTES + moff, A_BYTES / 2)
                                               : sdesc_k_sw128(base + A_BYTES + off);
                        const uint64_t bh = mn ? sdesc_mn_sw128(base + 2 * A_BYTES + moff, A_BYTES / 2)
                                               : sdesc_k_sw128(base + 2 * A_BYTES + off);
                        const uint64_t bl = mn ? sdesc_mn_sw128(base + 3 * A_BYTES + moff, A_BYTES / 2)
                                               : sdesc_k_sw128(base + 3 * A_BYTES + off);
                        if (d.split_b) {  // hi(A) once from shared memory for hi.hi and hi.lo
                            mma_bf16_pair_fill_a(dacc, ah, bh, id, (first && kk == 0) ? 0u : 1u);
                            mma_bf16_pair_lastuse_a(dacc, ah, bl, id, 1u);
                        } else {
                            mma_bf16_pair(dacc, ah, bh, id, (first && kk == 0) ? 0u : 1u);
                        }
                        mma_bf16_pair(dacc, al, bh, id, 1u);
                    }
                    mma_commit_pair(&sy.empty[st]);
                }
                mma_commit_pair(&sy.tfull[buf]);
            }
            sy.consumed = g;
        }
    } else {  // ---- epilogue: warps 2..9 of both CTAs ----
        // the EPI / 4 warps of a lane quarter split its 16 sub-chunks of 16 columns
        constexpr int PARTS = EPI / 4;
        const int e = warp - 2, wq = warp & 3, third = e >> 2;
        const int c_begin = (16 * third) / PARTS, c_end = (16 * (third + 1)) / PARTS;
        const int r = wq * 32 + lane;  // row of this CTA's 128-row half
        float *blk = blocks + (size_t)e * Cfg::BLK;  // this warp's 32 x 16 staging block, rows of 17
        const int tt = threadIdx.x - 64;  // 0..383
        const uint32_t tempty_even = mapa_shared(smem_u32(&sy.tempty[0]), 0);
        float *scr = src.scratch();  // running sums of P tiles' K chunks ([column][row])
        for (int n = first, idx = -1; n < last; ++n) {
            const int net = src.net(n);
            if (!src.active(net))
                continue;
            ++idx;
            const Dev &d = src.dev(net);
            const P2Item it = p2_item(src.tiles[n], d);
            if (it.chunk + 1 < it.nchunks) {  // a P tile's K chunk before the last: into the running sum
                const int buf = idx & 1;
                const bool ok = wait_bounded(&sy.tfull[buf], (uint32_t)(idx >> 1) & 1u, &sy.abort, d.ctl) &&
                                !*(volatile int *)&sy.abort;
                tc_fence_after();
                if (ok) {
                    const uint32_t tb = sy.tmem + buf * N2 + ((uint32_t)(wq * 32) << 16);
#pragma unroll 1
                    for (int c = c_begin; c < c_end; ++c) {  // this warp's 16-column sub-chunks
                        float v[16];
                        tmem_ld16(tb + c * 16, v);
                        float *sp = scr + (size_t)(c * 16) * 128 + r;
                        if (it.chunk == 0) {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                sp[q * 128] = v[q];
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q)
                                red_add(sp + q * 128, v[q]);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive_cluster(tempty_even + buf * (uint32_t)sizeof(uint64_t));
                }
                continue;
            }
            const int cur = src.cur(net);
            const float a = d.ctl->alpha, keep = 1.0f - a;
            // FP8MIX: C-tile accumulators hold products of W'^T scaled by f8[cur] on both sides; C' gets
            // an E4M3 copy scaled so that no entry saturates (bound from |C_k.| and |W'_.k|)
            const float sw = d.fp8 ? d.f8[cur] : 1.0f, ainv2 = 1.0f / (sw * sw);
            const float sC =
                d.fp8 ? e4m3_scale(fp8_bound_c(__uint_as_float(d.f8n[5]), __uint_as_float(d.f8n[3]))) : 1.0f;
            if (d.fp8 && threadIdx.x == 64)
                d.f8[2] = sC;  // the scale of C8 from here on (every writer stores the same value)
            const bool isP = it.isP;
            const int bm = it.bm, bn = it.bn;
            const int m0 = bm * N2 + 128 * (int)rank, n0 = bn * N2;
            const int nn = isP ? d.T : d.G, ld = isP ? d.Tp : d.Gp;
            const int nbk = ceil_div(ld, N2);  // 256-blocks: the column-role slots start here
            const float *nrm = isP ? d.rsqW : d.csqW;
            float *X = isP ? d.Poff : d.Coff;
            __nv_bfloat16 *Xh = isP ? d.Ph : d.Ch, *Xl = isP ? d.Pl : d.Cl;
            // BF16X3, BF16X2: C is held as its split pair alone (old values hi + lo, no FP32 store)
            const bool sst = !isP && d.c_split;
            const bool wlo = isP || d.split_b || sst;
            // split copies of the lower triangle: all of P (phase 1 reads its rows K-major), but of C
            // only inside diagonal 256-blocks (phase 1 reads the rest of C's lower triangle MN-major)
            const bool q8 = d.fp8 && !isP;
            const bool mirror = isP || bm == bn || q8;  // the E4M3 copy of C holds both triangles
            const float ascale = q8 ? ainv2 : 1.0f;
            const int buf = idx & 1;
            // everything that does not depend on the accumulator is fetched before waiting for it:
            // the tile's column norms (shared), this row's norm and its first old values
            if (tt < N2)
                colnrm[tt] = n0 + tt < nn ? nrm[n0 + tt] : 0.0f;
            const int k = m0 + r, k0 = m0 + wq * 32;
            const bool krow = k < nn;  // rows past the network (last block's padding) hold nothing
            const float nk_ = krow ? nrm[k] : 0.0f;
            // old values (rows past the network are padding inside the array; their values are never
            // used).  FP32: loaded coalesced (8 rows x 64 B per load), lane l takes columns
            // 4 (l & 3) .. + 3 of the warp's rows (l >> 2) + 8 i, i = 0..3, and each lane gets its own
            // row through the staging block.  A split-held C: each lane loads its own row, 32 bytes of
            // each half per sub-chunk, L2 fetching the row's 256-byte block at the first
            const size_t xo = sst ? (size_t)k * ld + n0 : (size_t)(k0 + (lane >> 2)) * ld + n0 + 4 * (lane & 3);
            const float *xblk = sst ? nullptr : X + xo;
            float4 nxt[4];
            if (n0 + c_begin * 16 < ld) {
                if (sst)
                    ld_row16_split(Xh + xo + c_begin * 16, Xl + xo + c_begin * 16, nxt);
                else
                    ld_rows4(xblk + c_begin * 16, ld, nxt);
            }
            epi_bar_p2<EPI>();
            // on a timed-out wait every epilogue warp still runs the named barriers below
            const bool live = wait_bounded(&sy.tfull[buf], (uint32_t)(idx >> 1) & 1u, &sy.abort, d.ctl) &&
                              !*(volatile int *)&sy.abort;
            tc_fence_after();
            float r1 = 0.0f, r2 = 0.0f, rv = 0.0f;
            // this warp's row sums of a column group, into its slot (zeros where nothing was summed)
            auto flush = [&](int grp) {
                rowred[(grp * NS + 0) * 128 + r] = r1;
                rowred[(grp * NS + 1) * 128 + r] = r2;
                if (SIM_SIGMA)
                    rowred[(grp * NS + 2) * 128 + r] = rv;
                r1 = r2 = rv = 0.0f;
            };
            for (int grp = p2_group(c_begin); grp <= p2_group(c_end - 1); ++grp)
                flush(grp);  // (all zero: a timed-out tile leaves no stale sums)
            const uint32_t tbase = sy.tmem + buf * N2 + ((uint32_t)(wq * 32) << 16);
            // accumulator columns one sub-chunk ahead: each sub-chunk's TMEM load is issued once the
            // previous one's arithmetic is done and lands while that one's stores go out
            uint32_t accr[16];
            if (live)
                tmem_ld16_nowait(tbase + c_begin * 16, accr);
#pragma unroll 1
            for (int c = c_begin; c < c_end && live; ++c) {  // this warp's 16-column sub-chunks
                const int cc = c * 16, j0 = n0 + cc;
                const bool inside = krow && j0 < ld;
                if (c > c_begin && p2_group(c) != p2_group(c - 1))
                    flush(p2_group(c - 1));
                float old[16], acc[16];
                if (sst) {  // this lane's own row
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        old[4 * i] = inside ? nxt[i].x : 0.0f;
                        old[4 * i + 1] = inside ? nxt[i].y : 0.0f;
                        old[4 * i + 2] = inside ? nxt[i].z : 0.0f;
                        old[4 * i + 3] = inside ? nxt[i].w : 0.0f;
                    }
                } else {  // to this lane's own row through the staging block
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        float *b = blk + ((lane >> 2) + 8 * i) * 17 + 4 * (lane & 3);
                        b[0] = nxt[i].x; b[1] = nxt[i].y; b[2] = nxt[i].z; b[3] = nxt[i].w;
                    }
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        old[q] = inside ? blk[lane * 17 + q] : 0.0f;
                    __syncwarp();  // the block takes the new values next
                }
                if (c + 1 < c_end && j0 + 16 < ld) {  // next sub-chunk's old values, in flight meanwhile
                    if (sst)
                        ld_row16_split(Xh + xo + (c + 1) * 16, Xl + xo + (c + 1) * 16, nxt);
                    else
                        ld_rows4(xblk + (c + 1) * 16, ld, nxt);
                }
                tmem_wait16(accr);
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    acc[q] = __uint_as_float(accr[q]) * ascale;
                if (it.nchunks > 1) {  // a P tile's last K chunk: add the running sum of the others
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        acc[q] = __ldcg(scr + (size_t)(cc + q) * 128 + r) + acc[q];  // L2: where the adds landed
                }
                if (c + 1 == c_end) {  // this warp is done with the accumulator: tell the even CTA
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0)
                        mbar_arrive_cluster(tempty_even + buf * (uint32_t)sizeof(uint64_t));
                }
                // interior sub-chunks of off-diagonal tiles are entirely valid
                uint32_t vmask = 0xffffu;
                if (!(k < j0 && j0 + 15 < nn)) {
                    vmask = 0;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        vmask |= (k < j0 + q && j0 + q < nn) ? (1u << q) : 0u;
                }
                if (vmask == 0xffffu) {  // interior: no masking
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 n4 = reinterpret_cast<const float4 *>(colnrm + cc)[q];
                        const float nj[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int e2 = 4 * q + u;
                            const float s = tanimoto_clamped(acc[e2], nk_, nj[u]);
                            const float v = fmaf(a, s, keep * old[e2]);
                            const float x = SIM_SIGMA ? s : v;
                            r1 += x;
                            r2 = fmaf(x, x, r2);
                            if (SIM_SIGMA)
                                rv = fmaf(v, v, rv);
                            old[e2] = v;
                            acc[e2] = x;
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const float s = tanimoto_fast(acc[q], nk_, colnrm[cc + q]);
                        const bool valid = (vmask >> q) & 1u;
                        const float v = valid ? fmaf(a, s, keep * old[q]) : old[q];
                        const float x = valid ? (SIM_SIGMA ? s : v) : 0.0f;
                        r1 += x;
                        r2 += x * x;
                        if (SIM_SIGMA)
                            rv += valid ? v * v : 0.0f;
                        old[q] = v;
                        acc[q] = x;
                    }
                }
                // column sums of s under D2 (from registers; v sums come from the staged block)
                if (SIM_SIGMA) {
                    float sq[16];  // old[] holds the new values, staged below; acc is consumed here
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        sq[q] = acc[q] * acc[q];
                    const float t1 = lane_transpose_sum16(sq);
                    const float t0 = lane_transpose_sum16(acc);
                    if (lane < 16) {
                        colred[(wq * NS + 1) * N2 + cc + lane] = t1;
                        colred[(wq * NS + 0) * N2 + cc + lane] = t0;
                    }
                }
                if (c + 1 < c_end)
                    tmem_ld16_nowait(tbase + cc + 16, accr);
                // stage the new values (0 where nothing is stored) in this warp's block
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    blk[lane * 17 + q] = (vmask >> q & 1u) ? old[q] : 0.0f;
                __syncwarp();
                // (a) row-major copies, coalesced.  A split-held C: lane l takes 8 columns of rows
                // (l >> 1) + 16 i, 16-byte stores of each half
                if (sst) {
#pragma unroll
                    for (int i2 = 0; i2 < 2; ++i2) {
                        const int rr = (lane >> 1) + 16 * i2, kk = k0 + rr, jj = j0 + 8 * (lane & 1);
                        float f[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            f[q] = blk[rr * 17 + 8 * (lane & 1) + q];
                        uint32_t h4[4], l4[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            split_pair(f[2 * q], f[2 * q + 1], h4[q], l4[q]);
                        const size_t ro = (size_t)kk * ld + jj;
                        if (kk < jj && jj + 7 < nn) {
                            *reinterpret_cast<uint4 *>(Xh + ro) = make_uint4(h4[0], h4[1], h4[2], h4[3]);
                            *reinterpret_cast<uint4 *>(Xl + ro) = make_uint4(l4[0], l4[1], l4[2], l4[3]);
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; ++q)
                                if (kk < jj + q && jj + q < nn) {
                                    reinterpret_cast<uint16_t *>(Xh)[ro + q] = (uint16_t)(h4[q >> 1] >> (16 * (q & 1)));
                                    reinterpret_cast<uint16_t *>(Xl)[ro + q] = (uint16_t)(l4[q >> 1] >> (16 * (q & 1)));
                                }
                        }
                    }
                }
#pragma unroll
                for (int i2 = 0; i2 < (sst ? 0 : 4); ++i2) {
                    const int rr = (lane >> 2) + 8 * i2, kk = k0 + rr, jj = j0 + 4 * (lane & 3);
                    float f[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        f[q] = blk[rr * 17 + 4 * (lane & 3) + q];
                    const size_t ro = (size_t)kk * ld + jj;
                    if (q8) {
                        if (kk < jj && jj + 3 < nn) {
                            *reinterpret_cast<float4 *>(X + ro) = make_float4(f[0], f[1], f[2], f[3]);
                            *reinterpret_cast<uint32_t *>(d.C8 + ro) =
                                e4m3x2(f[0], f[1], sC) | e4m3x2(f[2], f[3], sC) << 16;
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                if (kk < jj + q && jj + q < nn) {
                                    X[ro + q] = f[q];
                                    d.C8[ro + q] = (uint8_t)e4m3x2(f[q], 0.0f, sC);
                                }
                        }
                        continue;
                    }
                    uint32_t h2[2], l2[2];
                    split_pair(f[0], f[1], h2[0], l2[0]);
                    split_pair(f[2], f[3], h2[1], l2[1]);
                    if (kk < jj && jj + 3 < nn) {
                        if (!sst)
                            *reinterpret_cast<float4 *>(X + ro) = make_float4(f[0], f[1], f[2], f[3]);
                        *reinterpret_cast<uint2 *>(Xh + ro) = make_uint2(h2[0], h2[1]);
                        if (wlo)
                            *reinterpret_cast<uint2 *>(Xl + ro) = make_uint2(l2[0], l2[1]);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (kk < jj + q && jj + q < nn) {
                                if (!sst)
                                    X[ro + q] = f[q];
                                reinterpret_cast<uint16_t *>(Xh)[ro + q] = (uint16_t)(h2[q >> 1] >> (16 * (q & 1)));
                                if (wlo)
                                    reinterpret_cast<uint16_t *>(Xl)[ro + q] =
                                        (uint16_t)(l2[q >> 1] >> (16 * (q & 1)));
                            }
                    }
                }
                // (b) mirrored entries (j, k): lane l takes column (l & 15), rows 16 (l >> 4) + 0..15,
                //     and the column sums over the warp's 32 rows
                {
                    const int col = lane & 15, h16 = 16 * (lane >> 4);
                    float g[16];
#pragma unroll
                    for (int m = 0; m < 16; ++m)
                        g[m] = blk[(h16 + m) * 17 + col];
                    float c1 = 0.0f, c2 = 0.0f;
#pragma unroll
                    for (int m = 0; m < 16; ++m) {
                        c1 += g[m];
                        c2 += g[m] * g[m];
                    }
                    c1 += __shfl_xor_sync(0xffffffffu, c1, 16);
                    c2 += __shfl_xor_sync(0xffffffffu, c2, 16);
                    if (lane < 16) {
                        if (SIM_SIGMA) {
                            colred[(wq * NS + 2) * N2 + cc + lane] = c2;  // sum of v^2
                        } else {
                            colred[(wq * NS + 0) * N2 + cc + lane] = c1;
                            colred[(wq * NS + 1) * N2 + cc + lane] = c2;
                        }
                    }
                    if (mirror && q8) {
                        const int jm = j0 + col, km = k0 + h16;
                        const uint32_t mmask =
                            jm >= nn ? 0u : (km + 15 < jm ? 0xffffu : (km >= jm ? 0u : ((1u << (jm - km)) - 1u)));
                        if (mmask) {
                            uint32_t p8[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                p8[q] = e4m3x2(g[4 * q], g[4 * q + 1], sC) | e4m3x2(g[4 * q + 2], g[4 * q + 3], sC) << 16;
                            uint8_t *dst = d.C8 + (size_t)jm * ld + km;
                            if (mmask == 0xffffu) {
                                *reinterpret_cast<uint4 *>(dst) = make_uint4(p8[0], p8[1], p8[2], p8[3]);
                            } else {
#pragma unroll
                                for (int q = 0; q < 16; ++q)
                                    if (mmask >> q & 1u)
                                        dst[q] = (uint8_t)(p8[q >> 2] >> (8 * (q & 3)));
                            }
                        }
                    } else if (mirror) {
                        uint32_t hv[8], lv[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            split_pair(g[2 * q], g[2 * q + 1], hv[q], lv[q]);
                        const int jm = j0 + col, km = k0 + h16;
                        const uint32_t mmask =
                            jm >= nn ? 0u : (km + 15 < jm ? 0xffffu : (km >= jm ? 0u : ((1u << (jm - km)) - 1u)));
                        if (mmask) {
                            const size_t mo = (size_t)jm * ld + km;
                            st16_packed(Xh + mo, hv, mmask);
                            if (wlo)
                                st16_packed(Xl + mo, lv, mmask);
                        }
                    }
                }
                __syncwarp();  // the block is rewritten by the next sub-chunk
            }
            if (live)
                flush(p2_group(c_end - 1));
            epi_bar_p2<EPI>();
            if (live) {
#pragma unroll
                for (int w = 0; w < 3; ++w) {
                    float *S = w == 0 ? (isP ? d.ps_sum : d.cs_sum) : w == 1 ? (isP ? d.ps_sq : d.cs_sq)
                                                                            : (isP ? d.ps_vsq : d.cs_vsq);
                    const int wc = (!SIM_SIGMA && w == 2) ? 1 : w;  // sum of v^2 = sum of x^2 unless D2
                    // column role: tile column tt, summed over this CTA's 128 rows
                    if (tt < N2 && n0 + tt < ld)
                        S[(size_t)(nbk + 2 * bm + (int)rank) * ld + n0 + tt] =
                            ((colred[(0 * NS + wc) * N2 + tt] + colred[(1 * NS + wc) * N2 + tt]) +
                             colred[(2 * NS + wc) * N2 + tt]) + colred[(3 * NS + wc) * N2 + tt];
                    // row role: tile row tt of this CTA, summed over the 256 columns
                    if (tt < 128 && m0 + tt < ld) {
                        float rs = 0.0f;
#pragma unroll
                        for (int grp = 0; grp < P2_GROUPS; ++grp)
                            rs += rowred[(grp * NS + wc) * 128 + tt];
                        S[(size_t)bn * ld + m0 + tt] = rs;
                    }
                }
            }
            epi_bar_p2<EPI>();
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && rank == 0)  // loads counted here but not consumed (abort only)
        for (int g = sy.consumed; g < sy.consumed + ST2 && g < sy.issued; ++g)
            wait_bounded(&sy.full[g % ST2], (uint32_t)(g / ST2) & 1u, &sy.abort, ctl, true);
    cluster_sync();  // neither CTA leaves while the pair may still signal it
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(sy.tmem, 2 * N2);
    }
}

template <bool SIM_SIGMA, int EPI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EPI, 1)
    k_tc_phase2(const __grid_constant__ TcMaps maps, const __grid_constant__ Dev d, int cur,
                const int *__restrict__ sched_off, const int *__restrict__ sched)
{
    if (!d.ctl->active)  // both CTAs of a pair see the same value and leave together
        return;
    phase2_pair<SIM_SIGMA, EPI>(P2One{maps, d, cur, sched_off, sched}, d.ctl);
}

template <bool SIM_SIGMA, int EPI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EPI, 1) k_tc_phase2_set(const SetArgs a)
{
    phase2_pair<SIM_SIGMA, EPI>(P2Set{a, a.sched_off, a.sched}, a.devs[0].ctl);
}

// every network's control block into one array (one read-back per chunk of a set)
__global__ void k_gather_ctl(const Dev *devs, int n, Ctl *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n)
        out[k] = *devs[k].ctl;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Row-major BF16 matrix rows x cols (cols = K, contiguous), box 64 x box_rows,
// 128-byte swizzle.
cudaError_t make_map(CUtensorMap *m, const void *base, int rows, int cols, int box_rows)
{
    // box: 64 columns (128 B, the swizzle span) by box_rows rows
    auto fn = encode_fn();
    if (!fn)
        return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 8-bit [rows][cols] array (E4M3 bytes), boxes of 128 bytes by box_rows rows
cudaError_t make_map8(CUtensorMap *m, const void *base, int rows, int cols, int box_rows)
{
    auto fn = encode_fn();
    if (!fn)
        return cudaErrorNotSupported;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols};
    cuuint32_t box[2] = {128, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

constexpr size_t pair_smem() { return 1024 + (size_t)PAIR_ST * PAIR_STAGE + sizeof(SyncPair) + 16; }

struct TcHost {
    TcMaps maps;
    int *sched_off = nullptr;  // [grid2 + 1] offsets into sched
    int *sched = nullptr;      // packed phase-2 items (see P2Item)
    int *p1_off = nullptr;     // [grid1 / 2 + 1] offsets into p1_items
    int4 *p1_items = nullptr;  // phase-1 pieces (see build_p1)
    int clusters = 0;          // two-CTA clusters of phase 1 resident at once (occupancy calculator)
    int grid1 = 0, grid2 = 0;  // CTAs of the persistent phase-1 and phase-2 launches
    int epi2 = 12;             // epilogue warps of the phase-2 kernel (p2_epi)
};

// Cost of a phase-2 tile in MMA issue slots (a BF16 MMA of K = 16 and an E4M3
// MMA of K = 32 take the same time) plus a fixed epilogue share.
int tile_cost(const Dev &d, bool isP, int epi)
{
    const int terms = d.split_b ? 3 : 2;
    if (isP)
        return (d.Gp / BK) * 4 * terms + epi;
    if (d.fp8)
        return (d.Tp / (2 * BK)) * 4 + epi;
    return (d.Tp / BK) * 4 * terms + epi;
}

// Longest-processing-time assignment of weighted items to `pairs` lists
// (the heaviest item to the least loaded list); interleave: each list is then
// reordered heaviest, lightest, second heaviest, ... so that tensor-bound and
// memory-bound work alternate in time on every pair.
template <class Item>
void lpt_lists(std::vector<std::pair<long long, Item>> all, int pairs, bool interleave, std::vector<int> &off,
               std::vector<Item> &out)
{
    std::stable_sort(all.begin(), all.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    std::vector<std::vector<Item>> lists(std::max(pairs, 1));
    using L = std::pair<long long, int>;
    std::priority_queue<L, std::vector<L>, std::greater<L>> heap;
    for (int c = 0; c < (int)lists.size(); ++c)
        heap.push({0, c});
    for (const auto &t : all) {
        L top = heap.top();
        heap.pop();
        lists[top.second].push_back(t.second);
        heap.push({top.first + t.first, top.second});
    }
    off.assign(1, 0);
    out.clear();
    for (auto &l : lists) {
        if (interleave) {
            std::vector<Item> m;
            for (size_t i = 0, j = l.size(); i < j; ++i) {
                m.push_back(l[i]);
                if (i + 1 < j)
                    m.push_back(l[--j]);
            }
            l.swap(m);
        }
        out.insert(out.end(), l.begin(), l.end());
        off.push_back((int)out.size());
    }
}

// Bytes one phase-2 tile moves through HBM in its epilogue (old values read,
// new values and split copies written; operands come from L2), per entry.
int tile_epilogue_bytes(const Dev &d, bool isP)
{
    if (isP)
        return 16;  // FP32 old + FP32 new + split copy of both triangles
    if (d.fp8)
        return 10;  // FP32 old + new, E4M3 row and mirrored copies
    return d.c_split ? 8 : 12;  // split pair old + new (or FP32 old + new + split copy)
}

constexpr long long BYTES_PER_SLOT = 7200;  // HBM bytes per pair in one BF16 MMA slot (82 ns at the dense peak)

// Phase-2 candidates: cost model, epilogue weight, order
struct P2Spec {
    int roofline, epi, interleave;
    int other;  // 1: the phase-2 kernel configuration p2_epi does not pick (12 warps / 2 stages <-> 8 / 3)
};
const P2Spec TC_P2_SPEC[TC_P2_CANDS] = {{0, 192, 0, 0}, {1, 48, 0, 0},  {1, 192, 0, 0},
                                        {1, 192, 1, 0}, {1, 768, 0, 0}, {1, 192, 0, 1}};

int p2_epi(long long mma_slots);

// One phase-2 schedule of every network's upper-triangle P and C tiles (only
// the networks whose phase-2 kernel configuration p2_epi is epi, if epi > 0).
// A P tile is one unit of the LPT assignment (its whole K) and is listed as
// its K chunks, consecutively, on the pair it is assigned to (see P2Item).
void build_p2(const std::vector<const Dev *> &ds, int pairs, const P2Spec &sp, std::vector<int> &off,
              std::vector<int> &tiles, std::vector<int> &nets, int epi = 0)
{
    std::vector<std::pair<long long, std::pair<int, int>>> all;
    for (int k = 0; k < (int)ds.size(); ++k) {
        const Dev &d = *ds[k];
        if (epi > 0 && p2_epi(tile_cost(d, false, 0)) != epi)
            continue;
        for (int isP = 1; isP >= 0; --isP) {
            const int nb = ceil_div(isP ? d.Tp : d.Gp, N2);
            long long c = tile_cost(d, isP != 0, 0);
            if (sp.roofline)
                c = std::max(c, (long long)tile_epilogue_bytes(d, isP != 0) * N2 * N2 / BYTES_PER_SLOT);
            c += sp.epi;
            for (int bm = 0; bm < nb; ++bm)
                for (int bn = bm; bn < nb; ++bn)
                    all.push_back({c, {(int)((isP ? 0x80000000u : 0u) | ((uint32_t)bm << 16) | (uint32_t)bn), k}});
        }
    }
    std::vector<int> uoff;
    std::vector<std::pair<int, int>> units;
    lpt_lists(all, std::min<int>(pairs, (int)all.size()), sp.interleave != 0, uoff, units);
    off.assign(1, 0);
    tiles.clear();
    nets.clear();
    for (size_t p = 0; p + 1 < uoff.size(); ++p) {
        for (int q = uoff[p]; q < uoff[p + 1]; ++q) {
            const int code = units[q].first, net = units[q].second;
            const int nch = code < 0 ? p2_chunks(*ds[net]) : 1;
            for (int c = 0; c < nch; ++c) {
                tiles.push_back(code | (c << 24));
                nets.push_back(net);
            }
        }
        off.push_back((int)tiles.size());
    }
}

// One network: the first candidate (LPT on MMA slots, epilogue weight 192).
void build_schedule(const Dev &d, int pairs, std::vector<int> &off, std::vector<int> &tiles)
{
    std::vector<int> nets;
    build_p2({&d}, pairs, TC_P2_SPEC[0], off, tiles, nets);
}

// Phase-1 pieces of one network for `pairs` persistent CTA pairs, as lists
// (off, items) per pair; returns the number of tiles cut between two pairs.
// Whole tiles in rounds of the gene-block-major order (pair p: tiles p,
// p + pairs, ...) while every pair has one.  When the tile count leaves the
// last round more than about 1/20 of the work short (some pairs idle at the
// end), the tiles of the last full round and the partial one are instead
// taken TF-block-major, so
// that the pairs over the TF blocks of one gene block run side by side and
// share C's rows in L2, and their MMA work is cut into equal shares at
// chunk boundaries.  A tile straddling two shares becomes a head (chunks
// 0 .. b - 1) and a tail (chunks b .. , R-num, the epilogue) on the next
// pair, which waits for the head's flag; each entry's chunks are added in
// the same order as in an uncut tile (the result is the same to the bit).
// A pair runs its whole-tile rounds first (all pairs in step, so the TF
// blocks of a gene block still read C's rows together), then its head, its
// whole tiles of the cut rounds, and its tail last: a head waits for
// nothing, so no tail waits on work that cannot run.  cut_ok is false when
// not every pair is known to be resident at once (a tail could wait for a
// head that cannot start).
int build_p1(const Dev &d, int pairs, bool cut_ok, std::vector<int> &off, std::vector<int4> &items)
{
    const int nmt = d.Tp / 256, ntile = nmt * (d.Gp / 256);
    const int nA = d.Gp / (d.fp8 ? 2 * BK : BK), nR = d.Tp / BK, nc = (nA + P1_CHUNK - 1) / P1_CHUNK;
    pairs = std::max(1, std::min(pairs, ntile));
    std::vector<std::vector<int4>> rounds(pairs), head(pairs), body(pairs), tail(pairs);
    // whole tiles leave the busiest pair ceil(ntile / pairs) tiles against ntile / pairs on average;
    // under 5% more, cutting costs more than it saves (the cut rounds share C's rows in L2 less
    // well: 1600 x 30000, 1.2% to gain, ran phase 1 5% slower cut)
    const int most = (ntile + pairs - 1) / pairs;
    const bool cut = cut_ok && nc >= 2 && ntile > pairs && (double)most * pairs > 1.05 * ntile;
    const int ndp = cut ? (ntile / pairs - 1) * pairs : ntile;
    for (int q = 0; q < ndp; ++q)
        rounds[q % pairs].push_back(make_int4(q % nmt, q / nmt, nc << 16, -1));
    int cuts = 0;
    if (cut) {
        std::vector<std::pair<int, int>> sk;  // (mt, nt), TF-block-major
        for (int q = ndp; q < ntile; ++q)
            sk.push_back({q % nmt, q / nmt});
        std::sort(sk.begin(), sk.end());
        // MMA issue slots: a k-block is 4 MMAs of K = 16 per term (E4M3: K = 32, one term); the
        // epilogue after the last chunk is counted as 64 slots
        const long long wA = d.fp8 ? 4 : 4 * (d.split_b ? 3 : 2), wR = 4 * (d.split_b ? 3 : 2);
        std::vector<long long> cost(nc);
        long long per_tile = 0;
        for (int c = 0; c < nc; ++c) {
            cost[c] = wA * std::min(P1_CHUNK, nA - c * P1_CHUNK) + (c == nc - 1 ? wR * nR + 64 : 0);
            per_tile += cost[c];
        }
        const double share = (double)per_tile * (double)sk.size() / pairs;
        long long pos = 0;
        for (const auto &t : sk) {
            // owner of each chunk: the share holding its midpoint (at most two per tile: share >= one tile)
            std::vector<int> own(nc);
            for (int c = 0; c < nc; ++c) {
                own[c] = std::min(pairs - 1, (int)(((double)pos + 0.5 * (double)cost[c]) / share));
                pos += cost[c];
            }
            int b = 1;
            while (b < nc && own[b] == own[0])
                ++b;
            if (b == nc) {
                body[own[0]].push_back(make_int4(t.first, t.second, nc << 16, -1));
            } else {
                head[own[0]].push_back(make_int4(t.first, t.second, b << 16, cuts));
                tail[own[b]].push_back(make_int4(t.first, t.second, b | nc << 16, cuts));
                ++cuts;
            }
        }
    }
    off.assign(1, 0);
    items.clear();
    for (int p = 0; p < pairs; ++p) {
        for (auto *l : {&rounds[p], &head[p], &body[p], &tail[p]})
            items.insert(items.end(), l->begin(), l->end());
        off.push_back((int)items.size());
    }
    return cuts;
}

template <bool SIM, int EPI>
cudaError_t phase2_smem_limits()
{
    cudaError_t e = cudaFuncSetAttribute(k_tc_phase2<SIM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)phase2_smem<SIM, EPI>());
    return e ? e
             : cudaFuncSetAttribute(k_tc_phase2_set<SIM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)phase2_smem<SIM, EPI>());
}

// Epilogue warps of phase 2 for networks whose C' tiles take mma_slots MMA
// issue slots each (the largest over a set): 12 (two operand stages) while
// the MMAs are shorter than the epilogue, about 290 slots of the dense peak
// at 1000 x 17000 (1000 x 17000 under BF16X3: 192 slots), else 8 (three
// stages; 1600 x 30000: 336 slots)
int p2_epi(long long mma_slots) { return mma_slots > 256 ? 8 : 12; }

// One phase-2 launch of EPI epilogue warps
template <int EPI, class... Args>
void launch_p2_one(bool sim, int grid, cudaStream_t s, const Args &...args)
{
    if (sim)
        k_tc_phase2<true, EPI><<<grid, P2Cfg<true, EPI>::THREADS, phase2_smem<true, EPI>(), s>>>(args...);
    else
        k_tc_phase2<false, EPI><<<grid, P2Cfg<false, EPI>::THREADS, phase2_smem<false, EPI>(), s>>>(args...);
}
template <int EPI>
void launch_p2_set(bool sim, int grid, cudaStream_t s, const SetArgs &a)
{
    if (sim)
        k_tc_phase2_set<true, EPI><<<grid, P2Cfg<true, EPI>::THREADS, phase2_smem<true, EPI>(), s>>>(a);
    else
        k_tc_phase2_set<false, EPI><<<grid, P2Cfg<false, EPI>::THREADS, phase2_smem<false, EPI>(), s>>>(a);
}

cudaError_t set_smem_limits()
{
    static bool done = false;
    if (done)
        return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_tc_phase1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)phase1_smem())) ||
        (e = cudaFuncSetAttribute(k_tc_phase1_set, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)phase1_smem())) ||
        (e = phase2_smem_limits<false, 8>()) || (e = phase2_smem_limits<true, 8>()) ||
        (e = phase2_smem_limits<false, 12>()) || (e = phase2_smem_limits<true, 12>()))
        return e;
    constexpr size_t st_smem = 1024 + 3 * (4 * A_BYTES) + sizeof(Sync<3>) + 16;
    if ((e = cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_tc_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)pair_smem())))
        return e;
    done = true;
    return cudaSuccess;
}

// CTA pairs of the phase-1 launch of one network (one per SM pair), and
// whether all of them are resident at once (the occupancy calculator's count
// of co-resident two-CTA clusters).
cudaError_t phase1_pairs(int &pairs, bool &all_resident, int *clusters_out = nullptr)
{
    cudaError_t e = set_smem_limits();
    int dev = 0, nsm = 0;
    if (e || (e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
        return e;
    pairs = nsm / 2;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * pairs);
    cfg.blockDim = dim3(THREADS1);
    cfg.dynamicSmemBytes = phase1_smem();
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    all_resident = cudaOccupancyMaxActiveClusters(&clusters, (void *)k_tc_phase1, &cfg) == cudaSuccess &&
                   clusters >= pairs;
    cudaGetLastError();
    if (clusters_out)
        *clusters_out = clusters;
    return cudaSuccess;
}

}  // namespace

// Phase-1 candidates: the order of a network's tiles (LPT over persistent pairs by main-loop length)
const char *const TC_P1_NAMES[TC_P1_CANDS] = {"tiles of a gene block together (C rows shared in L2)",
                                              "tiles of a TF block together (W rows shared in L2)"};
// Phase-2 candidates (cost model, epilogue weight, order, kernel configuration), as in TC_P2_SPEC
const char *const TC_P2_NAMES[TC_P2_CANDS] = {
    "LPT on MMA slots + 192", "LPT on max(MMA, HBM) + 48", "LPT on max(MMA, HBM) + 192",
    "LPT on max(MMA, HBM) + 192, heavy and light tiles alternating", "LPT on max(MMA, HBM) + 768",
    "LPT on max(MMA, HBM) + 192, the other phase-2 kernel configuration (8 epilogue warps and 3 stages "
    "where the MMA-length model picks 12 and 2, or the reverse)"};

int tc_phase1_plan(const Dev &d, int pairs, bool cut_ok, std::vector<int> &off, std::vector<int4> &items)
{
    return build_p1(d, pairs, cut_ok, off, items);
}

int tc_phase1_layout(const Dev &d, int *pairs, int *clusters)
{
    const TcHost *h = static_cast<const TcHost *>(d.tc_host);
    if (!h)
        return -1;
    *pairs = h->grid1 / 2;
    *clusters = h->clusters;
    return d.p1_cuts;
}

int tc_phase1_cuts(const Dev &d)
{
    int pairs = 0;
    bool resident = false;
    if (phase1_pairs(pairs, resident))
        return -1;
    std::vector<int> off;
    std::vector<int4> items;
    return build_p1(d, pairs, resident, off, items);
}

bool tc_supported()
{
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess)
        return false;
    return major == 10 && minor == 3 && encode_fn() != nullptr;
}

cudaError_t tc_prepare(Dev &d, cudaStream_t s, bool fresh_scales)
{
    cudaError_t e = set_smem_limits();
    if (e)
        return e;
    const size_t TG = (size_t)d.Tp * d.Gp;
    // split copies of the current state (both W buffers get their maps; buffer 0 holds W now)
    for (int b = 0; b < 2; ++b)
        k_split<<<1024, 256, 0, s>>>(d.W[b], TG, d.Wh[b], d.Wl[b]);
    k_split<<<1024, 256, 0, s>>>(d.Poff, (size_t)d.Tp * d.Tp, d.Ph, d.Pl);
    if (d.fp8) {  // scales from the state's norms (or as restored), then the E4M3 copies
        if (fresh_scales)
            k_fp8_init<<<1, 1024, 0, s>>>(d);
        for (int b = 0; b < 2; ++b) {
            k_to_e4m3<<<1024, 256, 0, s>>>(d.W[b], TG, d.W8[b], d.f8 + b);
            k_to_e4m3<<<1024, 256, 0, s>>>(d.Wt[b], TG, d.Wt8[b], d.f8 + b);
        }
        k_to_e4m3<<<2048, 256, 0, s>>>(d.Coff, (size_t)d.Gp * d.Gp, d.C8, d.f8 + 2);
    } else if (d.Coff) {  // C's split pair from the FP32 C being derived (a restored pair is kept)
        k_split<<<2048, 256, 0, s>>>(d.Coff, (size_t)d.Gp * d.Gp, d.Ch, (d.split_b || d.c_split) ? d.Cl : nullptr);
    }
    if ((e = cudaGetLastError()))
        return e;
    if (!d.tc_host) {
        TcHost *h = new TcHost;
        TcMaps *m = &h->maps;
        std::memset(m, 0, sizeof *m);
        d.tc_host = h;
        if ((e = make_map(&m->Ph, d.Ph, d.Tp, d.Tp, 128)) || (e = make_map(&m->Pl, d.Pl, d.Tp, d.Tp, 128)))
            return e;
        if (d.fp8) {
            if ((e = make_map8(&m->C8, d.C8, d.Gp, d.Gp, 128)))
                return e;
            for (int b = 0; b < 2; ++b)
                if ((e = make_map8(&m->W8[b], d.W8[b], d.Tp, d.Gp, 128)) ||
                    (e = make_map8(&m->Wt8[b], d.Wt8[b], d.Gp, d.Tp, 128)))
                    return e;
        } else {
            if ((e = make_map(&m->Ch, d.Ch, d.Gp, d.Gp, 128)) || (e = make_map(&m->Chm, d.Ch, d.Gp, d.Gp, 64)))
                return e;
            if (d.split_b &&
                ((e = make_map(&m->Cl, d.Cl, d.Gp, d.Gp, 128)) || (e = make_map(&m->Clm, d.Cl, d.Gp, d.Gp, 64))))
                return e;
        }
        for (int b = 0; b < 2; ++b)
            if ((e = make_map(&m->Wh[b], d.Wh[b], d.Tp, d.Gp, 128)) ||
                (e = make_map(&m->Wl[b], d.Wl[b], d.Tp, d.Gp, 128)) ||
                (e = make_map(&m->Whm[b], d.Wh[b], d.Tp, d.Gp, 64)) ||
                (e = make_map(&m->Wlm[b], d.Wl[b], d.Tp, d.Gp, 64)))
                return e;
        int dev = 0, nsm = 0;
        if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
            return e;
        std::vector<int> off, tiles;
        build_schedule(d, nsm / 2, off, tiles);  // one list per CTA pair
        h->grid2 = 2 * ((int)off.size() - 1);
        h->epi2 = p2_epi(tile_cost(d, false, 0));
        int pairs = 0;
        bool resident = false;
        std::vector<int> off1;
        std::vector<int4> items1;
        if ((e = phase1_pairs(pairs, resident, &h->clusters)))
            return e;
        if (build_p1(d, pairs, resident, off1, items1) > d.p1_cuts)
            return cudaErrorInvalidValue;  // the memory plan made fewer cut slots (cannot happen)
        h->grid1 = 2 * ((int)off1.size() - 1);
        if ((e = cudaMalloc(&h->sched_off, off.size() * sizeof(int))) ||
            (e = cudaMalloc(&h->sched, tiles.size() * sizeof(int))) ||
            (e = cudaMemcpy(h->sched_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(h->sched, tiles.data(), tiles.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
            (e = cudaMalloc(&h->p1_off, off1.size() * sizeof(int))) ||
            (e = cudaMalloc(&h->p1_items, items1.size() * sizeof(int4))) ||
            (e = cudaMemcpy(h->p1_off, off1.data(), off1.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
            (e = cudaMemcpy(h->p1_items, items1.data(), items1.size() * sizeof(int4), cudaMemcpyHostToDevice)))
            return e;
    }
    return cudaSuccess;
}

void tc_release(Dev &d)
{
    TcHost *h = static_cast<TcHost *>(d.tc_host);
    if (h) {
        cudaFree(h->sched_off);
        cudaFree(h->sched);
        cudaFree(h->p1_off);
        cudaFree(h->p1_items);
        delete h;
    }
    d.tc_host = nullptr;
}

cudaError_t launch_iteration_tc(const Dev &d, int cur, cudaStream_t s, KernelEvents &ke)
{
    const TcHost &h = *static_cast<const TcHost *>(d.tc_host);
    const TcMaps &m = h.maps;
    ke.mark(s);
    k_tc_phase1<<<h.grid1, THREADS1, phase1_smem(), s>>>(m, d, cur, h.p1_items, h.p1_off);
    ke.mark(s);
    cudaError_t e = launch_reduce_wnorms(d, s);
    if (e)
        return e;
    ke.mark(s);
    if (h.epi2 == 8)
        launch_p2_one<8>(d.diag == 2, h.grid2, s, m, d, cur ^ 1, h.sched_off, h.sched);
    else
        launch_p2_one<12>(d.diag == 2, h.grid2, s, m, d, cur ^ 1, h.sched_off, h.sched);
    ke.mark(s);
    return launch_fin_tail(d, s, ke);
}

// ---- sets of networks: one launch per phase over all networks' tiles ---------------
struct TcSet {
    int n = 0, diag = 0, pairs = 0;
    Dev *devs = nullptr;      // device copies of the networks' Dev
    TcMaps *maps = nullptr;   // their tensor maps
    int *parity = nullptr;
    int2 *blocks = nullptr;
    int nblocks = 0;
    Ctl *gather = nullptr;
    float *acc = nullptr;     // phase 1: one running-sum slot per persistent CTA
    struct P1 {               // a phase-1 schedule: per pair, a list of (network, mt, nt, cost)
        int4 *items = nullptr;
        int *off = nullptr;
    };
    struct P2 {               // a phase-2 schedule: per pair, a list of packed tiles and their networks
        // one launch per phase-2 kernel configuration (p2_epi) among the networks, each network in
        // the configuration of its own single runs (the autotuner's last candidate swaps them; the
        // two give the same bits: see p2_group)
        struct Part {
            int epi2 = 12, pairs = 0;
            int *off = nullptr, *tiles = nullptr, *nets = nullptr;
        };
        Part part[2];
        int nparts = 0;
    };
    std::vector<P1> p1;
    std::vector<P2> p2;
};

namespace {
template <class T>
cudaError_t upload(T **dst, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(1, v.size()) * sizeof(T));
    if (!e && !v.empty())
        e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

}  // namespace

cudaError_t tc_set_create(const std::vector<const Dev *> &ds, TcSet **out)
{
    *out = nullptr;
    cudaError_t e = set_smem_limits();
    if (e)
        return e;
    TcSet *t = new TcSet;
    t->n = (int)ds.size();
    t->diag = ds[0]->diag;
    std::vector<Dev> hd;
    std::vector<TcMaps> hm;
    std::vector<int2> bl;
    for (int k = 0; k < t->n; ++k) {
        const Dev &d = *ds[k];
        hd.push_back(d);
        hm.push_back(static_cast<const TcHost *>(d.tc_host)->maps);
        for (int b = 0; b < set_norm_blocks(d.T, d.G); ++b)
            bl.push_back(make_int2(k, b));
    }
    t->nblocks = (int)bl.size();
    int dev = 0, nsm = 0;
    if (!(e = cudaGetDevice(&dev)) && !(e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) &&
        !(e = upload(&t->devs, hd)) && !(e = upload(&t->maps, hm)) && !(e = upload(&t->blocks, bl)) &&
        !(e = cudaMalloc(&t->parity, t->n * sizeof(int))) && !(e = cudaMemset(t->parity, 0, t->n * sizeof(int))) &&
        !(e = cudaMalloc(&t->gather, t->n * sizeof(Ctl))) &&
        !(e = cudaMalloc(&t->acc, sizeof(float) * P1_SLOT * (size_t)(nsm & ~1)))) {
        t->pairs = nsm / 2;
        for (int q = 0; q < TC_P1_CANDS && !e; ++q) {  // phase 1: persistent pairs over LPT lists
            std::vector<std::pair<long long, int4>> all;
            for (int k = 0; k < t->n; ++k) {
                const Dev &d = *ds[k];
                const int nk = d.Tp / BK + d.Gp / (d.fp8 ? 2 * BK : BK), nmt = d.Tp / 256, nnt = d.Gp / 256;
                for (int a = 0; a < (q == 0 ? nnt : nmt); ++a)
                    for (int b = 0; b < (q == 0 ? nmt : nnt); ++b)
                        all.push_back({nk, q == 0 ? make_int4(k, b, a, nk) : make_int4(k, a, b, nk)});
            }
            std::vector<int> off;
            std::vector<int4> items;
            lpt_lists(all, std::min<int>(t->pairs, (int)all.size()), false, off, items);
            off.resize(t->pairs + 1, off.back());  // pairs beyond the items get empty lists
            TcSet::P1 c;
            if (!(e = upload(&c.items, items)))
                e = upload(&c.off, off);
            t->p1.push_back(c);
        }
        bool has[2] = {false, false};  // networks whose phase 2 runs 12 / 8 epilogue warps
        for (const Dev *d : ds)
            has[p2_epi(tile_cost(*d, false, 0)) == 8] = true;
        for (int q = 0; q < TC_P2_CANDS && !e; ++q) {
            TcSet::P2 c;
            for (int g = 0; g < 2 && !e; ++g) {
                if (!has[g])
                    continue;
                std::vector<int> off, tiles, nets;
                TcSet::P2::Part &pt = c.part[c.nparts++];
                // the networks whose single runs use configuration g; the candidate may run the other
                build_p2(ds, t->pairs, TC_P2_SPEC[q], off, tiles, nets, g ? 8 : 12);
                pt.epi2 = (g != 0) != (TC_P2_SPEC[q].other != 0) ? 8 : 12;
                pt.pairs = (int)off.size() - 1;
                if (!(e = upload(&pt.off, off)) && !(e = upload(&pt.tiles, tiles)))
                    e = upload(&pt.nets, nets);
            }
            t->p2.push_back(c);
        }
    }
    if (e) {
        tc_set_destroy(t);
        return e;
    }
    *out = t;
    return cudaSuccess;
}

cudaError_t tc_set_parity(TcSet *t, const std::vector<int> &parity, cudaStream_t s)
{
    return cudaMemcpyAsync(t->parity, parity.data(), t->n * sizeof(int), cudaMemcpyHostToDevice, s);
}

cudaError_t tc_set_launch(TcSet *t, int p1, int p2, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                          cudaEvent_t ev2)
{
    const TcSet::P1 &a1 = t->p1[p1];
    const TcSet::P2 &c = t->p2[p2];
    SetArgs a{t->devs, t->maps, t->parity, a1.items, a1.off, t->acc, nullptr, nullptr, nullptr};
    if (ev0)
        cudaEventRecord(ev0, s);
    k_tc_phase1_set<<<2 * t->pairs, THREADS1, phase1_smem(), s>>>(a);
    cudaError_t e = launch_reduce_wnorms_set(t->devs, t->blocks, t->nblocks, s);
    if (e)
        return e;
    if (ev1)
        cudaEventRecord(ev1, s);
    for (int g = 0; g < c.nparts; ++g) {
        const TcSet::P2::Part &pt = c.part[g];
        a.sched_off = pt.off;
        a.sched = pt.tiles;
        a.sched_net = pt.nets;
        if (pt.epi2 == 8)
            launch_p2_set<8>(t->diag == 2, 2 * pt.pairs, s, a);
        else
            launch_p2_set<12>(t->diag == 2, 2 * pt.pairs, s, a);
    }
    if (ev2)
        cudaEventRecord(ev2, s);
    return launch_fin_tail_set(t->devs, t->blocks, t->nblocks, t->n, s);
}

cudaError_t tc_set_gather(TcSet *t, Ctl *host, cudaStream_t s)
{
    k_gather_ctl<<<ceil_div(t->n, 128), 128, 0, s>>>(t->devs, t->n, t->gather);
    cudaError_t e = cudaGetLastError();
    return e ? e : cudaMemcpyAsync(host, t->gather, t->n * sizeof(Ctl), cudaMemcpyDeviceToHost, s);
}

void tc_set_destroy(TcSet *t)
{
    if (!t)
        return;
    cudaFree(t->devs);
    cudaFree(t->maps);
    cudaFree(t->parity);
    cudaFree(t->blocks);
    cudaFree(t->gather);
    cudaFree(t->acc);
    for (auto &c : t->p1) {
        cudaFree(c.items);
        cudaFree(c.off);
    }
    for (auto &c : t->p2)
        for (auto &q : c.part) {
            cudaFree(q.off);
            cudaFree(q.tiles);
            cudaFree(q.nets);
        }
    delete t;
}

cudaError_t tc_gram(const __nv_bfloat16 *Zh, const __nv_bfloat16 *Zl, int Gp, int Kp, float *C, Ctl *ctl,
                    cudaStream_t s)
{
    cudaError_t e = set_smem_limits();
    if (e)
        return e;
    GemmMaps maps;
    if ((e = make_map(&maps.Ah, Zh, Gp, Kp, 128)) || (e = make_map(&maps.Al, Zl, Gp, Kp, 128)) ||
        (e = make_map(&maps.Bh, Zh, Gp, Kp, 128)) || (e = make_map(&maps.Bl, Zl, Gp, Kp, 128)))
        return e;
    k_tc_gemm_pair<<<dim3(Gp / 128, Gp / PAIR_N), THREADS, pair_smem(), s>>>(maps, Kp, Gp, C, ctl, 0, 0);
    return cudaGetLastError();
}

// D = A . B^T on the tensor-core pipeline (self-test support)
cudaError_t tc_selftest_gemm(int M, int N, int K, const float *A, const float *B, float *D, int terms,
                             int pair, int stall_kb, int *status)
{
    cudaError_t e = set_smem_limits();
    if (e)
        return e;
    // pair: 0 one CTA per tile, 1 CTA pairs, 2 pairs with B MN-major, 3 pairs on E4M3 operands (one term)
    const bool fp8 = pair == 3;
    const int Mp = round_up(M, pair ? 256 : 128), Np = round_up(N, pair ? PAIR_N : 128),
              Kp = round_up(K, fp8 ? 128 : 64);
    float *dA = nullptr, *dB = nullptr, *dD = nullptr;
    __nv_bfloat16 *Ah = nullptr, *Al = nullptr, *Bh = nullptr, *Bl = nullptr;
    Ctl *ctl = nullptr;
    GemmMaps maps;
    auto cleanup = [&]() {
        cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(Ah); cudaFree(Al); cudaFree(Bh); cudaFree(Bl);
        cudaFree(ctl);
    };
#define TRY(x)            \
    if ((e = (x))) {      \
        cleanup();        \
        return e;         \
    }
    TRY(cudaMalloc(&dA, (size_t)Mp * Kp * 4));
    TRY(cudaMalloc(&dB, (size_t)Np * Kp * 4));
    TRY(cudaMalloc(&dD, (size_t)Mp * Np * 4));
    TRY(cudaMalloc(&Ah, (size_t)Mp * Kp * 2));
    TRY(cudaMalloc(&Al, (size_t)Mp * Kp * 2));
    TRY(cudaMalloc(&Bh, (size_t)Np * Kp * 2));
    TRY(cudaMalloc(&Bl, (size_t)Np * Kp * 2));
    TRY(cudaMalloc(&ctl, sizeof(Ctl)));
    TRY(cudaMemset(ctl, 0, sizeof(Ctl)));
    TRY(cudaMemset(dA, 0, (size_t)Mp * Kp * 4));
    TRY(cudaMemset(dB, 0, (size_t)Np * Kp * 4));
    // pair 2: B held transposed and fed MN-major; 4: A and B; 5: A only
    const int mn = pair == 2 ? 1 : pair == 4 ? 3 : pair == 5 ? 2 : 0;
    if (mn & 2) {  // A^T, [Kp][Mp], for the MN-major A loads
        std::vector<float> at((size_t)K * M);
        for (int m = 0; m < M; ++m)
            for (int k = 0; k < K; ++k)
                at[(size_t)k * M + m] = A[(size_t)m * K + k];
        TRY(cudaMemcpy2D(dA, (size_t)Mp * 4, at.data(), (size_t)M * 4, (size_t)M * 4, K, cudaMemcpyHostToDevice));
    } else {
        TRY(cudaMemcpy2D(dA, (size_t)Kp * 4, A, (size_t)K * 4, (size_t)K * 4, M, cudaMemcpyHostToDevice));
    }
    if (mn & 1) {  // B^T, [Kp][Np], for the MN-major B loads
        std::vector<float> bt((size_t)K * N);
        for (int n = 0; n < N; ++n)
            for (int k = 0; k < K; ++k)
                bt[(size_t)k * N + n] = B[(size_t)n * K + k];
        TRY(cudaMemcpy2D(dB, (size_t)Np * 4, bt.data(), (size_t)N * 4, (size_t)N * 4, K, cudaMemcpyHostToDevice));
    } else {
        TRY(cudaMemcpy2D(dB, (size_t)Kp * 4, B, (size_t)K * 4, (size_t)K * 4, N, cudaMemcpyHostToDevice));
    }
    if (fp8) {  // E4M3 bytes in the hi buffers (each at least as large as an 8-bit copy)
        k_to_e4m3<<<256, 256>>>(dA, (size_t)Mp * Kp, reinterpret_cast<uint8_t *>(Ah), nullptr);
        k_to_e4m3<<<256, 256>>>(dB, (size_t)Np * Kp, reinterpret_cast<uint8_t *>(Bh), nullptr);
        TRY(cudaGetLastError());
        TRY(make_map8(&maps.Ah, Ah, Mp, Kp, 128));
        TRY(make_map8(&maps.Bh, Bh, Np, Kp, 128));
        k_tc_gemm_pair<<<dim3(Mp / 128, Np / PAIR_N), THREADS, pair_smem()>>>(maps, Kp, Np, dD, ctl, 0, 1);
        TRY(cudaGetLastError());
        TRY(cudaDeviceSynchronize());
        Ctl h;
        TRY(cudaMemcpy(&h, ctl, sizeof h, cudaMemcpyDeviceToHost));
        *status = h.status;
        TRY(cudaMemcpy2D(D, (size_t)N * 4, dD, (size_t)Np * 4, (size_t)N * 4, M, cudaMemcpyDeviceToHost));
        cleanup();
        return cudaSuccess;
    }
    k_split<<<256, 256>>>(dA, (size_t)Mp * Kp, Ah, Al);
    k_split<<<256, 256>>>(dB, (size_t)Np * Kp, Bh, Bl);
    TRY(cudaGetLastError());
    if (terms == 1) {  // hi only: zero the lo halves
        TRY(cudaMemset(Al, 0, (size_t)Mp * Kp * 2));
        TRY(cudaMemset(Bl, 0, (size_t)Np * Kp * 2));
    }
    if (mn & 2) {
        TRY(make_map(&maps.Ah, Ah, Kp, Mp, 64));
        TRY(make_map(&maps.Al, Al, Kp, Mp, 64));
    } else {
        TRY(make_map(&maps.Ah, Ah, Mp, Kp, 128));
        TRY(make_map(&maps.Al, Al, Mp, Kp, 128));
    }
    if (mn & 1) {
        TRY(make_map(&maps.Bh, Bh, Kp, Np, 64));
        TRY(make_map(&maps.Bl, Bl, Kp, Np, 64));
    } else {
        TRY(make_map(&maps.Bh, Bh, Np, Kp, 128));
        TRY(make_map(&maps.Bl, Bl, Np, Kp, 128));
    }
    constexpr size_t st_smem = 1024 + 3 * (4 * A_BYTES) + sizeof(Sync<3>) + 16;
    if (pair)
        k_tc_gemm_pair<<<dim3(Mp / 128, Np / PAIR_N), THREADS, pair_smem()>>>(maps, Kp, Np, dD, ctl, mn, 0);
    else
        k_tc_selftest<<<dim3(Mp / 128, Np / 128), THREADS, st_smem>>>(maps, Kp, Np, dD, ctl, stall_kb);
    TRY(cudaGetLastError());
    TRY(cudaDeviceSynchronize());
    Ctl h;
    TRY(cudaMemcpy(&h, ctl, sizeof h, cudaMemcpyDeviceToHost));
    *status = h.status;
    TRY(cudaMemcpy2D(D, (size_t)N * 4, dD, (size_t)Np * 4, (size_t)N * 4, M, cudaMemcpyDeviceToHost));
    cleanup();
#undef TRY
    return cudaSuccess;
}

}  // namespace panda
