// Internal declarations of libpanda_gb300 (not part of the C ABI).
//
// Device layout (all row-major, every dimension padded with zeros to a
// multiple of 128, or 256 on the tensor-core path, so that GEMM tiles never
// need bounds checks in their main loops; the epilogues mask by the true T
// and G):
//   W[2]   Tp x Gp  fp32   regulatory network, ping-pong (current / next)
//   Wt[2]  Gp x Tp  fp32   its transpose: written by the FP32 path's epilogue;
//                          on the tensor-core path made at create and load only
//                          (column norms, FP8MIX's E4M3 copy)
//   Poff   Tp x Tp  fp32   P with a zero diagonal (diagonal kept in pd)
//   Coff   Gp x Gp  fp32   C with a zero diagonal (diagonal kept in cd); in the
//                          BF16X3 and BF16X2 modes only while a create or
//                          set_state derives the state, which is then held as
//                          the split pair Ch + Cl alone
//   pd, cd          fp64   diagonals of P and C
//   rsqP, csqC      fp32   |P_i.|^2 and |C_.j|^2, diagonal included
//   rsqW, csqW      fp32   |W_i.|^2 and |W_.j|^2 of the current W
// plus per-tile partial sums (scratch) and a small control block.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <vector>
#include <cuda_bf16.h>
#include <stdint.h>

namespace panda {

constexpr int TILE = 128;          // padding granule and SIMT tile edge
constexpr int HIST_CAP = 1 << 16;  // iterations whose h is kept on the device

// Device control block, read by every kernel of an iteration.
struct Ctl {
    int active;     // kernels of an iteration do their work only while 1
    int iters;      // iterations done so far (the next one uses t = iters + 1)
    int stop_at;    // iteration count at which the current run stops
    int status;     // bit 0: non-finite state; bit 1: device wait timed out
    int converged;  // 1 when the last iteration gave h < tol
    float alpha;
    float pad0;
    double tol;
    double h_last;
};

enum : int { ST_NONFINITE = 1, ST_TIMEOUT = 2 };

// Pointers and shapes handed to kernels by value.
struct Dev {
    int T, G, Tp, Gp, nbT, nbG;  // true sizes, padded sizes, 128-blocks
    int diag;                    // panda_diag
    float *W[2], *Wt[2];         // Wt: FP32 and FP8MIX only (NULL under BF16X3 and BF16X2)
    float *Poff, *Coff;
    double *pd, *cd;
    float *pdf, *cdf;            // FP32 copies of the diagonals for epilogues
    float *rsqP, *csqC, *rsqW, *csqW;
    // scratch
    float *Rn;                   // Tp x Gp  P_off . W  (SIMT path)
    float *wrow_part;            // nbG x Tp
    float *wcol_part;            // nbT x Gp
    double *hpart;               // nbT * nbG
    float *ps_sum, *ps_sq, *ps_vsq;  // nsP x Tp  row partials of P'
    float *cs_sum, *cs_sq, *cs_vsq;  // nsC x Gp  row partials of C'
    int nsP, nsC;                    // partial-sum slots per row (0: one per 128-row block)
    int tri_slots;                   // 1: the tensor-core layout of those slots (row roles in
                                     // [0, nb), column roles from nb, nb = 256-blocks); 0: one
                                     // slot per 128-block, every slot written
    Ctl *ctl;
    double *hist;                // HIST_CAP
    double *e2tab;               // HIST_CAP + 1: e^{2 alpha t}, computed on the host
    // BF16 split copies (tensor-core path only; NULL otherwise)
    __nv_bfloat16 *Wh[2], *Wl[2];  // W^T operands are read from these MN-major
    __nv_bfloat16 *Ph, *Pl, *Ch, *Cl;
    // 1: C is held only as its split pair Ch + Cl (BF16X3, BF16X2): its upper
    // triangle and diagonal 256-blocks are the state, Coff is NULL between
    // calls (a staging buffer while a create or set_state derives the state)
    int c_split;
    // 1: B operands carry their lo halves too (BF16X3, hi.hi + hi.lo + lo.hi);
    // 0: B operands are BF16 hi only (BF16X2, hi.hi + lo.hi; C's lo half is never made)
    int split_b;
    // FP8MIX: E4M3 copies (one byte per entry) for W.C and W^T.W, and their scales
    int fp8;
    uint8_t *W8[2], *Wt8[2];     // W [Tp][Gp] and W^T [Gp][Tp], entries times f8[b]
    uint8_t *C8;                 // C_off [Gp][Gp], both triangles, entries times f8[2]
    float *f8;                   // [0], [1]: scale of W8/Wt8 buffer b; [2]: of C8; [3]: for the next W'
    unsigned *f8n;               // squared-norm maxima (float bits): [0..3] this iteration's
                                 // (rsqP, csqC, rsqW, csqW), [4..7] the state's, latched
    void *tc_host;               // host-side tensor maps of the split copies (tensor-core path)
    float *p1_acc;               // tensor-core phase 1: per CTA of its grid, a 128 x 256 slot for the
                                 // running sum of the availability numerator's chunks
    float *p1_fix;               // per tile cut between two CTA pairs (at most one per pair), a
                                 // 128 x 256 slot per CTA rank where its two pieces meet
    int *p1_flag;                // per cut tile and CTA rank: its head's adds have landed
    int p1_cuts;                 // cut tiles (slots and flag pairs above)
};

// Largest power of two s with s * bound <= 448 (the largest finite E4M3 value):
// bound >= every |x| that is scaled by s, so no entry saturates.
__host__ __device__ inline float e4m3_scale(float bound)
{
    if (!(bound > 0.0f) || !(bound < 3.0e38f))
        return 1.0f;
    const float x = 448.0f / bound;
    union { float f; unsigned u; } v{x};
    int e = (int)((v.u >> 23) & 0xffu) - 127;  // floor(log2 x) for normal x
    e = e < -100 ? -100 : (e > 100 ? 100 : e);
    v.u = (unsigned)(e + 127) << 23;
    return v.f;
}

// The alpha-free bounds behind the scales.  |Tan(x, y)| <= sqrt(|x| |y|) (Eq. 1);
// the damped updates are convex combinations, so |W'| <= max(|W|, (|R| + |A|) / 2)
// and |C'| <= max(|C|, |Tan|).  An entry is at most its row's norm.  The factor
// 1.25 covers E4M3 numerators, which may exceed the exact products by ~2^-4 per term.
__host__ __device__ inline float fp8_bound_w(float mrP, float mcC, float mrW, float mcW)
{
    const float t = 1.25f * 0.5f * (sqrtf(sqrtf(mrP) * sqrtf(mcW)) + sqrtf(sqrtf(mrW) * sqrtf(mcC)));
    return 1.001f * fmaxf(sqrtf(mrW), t);
}
__host__ __device__ inline float fp8_bound_c(float mcC, float mcW)
{
    return 1.001f * fmaxf(sqrtf(mcC), 1.25f * sqrtf(mcW));
}

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ inline int round_up(int a, int b) { return ceil_div(a, b) * b; }

// Eq. 1 from a numerator and the two squared norms (FP32, IEEE sqrt and
// division); 0 when the denominator is 0 (both vectors zero).
__device__ __forceinline__ float tanimoto_f(float num, float nx, float ny)
{
    float den = sqrtf((nx + ny) - fabsf(num));
    return den > 0.0f ? num / den : 0.0f;
}

// ---- FP32 error-free transforms --------------------------------------------
// This GPU's FP64 pipe issues about two operations per clock per SM, the FP32
// pipe 128, so sums and products that want more than FP32 accuracy run as
// FP32 pairs whose rounding errors are recovered exactly.

// Knuth's TwoSum: s + x = s' + e exactly (round to nearest, no overflow),
// s' = fl(s + x); the error e is added into the compensation c.
__device__ __forceinline__ void two_sum_add(float &s, float &c, float x)
{
    const float t = s + x;
    const float z = t - s;
    c += (s - (t - z)) + (x - z);
    s = t;
}

// a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// a * b = p + e exactly (the product's rounding error from one FMA), barring
// underflow of e
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ---- launchers (k_setup.cu) ------------------------------------------------
cudaError_t launch_check_finite_sym(const float *X, int rows, int cols, int ld, bool sym,
                                    int *flags, cudaStream_t s);
cudaError_t launch_zscore(float *X, int rows, int cols, int ld, double *stats, double *partials,
                          cudaStream_t s);
cudaError_t launch_split_diag(float *X, int n, int ld, double *d, float *df, cudaStream_t s);
cudaError_t launch_transpose(const float *X, int rows_p, int cols_p, float *Y, cudaStream_t s);
// out[j] = sum over the first `rows` rows of X[i][j]^2 (squared column norms, no transpose)
cudaError_t launch_col_norms(const float *X, int rows, int cols, int ld, float *out, cudaStream_t s);
cudaError_t launch_row_norms(const float *X, int rows, int cols, int ld, const double *diag,
                             float *out, cudaStream_t s);
cudaError_t launch_diag_to_float(const double *d, float *df, int n, cudaStream_t s);
cudaError_t launch_scan_nonfinite(const float *X, long long n, int *flag, cudaStream_t s);
// X[r][c] = X[c][r] for r > c: the full matrix from its upper triangle
cudaError_t launch_symmetrize(float *X, int n, int ld, cudaStream_t s);
// out (n x n, row stride ldo) = the symmetric matrix whose upper triangle is
// held as the BF16 split pair H + L (row stride ldi); diagonal entries are
// H + L too (callers put the FP64 diagonal in place afterwards)
cudaError_t launch_unsplit_sym(const __nv_bfloat16 *H, const __nv_bfloat16 *L, int n, int ldi, float *out, int ldo,
                              cudaStream_t s);
// Pearson initialisation (Sec. II-A): unit-norm centred rows of X (G x N) as a
// BF16 split [G][Kp]; flags[0] |= 1 (non-finite) / 2 (zero variance)
cudaError_t launch_standardize_rows(const float *X, int G, int N, __nv_bfloat16 *Zh, __nv_bfloat16 *Zl, int Kp,
                                    int *flags, cudaStream_t s);
cudaError_t launch_unit_diag(float *X, int n, int ld, cudaStream_t s);

// Optional per-kernel timing: when ev is not NULL, ev[0] is recorded before the
// first kernel of the iteration and ev[k + 1] after kernel k.
struct KernelEvents {
    cudaEvent_t *ev;
    int n;  // events recorded so far
    void mark(cudaStream_t s)
    {
        if (ev)  // external: inside a graph capture this becomes an event-record node
            cudaEventRecordWithFlags(ev[n++], s, cudaEventRecordExternal);
    }
};

// ---- one iteration, FP32 SIMT path (k_simt.cu) -----------------------------
constexpr int SIMT_KERNELS = 6;
extern const char *const SIMT_KERNEL_NAMES[SIMT_KERNELS];
cudaError_t launch_iteration_simt(const Dev &d, int cur, cudaStream_t s, KernelEvents &ke);
// shared tail of every path: diagonals, norms of P and C, h, stop test
cudaError_t launch_fin_tail(const Dev &d, cudaStream_t s, KernelEvents &ke);
// FP64 sums of the per-tile norm partials of W' (shared by both paths)
cudaError_t launch_reduce_wnorms(const Dev &d, cudaStream_t s);
// The same kernels over a set of networks (device arrays): blocks[b] = (network,
// that network's block), set_norm_blocks(T, G) blocks per network; one k_tail block per network.
cudaError_t launch_reduce_wnorms_set(const Dev *devs, const int2 *blocks, int nblocks, cudaStream_t s);
cudaError_t launch_fin_tail_set(const Dev *devs, const int2 *blocks, int nblocks, int nnets, cudaStream_t s);
int set_norm_blocks(int T, int G);
// FP32 FFMA throughput of the current device in TFLOP/s (best of several
// timed launches of a loop of independent FMAs on every SM)
cudaError_t measure_ffma_peak(double *tflops);

// ---- tensor-core path (k_tc.cu) --------------------------------------------
constexpr int TC_KERNELS = 5;
extern const char *const TC_KERNEL_NAMES[TC_KERNELS];
bool tc_supported();
// fresh_scales: derive the FP8MIX scales from the state's norms (false: keep those restored)
cudaError_t tc_prepare(Dev &d, cudaStream_t s, bool fresh_scales = true);  // split copies of the state, tensor maps
void tc_release(Dev &d);
// Tiles of one network's phase 1 cut between two CTA pairs (each needs a
// running-sum slot per CTA rank and a flag per rank); -1 on a CUDA error.
int tc_phase1_cuts(const Dev &d);
// The phase-1 launch of a prepared tensor-core context: CTA pairs, resident
// two-CTA clusters; returns its cut tiles (-1: not prepared).
int tc_phase1_layout(const Dev &d, int *pairs, int *clusters);
// The phase-1 pieces of one network (Dev needs Tp, Gp, fp8, split_b) for
// `pairs` CTA pairs: per pair p, items[off[p] .. off[p + 1]) of (mt, nt,
// c0 | c1 << 16, cut or -1); returns the number of cut tiles.  Host only.
int tc_phase1_plan(const Dev &d, int pairs, bool cut_ok, std::vector<int> &off, std::vector<int4> &items);
cudaError_t launch_iteration_tc(const Dev &d, int cur, cudaStream_t s, KernelEvents &ke);

// A set of networks (tensor-core modes, same options) iterated by one launch
// per phase: phases 1 and 2 persistent over LPT schedules of every network's
// tiles, the norm and stop kernels over all their rows.  Each network's W
// buffer is (parity + its iteration count) & 1.  A tile's result does not
// depend on which pair computes it or when, so every schedule gives the same
// bits and the fastest can be picked by timing real iterations.
// C (Gp x Gp, FP32, row stride Gp) = Z . Z^T with the three-term BF16 split of
// Z ([Gp][Kp] hi and lo, Gp a multiple of 256, Kp of 64) on CTA pairs; a
// timed-out wait sets ST_TIMEOUT in ctl (device memory).
cudaError_t tc_gram(const __nv_bfloat16 *Zh, const __nv_bfloat16 *Zl, int Gp, int Kp, float *C, Ctl *ctl,
                    cudaStream_t s);

struct TcSet;
// Schedule candidates of the set engine's autotuner: phase 1 (the order of each
// network's tiles in the persistent pairs' LPT lists) and phase 2 (cost model,
// epilogue weight, order of the LPT lists); TC_*_NAMES describe them.
constexpr int TC_P1_CANDS = 2, TC_P2_CANDS = 6;
extern const char *const TC_P1_NAMES[TC_P1_CANDS];
extern const char *const TC_P2_NAMES[TC_P2_CANDS];
cudaError_t tc_set_create(const std::vector<const Dev *> &ds, TcSet **out);
cudaError_t tc_set_parity(TcSet *t, const std::vector<int> &parity, cudaStream_t s);
// one iteration of every active network with phase-1 schedule p1 and phase-2
// schedule p2; events (each may be NULL) before phase 1, before phase 2, after phase 2
cudaError_t tc_set_launch(TcSet *t, int p1, int p2, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                          cudaEvent_t ev2);
cudaError_t tc_set_gather(TcSet *t, Ctl *host, cudaStream_t s);  // all control blocks to host (async)
void tc_set_destroy(TcSet *t);
// D (M x N, row-major) = A (M x K) . B (N x K)^T through the tcgen05 pipeline,
// host buffers; terms = 1 (hi only) or 3 (split).  *status: device status bits.
// stall_kb >= 0 plants a stage whose loads are never issued (timeout test).
cudaError_t tc_selftest_gemm(int M, int N, int K, const float *A, const float *B, float *D, int terms,
                             int pair, int stall_kb, int *status);

}  // namespace panda
