/*
 * libpanda_gb300: the PANDA message-passing iteration on one NVIDIA GB300.
 *
 * PANDA (Glass, Quackenbush, Kepner; "High Performance Computing of Gene
 * Regulatory Networks using a Message-Passing Model", Section II) iterates
 * three networks:
 *   W  T x G  regulatory network, TFs (effector nodes, N_e = T) to genes
 *             (affected nodes, N_a = G); not symmetric.
 *   P  T x T  cooperativity network between TFs; symmetric.
 *   C  G x G  co-regulatory network between genes; symmetric.
 * Each iteration t = 1, 2, ... computes
 *   R_ij = Tan(P_i., W_.j)                      (Eq. 3, responsibility)
 *   A_ij = Tan(W_i., C_.j)                      (Eq. 4, availability)
 *   W'   = (1-a) W + a/2 (R + A)                 (Eq. 2)
 *   h    = mean |W' - W|                         (Eq. 7)
 *   P'_im = (1-a) P_im + a Tan(W'_i., W'_m.)  for i != m          (Eq. 5)
 *   C'_kj = (1-a) C_kj + a Tan(W'_.k, W'_.j)  for k != j          (Eq. 5)
 *   P'_ii, C'_jj from the std of the off-diagonal entries of their row (Eq. 6)
 * with Tan(x, y) = x.y / sqrt(|x|^2 + |y|^2 - |x.y|) (Eq. 1), and stops when
 * h < tol (Section II-B, tested after the whole iteration).  Before the first
 * iteration each network is Z-scored (Section II-A, NormalizeNetwork).
 *
 * All matrices crossing this interface are dense, row-major, FP32, with no
 * padding: W has T*G entries, P has T*T, C has G*G (P and C include their
 * diagonals).  Host pointers are plain host memory (pageable or pinned);
 * device pointers are CUDA device memory of the current device.
 *
 * Return codes: 0 success; 1 PANDA_NOT_CONVERGED (max_iter reached, outputs
 * valid); negative values are errors and leave a message readable with
 * panda_last_error().  A context is used by one host thread at a time.
 */
#ifndef PANDA_GB300_H
#define PANDA_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

#define PANDA_OK 0
#define PANDA_NOT_CONVERGED 1
#define PANDA_EINVAL (-1)      /* bad argument: NULL, shape <= 0, alpha outside [0,1], tol < 0 */
#define PANDA_ENOMEM (-2)      /* device allocation failed (or the PANDA_ALLOC_LIMIT_BYTES cap) */
#define PANDA_ECUDA (-3)       /* a CUDA runtime or driver call failed */
#define PANDA_ENONFINITE (-4)  /* a non-finite input, or the state became non-finite */
#define PANDA_EASYM (-5)       /* P0 or C0 is not exactly symmetric */
#define PANDA_EDEGENERATE (-6) /* a network has zero standard deviation: Z-score undefined */
#define PANDA_ETIMEOUT (-7)    /* a bounded device-side wait expired */
#define PANDA_EUNSUPPORTED (-8)/* option not available in this build or on this device */

/* Arithmetic of the four products (the epilogues are FP32 in every mode).
 * State: W and P are FP32 in every mode, and so is C under PANDA_FP32 and
 * PANDA_FP8MIX.  Under PANDA_BF16X3 and PANDA_BF16X2 the library holds C only
 * as the split pair the products read, hi = bf16(x) and lo = bf16(x - hi) of
 * each FP32 entry x, the same 4 bytes per entry as FP32 (the paper's remark
 * on memory after Eq. 9: one copy of the largest network, not two).  BF16
 * keeps 8 significant bits, so hi + lo is within 2^-16 |x| of x: C entries
 * carry 16 significant bits instead of 24; panda_get and panda_get_state
 * return hi + lo (exact in FP32) with the diagonal from its FP64 vector. */
typedef enum {
    PANDA_FP32 = 0,   /* FP32 FFMA products (SIMT) */
    PANDA_BF16X3 = 1, /* tensor cores: x = hi + lo in BF16, hi*hi + hi*lo + lo*hi, FP32 accumulation */
    PANDA_BF16X2 = 2, /* tensor cores: A operands split hi + lo, B operands BF16 hi only: hi*hi + lo*hi
                         (about 2^-9 relative error on each B entry; 2/3 of BF16X3's tensor work) */
    PANDA_FP8MIX = 3  /* tensor cores: W.C and W^T.W on E4M3 copies (one term, FP32 accumulation,
                         one power-of-two scale per copy chosen from norm bounds so that no entry
                         saturates); P.W and W.W^T as BF16X3.  About 2^-4 relative error per E4M3
                         entry: W errors of order 1e-2 */
} panda_prec;

/* Reading of Eq. 6 (the paper prints no alpha on the diagonal increment). */
typedef enum {
    PANDA_DIAG_D1 = 0,         /* X_ii <- (1-a) X_ii + a N sigma_i e^{2 a t}  (default) */
    PANDA_DIAG_D0_LITERAL = 1, /* X_ii <- (1-a) X_ii +   N sigma_i e^{2 a t}  (as printed) */
    PANDA_DIAG_D2_SIM = 2      /* as D1, sigma over row i of the new similarity matrix */
} panda_diag;                  /* N = G (N_a) for P and T (N_e) for C, as Eq. 6 pairs them */

typedef struct {
    int prec;          /* panda_prec, default PANDA_FP32 */
    int diag;          /* panda_diag, default PANDA_DIAG_D1 */
    int normalize;     /* 1 (default): Z-score W0, P0, C0 at create; 0: use them as given */
    int t0;            /* iterations already done; the next iteration uses t = t0 + 1 (default 0) */
    int graph_iters;   /* iterations captured per CUDA-graph launch in panda_run (default 8; 0 = no graph) */
} panda_opts;

typedef struct panda_ctx panda_ctx;

/* 1 when precision mode prec (panda_prec) is built and runs on the current
 * device, else 0. */
int panda_precision_supported(int prec);

/* Fill *o with the defaults listed above. */
void panda_default_opts(panda_opts *o);

/* Create a context from host inputs (Section II-A: the three seed networks).
 * W0 is T x G, P0 is T x T, C0 is G x G, row-major FP32 host memory; they are
 * copied and not retained.  P0 and C0 must be exactly symmetric (PANDA_EASYM)
 * and every entry finite (PANDA_ENONFINITE).  With opts->normalize each
 * network is Z-scored with one global mean and population standard deviation
 * accurate to FP64 (compensated sums; PANDA_EDEGENERATE when that deviation is
 * 0); each Z-scored entry is within one FP32 ulp of the FP64 value rounded to
 * FP32, and equal to it except near a rounding midpoint.  o may be
 * NULL for the defaults.  The library owns all device state; it runs on the
 * current CUDA device and on its own non-blocking stream.  On error *out is
 * set to NULL and nothing is leaked. */
int panda_create(panda_ctx **out, int T, int G, const float *W0, const float *P0,
                 const float *C0, const panda_opts *o);

/* As panda_create, but W0, P0 and C0 are device pointers (not retained, not
 * freed) and every operation of the context runs on `stream` (a cudaStream_t;
 * NULL = the legacy default stream).  The inputs must stay valid until this
 * call returns. */
int panda_create_device(panda_ctx **out, int T, int G, const float *dW0, const float *dP0,
                        const float *dC0, const panda_opts *o, void *stream);

/* As panda_create, with the co-regulation prior computed on the GPU from
 * expression data (Sec. II-A): C0[g][h] = Pearson correlation of genes g and h
 * across the N samples of X (G x N, row-major host array, gene g's samples in
 * X[g*N .. g*N + N-1]), unit diagonal.  Each gene's centred samples are scaled
 * to unit norm in FP64 and the correlations are their Gram matrix on the
 * tensor cores (BF16 three-term split, FP32 accumulation: within 4.6e-5 of
 * the exact correlation, about 1e-6 with hundreds of samples), upper triangle mirrored so C0 is exactly symmetric.
 * P0 may be NULL: the identity (no interaction data).  Errors as panda_create,
 * plus PANDA_EDEGENERATE when a gene has zero variance across the samples,
 * PANDA_ENONFINITE for a non-finite sample, PANDA_EUNSUPPORTED off sm_103.
 * Temporary device memory of about 4 Gp^2 + 4 Gp N bytes (Gp = G rounded up to
 * 256) is freed before it returns. */
int panda_create_from_expression(panda_ctx **out, int T, int G, int N, const float *W0, const float *P0,
                                 const float *X, const panda_opts *o);

/* One message-passing iteration (Eqs. 2-7) with damping alpha in [0, 1].
 * *h_out (may be NULL) receives h of Eq. 7 in FP64.  Blocks until done. */
int panda_step(panda_ctx *ctx, float alpha, double *h_out);

/* Iterate until h < tol (strict, after a whole iteration) or max_iter
 * iterations (max_iter >= 0).  *iters_out (may be NULL) receives the number of
 * iterations run by this call, *h_last (may be NULL) the last h.  Returns 0
 * when converged, PANDA_NOT_CONVERGED when max_iter was reached first.
 * Blocks until done. */
int panda_run(panda_ctx *ctx, float alpha, double tol, int max_iter, int *iters_out,
              double *h_last);

/* Copy the current networks, diagonals included, into caller-allocated host
 * buffers (T*G, T*T and G*G floats, row-major); any pointer may be NULL to
 * skip that network. */
int panda_get(panda_ctx *ctx, float *W, float *P, float *C);

/* As panda_get, into device buffers; ordered on the context's stream and
 * complete when the call returns. */
int panda_get_device(panda_ctx *ctx, float *dW, float *dP, float *dC);

/* Networks plus the number of iterations done so far (*t, may be NULL); the
 * buffers may be host or device memory (of the context's device).
 * panda_set_state replaces the networks (taken as already normalised; P and
 * C must be exactly symmetric and finite) and the counter; the derived
 * vectors (row and column norms, FP64 diagonals) are recomputed from them, so
 * a run continued from panda_set_state matches an uninterrupted one to FP32
 * rounding.  For a bit-exact resume use panda_save / panda_load.  When
 * panda_set_state fails (for example PANDA_EASYM or PANDA_ENONFINITE on its
 * input) the context's previous state is gone: step, run, get, save and
 * batch runs then return PANDA_EINVAL until a panda_set_state or panda_load
 * succeeds.  The same holds for a panda_load that fails after its header
 * matched; one refused by the header check leaves the state untouched. */
int panda_get_state(panda_ctx *ctx, float *W, float *P, float *C, int *t);
int panda_set_state(panda_ctx *ctx, const float *W, const float *P, const float *C, int t);

/* Checkpoint and resume.  panda_checkpoint_bytes gives the size of a
 * checkpoint of ctx; panda_save writes the whole iteration state (networks,
 * FP64 diagonals, norm vectors, counters, h history) into a caller-allocated
 * host buffer of that size; panda_load restores it into a context of the
 * same shape and mode, after which the run continues bit-for-bit as if it
 * had never stopped. */
long long panda_checkpoint_bytes(const panda_ctx *ctx);
int panda_save(panda_ctx *ctx, void *buf, long long bytes);
int panda_load(panda_ctx *ctx, const void *buf, long long bytes);

/* h of every iteration done so far (oldest first) into h[0..cap); *n receives
 * the number of iterations recorded (which may exceed cap). */
int panda_get_history(panda_ctx *ctx, double *h, int cap, int *n);

/* Shape, mode and counters of a context. */
int panda_info(const panda_ctx *ctx, int *T, int *G, int *prec, int *t);

/* Bytes of device memory the context holds between calls. */
long long panda_device_bytes(const panda_ctx *ctx);

/* The most device memory the context has held at once: under PANDA_BF16X3
 * and PANDA_BF16X2 a create or panda_set_state also stages C in FP32 (4 G^2
 * bytes, padded) while it derives the split state, and frees it before it
 * returns.  PANDA_ALLOC_LIMIT_BYTES caps this peak. */
long long panda_device_bytes_peak(const panda_ctx *ctx);

/* Measurement support (the paper has no counterpart: it times the whole loop
 * only).  panda_set_profiling(ctx, 1) makes every later iteration record a
 * CUDA event before and after each of its kernels on the context's stream and
 * resets the per-kernel accumulators; panda_kernel_count gives the number of
 * kernels one iteration launches and panda_kernel_stats, for kernel i, its
 * name (NUL-terminated, truncated to name_cap), the summed device time in ms
 * and the number of launches that did work since profiling was switched on. */
int panda_set_profiling(panda_ctx *ctx, int on);
int panda_kernel_count(const panda_ctx *ctx);
int panda_kernel_stats(const panda_ctx *ctx, int i, char *name, int name_cap, double *total_ms,
                       long long *launches);

/* Self-test of the tensor-core pipeline (no paper counterpart): D = A . B^T
 * computed by the same TMA + tcgen05 + TMEM machinery the BF16X3 iteration
 * uses.  A is M x K, B is N x K, D is M x N, all row-major FP32 host buffers;
 * each operand is split into BF16 hi + lo and terms = 3 sums hi*hi + hi*lo +
 * lo*hi, terms = 1 uses hi*hi only; terms + 10 runs the same product on CTA
 * pairs (cta_group::2 MMAs over 256 x 256 tiles); terms + 20 does so with B
 * held transposed on the device ([K][N]) and fed to the MMAs MN-major, the
 * form the availability product reads the lower triangle of C in; terms + 40
 * holds both A ([K][M]) and B transposed and feeds both MN-major, terms + 50
 * A only; terms = 8
 * rounds A and B to E4M3 (nearest even, saturating) and sums their products
 * on CTA pairs with kind::f8f6f4 MMAs (FP32 accumulation).  PANDA_EINVAL on
 * other terms or non-positive sizes; PANDA_EUNSUPPORTED off sm_103. */
int panda_selftest_tc_gemm(int M, int N, int K, const float *A, const float *B, float *D, int terms);

/* Measurement support (no paper counterpart): the FP32 fused multiply-add
 * throughput of the current device, the roof of the FP32 path's products.
 * A loop of independent FMAs (8 chains per thread, 16 warps per scheduler) runs
 * on every SM; the best of ten launches timed by CUDA events after two
 * warm-up launches gives *tflops (FP32 TFLOP/s, 2 flop per FMA).  Allocates
 * and frees a few bytes of device memory.  PANDA_EINVAL for NULL,
 * PANDA_ECUDA when a CUDA call fails. */
int panda_measure_ffma_peak(double *tflops);

/* Test of the bounded device waits (no paper counterpart): runs the
 * tensor-core self-test product with one pipeline stage armed but never
 * loaded, so its barrier never completes; the kernel's bounded waits give up
 * after about a second, drain, release TMEM and exit.  Returns
 * PANDA_ETIMEOUT when that happened as intended (the device stays usable),
 * 0 if the wait unexpectedly completed, another error otherwise. */
int panda_selftest_timeout(void);

/* The context's stream as a cudaStream_t. */
void *panda_stream(const panda_ctx *ctx);

/* Message of the last error on ctx (or, when ctx is NULL, of the last failed
 * create or panda_step_static on this thread); never NULL. */
const char *panda_last_error(const panda_ctx *ctx);

/* Free everything the context owns.  NULL is ignored. */
void panda_destroy(panda_ctx *ctx);

/* ---- sets of networks ----------------------------------------------------------
 * The paper's applications compare sets of networks, one per condition or
 * sample (Section I).  A batch holds n independent networks of their own
 * sizes, each a context of its own (own device state), created with the same
 * options; each stops on its own h < tol (or max_iter).
 * Tensor-core modes: panda_batch_run iterates all of them together with one
 * launch per phase over every network's tiles (phase 1 over all their W'
 * tiles, phase 2 persistent over one longest-first schedule of all their P and
 * C tiles, then the norm and stop kernels over all their rows), a chunk of
 * iterations captured as one CUDA graph.  The schedules of both phases are
 * autotuned on the first iterations a batch runs (panda_batch_schedule).  A tile's result does
 * not depend on the schedule, so every network's results equal, bit for bit,
 * those of the same network run alone.
 * FP32: every network queues its chunks (a CUDA graph each) on its own stream. */
typedef struct panda_batch panda_batch;

/* T[k], G[k], W0[k], P0[k], C0[k] as in panda_create for network k (host
 * pointers, copied).  On error nothing is kept and panda_last_error(NULL)
 * names the failing network. */
int panda_batch_create(panda_batch **out, int n, const int *T, const int *G, const float *const *W0,
                       const float *const *P0, const float *const *C0, const panda_opts *o);

/* Run every network until its own h < tol or max_iter iterations.
 * iters_out[k] and h_last[k] (each may be NULL, else n entries) receive the
 * iterations run and the last h of network k.  Returns 0 when every network
 * converged, PANDA_NOT_CONVERGED when at least one reached max_iter. */
int panda_batch_run(panda_batch *b, float alpha, double tol, int max_iter, int *iters_out, double *h_last);

/* Network k's current W, P, C (as panda_get). */
int panda_batch_get(panda_batch *b, int k, float *W, float *P, float *C);

/* Number of networks; network k's context (owned by the batch: do not
 * destroy it; it accepts the per-context calls such as panda_get_history). */
int panda_batch_size(const panda_batch *b);
panda_ctx *panda_batch_context(panda_batch *b, int k);

/* The schedule autotuning of a tensor-core batch (no paper counterpart).
 * Both phases run on persistent CTA pairs over longest-first (LPT) lists of
 * every network's tiles; the candidates differ in the order of a network's
 * phase-1 tiles (which operand rows neighbouring tiles share in L2) and in
 * the phase-2 cost model (MMA slots, or the larger of MMA and HBM time),
 * epilogue weight and list order (panda_batch_schedule_name describes each).
 * The first iterations a batch runs are the trials: one warm-up, then three
 * iterations per phase-1 candidate (timing phase 1), the fastest by median
 * kept, then three per phase-2 candidate (timing phase 2).  *p1, *p2 receive
 * the candidates in use; p1_ms[q] (n1 entries) and p2_ms[q] (n2 entries),
 * each may be NULL, the median trial times in ms (0 while not yet run);
 * *done whether the trials are over.  Returns 1 for a tensor-core batch, 0 for
 * an FP32 batch (no schedules), PANDA_EINVAL for NULL b. */
int panda_batch_schedule(const panda_batch *b, int *p1, int *p2, float *p1_ms, int n1, float *p2_ms, int n2,
                         int *done);

/* Description of schedule candidate k of phase 1 (phase = 1) or phase 2
 * (phase = 2); NULL past the last candidate. */
const char *panda_batch_schedule_name(int phase, int k);

/* How phase 1 of one network of T TFs and G genes would be spread over
 * `pairs` persistent CTA pairs in tensor-core mode prec (a host computation:
 * no device is needed).  Phase 1 computes the W' tiles of Eqs. 2-3 and 7;
 * each 256 x 256 tile sums the availability numerator W.C over all genes in
 * chunks of 32 k-blocks (64 genes each; 128 under PANDA_FP8MIX), then the
 * responsibility numerator and the epilogue.  Whole tiles run in rounds;
 * when that leaves the busiest pair more than 5% above the average, the
 * tiles of the last two rounds are cut at chunk boundaries into equal
 * shares of MMA work.  A cut tile's head (chunks 0 .. b - 1) runs on its
 * pair right after the whole-tile rounds, its tail (chunks b .. n - 1, the
 * responsibility numerator, the epilogue) last on another pair, which waits
 * (bounded) for the head: all_resident = 0 (not every pair known to be
 * resident at once) makes no cuts.  Up to cap pieces are written to pieces,
 * six ints each, in the order each pair runs them, pair by pair: pair, TF
 * block mt, gene block nt, first chunk c0, end chunk c1 (c1 = n for a piece
 * that ends the tile), cut index (-1 for a whole tile).  *n_pieces receives
 * the total count.  Returns the number of cut tiles, or PANDA_EINVAL (T or G
 * < 1, prec not a tensor-core mode, pairs < 1, n_pieces NULL, or pieces NULL
 * with cap > 0). */
int panda_phase1_plan(int T, int G, int prec, int pairs, int all_resident, int *pieces, int cap, int *n_pieces);

/* The phase-1 launch a tensor-core context uses (see panda_phase1_plan):
 * *pairs its persistent CTA pairs, *clusters the two-CTA clusters the
 * device holds at once for that kernel (cuts are made only when every pair
 * is resident), *cuts the tiles cut between two pairs; any pointer may be
 * NULL.  Returns 0, or PANDA_EINVAL for NULL c or an FP32 context. */
int panda_phase1_layout(const panda_ctx *c, int *pairs, int *clusters, int *cuts);

const char *panda_batch_last_error(const panda_batch *b);
void panda_batch_destroy(panda_batch *b);

/* ---- allocation-free single iteration ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that are not allowed to allocate device memory: code running inside a host
 * framework that hands out all device memory from its own pool or budget,
 * plug-ins that must not call cudaMalloc once the process is running, or
 * loops where cudaMalloc's implicit device synchronisation is not
 * acceptable.  panda_step_static runs one message-passing iteration (the same
 * FP32 kernels as panda_step, so the same results) directly on the caller's
 * device networks and calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * dW (T x G), dP (T x T) and dC (G x G) are dense row-major FP32 device
 * buffers, diagonals included, owned by the caller and updated in place.
 * They are used as given: no Z-score is applied (normalise them first, or
 * take them from panda_get).  dP and dC must be exactly symmetric
 * (PANDA_EASYM) and finite (PANDA_ENONFINITE).  alpha in [0, 1]; t >= 1 is
 * the 1-based iteration index used in the diagonal growth factor
 * e^{2 alpha t}; diag is a panda_diag rule.  *h_out (may be NULL) receives
 * h.  The call runs on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and blocks until the iteration is done.  When it returns an error
 * (PANDA_ENONFINITE included) dW, dP and dC hold what they held before.
 *
 * Working memory is one file-scope device array of about 7.4 MB, sized for
 * T, G <= PANDA_STATIC_MAX_NODES; larger shapes are rejected with
 * PANDA_EINVAL before any GPU work.  Every GPU that loads the library's
 * device code holds the array until the process exits; with CUDA's lazy
 * module loading (the default) that happens at the first call on the
 * device, so a caller with a fixed memory budget makes that call at
 * start-up.  The first call on each device also looks up the array's device
 * address (with that device current); make that first call before any
 * stream capture.  All calls share the array and clear it at
 * their start, so calls that overlap on the GPU (for example on two streams)
 * race and must be serialised by the caller.  Errors are reported by the
 * return code and panda_last_error(NULL). */
#define PANDA_STATIC_MAX_NODES 512
int panda_step_static(int T, int G, float *dW, float *dP, float *dC, float alpha, int t, int diag,
                      double *h_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
