// The C ABI of libpanda_gb300 (declared in include/panda.h): context
// creation with validation and Z-score normalisation (Section II-A), the
// iteration driver with its stop test (Section II-B), state access,
// checkpointing, and the device memory plan.
#include "panda.h"
#include "panda_internal.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace panda;

struct panda_ctx {
    int T = 0, G = 0, Tp = 0, Gp = 0, nbT = 0, nbG = 0;
    int prec = PANDA_FP32, diag = PANDA_DIAG_D1, normalize = 1, graph_iters = 8;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int cur = 0;  // which W buffer holds the current network
    // false once panda_set_state or panda_load has rejected its input or failed midway: the
    // device then holds no valid state, and everything that reads it refuses until one of
    // them succeeds
    bool state_ok = true;
    Dev d{};
    Ctl *h_ctl = nullptr;  // pinned mirror of the device control block
    std::vector<void *> allocs;
    long long bytes = 0;       // device memory held between calls
    long long peak = 0;        // the most held at once (staging buffers included)
    long long limit = -1;
    float *c_stage = nullptr;  // FP32 C while a create or set_state derives a split-held state
    float e2_alpha = -1.0f;  // alpha for which d.e2tab is filled
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int *d_flags = nullptr;
    double *d_stats = nullptr, *d_partials = nullptr;
    // per-kernel timing (panda_set_profiling)
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // graph_iters (or 1) x (kernels + 1)
    double k_ms[16] = {};
    long long k_launches[16] = {};
    std::string err;
};

namespace {

thread_local std::string g_create_error = "no error";

// An NVTX range over one API call, for timeline tools (no cost without one attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

// the modes that run on the tensor-core path (k_tc.cu)
bool tensor_prec(int prec) { return prec == PANDA_BF16X3 || prec == PANDA_BF16X2 || prec == PANDA_FP8MIX; }

struct Fail {
    int code;
};

int set_err(panda_ctx *c, int code, const std::string &msg)
{
    if (c)
        c->err = msg;
    else
        g_create_error = msg;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return set_err(c, e_ == cudaErrorMemoryAllocation ? PANDA_ENOMEM : PANDA_ECUDA,  \
                           std::string(#call) + ": " + cudaGetErrorString(e_));               \
    } while (0)

long long alloc_limit_from_env()
{
    const char *s = std::getenv("PANDA_ALLOC_LIMIT_BYTES");
    if (!s || !*s)
        return -1;
    return std::atoll(s);
}

template <typename T>
int dalloc(panda_ctx *c, T **p, size_t count)
{
    size_t bytes = count * sizeof(T);
    if (bytes == 0)
        bytes = 16;
    if (c->limit >= 0 && c->bytes + (long long)bytes > c->limit) {
        *p = nullptr;
        return set_err(c, PANDA_ENOMEM, "device memory plan exceeds PANDA_ALLOC_LIMIT_BYTES");
    }
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, PANDA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    c->allocs.push_back(q);
    c->bytes += (long long)bytes;
    c->peak = c->bytes > c->peak ? c->bytes : c->peak;
    e = cudaMemsetAsync(q, 0, bytes, c->stream);
    if (e != cudaSuccess)
        return set_err(c, PANDA_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    *p = static_cast<T *>(q);
    return 0;
}

#define DALLOC(ptr, n)                     \
    do {                                   \
        int r_ = dalloc(c, &(ptr), (n));   \
        if (r_)                            \
            return r_;                     \
    } while (0)

int plan_memory(panda_ctx *c)
{
    Dev &d = c->d;
    const size_t Tp = c->Tp, Gp = c->Gp;
    d.T = c->T; d.G = c->G; d.Tp = c->Tp; d.Gp = c->Gp; d.nbT = c->nbT; d.nbG = c->nbG;
    d.diag = c->diag;
    d.split_b = c->prec == PANDA_BF16X2 ? 0 : 1;  // the BF16 products of FP8MIX are BF16X3
    d.fp8 = c->prec == PANDA_FP8MIX ? 1 : 0;
    // BF16X3 and BF16X2 hold C as its split pair only (FP32 C is staged while the state is derived)
    d.c_split = (c->prec == PANDA_BF16X3 || c->prec == PANDA_BF16X2) ? 1 : 0;
    for (int b = 0; b < 2; ++b) {
        DALLOC(d.W[b], Tp * Gp);
        if (!d.c_split)  // the FP32 path's operand, FP8MIX's source of its E4M3 transposes
            DALLOC(d.Wt[b], Gp * Tp);
    }
    DALLOC(d.Poff, Tp * Tp);
    if (!d.c_split)
        DALLOC(d.Coff, Gp * Gp);
    DALLOC(d.pd, Tp);
    DALLOC(d.cd, Gp);
    DALLOC(d.pdf, Tp);
    DALLOC(d.cdf, Gp);
    DALLOC(d.rsqP, Tp);
    DALLOC(d.csqC, Gp);
    DALLOC(d.rsqW, Tp);
    DALLOC(d.csqW, Gp);
    if (c->prec == PANDA_FP32)
        DALLOC(d.Rn, Tp * Gp);
    DALLOC(d.wrow_part, (size_t)c->nbG * Tp);
    DALLOC(d.wcol_part, (size_t)c->nbT * Gp);
    DALLOC(d.hpart, (size_t)c->nbT * c->nbG);
    // partial-sum slots: one per 128-row block (FP32 path); on the tensor-core
    // path one per 256-column block for the row role plus one per 128-row half
    // for the column role (see k_tc.cu)
    d.nsP = tensor_prec(c->prec) ? 3 * ceil_div(c->Tp, 256) : c->nbT;
    d.nsC = tensor_prec(c->prec) ? 3 * ceil_div(c->Gp, 256) : c->nbG;
    d.tri_slots = tensor_prec(c->prec) ? 1 : 0;
    DALLOC(d.ps_sum, (size_t)d.nsP * Tp);
    DALLOC(d.ps_sq, (size_t)d.nsP * Tp);
    DALLOC(d.ps_vsq, (size_t)d.nsP * Tp);
    DALLOC(d.cs_sum, (size_t)d.nsC * Gp);
    DALLOC(d.cs_sq, (size_t)d.nsC * Gp);
    DALLOC(d.cs_vsq, (size_t)d.nsC * Gp);
    DALLOC(d.ctl, 1);
    DALLOC(d.hist, HIST_CAP);
    DALLOC(d.e2tab, HIST_CAP + 1);
    DALLOC(c->d_flags, 4);
    DALLOC(c->d_stats, 4);
    DALLOC(c->d_partials, 1024);
    if (tensor_prec(c->prec)) {
        for (int b = 0; b < 2; ++b) {
            DALLOC(d.Wh[b], Tp * Gp);
            DALLOC(d.Wl[b], Tp * Gp);
        }
        DALLOC(d.Ph, Tp * Tp);
        DALLOC(d.Pl, Tp * Tp);
        // running sums of the long products' K chunks: one 128 x 256 slot per CTA of the
        // persistent phase-1 and phase-2 launches (at most one CTA per SM)
        int nsm = 0;
        CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
        DALLOC(d.p1_acc, (size_t)nsm * 128 * 256);
        d.p1_cuts = tc_phase1_cuts(d);  // tiles cut between two pairs: a slot and a flag per CTA rank
        if (d.p1_cuts < 0)
            return set_err(c, PANDA_ECUDA, "cudaOccupancyMaxActiveClusters failed");
        if (d.p1_cuts > 0) {
            DALLOC(d.p1_fix, (size_t)d.p1_cuts * 2 * 128 * 256);
            DALLOC(d.p1_flag, (size_t)d.p1_cuts * 2);
        }
        if (d.fp8) {  // W.C and W^T.W on E4M3 copies; no BF16 copy of C
            for (int b = 0; b < 2; ++b) {
                DALLOC(d.W8[b], Tp * Gp);
                DALLOC(d.Wt8[b], Gp * Tp);
            }
            DALLOC(d.C8, Gp * Gp);
            DALLOC(d.f8, 4);
            DALLOC(d.f8n, 8);
        } else {  // C's state: hi and lo (BF16X2 keeps lo too, for the state, not as an operand)
            DALLOC(d.Ch, Gp * Gp);
            DALLOC(d.Cl, Gp * Gp);
        }
    }
    return 0;
}

// A split-held C (d.c_split) is derived from an FP32 copy: stage_c gives Coff
// a zeroed Gp x Gp FP32 buffer for that (within PANDA_ALLOC_LIMIT_BYTES,
// counted in the peak, not in the memory held between calls), unstage_c frees
// it once the split pair is written.
int stage_c(panda_ctx *c)
{
    Dev &d = c->d;
    if (!d.c_split || c->c_stage)
        return 0;
    const size_t bytes = sizeof(float) * (size_t)c->Gp * c->Gp;
    if (c->limit >= 0 && c->bytes + (long long)bytes > c->limit)
        return set_err(c, PANDA_ENOMEM, "device memory plan exceeds PANDA_ALLOC_LIMIT_BYTES");
    CU(cudaMalloc(&c->c_stage, bytes));
    const long long held = c->bytes + (long long)bytes;
    c->peak = held > c->peak ? held : c->peak;
    CU(cudaMemsetAsync(c->c_stage, 0, bytes, c->stream));
    d.Coff = c->c_stage;
    return 0;
}

int unstage_c(panda_ctx *c)
{
    if (!c->c_stage)
        return 0;
    CU(cudaStreamSynchronize(c->stream));
    CU(cudaFree(c->c_stage));
    c->c_stage = nullptr;
    c->d.Coff = nullptr;
    return 0;
}

int push_ctl(panda_ctx *c)
{
    CU(cudaMemcpyAsync(c->d.ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, c->stream));
    return 0;
}

// Copy a rows x cols row-major matrix (host or device) into a padded buffer.
// src: host or device (cudaMemcpyDefault), row stride src_ld (0: cols)
int upload(panda_ctx *c, float *dst, int ld, const float *src, int rows, int cols, int src_ld = 0)
{
    const size_t spitch = (size_t)(src_ld > 0 ? src_ld : cols) * sizeof(float);
    CU(cudaMemcpy2DAsync(dst, (size_t)ld * sizeof(float), src, spitch, (size_t)cols * sizeof(float), rows,
                         cudaMemcpyDefault, c->stream));
    return 0;
}

int download(panda_ctx *c, float *dst, const float *src, int ld, int rows, int cols)
{
    CU(cudaMemcpy2DAsync(dst, (size_t)cols * sizeof(float), src, (size_t)ld * sizeof(float),
                         (size_t)cols * sizeof(float), rows, cudaMemcpyDefault, c->stream));
    return 0;
}

// Validate the freshly uploaded networks: finite entries, exact symmetry.
int validate(panda_ctx *c)
{
    Dev &d = c->d;
    int flags[4];
    CU(cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), c->stream));
    CU(launch_check_finite_sym(d.W[c->cur], c->T, c->G, c->Gp, false, c->d_flags, c->stream));
    CU(launch_check_finite_sym(d.Poff, c->T, c->T, c->Tp, true, c->d_flags, c->stream));
    CU(launch_check_finite_sym(d.Coff, c->G, c->G, c->Gp, true, c->d_flags, c->stream));
    CU(cudaMemcpyAsync(flags, c->d_flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (flags[0])
        return set_err(c, PANDA_ENONFINITE, "an input network has a non-finite entry");
    if (flags[1])
        return set_err(c, PANDA_EASYM, "P0 or C0 is not exactly symmetric");
    return 0;
}

int zscore_all(panda_ctx *c)
{
    Dev &d = c->d;
    struct { float *X; int rows, cols, ld; const char *name; } nets[3] = {
        {d.W[c->cur], c->T, c->G, c->Gp, "W0"},
        {d.Poff, c->T, c->T, c->Tp, "P0"},
        {d.Coff, c->G, c->G, c->Gp, "C0"}};
    for (auto &n : nets) {
        double st[2];
        CU(launch_zscore(n.X, n.rows, n.cols, n.ld, c->d_stats, c->d_partials, c->stream));
        CU(cudaMemcpyAsync(st, c->d_stats, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        if (!(st[1] > 0.0))
            return set_err(c, PANDA_EDEGENERATE,
                           std::string(n.name) + " has zero standard deviation; its Z-score is undefined");
        if (!std::isfinite(st[0]) || !std::isfinite(st[1]))
            return set_err(c, PANDA_ENONFINITE, std::string(n.name) + " statistics are not finite");
    }
    return 0;
}

// From full W (in W[cur]), P and C (diagonals in place): strip diagonals,
// transposed W, squared norms, split copies.
int derive_state(panda_ctx *c, bool split_diag)
{
    Dev &d = c->d;
    if (split_diag) {
        CU(launch_split_diag(d.Poff, c->T, c->Tp, d.pd, d.pdf, c->stream));
        CU(launch_split_diag(d.Coff, c->G, c->Gp, d.cd, d.cdf, c->stream));
    }
    CU(launch_row_norms(d.W[c->cur], c->T, c->G, c->Gp, nullptr, d.rsqW, c->stream));
    if (d.Wt[c->cur]) {
        CU(launch_transpose(d.W[c->cur], c->Tp, c->Gp, d.Wt[c->cur], c->stream));
        CU(launch_row_norms(d.Wt[c->cur], c->G, c->T, c->Tp, nullptr, d.csqW, c->stream));  // columns of W
    } else {
        CU(launch_col_norms(d.W[c->cur], c->T, c->G, c->Gp, d.csqW, c->stream));
    }
    CU(launch_row_norms(d.Poff, c->T, c->T, c->Tp, d.pd, d.rsqP, c->stream));
    CU(launch_row_norms(d.Coff, c->G, c->G, c->Gp, d.cd, d.csqC, c->stream));
    if (tensor_prec(c->prec))
        CU(tc_prepare(d, c->stream));
    return 0;
}

void drop_graphs(panda_ctx *c)
{
    for (auto &g : c->gexec)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

int n_kernels(const panda_ctx *c) { return tensor_prec(c->prec) ? TC_KERNELS : SIMT_KERNELS; }

const char *kernel_name(const panda_ctx *c, int i)
{
    return tensor_prec(c->prec) ? TC_KERNEL_NAMES[i] : SIMT_KERNEL_NAMES[i];
}

// slot: which iteration of a graph (or chunk) this is, for the timing events
int launch_iteration(panda_ctx *c, int cur, int slot)
{
    KernelEvents ke{c->prof ? c->ev.data() + (size_t)slot * (n_kernels(c) + 1) : nullptr, 0};
    cudaError_t e = tensor_prec(c->prec) ? launch_iteration_tc(c->d, cur, c->stream, ke)
                                            : launch_iteration_simt(c->d, cur, c->stream, ke);
    if (e != cudaSuccess)
        return set_err(c, PANDA_ECUDA, std::string("iteration launch: ") + cudaGetErrorString(e));
    return 0;
}

int ensure_graph(panda_ctx *c, int cur)
{
    if (c->gexec[cur])
        return 0;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int k = 0; k < c->graph_iters && !rc; ++k)
        rc = launch_iteration(c, cur ^ (k & 1), k);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc) {
        if (g)
            cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess)
        return set_err(c, PANDA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec[cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[cur] = nullptr;
        return set_err(c, PANDA_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return 0;
}

int fill_e2(panda_ctx *c, float alpha)
{
    if (c->e2_alpha == alpha)
        return 0;
    std::vector<double> tab(HIST_CAP + 1);
    for (int t = 0; t <= HIST_CAP; ++t)
        tab[t] = std::exp(2.0 * (double)alpha * (double)t);  // e^{2 alpha t} of Eq. 6
    CU(cudaMemcpyAsync(c->d.e2tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice,
                       c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->e2_alpha = alpha;
    return 0;
}

// The driver, in three parts so that several contexts can run concurrently:
// drive_begin arms the device control block for up to max_iter iterations,
// drive_launch queues one chunk (a graph of graph_iters iterations, or that
// many plain launches) without waiting, drive_collect waits for it and
// reads the control block back.  Kernels of iterations past the stop do no
// work, so a chunk never overshoots.
struct DriveState {
    int start = 0, before = 0;
    bool use_graph = false;
};

int drive_begin(panda_ctx *c, float alpha, double tol, int max_iter, bool use_graph, DriveState &ds)
{
    int rc = fill_e2(c, alpha);
    if (rc)
        return rc;
    Ctl &h = *c->h_ctl;
    ds.start = ds.before = h.iters;
    ds.use_graph = use_graph && c->graph_iters > 0 && c->stream != nullptr;  // the legacy NULL stream cannot be captured
    if ((long long)ds.start + max_iter > (long long)HIST_CAP)
        return set_err(c, PANDA_EINVAL, "iteration count would exceed the supported maximum (65536)");
    h.active = max_iter > 0;
    h.stop_at = ds.start + max_iter;
    if (c->d.p1_flag)  // a run that gave up (a bounded wait ran out) may have left a cut tile's flag raised
        CU(cudaMemsetAsync(c->d.p1_flag, 0, (size_t)c->d.p1_cuts * 2 * sizeof(int), c->stream));
    h.status = 0;
    h.converged = 0;
    h.alpha = alpha;
    h.tol = tol;
    return push_ctl(c);
}

int drive_launch(panda_ctx *c, DriveState &ds)
{
    Ctl &h = *c->h_ctl;
    ds.before = h.iters;
    const int cur = c->cur ^ ((ds.before - ds.start) & 1);
    int rc;
    if (ds.use_graph) {
        if ((rc = ensure_graph(c, cur)))
            return rc;
        CU(cudaGraphLaunch(c->gexec[cur], c->stream));
    } else {
        const int K = c->graph_iters;
        int chunk = K > 0 ? K : 1;
        if (chunk > h.stop_at - ds.before)
            chunk = h.stop_at - ds.before;
        for (int k = 0; k < chunk; ++k)
            if ((rc = launch_iteration(c, cur ^ (k & 1), k)))
                return rc;
    }
    CU(cudaMemcpyAsync(c->h_ctl, c->d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
    return 0;
}

// Returns 0 with *more set while the run continues.
int drive_collect(panda_ctx *c, DriveState &ds, bool *more)
{
    CU(cudaStreamSynchronize(c->stream));
    Ctl &h = *c->h_ctl;
    if (c->prof) {  // iterations that did work in this chunk: their kernel times
        const int nk = n_kernels(c);
        for (int k = 0; k < h.iters - ds.before; ++k) {
            cudaEvent_t *e = c->ev.data() + (size_t)k * (nk + 1);
            for (int q = 0; q < nk; ++q) {
                float ms = 0.0f;
                CU(cudaEventElapsedTime(&ms, e[q], e[q + 1]));
                c->k_ms[q] += ms;
                c->k_launches[q] += 1;
            }
        }
    }
    *more = h.active != 0;
    if (!*more) {
        c->cur ^= ((h.iters - ds.start) & 1);
        if (h.status & ST_NONFINITE)
            return set_err(c, PANDA_ENONFINITE, "the state became non-finite");
        if (h.status & ST_TIMEOUT)
            return set_err(c, PANDA_ETIMEOUT, "a bounded device wait expired");
    }
    return 0;
}

// Run up to max_iter iterations (stopping early when h < tol).
int drive(panda_ctx *c, float alpha, double tol, int max_iter, bool use_graph, int *n_done)
{
    *n_done = 0;
    if (max_iter <= 0)
        return 0;
    DriveState ds;
    int rc = drive_begin(c, alpha, tol, max_iter, use_graph, ds);
    bool more = true;
    while (!rc && more) {
        rc = drive_launch(c, ds);
        if (!rc)
            rc = drive_collect(c, ds, &more);
    }
    *n_done = c->h_ctl->iters - ds.start;
    return rc;
}

int check_ctx(const panda_ctx *c) { return c ? 0 : PANDA_EINVAL; }

int check_state(panda_ctx *c)
{
    return c->state_ok ? 0
                       : set_err(c, PANDA_EINVAL,
                                 "the context holds no valid state (a panda_set_state or panda_load failed): "
                                 "give it one with panda_set_state or panda_load");
}

void free_all(panda_ctx *c)
{
    if (!c)
        return;
    drop_graphs(c);
    if (c->stream)
        cudaStreamSynchronize(c->stream);
    tc_release(c->d);
    if (c->c_stage)
        cudaFree(c->c_stage);
    c->c_stage = nullptr;
    for (void *p : c->allocs)
        cudaFree(p);
    c->allocs.clear();
    if (c->h_ctl)
        cudaFreeHost(c->h_ctl);
    for (auto &ev : c->ev)
        if (ev)
            cudaEventDestroy(ev);
    c->ev.clear();
    if (c->own_stream && c->stream)
        cudaStreamDestroy(c->stream);
}

// C0's row stride is ldc (0: G); the sources may be host or device memory.
int create_common(panda_ctx **out, int T, int G, const float *W0, const float *P0, const float *C0,
                  const panda_opts *o, void *stream, bool device_ptrs, int ldc = 0)
{
    if (!out)
        return set_err(nullptr, PANDA_EINVAL, "out is NULL");
    *out = nullptr;
    if (T <= 0 || G <= 0)
        return set_err(nullptr, PANDA_EINVAL, "T and G must be positive");
    if (!W0 || !P0 || !C0)
        return set_err(nullptr, PANDA_EINVAL, "W0, P0 and C0 must not be NULL");
    if ((long long)G > 46000 || (long long)T > 46000)
        return set_err(nullptr, PANDA_EINVAL, "T and G must be at most 46000");
    panda_opts opts;
    panda_default_opts(&opts);
    if (o)
        opts = *o;
    if (opts.prec != PANDA_FP32 && !tensor_prec(opts.prec))
        return set_err(nullptr, PANDA_EUNSUPPORTED, "unknown precision mode");
    if (opts.diag < 0 || opts.diag > 2 || opts.t0 < 0 || opts.t0 >= HIST_CAP || opts.graph_iters < 0)
        return set_err(nullptr, PANDA_EINVAL, "bad option value");
    if (tensor_prec(opts.prec) && !tc_supported())
        return set_err(nullptr, PANDA_EUNSUPPORTED, "the tensor-core modes need an sm_103 device");

    panda_ctx *c = new panda_ctx();
    c->T = T; c->G = G;
    // the tensor-core path works on 256-row tiles of CTA pairs: pad to 256 there
    const int granule = tensor_prec(opts.prec) ? 2 * TILE : TILE;
    c->Tp = round_up(T, granule); c->Gp = round_up(G, granule);
    c->nbT = c->Tp / TILE; c->nbG = c->Gp / TILE;
    c->prec = opts.prec; c->diag = opts.diag; c->normalize = opts.normalize;
    c->graph_iters = (opts.graph_iters + 1) & ~1;  // even: a graph returns to its start buffer
    c->limit = alloc_limit_from_env();
    int rc = 0;
    auto fail = [&](int code) {
        std::string msg = c->err;
        free_all(c);
        delete c;
        g_create_error = msg;
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        c->err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return fail(PANDA_ECUDA);
    }
    if (device_ptrs) {
        c->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c->err = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            return fail(PANDA_ECUDA);
        }
        c->own_stream = true;
    }
    e = cudaMallocHost(&c->h_ctl, sizeof(Ctl));
    if (e != cudaSuccess) {
        c->err = std::string("cudaMallocHost: ") + cudaGetErrorString(e);
        return fail(PANDA_ENOMEM);
    }
    std::memset(c->h_ctl, 0, sizeof(Ctl));
    c->h_ctl->iters = opts.t0;
    c->ev.resize((size_t)(c->graph_iters > 0 ? c->graph_iters : 1) * 17, nullptr);
    for (auto &ev : c->ev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) {
            c->err = std::string("cudaEventCreate: ") + cudaGetErrorString(e);
            return fail(PANDA_ECUDA);
        }
    if ((rc = plan_memory(c)) || (rc = stage_c(c)))
        return fail(rc);
    if ((rc = upload(c, c->d.W[0], c->Gp, W0, T, G)) || (rc = upload(c, c->d.Poff, c->Tp, P0, T, T)) ||
        (rc = upload(c, c->d.Coff, c->Gp, C0, G, G, ldc)))
        return fail(rc);
    if ((rc = validate(c)))
        return fail(rc);
    if (c->normalize && (rc = zscore_all(c)))
        return fail(rc);
    if ((rc = derive_state(c, true)) || (rc = push_ctl(c)) || (rc = unstage_c(c)))
        return fail(rc);
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        c->err = std::string("create: ") + cudaGetErrorString(e);
        return fail(PANDA_ECUDA);
    }
    *out = c;
    return 0;
}

}  // namespace

namespace panda {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace panda

extern "C" {

int panda_precision_supported(int prec)
{
    if (prec == PANDA_FP32) {
        int n = 0;
        return cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
    }
    if (tensor_prec(prec))
        return tc_supported() ? 1 : 0;
    return 0;
}

void panda_default_opts(panda_opts *o)
{
    if (!o)
        return;
    o->prec = PANDA_FP32;
    o->diag = PANDA_DIAG_D1;
    o->normalize = 1;
    o->t0 = 0;
    o->graph_iters = 8;
}

int panda_create(panda_ctx **out, int T, int G, const float *W0, const float *P0, const float *C0,
                 const panda_opts *o)
{
    Range r("panda_create");
    return create_common(out, T, G, W0, P0, C0, o, nullptr, false);
}

int panda_create_device(panda_ctx **out, int T, int G, const float *dW0, const float *dP0,
                        const float *dC0, const panda_opts *o, void *stream)
{
    Range r("panda_create_device");
    return create_common(out, T, G, dW0, dP0, dC0, o, stream, true);
}

int panda_create_from_expression(panda_ctx **out, int T, int G, int N, const float *W0, const float *P0,
                                 const float *X, const panda_opts *o)
{
    Range range("panda_create_from_expression");
    if (!out)
        return set_err(nullptr, PANDA_EINVAL, "out is NULL");
    *out = nullptr;
    if (T <= 0 || G <= 0 || N <= 0 || !W0 || !X)
        return set_err(nullptr, PANDA_EINVAL, "T, G, N must be positive; W0 and X must not be NULL");
    if (G > 46000 || T > 46000)
        return set_err(nullptr, PANDA_EINVAL, "T and G must be at most 46000");
    if (!tc_supported())
        return set_err(nullptr, PANDA_EUNSUPPORTED, "the GPU Pearson initialisation needs an sm_103 device");
    const int Gp = round_up(G, 2 * TILE), Kp = round_up(N, 64);
    cudaStream_t s = nullptr;
    float *dX = nullptr, *dC = nullptr;
    __nv_bfloat16 *Zh = nullptr, *Zl = nullptr;
    int *flags = nullptr;
    Ctl *ctl = nullptr;
    std::vector<float> eye;
    auto cleanup = [&]() {
        if (s)
            cudaStreamSynchronize(s);
        cudaFree(dX); cudaFree(dC); cudaFree(Zh); cudaFree(Zl); cudaFree(flags); cudaFree(ctl);
        if (s)
            cudaStreamDestroy(s);
    };
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) ||
        (e = cudaMalloc(&dX, sizeof(float) * (size_t)G * N)) ||
        (e = cudaMalloc(&dC, sizeof(float) * (size_t)Gp * Gp)) ||
        (e = cudaMalloc(&Zh, sizeof(__nv_bfloat16) * (size_t)Gp * Kp)) ||
        (e = cudaMalloc(&Zl, sizeof(__nv_bfloat16) * (size_t)Gp * Kp)) || (e = cudaMalloc(&flags, sizeof(int))) ||
        (e = cudaMalloc(&ctl, sizeof(Ctl)))) {
        const int code = e == cudaErrorMemoryAllocation ? PANDA_ENOMEM : PANDA_ECUDA;
        cleanup();
        return set_err(nullptr, code, std::string("panda_create_from_expression: ") + cudaGetErrorString(e));
    }
    int hflags = 0;
    Ctl hctl{};
    if ((e = cudaMemsetAsync(Zh, 0, sizeof(__nv_bfloat16) * (size_t)Gp * Kp, s)) ||
        (e = cudaMemsetAsync(Zl, 0, sizeof(__nv_bfloat16) * (size_t)Gp * Kp, s)) ||
        (e = cudaMemsetAsync(flags, 0, sizeof(int), s)) || (e = cudaMemsetAsync(ctl, 0, sizeof(Ctl), s)) ||
        (e = cudaMemcpyAsync(dX, X, sizeof(float) * (size_t)G * N, cudaMemcpyDefault, s)) ||
        (e = launch_standardize_rows(dX, G, N, Zh, Zl, Kp, flags, s)) ||
        (e = cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        cleanup();
        return set_err(nullptr, PANDA_ECUDA, std::string("panda_create_from_expression: ") + cudaGetErrorString(e));
    }
    if (hflags) {
        cleanup();
        return set_err(nullptr, hflags & 1 ? PANDA_ENONFINITE : PANDA_EDEGENERATE,
                       hflags & 1 ? "panda_create_from_expression: a sample is not finite"
                                  : "panda_create_from_expression: a gene has zero variance across the samples");
    }
    // correlations: the Gram of the unit-norm centred rows, its upper triangle mirrored, unit diagonal
    if ((e = tc_gram(Zh, Zl, Gp, Kp, dC, ctl, s)) || (e = launch_symmetrize(dC, G, Gp, s)) ||
        (e = launch_unit_diag(dC, G, Gp, s)) ||
        (e = cudaMemcpyAsync(&hctl, ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s))) {
        cleanup();
        return set_err(nullptr, PANDA_ECUDA, std::string("panda_create_from_expression: ") + cudaGetErrorString(e));
    }
    if (hctl.status & ST_TIMEOUT) {
        cleanup();
        return set_err(nullptr, PANDA_ETIMEOUT, "panda_create_from_expression: a bounded device wait expired");
    }
    if (!P0) {  // no interaction data: the identity (Sec. II-A)
        eye.assign((size_t)T * T, 0.0f);
        for (int i = 0; i < T; ++i)
            eye[(size_t)i * T + i] = 1.0f;
        P0 = eye.data();
    }
    const int rc = create_common(out, T, G, W0, P0, dC, o, nullptr, false, Gp);
    cleanup();
    return rc;
}

int panda_step(panda_ctx *c, float alpha, double *h_out)
{
    Range r("panda_step");
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (int rc = check_state(c))
        return rc;
    if (!(alpha >= 0.0f && alpha <= 1.0f))
        return set_err(c, PANDA_EINVAL, "alpha must be in [0, 1]");
    int n = 0;
    int rc = drive(c, alpha, -1.0, 1, false, &n);
    if (rc)
        return rc;
    if (h_out)
        *h_out = c->h_ctl->h_last;
    return 0;
}

int panda_run(panda_ctx *c, float alpha, double tol, int max_iter, int *iters_out, double *h_last)
{
    Range r("panda_run");
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (int rc = check_state(c))
        return rc;
    if (!(alpha >= 0.0f && alpha <= 1.0f))
        return set_err(c, PANDA_EINVAL, "alpha must be in [0, 1]");
    if (!(tol >= 0.0) || max_iter < 0)
        return set_err(c, PANDA_EINVAL, "tol must be >= 0 and max_iter >= 0");
    int n = 0;
    int rc = drive(c, alpha, tol, max_iter, c->graph_iters > 0, &n);
    if (iters_out)
        *iters_out = n;
    if (h_last)
        *h_last = c->h_ctl->h_last;
    if (rc)
        return rc;
    return c->h_ctl->converged ? PANDA_OK : PANDA_NOT_CONVERGED;
}

// The tensor-core path keeps only the upper triangle of FP32 P and C current.
static int full_matrices(panda_ctx *c)
{
    if (tensor_prec(c->prec)) {
        CU(launch_symmetrize(c->d.Poff, c->T, c->Tp, c->stream));
        if (!c->d.c_split)
            CU(launch_symmetrize(c->d.Coff, c->G, c->Gp, c->stream));
    }
    return 0;
}

// Whether p is device (or managed) memory of the current device.
static bool device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// C (G x G, dense, host or device) from its split pair: straight into device
// memory, through a temporary device buffer into host memory.
static int get_split_c(panda_ctx *c, float *C)
{
    Dev &d = c->d;
    const int G = c->G;
    if (device_pointer(C)) {
        CU(launch_unsplit_sym(d.Ch, d.Cl, G, c->Gp, C, G, c->stream));
        return 0;
    }
    float *tmp = nullptr;
    CU(cudaMalloc(&tmp, sizeof(float) * (size_t)G * G));
    cudaError_t e = launch_unsplit_sym(d.Ch, d.Cl, G, c->Gp, tmp, G, c->stream);
    if (!e)
        e = cudaMemcpyAsync(C, tmp, sizeof(float) * (size_t)G * G, cudaMemcpyDeviceToHost, c->stream);
    if (!e)
        e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    CU(e);
    return 0;
}

static int get_impl(panda_ctx *c, float *W, float *P, float *C)
{
    if (int rc = check_state(c))
        return rc;
    Dev &d = c->d;
    if ((P || C) && full_matrices(c))
        return PANDA_ECUDA;
    if (W) {
        int rc = download(c, W, d.W[c->cur], c->Gp, c->T, c->G);
        if (rc)
            return rc;
    }
    struct { float *dst; const float *src; const double *diag; int n, ld; } nets[2] = {
        {P, d.Poff, d.pd, c->T, c->Tp}, {C, d.Coff, d.cd, c->G, c->Gp}};
    for (auto &n : nets) {
        if (!n.dst)
            continue;
        int rc = (n.dst == C && d.c_split) ? get_split_c(c, C) : download(c, n.dst, n.src, n.ld, n.n, n.n);
        if (rc)
            return rc;
        // diagonal entries, rounded from the FP64 diagonal
        std::vector<double> dg(n.n);
        CU(cudaMemcpyAsync(dg.data(), n.diag, n.n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
        std::vector<float> f(n.n);
        for (int i = 0; i < n.n; ++i)
            f[i] = (float)dg[i];
        CU(cudaMemcpy2DAsync(n.dst, (size_t)(n.n + 1) * sizeof(float), f.data(), sizeof(float),
                             sizeof(float), n.n, cudaMemcpyDefault, c->stream));
        CU(cudaStreamSynchronize(c->stream));  // f is released at the end of this scope
    }
    CU(cudaStreamSynchronize(c->stream));
    return 0;
}

int panda_get(panda_ctx *c, float *W, float *P, float *C)
{
    Range r("panda_get");
    if (check_ctx(c))
        return PANDA_EINVAL;
    return get_impl(c, W, P, C);
}

int panda_get_device(panda_ctx *c, float *dW, float *dP, float *dC)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    return get_impl(c, dW, dP, dC);
}

int panda_get_state(panda_ctx *c, float *W, float *P, float *C, int *t)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    int rc = get_impl(c, W, P, C);
    if (!rc && t)
        *t = c->h_ctl->iters;
    return rc;
}

int panda_set_state(panda_ctx *c, const float *W, const float *P, const float *C, int t)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (!W || !P || !C || t < 0 || t >= HIST_CAP)
        return set_err(c, PANDA_EINVAL, "W, P, C must be non-NULL and 0 <= t < 65536");
    drop_graphs(c);
    Dev &d = c->d;
    c->cur = 0;
    c->state_ok = false;  // until the new networks are in, validated and their vectors derived
    int rc;
    if ((rc = stage_c(c)))
        return rc;
    if ((rc = upload(c, d.W[0], c->Gp, W, c->T, c->G)) || (rc = upload(c, d.Poff, c->Tp, P, c->T, c->T)) ||
        (rc = upload(c, d.Coff, c->Gp, C, c->G, c->G)) || (rc = validate(c)) || (rc = derive_state(c, true))) {
        unstage_c(c);
        return rc;
    }
    if ((rc = unstage_c(c)))
        return rc;
    c->h_ctl->iters = t;
    c->h_ctl->active = 0;
    c->h_ctl->status = 0;
    if ((rc = push_ctl(c)))
        return rc;
    CU(cudaStreamSynchronize(c->stream));
    c->state_ok = true;
    return 0;
}

// ---- checkpoints -------------------------------------------------------------
namespace {
struct CkptHeader {
    char magic[8];
    int version, T, G, prec, diag, iters;
    int pad;
};

struct CkptItem {
    void *dev;
    size_t bytes;
};

std::vector<CkptItem> ckpt_items(panda_ctx *c)
{
    Dev &d = c->d;
    const size_t Tp = c->Tp, Gp = c->Gp;
    std::vector<CkptItem> v = {{d.W[c->cur], Tp * Gp * 4}, {d.Poff, Tp * Tp * 4}};
    if (d.c_split) {  // C as held: its split pair (the same 4 bytes per entry)
        v.push_back({d.Ch, Gp * Gp * 2});
        v.push_back({d.Cl, Gp * Gp * 2});
    } else {
        v.push_back({d.Coff, Gp * Gp * 4});
    }
    for (CkptItem it : {CkptItem{d.pd, Tp * 8}, CkptItem{d.cd, Gp * 8}, CkptItem{d.rsqP, Tp * 4},
                        CkptItem{d.csqC, Gp * 4}, CkptItem{d.rsqW, Tp * 4}, CkptItem{d.csqW, Gp * 4},
                        CkptItem{d.hist, (size_t)HIST_CAP * 8}})
        v.push_back(it);
    if (d.fp8) {  // the E4M3 scales and latched norm maxima, so that a resumed run continues bit for bit
        v.push_back({d.f8, 4 * sizeof(float)});
        v.push_back({d.f8n, 8 * sizeof(unsigned)});
    }
    return v;
}
}  // namespace

long long panda_checkpoint_bytes(const panda_ctx *cc)
{
    if (!cc)
        return 0;
    panda_ctx *c = const_cast<panda_ctx *>(cc);
    long long n = sizeof(CkptHeader);
    for (auto &it : ckpt_items(c))
        n += (long long)it.bytes;
    return n;
}

int panda_save(panda_ctx *c, void *buf, long long bytes)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (int rc = check_state(c))
        return rc;
    if (!buf || bytes < panda_checkpoint_bytes(c))
        return set_err(c, PANDA_EINVAL, "checkpoint buffer too small");
    CkptHeader h{};
    std::memcpy(h.magic, "PANDAGB", 8);
    h.version = 1; h.T = c->T; h.G = c->G; h.prec = c->prec; h.diag = c->diag; h.iters = c->h_ctl->iters;
    if (full_matrices(c))
        return PANDA_ECUDA;
    char *p = static_cast<char *>(buf);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    for (auto &it : ckpt_items(c)) {
        CU(cudaMemcpyAsync(p, it.dev, it.bytes, cudaMemcpyDeviceToHost, c->stream));
        p += it.bytes;
    }
    CU(cudaStreamSynchronize(c->stream));
    return 0;
}

int panda_load(panda_ctx *c, const void *buf, long long bytes)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (!buf || bytes < panda_checkpoint_bytes(c))
        return set_err(c, PANDA_EINVAL, "checkpoint buffer too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof h);
    if (std::memcmp(h.magic, "PANDAGB", 8) || h.version != 1 || h.T != c->T || h.G != c->G ||
        h.prec != c->prec || h.diag != c->diag)
        return set_err(c, PANDA_EINVAL, "checkpoint does not match this context");
    drop_graphs(c);
    c->state_ok = false;  // until every item is back
    const char *p = static_cast<const char *>(buf) + sizeof h;
    for (auto &it : ckpt_items(c)) {
        CU(cudaMemcpyAsync(it.dev, p, it.bytes, cudaMemcpyHostToDevice, c->stream));
        p += it.bytes;
    }
    Dev &d = c->d;
    if (d.Wt[c->cur])
        CU(launch_transpose(d.W[c->cur], c->Tp, c->Gp, d.Wt[c->cur], c->stream));
    CU(launch_diag_to_float(d.pd, d.pdf, c->T, c->stream));
    CU(launch_diag_to_float(d.cd, d.cdf, c->G, c->stream));
    if (tensor_prec(c->prec))
        CU(tc_prepare(d, c->stream, false));  // keep the saved E4M3 scales
    c->h_ctl->iters = h.iters;
    c->h_ctl->active = 0;
    c->h_ctl->status = 0;
    int rc = push_ctl(c);
    if (rc)
        return rc;
    CU(cudaStreamSynchronize(c->stream));
    c->state_ok = true;
    return 0;
}

int panda_get_history(panda_ctx *c, double *hh, int cap, int *n)
{
    if (check_ctx(c) || (cap > 0 && !hh))
        return PANDA_EINVAL;
    int m = c->h_ctl->iters;
    if (n)
        *n = m;
    int k = m < cap ? m : cap;
    if (k > HIST_CAP)
        k = HIST_CAP;
    if (k > 0) {
        CU(cudaMemcpyAsync(hh, c->d.hist, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return 0;
}

int panda_info(const panda_ctx *c, int *T, int *G, int *prec, int *t)
{
    if (!c)
        return PANDA_EINVAL;
    if (T) *T = c->T;
    if (G) *G = c->G;
    if (prec) *prec = c->prec;
    if (t) *t = c->h_ctl->iters;
    return 0;
}

long long panda_device_bytes(const panda_ctx *c) { return c ? c->bytes : 0; }

long long panda_device_bytes_peak(const panda_ctx *c) { return c ? c->peak : 0; }

int panda_set_profiling(panda_ctx *c, int on)
{
    if (check_ctx(c))
        return PANDA_EINVAL;
    if (c->prof != (on != 0))
        drop_graphs(c);  // graphs are captured with or without the timing events
    c->prof = on != 0;
    for (int q = 0; q < 16; ++q) {
        c->k_ms[q] = 0.0;
        c->k_launches[q] = 0;
    }
    return 0;
}

int panda_kernel_count(const panda_ctx *c) { return c ? n_kernels(c) : 0; }

int panda_selftest_timeout(void)
{
    if (!tc_supported())
        return set_err(nullptr, PANDA_EUNSUPPORTED, "panda_selftest_timeout: needs an sm_103 device");
    const int M = 128, N = 128, K = 256;
    std::vector<float> A((size_t)M * K, 1.0f), B((size_t)N * K, 1.0f), D((size_t)M * N, 0.0f);
    int status = 0;
    cudaError_t e = tc_selftest_gemm(M, N, K, A.data(), B.data(), D.data(), 1, 0, 0, &status);
    if (e != cudaSuccess)
        return set_err(nullptr, PANDA_ECUDA, std::string("panda_selftest_timeout: ") + cudaGetErrorString(e));
    if (status & ST_TIMEOUT)
        return set_err(nullptr, PANDA_ETIMEOUT, "panda_selftest_timeout: the planted wait expired as intended");
    return 0;
}

int panda_measure_ffma_peak(double *tflops)
{
    if (!tflops)
        return set_err(nullptr, PANDA_EINVAL, "panda_measure_ffma_peak: NULL output");
    cudaError_t e = measure_ffma_peak(tflops);
    if (e != cudaSuccess)
        return set_err(nullptr, PANDA_ECUDA, std::string("panda_measure_ffma_peak: ") + cudaGetErrorString(e));
    return 0;
}

int panda_selftest_tc_gemm(int M, int N, int K, const float *A, const float *B, float *D, int terms)
{
    // terms + 10: the same product on CTA pairs (cta_group::2, 256 x 256 tiles);
    // terms + 20: on CTA pairs with B stored transposed and loaded MN-major;
    // terms + 40: A and B both so; terms + 50: A only;
    // terms = 8: E4M3 operands, one term, on CTA pairs
    int pair = terms / 10;
    terms %= 10;
    if (terms == 8 && pair == 0) {
        pair = 3;
        terms = 1;
    } else if (pair == 3 || pair > 5) {
        return set_err(nullptr, PANDA_EINVAL, "panda_selftest_tc_gemm: bad argument");
    }
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !D || (terms != 1 && terms != 3))
        return set_err(nullptr, PANDA_EINVAL, "panda_selftest_tc_gemm: bad argument");
    if (!tc_supported())
        return set_err(nullptr, PANDA_EUNSUPPORTED, "panda_selftest_tc_gemm: needs an sm_103 device");
    int status = 0;
    cudaError_t e = tc_selftest_gemm(M, N, K, A, B, D, terms, pair, -1, &status);
    if (e != cudaSuccess)
        return set_err(nullptr, PANDA_ECUDA, std::string("panda_selftest_tc_gemm: ") + cudaGetErrorString(e));
    if (status & ST_TIMEOUT)
        return set_err(nullptr, PANDA_ETIMEOUT, "panda_selftest_tc_gemm: a bounded device wait expired");
    return 0;
}

int panda_kernel_stats(const panda_ctx *c, int i, char *name, int name_cap, double *total_ms,
                       long long *launches)
{
    if (!c || i < 0 || i >= n_kernels(c))
        return PANDA_EINVAL;
    if (name && name_cap > 0) {
        std::strncpy(name, kernel_name(c, i), (size_t)name_cap - 1);
        name[name_cap - 1] = 0;
    }
    if (total_ms)
        *total_ms = c->k_ms[i];
    if (launches)
        *launches = c->k_launches[i];
    return 0;
}

void *panda_stream(const panda_ctx *c) { return c ? (void *)c->stream : nullptr; }

const char *panda_last_error(const panda_ctx *c) { return c ? c->err.c_str() : g_create_error.c_str(); }

void panda_destroy(panda_ctx *c)
{
    if (!c)
        return;
    free_all(c);
    delete c;
}

// ---- sets of networks ----------------------------------------------------------
struct panda_batch {
    std::vector<panda_ctx *> nets;
    std::string err;
    // tensor-core modes: the set engine (one launch per phase for all networks)
    TcSet *set = nullptr;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_iters = 8;
    Ctl *h_ctls = nullptr;               // pinned: every network's control block after a chunk
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    // schedule autotuning: one warm-up iteration, then TUNE_REPS iterations per phase-1
    // candidate (phase-1 time), then per phase-2 candidate (phase-2 time); medians decide
    static constexpr int TUNE_REPS = 3;
    int tune_step = 0;                   // trial iterations run so far
    int p1 = 0, p2 = 0;                  // the schedules in use
    float p1_ms[TC_P1_CANDS][TUNE_REPS] = {}, p2_ms[TC_P2_CANDS][TUNE_REPS] = {};
    float p1_med[TC_P1_CANDS] = {}, p2_med[TC_P2_CANDS] = {};
    static constexpr int TUNE_STEPS = 1 + (TC_P1_CANDS + TC_P2_CANDS) * TUNE_REPS;
};

namespace {
void batch_free_set(panda_batch *b)
{
    if (b->gexec)
        cudaGraphExecDestroy(b->gexec);
    tc_set_destroy(b->set);
    if (b->h_ctls)
        cudaFreeHost(b->h_ctls);
    for (cudaEvent_t &e : b->ev)
        if (e)
            cudaEventDestroy(e);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    b->set = nullptr;
    b->gexec = nullptr;
    b->h_ctls = nullptr;
    b->stream = nullptr;
}

// The set engine's graph: graph_iters iterations of every network, the chosen schedule.
int batch_graph(panda_batch *b)
{
    if (b->gexec)
        return 0;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    for (int k = 0; k < b->graph_iters && !e; ++k)
        e = tc_set_launch(b->set, b->p1, b->p2, b->stream, nullptr, nullptr, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (!e)
        e = e2;
    if (!e)
        e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (g)
        cudaGraphDestroy(g);
    if (e) {
        b->gexec = nullptr;
        b->err = std::string("set graph: ") + cudaGetErrorString(e);
        return PANDA_ECUDA;
    }
    return 0;
}

float median3(const float (&v)[panda_batch::TUNE_REPS])
{
    float a[panda_batch::TUNE_REPS];
    std::copy(v, v + panda_batch::TUNE_REPS, a);
    std::sort(a, a + panda_batch::TUNE_REPS);
    return a[panda_batch::TUNE_REPS / 2];
}

// One chunk of the set engine: while the schedule autotuning is unfinished, a
// single iteration with the next trial's schedules, its phases timed by CUDA
// events (the warm-up first, then TUNE_REPS iterations of each phase-1
// candidate with the default phase 2, the fastest by median kept, then of each
// phase-2 candidate); afterwards the captured graph with the chosen pair.
// Every schedule gives the same results.  Then all control blocks are read back.
int batch_chunk(panda_batch *b)
{
    cudaError_t e;
    constexpr int R = panda_batch::TUNE_REPS;
    const int step = b->tune_step;
    const bool tuning = step < panda_batch::TUNE_STEPS;
    int which = -1, cand = -1;  // phase being tried (1 or 2) and its candidate
    if (tuning) {
        int p1 = b->p1, p2 = b->p2;
        if (step >= 1 && step < 1 + TC_P1_CANDS * R) {
            which = 1, cand = (step - 1) / R, p1 = cand;
        } else if (step >= 1 + TC_P1_CANDS * R) {
            which = 2, cand = (step - 1 - TC_P1_CANDS * R) / R, p2 = cand;
        }
        if ((e = tc_set_launch(b->set, p1, p2, b->stream, b->ev[0], b->ev[1], b->ev[2])))
            return b->err = std::string("set launch: ") + cudaGetErrorString(e), PANDA_ECUDA;
    } else {
        int rc = batch_graph(b);
        if (rc)
            return rc;
        if ((e = cudaGraphLaunch(b->gexec, b->stream)))
            return b->err = std::string("set graph launch: ") + cudaGetErrorString(e), PANDA_ECUDA;
    }
    if ((e = tc_set_gather(b->set, b->h_ctls, b->stream)) || (e = cudaStreamSynchronize(b->stream)))
        return b->err = std::string("set chunk: ") + cudaGetErrorString(e), PANDA_ECUDA;
    if (tuning) {
        b->tune_step++;
        float ms = 0.0f;
        if (which > 0 && (e = cudaEventElapsedTime(&ms, b->ev[which - 1], b->ev[which])))
            return b->err = std::string("set timing: ") + cudaGetErrorString(e), PANDA_ECUDA;
        const int rep = (step - 1) % R;
        if (which == 1) {
            b->p1_ms[cand][rep] = ms;
            if (rep == R - 1)
                b->p1_med[cand] = median3(b->p1_ms[cand]);
            if (step == TC_P1_CANDS * R)  // the last phase-1 trial: keep the fastest
                b->p1 = (int)(std::min_element(b->p1_med, b->p1_med + TC_P1_CANDS) - b->p1_med);
        } else if (which == 2) {
            b->p2_ms[cand][rep] = ms;
            if (rep == R - 1)
                b->p2_med[cand] = median3(b->p2_ms[cand]);
            if (step == panda_batch::TUNE_STEPS - 1)
                b->p2 = (int)(std::min_element(b->p2_med, b->p2_med + TC_P2_CANDS) - b->p2_med);
        }
    }
    return 0;
}

int batch_run_set(panda_batch *b, float alpha, double tol, int max_iter, int *iters_out, double *h_last)
{
    const size_t n = b->nets.size();
    std::vector<DriveState> ds(n);
    std::vector<int> parity(n);
    for (size_t k = 0; k < n; ++k) {  // arm every control block, as a single run does
        panda_ctx *c = b->nets[k];
        int rc = drive_begin(c, alpha, tol, max_iter, false, ds[k]);
        if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess)
            rc = set_err(c, PANDA_ECUDA, "stream synchronize failed");
        if (rc) {
            b->err = "network " + std::to_string(k) + ": " + c->err;
            return rc;
        }
        parity[k] = (c->cur - ds[k].start) & 1;
    }
    cudaError_t e = tc_set_parity(b->set, parity, b->stream);
    if (e)
        return b->err = std::string("set parity: ") + cudaGetErrorString(e), PANDA_ECUDA;
    bool any = max_iter > 0;
    int rc = 0;
    while (any && !rc) {
        if ((rc = batch_chunk(b)))
            break;
        any = false;
        for (size_t k = 0; k < n; ++k)
            any = any || b->h_ctls[k].active;
    }
    if (rc) {
        cudaStreamSynchronize(b->stream);
        return rc;
    }
    bool all = true;
    for (size_t k = 0; k < n; ++k) {
        panda_ctx *c = b->nets[k];
        if (max_iter > 0)
            *c->h_ctl = b->h_ctls[k];
        const Ctl &h = *c->h_ctl;
        c->cur ^= ((h.iters - ds[k].start) & 1);
        if (h.status & ST_NONFINITE)
            rc = set_err(c, PANDA_ENONFINITE, "the state became non-finite");
        else if (h.status & ST_TIMEOUT)
            rc = set_err(c, PANDA_ETIMEOUT, "a bounded device wait expired");
        if (rc) {
            b->err = "network " + std::to_string(k) + ": " + c->err;
            return rc;
        }
        if (iters_out)
            iters_out[k] = h.iters - ds[k].start;
        if (h_last)
            h_last[k] = h.h_last;
        all = all && h.converged;
    }
    return all ? PANDA_OK : PANDA_NOT_CONVERGED;
}
}  // namespace

int panda_batch_create(panda_batch **out, int n, const int *T, const int *G, const float *const *W0,
                       const float *const *P0, const float *const *C0, const panda_opts *o)
{
    if (!out)
        return set_err(nullptr, PANDA_EINVAL, "out is NULL");
    *out = nullptr;
    if (n <= 0 || !T || !G || !W0 || !P0 || !C0)
        return set_err(nullptr, PANDA_EINVAL, "panda_batch_create: n > 0 and non-NULL arrays required");
    panda_batch *b = new panda_batch();
    for (int k = 0; k < n; ++k) {
        panda_ctx *c = nullptr;
        int rc = create_common(&c, T[k], G[k], W0[k], P0[k], C0[k], o, nullptr, false);
        if (rc) {
            std::string msg = "network " + std::to_string(k) + ": " + g_create_error;
            for (panda_ctx *x : b->nets)
                panda_destroy(x);
            delete b;
            return set_err(nullptr, rc, msg);
        }
        b->nets.push_back(c);
    }
    if (tensor_prec(b->nets[0]->prec)) {  // the set engine
        std::vector<const Dev *> ds;
        for (panda_ctx *c : b->nets)
            ds.push_back(&c->d);
        b->graph_iters = b->nets[0]->graph_iters > 0 ? b->nets[0]->graph_iters : 2;
        cudaError_t e = tc_set_create(ds, &b->set);
        if (!e)
            e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (!e)
            e = cudaMallocHost(&b->h_ctls, n * sizeof(Ctl));
        for (int q = 0; q < 3 && !e; ++q)
            e = cudaEventCreate(&b->ev[q]);
        if (e) {
            std::string msg = std::string("panda_batch_create: set engine: ") + cudaGetErrorString(e);
            batch_free_set(b);
            for (panda_ctx *x : b->nets)
                panda_destroy(x);
            delete b;
            return set_err(nullptr, PANDA_ECUDA, msg);
        }
    }
    *out = b;
    return 0;
}

int panda_batch_run(panda_batch *b, float alpha, double tol, int max_iter, int *iters_out, double *h_last)
{
    Range r("panda_batch_run");
    if (!b)
        return PANDA_EINVAL;
    if (!(alpha >= 0.0f && alpha <= 1.0f) || !(tol >= 0.0) || max_iter < 0) {
        b->err = "alpha must be in [0, 1], tol >= 0 and max_iter >= 0";
        return PANDA_EINVAL;
    }
    for (size_t k = 0; k < b->nets.size(); ++k)
        if (int rc = check_state(b->nets[k])) {
            b->err = "network " + std::to_string(k) + ": " + b->nets[k]->err;
            return rc;
        }
    if (b->set)
        return batch_run_set(b, alpha, tol, max_iter, iters_out, h_last);
    const size_t n = b->nets.size();
    std::vector<DriveState> ds(n);
    std::vector<char> more(n, max_iter > 0 ? 1 : 0);
    int rc = 0;
    for (size_t k = 0; k < n && !rc; ++k) {
        panda_ctx *c = b->nets[k];
        if ((rc = drive_begin(c, alpha, tol, max_iter, c->graph_iters > 0, ds[k])))
            b->err = "network " + std::to_string(k) + ": " + c->err;
    }
    bool any = max_iter > 0;
    while (!rc && any) {
        for (size_t k = 0; k < n && !rc; ++k)  // every active network queues a chunk on its own stream
            if (more[k] && (rc = drive_launch(b->nets[k], ds[k])))
                b->err = "network " + std::to_string(k) + ": " + b->nets[k]->err;
        any = false;
        for (size_t k = 0; k < n && !rc; ++k) {
            if (!more[k])
                continue;
            bool m = false;
            if ((rc = drive_collect(b->nets[k], ds[k], &m)))
                b->err = "network " + std::to_string(k) + ": " + b->nets[k]->err;
            more[k] = m;
            any = any || m;
        }
    }
    if (rc) {  // leave every stream idle before reporting
        for (panda_ctx *c : b->nets)
            cudaStreamSynchronize(c->stream);
        return rc;
    }
    bool all = true;
    for (size_t k = 0; k < n; ++k) {
        const Ctl &h = *b->nets[k]->h_ctl;
        if (iters_out)
            iters_out[k] = h.iters - ds[k].start;
        if (h_last)
            h_last[k] = h.h_last;
        all = all && h.converged;
    }
    return all ? PANDA_OK : PANDA_NOT_CONVERGED;
}

int panda_batch_get(panda_batch *b, int k, float *W, float *P, float *C)
{
    if (!b || k < 0 || k >= (int)b->nets.size())
        return PANDA_EINVAL;
    int rc = get_impl(b->nets[k], W, P, C);
    if (rc)
        b->err = b->nets[k]->err;
    return rc;
}

int panda_batch_size(const panda_batch *b) { return b ? (int)b->nets.size() : 0; }

panda_ctx *panda_batch_context(panda_batch *b, int k)
{
    if (!b || k < 0 || k >= (int)b->nets.size())
        return nullptr;
    return b->nets[k];
}

int panda_batch_schedule(const panda_batch *b, int *p1, int *p2, float *p1_ms, int n1, float *p2_ms, int n2,
                         int *done)
{
    if (!b)
        return PANDA_EINVAL;
    if (!b->set)
        return 0;
    if (p1)
        *p1 = b->p1;
    if (p2)
        *p2 = b->p2;
    for (int q = 0; p1_ms && q < n1 && q < TC_P1_CANDS; ++q)
        p1_ms[q] = b->p1_med[q];
    for (int q = 0; p2_ms && q < n2 && q < TC_P2_CANDS; ++q)
        p2_ms[q] = b->p2_med[q];
    if (done)
        *done = b->tune_step >= panda_batch::TUNE_STEPS;
    return 1;
}

const char *panda_batch_schedule_name(int phase, int k)
{
    if (phase == 1 && k >= 0 && k < TC_P1_CANDS)
        return TC_P1_NAMES[k];
    if (phase == 2 && k >= 0 && k < TC_P2_CANDS)
        return TC_P2_NAMES[k];
    return nullptr;
}

int panda_phase1_layout(const panda_ctx *c, int *pairs, int *clusters, int *cuts)
{
    if (!c || !tensor_prec(c->prec))
        return set_err(nullptr, PANDA_EINVAL, "panda_phase1_layout: no tensor-core context");
    int p = 0, k = 0;
    const int n = tc_phase1_layout(c->d, &p, &k);
    if (n < 0)
        return set_err(nullptr, PANDA_EINVAL, "panda_phase1_layout: the context is not prepared");
    if (pairs)
        *pairs = p;
    if (clusters)
        *clusters = k;
    if (cuts)
        *cuts = n;
    return 0;
}

int panda_phase1_plan(int T, int G, int prec, int pairs, int all_resident, int *pieces, int cap, int *n_pieces)
{
    if (T < 1 || G < 1 || !tensor_prec(prec) || pairs < 1 || !n_pieces || (cap > 0 && !pieces))
        return set_err(nullptr, PANDA_EINVAL, "panda_phase1_plan: bad argument");
    Dev d{};
    d.T = T; d.G = G;
    d.Tp = round_up(T, 2 * TILE); d.Gp = round_up(G, 2 * TILE);
    d.split_b = prec == PANDA_BF16X2 ? 0 : 1;
    d.fp8 = prec == PANDA_FP8MIX ? 1 : 0;
    std::vector<int> off;
    std::vector<int4> items;
    const int cuts = tc_phase1_plan(d, pairs, all_resident != 0, off, items);
    *n_pieces = (int)items.size();
    int k = 0;
    for (int p = 0; p + 1 < (int)off.size(); ++p)
        for (int q = off[p]; q < off[p + 1]; ++q, ++k)
            if (k < cap) {
                const int4 w = items[q];
                int *o = pieces + 6 * (size_t)k;
                o[0] = p; o[1] = w.x; o[2] = w.y; o[3] = w.z & 0xffff; o[4] = w.z >> 16; o[5] = w.w;
            }
    return cuts;
}

const char *panda_batch_last_error(const panda_batch *b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void panda_batch_destroy(panda_batch *b)
{
    if (!b)
        return;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    batch_free_set(b);
    for (panda_ctx *c : b->nets)
        panda_destroy(c);
    delete b;
}

}  // extern "C"
