// panda_step_static: one message-passing iteration on caller-owned device
// networks that allocates no device memory at all.
//
// Some callers cannot call cudaMalloc: code that must run within a fixed
// device-memory budget handed out by a host framework's own allocator or
// pool, plug-ins loaded into a process that forbids allocation once it is
// running, or latency-critical loops where a cudaMalloc (an implicit device
// synchronisation) is not acceptable.  For them this entry point takes its
// working memory from one file-scope device array of fixed size instead.
//
// The array is `g_scratch` below: STATIC_BYTES bytes (about 7.4 MB), sized
// for networks of at most PANDA_STATIC_MAX_NODES TFs and genes.  Every GPU
// that loads the library's device code holds it until the process exits (with
// CUDA's lazy module loading that happens at the first call on the device, so
// a caller with a fixed budget makes that call at start-up).  In host code its
// name only stands for the device array; the device address is looked up once
// per device with cudaGetSymbolAddress, with that device current, on the
// first call made on it.  All calls share the array and each call clears it
// first, so two calls that overlap on the GPU (for example on two streams)
// race with each other.
//
// The iteration itself is the FP32 SIMT path of panda_step (the same kernels,
// so the same results), run on a copy of the caller's networks laid out in
// the array.
#include "panda.h"
#include "panda_internal.cuh"

#include <cmath>
#include <mutex>
#include <string>

namespace panda {

// Sets the message panda_last_error(NULL) returns (defined in panda_api.cu).
void set_global_error(const std::string &msg);

namespace {

constexpr int SMAX = PANDA_STATIC_MAX_NODES;  // a multiple of TILE
constexpr int SNB = SMAX / TILE;
constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t SQ = al256(sizeof(float) * SMAX * SMAX);  // one padded square matrix
constexpr size_t VF = al256(sizeof(float) * SMAX);
constexpr size_t VD = al256(sizeof(double) * SMAX);
constexpr size_t PART = al256(sizeof(float) * SNB * SMAX);
constexpr size_t STATIC_BYTES = 7 * SQ                  // W[2], Wt[2], Poff, Coff, Rn
                                + 2 * VD + 6 * VF       // pd, cd; pdf, cdf, rsqP, csqC, rsqW, csqW
                                + 8 * PART              // wrow, wcol, ps_sum/sq/vsq, cs_sum/sq/vsq
                                + al256(sizeof(double) * SNB * SNB)  // hpart
                                + al256(sizeof(Ctl)) + 2 * al256(2 * sizeof(double))  // ctl, hist, e2tab
                                + al256(4 * sizeof(int));            // validation flags

__device__ __align__(256) unsigned char g_scratch[STATIC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char *g_addr[MAX_DEVICES] = {};

// Device address of g_scratch on the current device (looked up once).
cudaError_t scratch_address(int dev, unsigned char **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess)
            return e;
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

__global__ void k_put_diag(float *X, int n, int ld, const double *d)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        X[(size_t)i * ld + i] = (float)d[i];
}

int fail(int code, const std::string &msg)
{
    set_global_error(msg);
    return code;
}

}  // namespace
}  // namespace panda

using namespace panda;

#define SCU(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(PANDA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

extern "C" int panda_step_static(int T, int G, float *dW, float *dP, float *dC, float alpha, int t,
                                 int diag, double *h_out, void *stream)
{
    if (T < 1 || G < 1 || T > SMAX || G > SMAX)
        return fail(PANDA_EINVAL, "panda_step_static: T and G must be in [1, " +
                                      std::to_string(SMAX) + "] (the size of its static scratch)");
    if (!dW || !dP || !dC)
        return fail(PANDA_EINVAL, "panda_step_static: W, P and C must not be NULL");
    if (!(alpha >= 0.0f && alpha <= 1.0f) || t < 1 || diag < 0 || diag > 2)
        return fail(PANDA_EINVAL, "panda_step_static: need alpha in [0, 1], t >= 1, diag in 0..2");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    SCU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES)
        return fail(PANDA_EUNSUPPORTED, "panda_step_static: device index out of range");
    unsigned char *base = nullptr;
    SCU(scratch_address(dev, &base));

    // carve the array (every region sized for the maximum network)
    Dev d{};
    d.T = T; d.G = G;
    d.Tp = round_up(T, TILE); d.Gp = round_up(G, TILE);
    d.nbT = d.Tp / TILE; d.nbG = d.Gp / TILE;
    d.diag = diag;
    unsigned char *p = base;
    auto take = [&p](size_t bytes) { unsigned char *q = p; p += bytes; return q; };
    for (int b = 0; b < 2; ++b) {
        d.W[b] = (float *)take(SQ);
        d.Wt[b] = (float *)take(SQ);
    }
    d.Poff = (float *)take(SQ);
    d.Coff = (float *)take(SQ);
    d.Rn = (float *)take(SQ);
    d.pd = (double *)take(VD);
    d.cd = (double *)take(VD);
    d.pdf = (float *)take(VF);
    d.cdf = (float *)take(VF);
    d.rsqP = (float *)take(VF);
    d.csqC = (float *)take(VF);
    d.rsqW = (float *)take(VF);
    d.csqW = (float *)take(VF);
    d.wrow_part = (float *)take(PART);
    d.wcol_part = (float *)take(PART);
    d.ps_sum = (float *)take(PART);
    d.ps_sq = (float *)take(PART);
    d.ps_vsq = (float *)take(PART);
    d.cs_sum = (float *)take(PART);
    d.cs_sq = (float *)take(PART);
    d.cs_vsq = (float *)take(PART);
    d.hpart = (double *)take(al256(sizeof(double) * SNB * SNB));
    d.ctl = (Ctl *)take(al256(sizeof(Ctl)));
    d.hist = (double *)take(al256(2 * sizeof(double)));
    d.e2tab = (double *)take(al256(2 * sizeof(double)));
    int *flags = (int *)take(al256(4 * sizeof(int)));

    // zero everything: padding, partial sums, flags
    SCU(cudaMemsetAsync(base, 0, STATIC_BYTES, s));
    SCU(cudaMemcpy2DAsync(d.W[0], (size_t)d.Gp * 4, dW, (size_t)G * 4, (size_t)G * 4, T,
                          cudaMemcpyDeviceToDevice, s));
    SCU(cudaMemcpy2DAsync(d.Poff, (size_t)d.Tp * 4, dP, (size_t)T * 4, (size_t)T * 4, T,
                          cudaMemcpyDeviceToDevice, s));
    SCU(cudaMemcpy2DAsync(d.Coff, (size_t)d.Gp * 4, dC, (size_t)G * 4, (size_t)G * 4, G,
                          cudaMemcpyDeviceToDevice, s));
    SCU(launch_check_finite_sym(d.W[0], T, G, d.Gp, false, flags, s));
    SCU(launch_check_finite_sym(d.Poff, T, T, d.Tp, true, flags, s));
    SCU(launch_check_finite_sym(d.Coff, G, G, d.Gp, true, flags, s));
    int hflags[4] = {0, 0, 0, 0};
    SCU(cudaMemcpyAsync(hflags, flags, sizeof hflags, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    if (hflags[0])
        return fail(PANDA_ENONFINITE, "panda_step_static: a network has a non-finite entry");
    if (hflags[1])
        return fail(PANDA_EASYM, "panda_step_static: P or C is not exactly symmetric");

    // derived state, exactly as a context builds it
    SCU(launch_split_diag(d.Poff, T, d.Tp, d.pd, d.pdf, s));
    SCU(launch_split_diag(d.Coff, G, d.Gp, d.cd, d.cdf, s));
    SCU(launch_transpose(d.W[0], d.Tp, d.Gp, d.Wt[0], s));
    SCU(launch_row_norms(d.W[0], T, G, d.Gp, nullptr, d.rsqW, s));
    SCU(launch_row_norms(d.Wt[0], G, T, d.Tp, nullptr, d.csqW, s));  // columns of W
    SCU(launch_row_norms(d.Poff, T, T, d.Tp, d.pd, d.rsqP, s));
    SCU(launch_row_norms(d.Coff, G, G, d.Gp, d.cd, d.csqC, s));

    // one iteration at index t: counter 0, growth factor e^{2 alpha t} in slot 1
    Ctl hc{};
    hc.active = 1;
    hc.iters = 0;
    hc.stop_at = 1;
    hc.alpha = alpha;
    hc.tol = -1.0;
    const double e2[2] = {1.0, std::exp(2.0 * (double)alpha * (double)t)};
    SCU(cudaMemcpyAsync(d.ctl, &hc, sizeof hc, cudaMemcpyHostToDevice, s));
    SCU(cudaMemcpyAsync(d.e2tab, e2, sizeof e2, cudaMemcpyHostToDevice, s));
    KernelEvents ke{nullptr, 0};
    SCU(launch_iteration_simt(d, 0, s, ke));
    SCU(cudaMemcpyAsync(&hc, d.ctl, sizeof hc, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    // a failed iteration leaves the caller's networks as they were
    if (hc.status & ST_NONFINITE)
        return fail(PANDA_ENONFINITE, "panda_step_static: the networks became non-finite (left unchanged)");

    // results back into the caller's buffers, diagonals from the FP64 vectors
    SCU(cudaMemcpy2DAsync(dW, (size_t)G * 4, d.W[1], (size_t)d.Gp * 4, (size_t)G * 4, T,
                          cudaMemcpyDeviceToDevice, s));
    SCU(cudaMemcpy2DAsync(dP, (size_t)T * 4, d.Poff, (size_t)d.Tp * 4, (size_t)T * 4, T,
                          cudaMemcpyDeviceToDevice, s));
    SCU(cudaMemcpy2DAsync(dC, (size_t)G * 4, d.Coff, (size_t)d.Gp * 4, (size_t)G * 4, G,
                          cudaMemcpyDeviceToDevice, s));
    k_put_diag<<<ceil_div(T, 256), 256, 0, s>>>(dP, T, T, d.pd);
    k_put_diag<<<ceil_div(G, 256), 256, 0, s>>>(dC, G, G, d.cd);
    SCU(cudaGetLastError());
    SCU(cudaStreamSynchronize(s));
    if (h_out)
        *h_out = hc.h_last;
    return PANDA_OK;
}
