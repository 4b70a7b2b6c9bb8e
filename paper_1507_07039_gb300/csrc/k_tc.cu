// Tensor-core (tcgen05) path: placeholder until the BF16X3 kernels land.
#include "panda_internal.cuh"

namespace panda {

const char *const TC_KERNEL_NAMES[TC_KERNELS] = {"", "", "", "", "", ""};
bool tc_supported() { return false; }
cudaError_t tc_prepare(Dev &, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_iteration_tc(const Dev &, int, cudaStream_t, KernelEvents &) { return cudaErrorNotSupported; }

}  // namespace panda
