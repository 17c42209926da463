// mdls_wait_check: a diagnostic of the bounded device waits that the
// Householder panel uses between its column blocks (failure detection).  It
// runs the same wait_flag as the panel, with a limit the caller chooses, on a
// flag that is published or never published, so a caller (or a test) can see
// the wait give up with MDLS_ERR_TIMEOUT and leave the GPU usable.
#include <cuda_runtime.h>

#include "../../include/mdls.h"
#include "kernels.cuh"

namespace {
__global__ void header_init_kernel(mdls::WsHeader* h, unsigned long long wait_ns) {
    if (threadIdx.x == 0 && blockIdx.x == 0) h->wait_ns = wait_ns;
}
}  // namespace

extern "C" int mdls_wait_check(void* ws, size_t ws_bytes, uint64_t limit_ns, int publish, void* stream) {
    if (!ws || ws_bytes < MDLS_WAIT_CHECK_WORKSPACE || (reinterpret_cast<uintptr_t>(ws) & 255) != 0)
        return MDLS_ERR_WORKSPACE;
    if (limit_ns < 1000 || limit_ns > 10000000000ull || (publish != 0 && publish != 1)) return MDLS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(ws);
    auto* h = reinterpret_cast<mdls::WsHeader*>(w);
    auto* flag = reinterpret_cast<unsigned int*>(w + 256);
    if (cudaMemsetAsync(w, 0, MDLS_WAIT_CHECK_WORKSPACE, st) != cudaSuccess) return MDLS_ERR_CUDA;
    header_init_kernel<<<1, 32, 0, st>>>(h, (unsigned long long)limit_ns);
    if (cudaGetLastError() != cudaSuccess) return MDLS_ERR_CUDA;
    void* args[] = {&flag, &h, &publish};
    if (cudaLaunchCooperativeKernel((const void*)mdls::wait_check_kernel, dim3(2), dim3(32), args, 0, st) !=
        cudaSuccess)
        return MDLS_ERR_CUDA;
    return MDLS_OK;
}
