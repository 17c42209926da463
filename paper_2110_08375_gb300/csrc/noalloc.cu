// mdls_backsub_noalloc: the tiled back substitution with its scratch in a
// fixed device array of this library instead of a caller workspace.
//
// Some callers cannot allocate device memory when they call us: a plugin
// inside a host framework that owns all device memory through its own
// allocator, a real-time or embedded loop whose memory budget is fixed at
// start-up, or code that must not risk the implicit device synchronisation a
// cudaMalloc can cause.  For them this entry point takes only inputs and
// outputs.  Its scratch (status word, inverted diagonal tiles, working right-
// hand side) is the file-scope array below; every GPU that loads the library
// keeps it (MDLS_BACKSUB_NOALLOC_MAX_BYTES) until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mdls.h"
#include "layout.h"

namespace mdls {
int bs_entry_p2(int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*, int64_t,
                int, void*, cudaStream_t);
int bs_entry_p4(int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*, int64_t,
                int, void*, cudaStream_t);
int bs_entry_p8(int64_t, const double*, int64_t, int64_t, const double*, int64_t, double*, int64_t,
                int, void*, cudaStream_t);
}  // namespace mdls

namespace {

// The shared scratch.  In host code this name is only a stand-in for the
// device symbol, never a device address: the address comes from
// cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_backsub_scratch[MDLS_BACKSUB_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Set-up, once per device, with that device current.
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MDLS_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (g_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_backsub_scratch) != cudaSuccess || p == nullptr)
            return MDLS_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MDLS_OK;
}

}  // namespace

extern "C" int mdls_backsub_noalloc(int prec, int64_t n, const double* R, int64_t ldr, int64_t psr,
                                    const double* y, int64_t psy, double* x, int64_t psx, int tile,
                                    int* status, void* stream) {
    if (prec != 2 && prec != 4 && prec != 8) return MDLS_ERR_PREC;
    if (!R || !y || !x || n < 1 || ldr < n || psr < ldr * n || psy < n || psx < n)
        return MDLS_ERR_ARG;
    const int t = mdls::norm_tile_bs(tile, n, prec);
    if (t < 1) return MDLS_ERR_ARG;
    const size_t need = mdls_backsub_workspace(prec, n, tile);
    if (need == 0 || need > (size_t)MDLS_BACKSUB_NOALLOC_MAX_BYTES) return MDLS_ERR_WORKSPACE;
    void* ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc != MDLS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the status word at the start of the scratch is cleared by the call itself
    switch (prec) {
        case 2: rc = mdls::bs_entry_p2(n, R, ldr, psr, y, psy, x, psx, t, ws, st); break;
        case 4: rc = mdls::bs_entry_p4(n, R, ldr, psr, y, psy, x, psx, t, ws, st); break;
        default: rc = mdls::bs_entry_p8(n, R, ldr, psr, y, psy, x, psx, t, ws, st); break;
    }
    if (rc != MDLS_OK) return rc;
    if (status && cudaMemcpyAsync(status, ws, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return MDLS_ERR_CUDA;
    return MDLS_OK;
}
