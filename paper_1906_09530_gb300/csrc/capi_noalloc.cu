// capi_noalloc.cu -- lbm_diag_noalloc: the diagnostics of lbm_diag with the
// reduction's per-block partial sums kept in a fixed array that is part of the
// library's device image, so that the call itself allocates nothing.
//
// Callers that cannot call cudaMalloc (code running under an allocator that
// owns all device memory, or a host environment whose policy forbids device
// allocations after start-up) can still take the run's diagnostics: they pass
// the context (whose workspace they obtained from their own pool) and host
// outputs, and nothing is allocated here.  Like lbm_diag, the call copies its
// four results to the host and waits for the context's stream before it
// returns.  So no call can be captured into a CUDA graph, and none may be made
// while the context's stream is capturing.
//
// The array g_diag_partials is a file-scope __device__ variable: every GPU that
// loads the library holds its 512 KB until the process exits.  In host code its
// name is only a host-side stand-in, so the device address is taken once per
// device with cudaGetSymbolAddress (with that device current) and passed to the
// kernels.  That set-up happens on the first call on each device; make that
// first call before any stream capture.  All calls share the array and it keeps
// the last call's contents: every slot a call reads is written by the same call
// first, so nothing needs clearing, but calls that overlap on the GPU (several
// streams or threads at once) race on it.
#include <cstring>
#include <mutex>

#include "cplbm_internal.cuh"

namespace {

// One partial record (4 doubles) per block of 256 threads, each block covering
// kNodesPerBlock nodes; at most kMaxParts records, i.e. grids up to
// kMaxParts * kNodesPerBlock = 33,554,432 nodes.
constexpr int kNodesPerBlock = 2048;
constexpr int kMaxParts = 16384;

__device__ __align__(256) double g_diag_partials[4 * kMaxParts];

constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

cudaError_t partials_on_device(int dev, double** out) {
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_diag_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = static_cast<double*>(p);
    }
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

// Defined in capi.cu: the shared body of lbm_diag with caller-chosen partials.
lbm_status cplbm_diag_with_partials(lbm_ctx* c, double* partials, int nparts, double* mass,
                                    double* max_v, double* rho_min, double* rho_max);
int cplbm_ctx_device(const lbm_ctx* c);
size_t cplbm_ctx_nodes(const lbm_ctx* c);

extern "C" lbm_status lbm_diag_noalloc(lbm_ctx* ctx, double* mass, double* max_v,
                                       double* rho_min, double* rho_max) {
    if (!ctx) return LBM_EINVAL;
    const size_t N = cplbm_ctx_nodes(ctx);
    const size_t parts = (N + kNodesPerBlock - 1) / kNodesPerBlock;
    if (parts > (size_t)kMaxParts) return LBM_EINVAL;  // grid above 33,554,432 nodes
    const int dev = cplbm_ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return LBM_ECUDA;
    double* partials = nullptr;
    if (partials_on_device(dev, &partials) != cudaSuccess) return LBM_ECUDA;
    return cplbm_diag_with_partials(ctx, partials, (int)parts, mass, max_v, rho_min, rho_max);
}
