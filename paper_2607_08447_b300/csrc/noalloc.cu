// Allocation-free variant of the Hellmann-Feynman backward.
//
// khp_eigs_backward reduces the gate-lever gradient dL/dalpha_g through a
// scratch array of per-block partial sums that it allocates on the stream
// for every call.  Some callers cannot allow that: a process that has handed
// the whole device to a pooling allocator (cudaMalloc would fail or fragment
// the pool), code on a latency-critical path where an allocation or free may
// synchronise the device, or an embedding that forbids the library from
// owning device memory between calls.  khp_eigs_backward_noalloc gives them
// the same computation with its scratch in one fixed, file-scope device
// array, so the call itself never allocates or frees.
//
// The array holds KHP_NOALLOC_BLOCKS x KHP_MAX_GATES partial sums plus the
// KHP_MAX_GATES results (38 KB of doubles).  Every GPU that loads the
// library keeps it until the process exits.  All calls share it: two calls
// whose kernels overlap on the GPU (different streams, or different host
// threads without ordering) race on it.  Each call overwrites every entry
// it reads, so nothing has to be cleared between calls.
#include <cmath>
#include <mutex>
#include <string>

#include "khp_common.cuh"
#include "khp_internal.h"

#define KHP_NOALLOC_BLOCKS 296
#define KHP_NOALLOC_DEVICES 64

static __device__ __align__(256) double khp_noalloc_scratch[KHP_NOALLOC_BLOCKS * KHP_MAX_GATES + KHP_MAX_GATES];

namespace {

std::mutex g_mu;
double* g_scratch[KHP_NOALLOC_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
cudaError_t scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, khp_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" khp_status khp_eigs_backward_noalloc(khp_handle g, const void* evecs_dev, const double* evals_host,
                                                int n, const double* dLdE_host, double* dLdV_dev,
                                                double* dLdstrain_dev, const double* levers_dev, int n_gates,
                                                double* dLdalpha_host) {
    using namespace khp;
    khp_clear_error();
    if (!g) return khp_set_error(KHP_ERR_INVALID_ARG, "handle is NULL");
    if (!evecs_dev || !evals_host || !dLdE_host || !dLdV_dev)
        return khp_set_error(KHP_ERR_INVALID_ARG, "NULL argument");
    if (n < 1 || n > KHP_MAX_M) return khp_set_error(KHP_ERR_INVALID_ARG, "n out of range 1..64");
    if (n_gates < 0 || n_gates > KHP_MAX_GATES)
        return khp_set_error(KHP_ERR_INVALID_ARG,
                             "n_gates exceeds the fixed scratch of khp_eigs_backward_noalloc (max 16)");
    if (n_gates > 0 && (!levers_dev || !dLdalpha_host))
        return khp_set_error(KHP_ERR_INVALID_ARG, "levers/alpha output NULL");
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(dLdE_host[i]) || !std::isfinite(evals_host[i]))
            return khp_set_error(KHP_ERR_INVALID_ARG, "non-finite input");
    for (int i = 0; i < n;) {
        int j = i + 1;
        while (j < n && evals_host[j] - evals_host[j - 1] <= 1e-6) ++j;
        for (int k = i + 1; k < j; ++k) {
            const double d = dLdE_host[k] - dLdE_host[i];
            const double s = dLdE_host[i] < 0 ? -dLdE_host[i] : dLdE_host[i];
            if ((d < 0 ? -d : d) > 1e-12 * (s > 1.0 ? s : 1.0))
                return khp_set_error(KHP_ERR_DEGENERATE, "dL/dE differs inside a degenerate cluster");
        }
        i = j;
    }
    if (g->device < 0 || g->device >= KHP_NOALLOC_DEVICES)
        return khp_set_error(KHP_ERR_INVALID_ARG, "device index beyond the scratch table");
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return khp_set_error(KHP_ERR_CUDA, "cudaGetDevice failed");
    if (prev != g->device && cudaSetDevice(g->device) != cudaSuccess)
        return khp_set_error(KHP_ERR_CUDA, "cudaSetDevice failed");
    double* scratch = nullptr;
    cudaError_t e = scratch_address(g->device, &scratch);
    if (e == cudaSuccess) {
        double* partial = scratch;
        double* dalpha = scratch + KHP_NOALLOC_BLOCKS * KHP_MAX_GATES;
        e = launch_backward((const double2*)evecs_dev, g->np, n, dLdE_host, g->De, dLdV_dev, dLdstrain_dev,
                            n_gates ? levers_dev : nullptr, n_gates, partial, KHP_NOALLOC_BLOCKS, dalpha,
                            g->stream, g->nb);
        if (e == cudaSuccess && n_gates > 0) {
            e = cudaMemcpyAsync(dLdalpha_host, dalpha, sizeof(double) * n_gates, cudaMemcpyDeviceToHost,
                                g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        }
    }
    if (prev != g->device) cudaSetDevice(prev);
    if (e != cudaSuccess)
        return khp_set_error(KHP_ERR_CUDA, std::string("backward (no-alloc): ") + cudaGetErrorString(e));
    return KHP_OK;
}
