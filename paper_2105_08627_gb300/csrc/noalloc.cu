// noalloc.cu -- the operator product for callers that cannot allocate device memory.
//
// svh_matvec grows its intermediate grids with cudaMalloc on first use for a
// given batch size. Some callers cannot allow that at call time: a plug-in
// running inside a host application that owns the whole device-memory
// budget, or a latency-critical loop that must not enter the allocator
// (cudaMalloc may synchronise the device). svh_matvec_noalloc runs the same
// kernels on a fixed scratch array that lives in the library's own device
// image instead, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <mutex>

#include "svh_internal.h"

namespace svh {

// The scratch of svh_matvec_noalloc. Every device that loads this library's
// device code holds these SVH_NOALLOC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SVH_NOALLOC_SCRATCH_BYTES];

// In host code g_noalloc_scratch names a host-side stand-in, not device
// memory, so kernels get its device address, looked up once per device.
constexpr int kMaxDevices = 256;
static std::mutex g_scratch_mu;
static void* g_scratch_dev[kMaxDevices] = {};

static int noalloc_scratch(Handle* h, void** out) {
    if (h->device < 0 || h->device >= kMaxDevices)
        return set_err(h, SVH_ERR_ARG, "svh_matvec_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_dev[h->device]) {
        // the handle's device is current (set by the caller of this function)
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err(h, e, "svh_matvec_noalloc: cudaGetSymbolAddress");
        g_scratch_dev[h->device] = p;
    }
    *out = g_scratch_dev[h->device];
    return SVH_OK;
}

}  // namespace svh

using namespace svh;

extern "C" int svh_matvec_noalloc(svh_handle* hh, double omega, int nb, const void* x, void* y, int precision) {
    Handle* h = reinterpret_cast<Handle*>(hh);
    if (!h) return SVH_ERR_ARG;
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_err(h, e, "cudaSetDevice");
    if (!h->have_grid || !h->have_kernels)
        return set_err(h, SVH_ERR_STATE, "svh_matvec_noalloc: grid and kernels must be set up first");
    if (!(omega > 0) || nb <= 0 || !x || !y || (precision != SVH_FP32 && precision != SVH_FP64))
        return set_err(h, SVH_ERR_ARG, "svh_matvec_noalloc: bad omega, nb, pointers or precision");
    const size_t bytes = (size_t)nb * (5 * h->K + h->M) * (precision == SVH_FP32 ? 8 : 16);
    const char* xc = static_cast<const char*>(x);
    const char* yc = static_cast<const char*>(y);
    if (xc < yc + bytes && yc < xc + bytes) return set_err(h, SVH_ERR_ARG, "svh_matvec_noalloc: x and y overlap");
    bool tucker = false;
    for (int u = 0; u < 7; ++u) tucker = tucker || h->tucker_on[u];
    if (precision == SVH_FP32 && h->kernel_mode == SVH_KERNELS_TUCKER_REBUILD && tucker &&
        h->spec32_tk_version != h->tk_version)
        return set_err(h, SVH_ERR_STATE,
                       "svh_matvec_noalloc: in Tucker-restore mode the restored spectra must be on the device "
                       "(call svh_rebuild_spectra first)");
    size_t b1, b2;
    matvec_scratch_bytes(h, nb, precision, &b1, &b2);
    const size_t b1a = (b1 + 255) & ~(size_t)255;
    if (b1a + b2 > (size_t)SVH_NOALLOC_SCRATCH_BYTES)
        return set_err(h, SVH_ERR_ARG,
                       "svh_matvec_noalloc: this grid and batch need more than the fixed 64 MiB of scratch "
                       "(use svh_matvec, or fewer right-hand sides per call)");
    void* base = nullptr;
    int rc = noalloc_scratch(h, &base);
    if (rc) return rc;
    // Every scratch element read by the passes is written earlier in the same
    // call, so nothing left from a previous call needs clearing.
    char* p = static_cast<char*>(base);
    return launch_matvec_on(h, omega, nb, x, y, precision, p, p + b1a);
}
