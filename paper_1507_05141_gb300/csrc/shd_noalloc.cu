// shd_project_noalloc: the projection stage (a1) into caller-owned device
// memory with no allocation of any kind.
//
// Some callers cannot call cudaMalloc at the point where they need the
// moments: a host program whose device memory is owned by another allocator
// (a framework's memory pool that must see every byte), a time-critical loop
// that must not meet the allocator's implicit device synchronisation, or a
// process already at its device-memory limit.  For them this entry point
// keeps the comoving intensities of moving nodes -- the only scratch the
// projection needs -- in a fixed file-scope device array instead of the
// context's buffer.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "shd_internal.cuh"

using namespace shd;

// The scratch: one fixed array per device that loads this library, held until
// the process exits.  In host code the symbol is only a stand-in; kernels get
// its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SHD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

thread_local char g_msg[256] = "";

// Device address of the scratch on the current device (looked up once per
// device, on the first call made with that device current).
cudaError_t scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// The body of shd_project_noalloc with c->device current.
static int project_noalloc(shd_ctx *c, void *dev_Ish, void *dev_mom, void *cuda_stream)
{
    // the same readiness check as shd_get_moments (configured, every stage's
    // shared memory within the limit); it allocates nothing
    int rc = check_ready(c);
    if (rc != SHD_OK) {
        snprintf(g_msg, sizeof(g_msg), "%s", shd_last_error());
        return rc;
    }
    if (!c->have_state) {
        snprintf(g_msg, sizeof(g_msg), "state not set");
        return SHD_ERR_STATE;
    }
    if (c->nmoving > 0) {
        size_t need = (size_t)2 * c->nmoving * c->G * c->N * c->esize;
        if (need > (size_t)SHD_NOALLOC_SCRATCH_BYTES) {
            snprintf(g_msg, sizeof(g_msg), "needs %zu bytes of scratch, the static scratch holds %zu", need,
                     (size_t)SHD_NOALLOC_SCRATCH_BYTES);
            return SHD_ERR_ARG;
        }
    }
    void *scratch = nullptr;
    cudaError_t e = scratch_address(c->device, &scratch);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return SHD_ERR_CUDA;
    }
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
    if (c->precision == SHD_FP64)
        e = launch_project_scratch<double>(c, (const double *)c->d_I, (double *)dev_Ish, (double *)dev_mom,
                                           (double *)scratch, st);
    else
        e = launch_project_scratch<float>(c, (const float *)c->d_I, (float *)dev_Ish, (float *)dev_mom,
                                          (float *)scratch, st);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "launch: %s", cudaGetErrorString(e));
        return SHD_ERR_CUDA;
    }
    return SHD_OK;
}

extern "C" int shd_project_noalloc(shd_ctx *c, void *dev_Ish, void *dev_mom, void *cuda_stream)
{
    g_msg[0] = 0;
    if (!c || !dev_Ish || !dev_mom) {
        snprintf(g_msg, sizeof(g_msg), "null context or output pointer");
        return SHD_ERR_ARG;
    }
    if (c->device < 0 || c->device >= kMaxDevices) {
        snprintf(g_msg, sizeof(g_msg), "device %d out of range", c->device);
        return SHD_ERR_ARG;
    }
    // run with the context's device current, then give the caller back theirs
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != c->device) e = cudaSetDevice(c->device);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "cudaSetDevice: %s", cudaGetErrorString(e));
        return SHD_ERR_CUDA;
    }
    int rc = project_noalloc(c, dev_Ish, dev_mom, cuda_stream);
    if (prev != c->device && prev >= 0) {
        e = cudaSetDevice(prev);
        if (e != cudaSuccess && rc == SHD_OK) {
            snprintf(g_msg, sizeof(g_msg), "restoring device %d: %s", prev, cudaGetErrorString(e));
            rc = SHD_ERR_CUDA;
        }
    }
    return rc;
}

extern "C" const char *shd_noalloc_last_error(void) { return g_msg; }
