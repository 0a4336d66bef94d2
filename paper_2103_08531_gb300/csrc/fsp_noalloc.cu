// fsp_noalloc.cu -- a solve entry point that needs no caller-provided workspace.
//
// fsp_solve needs a device workspace that the caller allocates (cudaMalloc,
// a torch tensor, a pool).  Some callers cannot allocate device memory at the
// point where they solve: code running while a framework owns the allocator
// (a plugin or callback inside a host application with its own memory pool
// and no allocation allowed from libraries), real-time or embedded loops whose
// memory budget is fixed at start-up, and code paths that must not call
// cudaMalloc because it can synchronise the device.  fsp_solve_noalloc serves
// them: its scratch is a fixed, file-scope device array that exists for as
// long as the library is loaded, on every GPU that loads it.
#include "fsp_internal.h"

#include <cstdint>
#include <mutex>

namespace fsp {
int run_forward(const Plan &p, void *ws, const float *rho, float *phi, float *E, cudaStream_t st);
}

// The shared scratch: FSP_NOALLOC_SCRATCH_BYTES on each device, alive until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FSP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};   // device address of g_noalloc_scratch, per device
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).  Returns FSP_OK or an error code.
static int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return FSP_ERR_CUDA;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return FSP_OK;
}

extern "C" int fsp_solve_noalloc(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream)
{
    if (!plan || !rho || (!phi && !E)) return FSP_ERR_INVALID;
    if (((uintptr_t)rho % 16) || ((uintptr_t)phi % 16) || ((uintptr_t)E % 16)) return FSP_ERR_INVALID;
    const fsp::Plan &p = plan->p;
    if (fsp_plan_workspace_bytes(plan, E != nullptr, 1) > (size_t)FSP_NOALLOC_SCRATCH_BYTES)
        return FSP_ERR_WORKSPACE;   // grid too large for the fixed scratch
    void *ws = nullptr;
    int rc = scratch_address(&ws);
    if (rc != FSP_OK) return rc;
    return fsp::run_forward(p, ws, (const float *)rho, (float *)phi, (float *)E, (cudaStream_t)cuda_stream);
}
