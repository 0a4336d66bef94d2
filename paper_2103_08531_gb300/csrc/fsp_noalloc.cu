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

#include <cuda.h>
#include <cstdint>
#include <mutex>

// The shared scratch: FSP_NOALLOC_SCRATCH_BYTES on each device, alive until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FSP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Slot {
    void *ptr = nullptr;             // device address of g_noalloc_scratch
    unsigned long long ctx_id = 0;   // context it was looked up in (0: unknown)
};
Slot g_slot[kMaxDevices];

// Unique id of the calling thread's current CUDA context (cuCtxGetId), or 0
// where the driver does not offer it.  A device reset replaces the primary
// context and with it the id, so a cached address is never reused across it.
unsigned long long current_context_id()
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(f1);
            get_id = reinterpret_cast<GetId>(f2);
        }
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
    return 0;
}
} // namespace

// Device address of the scratch array on the current device, looked up with
// that device current (cudaGetSymbolAddress) the first time the device is
// used, and again whenever its CUDA context has changed since (after
// cudaDeviceReset).  Returns FSP_OK or an error code.
static int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FSP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    Slot &s = g_slot[dev];
    if (!s.ptr || (ctx && ctx != s.ctx_id)) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            s.ptr = nullptr;
            return FSP_ERR_CUDA;
        }
        s.ptr = ptr;
        s.ctx_id = ctx;
    }
    *out = s.ptr;
    return FSP_OK;
}

static int solve_noalloc(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream)
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

extern "C" int fsp_solve_noalloc(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream)
{
    return fsp::record_error(solve_noalloc(plan, rho, phi, E, cuda_stream));
}
