// fsp_host.cu -- solves of host-resident grids: copy-in, solve and copy-out
// on three library-owned streams, so that the transfers of neighbouring
// solves run under each other's kernels (C ABI: fsp_host_pipe_*).
//
// Slot k of `depth` device buffer sets: the copy-in stream waits until the
// slot's previous outputs have left (freed[k]), copies rho in and records
// loaded[k]; the compute stream waits for loaded[k], runs the plan's passes
// on the plan's workspace (which serialises solves there) and records
// solved[k]; the copy-out stream waits for solved[k], copies phi and E out
// and records freed[k].  The first copy waits for the work already queued on
// the caller's stream; the caller's stream waits for the last copy-out.
#include "fsp_internal.h"

#include <cstdint>
#include <new>
#include <vector>

struct fsp_host_pipe {
    fsp_plan *plan = nullptr;
    int depth = 0, with_phi = 0, with_E = 0;
    size_t grid_bytes = 0;   // one real grid in the plan's precision
    std::vector<void *> rho, phi, E;
    cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> loaded, solved, freed;
    cudaEvent_t start = nullptr, done = nullptr;
};

static void pipe_free(fsp_host_pipe *p)
{
    for (void *b : p->rho) cudaFree(b);
    for (void *b : p->phi) cudaFree(b);
    for (void *b : p->E) cudaFree(b);
    for (auto *v : {&p->loaded, &p->solved, &p->freed})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    if (p->start) cudaEventDestroy(p->start);
    if (p->done) cudaEventDestroy(p->done);
    for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
        if (s) cudaStreamDestroy(s);
    delete p;
}

extern "C" fsp_host_pipe *fsp_host_pipe_create(fsp_plan *plan, int depth, int with_phi, int with_E)
{
    if (!plan || depth < 1 || depth > 8 || (!with_phi && !with_E)) {
        fsp::record_error(FSP_ERR_INVALID);
        return nullptr;
    }
    fsp_host_pipe *p = fsp::inject_fault("alloc") ? nullptr : new (std::nothrow) fsp_host_pipe();
    if (!p) {
        fsp::record_error(FSP_ERR_NOMEM);
        return nullptr;
    }
    const fsp::Plan &q = plan->p;
    p->plan = plan;
    p->depth = depth;
    p->with_phi = with_phi != 0;
    p->with_E = with_E != 0;
    const size_t cells = (size_t)q.n[0] * q.n[1] * (q.dim == 3 ? q.n[2] : 1);
    p->grid_bytes = cells * (q.dtype == FSP_F64 ? sizeof(double) : sizeof(float));
    int rc = FSP_OK;
    p->rho.assign(depth, nullptr);
    p->phi.assign(depth, nullptr);
    p->E.assign(depth, nullptr);
    for (int k = 0; k < depth && rc == FSP_OK; ++k) {
        if (cudaMalloc(&p->rho[k], p->grid_bytes) != cudaSuccess) rc = FSP_ERR_NOMEM;
        if (rc == FSP_OK && p->with_phi && cudaMalloc(&p->phi[k], p->grid_bytes) != cudaSuccess) rc = FSP_ERR_NOMEM;
        if (rc == FSP_OK && p->with_E && cudaMalloc(&p->E[k], q.dim * p->grid_bytes) != cudaSuccess)
            rc = FSP_ERR_NOMEM;
    }
    for (cudaStream_t *s : {&p->s_in, &p->s_run, &p->s_out})
        if (rc == FSP_OK && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess) rc = FSP_ERR_CUDA;
    for (auto *v : {&p->loaded, &p->solved, &p->freed}) {
        v->assign(depth, nullptr);
        for (int k = 0; k < depth && rc == FSP_OK; ++k)
            if (cudaEventCreateWithFlags(&(*v)[k], cudaEventDisableTiming) != cudaSuccess) rc = FSP_ERR_CUDA;
    }
    if (rc == FSP_OK && (cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess))
        rc = FSP_ERR_CUDA;
    // every slot starts free
    for (int k = 0; k < depth && rc == FSP_OK; ++k)
        if (cudaEventRecord(p->freed[k], p->s_out) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc != FSP_OK) {
        pipe_free(p);
        fsp::record_error(rc);
        return nullptr;
    }
    fsp::record_error(FSP_OK);
    return p;
}

static int pipe_solve(fsp_host_pipe *p, int count, const void *const *rho_host, void *const *phi_host,
                      void *const *E_host, cudaStream_t caller)
{
    if (!p || count < 0 || (count > 0 && !rho_host)) return FSP_ERR_INVALID;
    if ((p->with_phi && count > 0 && !phi_host) || (p->with_E && count > 0 && !E_host)) return FSP_ERR_INVALID;
    for (int i = 0; i < count; ++i) {
        if (!rho_host[i] || (p->with_phi && !phi_host[i]) || (p->with_E && !E_host[i])) return FSP_ERR_INVALID;
    }
    const fsp::Plan &q = p->plan->p;
    if (!q.ws || q.ws_bytes < fsp_plan_workspace_bytes(p->plan, p->with_E, 1)) return FSP_ERR_WORKSPACE;
    const size_t gb = p->grid_bytes;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaEventRecord(p->start, caller)) || !ok(cudaStreamWaitEvent(p->s_in, p->start, 0))) return FSP_ERR_CUDA;
    for (int i = 0; i < count; ++i) {
        const int k = i % p->depth;
        if (!ok(cudaStreamWaitEvent(p->s_in, p->freed[k], 0)) ||
            !ok(cudaMemcpyAsync(p->rho[k], rho_host[i], gb, cudaMemcpyHostToDevice, p->s_in)) ||
            !ok(cudaEventRecord(p->loaded[k], p->s_in)) || !ok(cudaStreamWaitEvent(p->s_run, p->loaded[k], 0)))
            return FSP_ERR_CUDA;
        const int rc = fsp::run_forward(q, q.ws, (const float *)p->rho[k], (float *)p->phi[k], (float *)p->E[k],
                                        p->s_run);
        if (rc != FSP_OK) return rc;
        if (!ok(cudaEventRecord(p->solved[k], p->s_run)) || !ok(cudaStreamWaitEvent(p->s_out, p->solved[k], 0)))
            return FSP_ERR_CUDA;
        if (p->with_phi && !ok(cudaMemcpyAsync(phi_host[i], p->phi[k], gb, cudaMemcpyDeviceToHost, p->s_out)))
            return FSP_ERR_CUDA;
        if (p->with_E && !ok(cudaMemcpyAsync(E_host[i], p->E[k], q.dim * gb, cudaMemcpyDeviceToHost, p->s_out)))
            return FSP_ERR_CUDA;
        if (!ok(cudaEventRecord(p->freed[k], p->s_out))) return FSP_ERR_CUDA;
    }
    // the caller's stream resumes after the last copy-out (and after the copy-in
    // and compute streams, which the copy-out stream has waited for)
    if (!ok(cudaEventRecord(p->done, p->s_out)) || !ok(cudaStreamWaitEvent(caller, p->done, 0))) return FSP_ERR_CUDA;
    return FSP_OK;
}

extern "C" int fsp_host_pipe_solve(fsp_host_pipe *pipe, int count, const void *const *rho_host,
                                   void *const *phi_host, void *const *E_host, void *cuda_stream)
{
    return fsp::record_error(pipe_solve(pipe, count, rho_host, phi_host, E_host, (cudaStream_t)cuda_stream));
}

extern "C" void fsp_host_pipe_destroy(fsp_host_pipe *pipe)
{
    if (!pipe) return;
    cudaStreamSynchronize(pipe->s_in);
    cudaStreamSynchronize(pipe->s_run);
    cudaStreamSynchronize(pipe->s_out);
    pipe_free(pipe);
}
