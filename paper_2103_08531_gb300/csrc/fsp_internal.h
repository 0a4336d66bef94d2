// fsp_internal.h -- plan object and launcher declarations shared by the .cu files.
#pragma once

#include "../../include/fsp.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

struct fsp_plan;

namespace fsp {

struct PassArgs;

struct Plan {
    int dim;          // 2 or 3
    int n[3];         // cells per physical axis (n[2] = 0 in 2D)
    double h[3];
    int method;
    double L;         // VGF truncation radius (0 for HE)
    int M[3];         // VGF oversampled grid (0 for HE)
    double g0;        // HE value replacing G(0)
    // pass geometry: n0 x n1 x n2 with axis 2 contiguous (2D: n1 = 1)
    int n0, n1, n2, rows1, three_d;
    float k0s, k1s, k2s;
    float2 *tw0, *tw1, *tw2;  // device twiddle tables for 2 n0, 2 n1, 2 n2
    float *K;                 // device FP32 kernel octant
    size_t K_count;
    size_t buf_elems;         // complex elements of one intermediate buffer
    void *ws;
    size_t ws_bytes;
    int device;
    cudaEvent_t pass_ev[8];   // optional per-pass timing events (see fsp_plan_set_pass_events)
    int n_pass_ev;
    // direct-sum path (fsp_direct.cu): sizes the fast passes do not cover, and FP64
    int dtype;                // FSP_F32 or FSP_F64
    int direct;               // 1: solves run the direct-sum DFT path
    double *K64;              // FP64 kernel octant (FP64 plans)
    double2 *dtw[3];          // FP64 twiddles exp(2 pi i m / (2 n_a)) per pass axis (direct plans)
    double kd[3];             // 2 pi / (2 n_a h_a) per pass axis, FP64
    int *status;              // device status word (FSP_OK, or FSP_ERR_TIMEOUT from a bounded wait)
    int plane_group;          // > 0: P2-P4 of single 3D solves run in groups of this many k0 planes
};

// fsp_precompute.cu
int make_twiddles(float2 *tw, int N, cudaStream_t st);
int make_twiddles_aux(float2 *tw, int N, cudaStream_t st);    // fsp_axis2.cu
int make_twiddles_gall(float2 *tw, int N, cudaStream_t st);   // fsp_axis2.cu
int twiddle_gall_entries(int N);                              // fsp_axis2.cu
int has_radix_plan_b(int N);   // 1: length N has a second radix split (Plan16B), fsp_axis2.cu
constexpr int TW_AUX = 1024;   // gathered-twiddle entries after each N-entry table (N <= 512)
inline size_t twiddle_entries(int N)
{
    const int g = twiddle_gall_entries(N);
    return (size_t)N + (size_t)(g > TW_AUX ? g : TW_AUX);
}
int build_kernel_spectrum(Plan *p, cudaStream_t st);

// pass kinds
enum PassKind { PASS_P1F = 0, PASS_P1A, PASS_P2F, PASS_P2A, PASS_P3F, PASS_P3A, PASS_P4F, PASS_P5F };

// launchers (return 0 or a cudaError_t value).  Each runs one pass of padded
// length N over items[0..n) in one launch per BATCH_MAX items; flag is withE
// (forward) or hasE (adjoint) where the pass takes one.
int supported_axis0(int N);
int supported_axis1(int N);
int supported_axis2(int N);
int prepare_axis0(int N);
int prepare_axis1(int N);
int prepare_axis2(int N);
// var: tuning variant bits (1 = 8 values per thread in column tiles, 2 = one
// CTA per SM in persistent launches, 4 = the cp.async block-synchronous column
// tiles instead of the TMA-staged group tiles); chosen by the autotuner
// (fsp_autotune.cu).  Column passes of 2n <= 512 run the TMA-staged tiles
// (single solves and batches) unless bit 4 is set; longer columns run the
// block and staged long-column kernels.
int launch_axis0(int kind, int N, const PassArgs *items, int n, int var, cudaStream_t st);
int launch_axis1(int kind, int N, const PassArgs *items, int n, int flag, int var, cudaStream_t st);
int launch_axis2(int kind, int N, const PassArgs *items, int n, int flag, int var, cudaStream_t st);

// fsp_direct.cu: the direct-sum DFT path (any size, FP32 or FP64)
constexpr int DIRECT_MAX_N = 512;   // cells per axis
size_t direct_workspace_bytes(const Plan &p);
int run_direct_forward(const Plan &p, void *ws, const void *rho, void *phi, void *E, cudaStream_t st);
int run_direct_adjoint(const Plan &p, void *ws, const void *g_phi, const void *g_E, void *g_rho, cudaStream_t st);
int make_direct_twiddles(double2 *tw, int N, cudaStream_t st);   // fsp_precompute.cu

// fsp_api.cu: the forward and adjoint pipelines of one plan on workspace ws
int run_forward(const Plan &p, void *ws, const float *rho, float *phi, float *E, cudaStream_t st);
int run_adjoint(const Plan &p, void *ws, const float *g_phi, const float *g_E, float *g_rho, cudaStream_t st);
// Store status s as the calling thread's fsp_last_error() and return it; every
// C entry point returns through this.
int record_error(int s);

// fsp_tma_host.cu: a tiled tensor map over a row-major array (dims[0] contiguous;
// strides in bytes of dims 1 .. rank-1), 128-byte swizzle, box `box`; elem_bytes
// 4 or 8.  Returns 0 or a CUresult.
int encode_tensor_map(void *map, const void *base, int rank, int elem_bytes, const unsigned long long *dims,
                      const unsigned long long *strides, const unsigned *box);

// NVTX range around a solve or a pass (host-side enqueue; shown by Nsight tools,
// free when no tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

// Host-side fault injection for tests of the error paths: when the
// environment variable FSP_FAULT_INJECT names `what` ("alloc": the
// allocations of plan, batch and host-pipe creation), the call fails as if
// the allocation had failed.  Nothing on the GPU is involved.
inline bool inject_fault(const char *what)
{
    const char *v = getenv("FSP_FAULT_INJECT");
    return v && strcmp(v, what) == 0;
}

// fsp_autotune.cu: the variant chosen for a pass kind at padded length N (0 if untuned)
int tuned_variant(int kind, int N);
constexpr int PASS_KINDS = 8;

} // namespace fsp

struct fsp_plan {
    fsp::Plan p;
};
