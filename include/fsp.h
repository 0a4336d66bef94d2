/*
 * fsp.h -- C ABI of the GB300 free-space Poisson solver.
 *
 * Solves Laplacian(phi) = -rho with free-space boundary conditions and returns
 * phi and E = -grad(phi) on a uniform cell-centred grid (paper Sec. 1,
 * Eq. "eq:Poisson" and "eq:convolution"), by the zero-padded FFT convolution of
 * Hockney and Eastwood (HE, paper Sec. 1) or of Vico, Greengard and Ferrando
 * (VGF, paper Sec. 2).  The two differ only in the Green's function that is
 * convolved (paper Sec. 2, last paragraph): HE samples G with a finite value at
 * r = 0, VGF uses the truncated kernel G^L whose transform is given in closed
 * form (Eqs. GLFourier2D, GLFourier3D), brought to the 2N grid through an
 * oversampled inverse transform.  Both run on the same GPU machinery:
 *
 *     phi = prod(h) IFFT_2N( FFT_2N(rho padded) FFT_2N(g) ) cropped to N,
 *     E_a = prod(h) IFFT_2N( -i k_a FFT_2N(rho padded) FFT_2N(g) ) cropped,
 *
 * with k_a = 2 pi m / (2 n_a h_a), m in [-n_a, n_a), and k_a = 0 at the
 * unpaired index m = -n_a (Fourier differentiation, paper Sec. 3).
 *
 * Units follow the paper: G = 1/(4 pi r) in 3D and -ln(r)/(2 pi) in 2D.
 *
 * Layouts.  All arrays are row-major with the last axis contiguous:
 *   3D rho, phi: real [nx][ny][nz];   E: real [3][nx][ny][nz]
 *   2D rho, phi: real [nx][ny];       E: real [2][nx][ny]
 * "real" is float for FSP_F32 plans and double for FSP_F64 plans.
 * Device pointers must be 16-byte aligned; the caller owns every buffer.
 *
 * Execution.  Solves are asynchronous on the given CUDA stream (a
 * cudaStream_t passed as void*, NULL = legacy default stream); they never
 * synchronise and never allocate, so they can be captured in a CUDA graph.
 * Argument errors are reported synchronously through the return code.  A plan
 * owns one workspace, so a plan must not be used by two overlapping solves.
 *
 * Errors.  Functions returning int return an fsp_status.  fsp_plan_create and
 * fsp_batch_create return NULL on failure and leave the code in
 * fsp_last_error() (thread-local).
 */
#ifndef FSP_H
#define FSP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsp_plan fsp_plan;
typedef struct fsp_batch fsp_batch;

enum fsp_method {
    FSP_HE = 0,         /* Hockney-Eastwood, G(0) replaced by 1 (3D) or 1/(2 pi) (2D): paper Sec. 1, Sec. 3 */
    FSP_VGF = 1,        /* Vico-Greengard-Ferrando truncated kernel: paper Sec. 2 */
    FSP_HE_NEARBY = 2,  /* HE with G(0) := G(min_a h_a) ("nearby value" variant, paper Sec. 3) */
    FSP_HE_CELLAVG = 3  /* HE with G(0) := mean of G over the cell ("cell average" variant, paper Sec. 3) */
};

enum fsp_dtype { FSP_F32 = 0, FSP_F64 = 1 };

enum fsp_status {
    FSP_OK = 0,
    FSP_ERR_INVALID = 1,          /* bad argument: NULL, misaligned, out of range */
    FSP_ERR_UNSUPPORTED_SIZE = 2, /* grid size the FFT passes do not cover */
    FSP_ERR_CUDA = 3,             /* a CUDA runtime call failed */
    FSP_ERR_NOMEM = 4,            /* allocation at plan creation failed */
    FSP_ERR_WORKSPACE = 5,        /* no workspace set, or too small */
    FSP_ERR_TIMEOUT = 6           /* a bounded device-side wait gave up */
};

/*
 * Create a plan for one grid geometry: nx x ny x nz cells (nz = 0 for a 2D
 * nx x ny problem; hz is then ignored) with spacings hx, hy, hz.  Runs the
 * once-per-geometry kernel precomputation on the current CUDA device in FP64
 * (paper Sec. 2, last paragraph: transform of G^L on an oversampled grid,
 * restricted to the 2N grid) and stores the real, even FP32 spectrum of the
 * kernel with prod(h)/prod(2n) folded in.  Blocks until the precomputation
 * has finished.
 *
 * Two solve paths.  The FFT passes (FP32) cover the padded lengths 2 n_a in
 * {32, 64, 96, 128, 192, 256, 384, 512, 768, 1024} on every 3D axis and, in 2D,
 * also 1536, 2048, 3072, 4096, 6144 and 8192 (the powers of two and three times
 * the powers of two); the contiguous axis (nz in 3D, ny in 2D) needs a cell
 * count that is a multiple of 32.  Every other size
 * with 1 <= n_a <= 512, and every FSP_F64 plan, runs the direct-sum path: the
 * same pruned convolution with each 1D transform taken by its definition
 * (O(N^2) per line), in the plan's precision -- the paper's convergence
 * studies use N = 10 ... 100 per axis (Sec. 3), 2 N often with large prime
 * factors.  Larger odd-size grids: FSP_ERR_UNSUPPORTED_SIZE.
 * dtype: FSP_F32 (float buffers) or FSP_F64 (double buffers everywhere a
 * solve, adjoint or gradient takes a grid).
 * Returns NULL on failure (see fsp_last_error()).
 */
fsp_plan *fsp_plan_create(int nx, int ny, int nz, double hx, double hy, double hz, int method, int dtype);

enum fsp_plan_flags {
    FSP_PLAN_DIRECT = 1   /* run the direct-sum path even where the FFT passes cover the size */
};

/*
 * As fsp_plan_create, with the VGF truncation radius scaled by lambda (L =
 * lambda * box diagonal; lambda <= 0 means 1), for the HE methods an explicit
 * value g0 for G(0) (NaN means the method's default), and flags (a set of
 * fsp_plan_flags; unknown bits: FSP_ERR_INVALID).
 */
fsp_plan *fsp_plan_create_ex(int nx, int ny, int nz, double hx, double hy, double hz, int method, int dtype,
                             double lambda, double g0, int flags);

int fsp_last_error(void);
const char *fsp_error_string(int status);

/*
 * Geometry chosen by the plan: n[3], h[3], the VGF truncation radius L and
 * oversampled grid M[3] (0 for HE), and the dimension (2 or 3).  Any output
 * pointer may be NULL.
 */
int fsp_plan_geometry(const fsp_plan *plan, int *dim, int *n, double *h, double *L, int *M);

/*
 * Device workspace one solve needs, in bytes; batch >= 1 multiplies it.
 * with_E = 0 sizes it for solves without E (and adjoints without g_E): a 2D
 * FFT-path plan then needs one intermediate buffer instead of two; 3D and
 * direct-sum plans need the same either way.  Returns 0 for a NULL plan or
 * batch < 1.
 */
size_t fsp_plan_workspace_bytes(const fsp_plan *plan, int with_E, int batch);

/*
 * Hand the plan a device workspace (the caller keeps ownership; 256-byte
 * aligned, else FSP_ERR_INVALID).  bytes below fsp_plan_workspace_bytes(plan,
 * 0, 1) is FSP_ERR_WORKSPACE; each solve checks the size it needs for its own
 * outputs and returns FSP_ERR_WORKSPACE if the workspace is smaller.
 */
int fsp_plan_set_workspace(fsp_plan *plan, void *dev_ptr, size_t bytes);

/*
 * One solve.  rho: device real grid.  phi: device real grid or NULL.
 * E: device real [dim][grid] or NULL.  phi and E must not both be NULL.
 */
int fsp_solve(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream);

/*
 * Adjoint of the linear map rho -> (phi, E):
 *     g_rho = A^T g_phi + sum_a B_a^T g_E[a] = A g_phi - sum_a B_a g_E[a],
 * A symmetric because the kernel is even, B_a antisymmetric because -i k_a is
 * odd with the Nyquist entry zero.  g_phi or g_E may be NULL (zero).
 */
int fsp_solve_adjoint(fsp_plan *plan, const void *g_phi, const void *g_E, void *g_rho, void *cuda_stream);

/*
 * Many independent solves of different geometries, one launch per pass over
 * all of them.  plans[i] must be distinct plans, each with its own workspace
 * set; rho/phi/E as for fsp_solve (phi[i] or E[i] may be NULL consistently for
 * all i: with_E is taken from E != NULL).  Direct-path plans (see
 * fsp_plan_create) are solved one after another after the batched launches.
 */
int fsp_solve_batched(fsp_plan *const *plans, int count, const void *const *rho, void *const *phi,
                      void *const *E, void *cuda_stream);

/*
 * Prebuilt batch: the device work lists of fsp_solve_batched built once, so
 * that repeated launches (or a captured CUDA graph) do no host work.
 * fsp_batch_create copies the pointer arrays; they must stay valid device
 * buffers for the life of the batch.  It also creates a few CUDA streams and
 * events of its own: the launches of one pass that serve different padded
 * lengths are independent, so fsp_batch_solve forks them onto those streams
 * from the caller's stream and joins them back before the next pass (in a
 * captured graph: parallel branches).  The caller's stream sees the usual
 * stream order: the solve starts after earlier work on it and later work
 * starts after the solve.
 */
fsp_batch *fsp_batch_create(fsp_plan *const *plans, int count, const void *const *rho, void *const *phi,
                            void *const *E);
int fsp_batch_solve(fsp_batch *batch, void *cuda_stream);
void fsp_batch_destroy(fsp_batch *batch);
/* Number of kernels one fsp_batch_solve of this batch launches (a report for
 * benchmarks and tests, not part of the paper's method): the solve is captured
 * once on a private stream into a CUDA graph whose kernel nodes are counted;
 * nothing runs on the GPU.  *count is written on FSP_OK.  FSP_ERR_INVALID for
 * a NULL argument, FSP_ERR_CUDA if the capture fails.  Set-up, not a solve:
 * do not call it while the calling thread captures a stream. */
int fsp_batch_kernel_count(fsp_batch *batch, int *count);

/*
 * Measurement hook: when count > 0, every later fsp_solve / fsp_solve_adjoint
 * on this plan records events[i] (cudaEvent_t values created by the caller) on
 * its stream just before pass i, and events[passes] after the last pass
 * (passes = 5 in 3D, 3 in 2D; count must be >= passes + 1).  events = NULL or
 * count = 0 turns it off.  The array is copied; the events stay the caller's.
 * Plans on the direct-sum path have no such passes: FSP_ERR_INVALID.
 */
int fsp_plan_set_pass_events(fsp_plan *plan, void *const *events, int count);

/*
 * E = -grad(phi) by centred finite differences on the plan's grid, the
 * alternative to Fourier differentiation that the paper compares for HE
 * (Sec. 3, two-dimensional example): (phi[i+1] - phi[i-1]) / (2 h) inside,
 * second-order one-sided differences on the first and last cell of each axis.
 * phi: device real grid; E: device real [dim][grid].  Asynchronous on the
 * stream; allocates nothing.
 */
int fsp_gradient_fd(const fsp_plan *plan, const void *phi, void *E, void *cuda_stream);

/*
 * Autotuner.  Each pass has launch variants (bit 4: the cp.async column tiles
 * instead of the TMA-staged ones, and for middle passes of 1024-, 2048- and
 * 8192-point lines the block-synchronous line kernel instead of the
 * multi-warp or four-step one; bit 1, with bit 4: 8 instead of 16 values per
 * thread in column tiles; bit 2: one CTA per SM in persistent launches; bit 8,
 * without bit 4, at padded lengths 128, 256 and 512: a second radix split of
 * the transforms, 8 x 16, 8 x 8 x 4 and 8 x 8 x 8 instead of 16 x 8, 16 x 16
 * and 16 x 16 x 2, in the TMA column tiles and the single-solve middle pass,
 * and for 1024-point middle lines two warp-synchronous 512-point halves); the
 * choice is a process-wide table keyed by pass and padded length, read by
 * every solve.  fsp_autotune fills it for the passes this plan uses:
 * mode 0 reads the JSON cache at cache_path (may be NULL) only; mode 1 reads
 * it and times the missing passes on this plan's geometry; mode 2 times all
 * of them.  With a cache_path the table is written back, keyed by GPU
 * architecture.  With FSP_TUNE_LOG set in the environment every timed variant
 * is reported on stderr.  This call allocates scratch buffers and synchronises (it is
 * set-up, not a solve).  fsp_tuned_variant reports an entry: kind is 0..7 for
 * p1_fwd, p1_adj, p2_fwd, p2_adj, p3_fwd, p3_adj, p4_fwd, p5_fwd.  Direct-path
 * plans have nothing to tune (mode 0 behaviour).
 */
int fsp_autotune(fsp_plan *plan, const char *cache_path, int mode);
int fsp_tuned_variant(int kind, int N);

/*
 * Host-resident grids.  A pipe owns `depth` device buffer sets (rho, and phi
 * and/or E as chosen at creation) and three CUDA streams: copy-in,
 * compute and copy-out.  fsp_host_pipe_solve enqueues `count` solves of host
 * grids rho_host[i] -> phi_host[i], E_host[i] (layouts as for fsp_solve, in
 * the plan's precision) through slot i % depth: the copy of rho in, the
 * solve (the plan's passes on the plan's workspace), the copy of the outputs
 * out; the transfers of one solve overlap the kernels of its neighbours.  It
 * returns once everything is queued (asynchronous): the copies start after
 * the work already queued on cuda_stream, and cuda_stream waits for the last
 * copy-out, so an event recorded on cuda_stream after the call, or a
 * synchronisation of it, covers every copy and solve.  Host buffers should be
 * page-locked (cudaMallocHost / cudaHostRegister) for the copies to overlap;
 * pageable buffers still give correct results.  They must stay valid until
 * cuda_stream has passed the call.  phi_host (E_host) must be non-NULL,
 * with non-NULL entries, exactly when the pipe was created with with_phi
 * (with_E).  The plan needs its workspace set (FSP_ERR_WORKSPACE otherwise)
 * and must not run other solves while the pipe works.  fsp_host_pipe_create
 * allocates (set-up); fsp_host_pipe_solve does not.  depth: 1 .. 8.
 * fsp_host_pipe_destroy waits for the pipe's streams, then frees it.
 * Not part of the paper's method: it is how a caller with host data reaches
 * the solver end to end.
 */
typedef struct fsp_host_pipe fsp_host_pipe;
fsp_host_pipe *fsp_host_pipe_create(fsp_plan *plan, int depth, int with_phi, int with_E);
int fsp_host_pipe_solve(fsp_host_pipe *pipe, int count, const void *const *rho_host, void *const *phi_host,
                        void *const *E_host, void *cuda_stream);
void fsp_host_pipe_destroy(fsp_host_pipe *pipe);

/*
 * Schedule of single 3D solves: with planes > 0 the three middle passes (axis
 * 1 forward, axis 2 forward-multiply-inverse, axis 1 inverse) run in turn on
 * groups of `planes` k0 planes of the half spectrum instead of each over all
 * n0 + 1 planes, so that one group's intermediates (about 2.5 MB per plane at
 * 256^3) can stay in the 129 MB L2 from one pass to the next; 0 (the default)
 * turns it off.  It applies where those passes are the single-solve kernels
 * with plane ranges (2 n_y, 2 n_z <= 512, TMA column tiles); elsewhere it is
 * ignored.  Results are the same bit for bit.  Not a step of the paper's
 * method: a memory-traffic schedule for the same arithmetic.
 */
int fsp_plan_set_plane_group(fsp_plan *plan, int planes);

/*
 * Device-side status of the plan's solves: FSP_OK, or FSP_ERR_TIMEOUT if a
 * kernel's bounded wait (the shared-memory tile barriers of the TMA-staged
 * passes, which give up after about 2 s) failed in some solve since the last
 * clear; that solve's outputs are then not valid.  Synchronises with the
 * device (a blocking copy of one word); clear != 0 resets the word.  The
 * solve calls never return this code themselves, since they do not wait.
 */
int fsp_plan_device_status(fsp_plan *plan, int clear);

/*
 * Test hook for the bounded device waits: runs one small kernel whose wait on
 * a shared-memory barrier can never complete (a transaction count that no
 * copy fills; no copy is in flight) with a limit of limit_seconds (0 < limit
 * <= 10), and returns the status that kernel recorded: FSP_ERR_TIMEOUT when
 * the wait gave up as it should; FSP_ERR_INVALID for a bad limit,
 * FSP_ERR_CUDA if a CUDA call failed.  Synchronises the device.  The same
 * bounded wait guards every tile of the TMA-staged passes (about 2 s there).
 */
int fsp_selftest_wait_timeout(double limit_seconds);

/*
 * Test hook: copy the plan's FP32 kernel spectrum to host memory, layout
 * [nx+1][ny+1][nz+1] (2D: [nx+1][ny+1]), entry (kx,ky,kz) = prod(h)/prod(2n)
 * times the DFT of the padded kernel at index k (indices k and 2n-k share it).
 */
int fsp_plan_kernel_spectrum(const fsp_plan *plan, void *host_out, size_t bytes);

/*
 * Test hooks for the intermediates of the padded convolution (paper Sec. 1,
 * the HE formula: pad, transform, product, inverse, crop, here one axis per
 * pass).  fsp_plan_run_passes runs the first `passes` of a forward solve of
 * rho (device, [nx][ny][nz]) on the plan's workspace, asynchronously on
 * cuda_stream, and stops: 3D passes 1..4 of P1 (axis 0 pad + R2C), P2
 * (axis 1 forward), P3 (axis 2 forward, product with the kernel spectrum and,
 * with with_E, with -i k_2 too, inverse, crop), P4 (axis 1 inverse and crop,
 * with with_E the -i k_1 stream); 2D passes 1..2 of P1 and P3.  The last pass
 * (C2R to the outputs) is what fsp_solve adds.  Plane groups are not used.
 * FSP_ERR_INVALID for a NULL or misaligned rho, a direct-path plan or passes
 * outside that range; FSP_ERR_WORKSPACE without a large enough workspace.
 *
 * fsp_plan_workspace_layout: the two intermediate buffers of the workspace,
 * buf0 at byte 0 and buf1 at *buf1_offset, each complex64 [dims[0]][dims[1]]
 * [dims[2]] = [nx+1][2 ny][nz] (2D: [nx+1][1][ny]), last index fastest; the
 * first index is k_0 of the half spectrum, the second the axis-1 position
 * (frequency after P2, cell after P4; rows ny.. hold the -i k_1 stream after
 * P4), the third the axis-2 position.  After P1 (3D) the spectrum of the
 * padded axis 0 is in buf1 rows 0..ny-1 (2D: buf0); after P2 the axis-1
 * spectrum is in buf0; after P3 the phi stream is in buf0 and the -i k_2
 * stream in buf1; after P4 the phi stream is in buf0 rows 0..ny-1, the -i k_1
 * stream in buf0 rows ny..2ny-1 and the -i k_2 stream in buf1 rows 0..ny-1.
 * Values carry prod(h)/prod(2n) from the kernel spectrum from P3 on.
 * FSP_ERR_INVALID for NULL arguments or a direct-path plan.
 */
int fsp_plan_run_passes(fsp_plan *plan, const void *rho, int passes, int with_E, void *cuda_stream);
int fsp_plan_workspace_layout(const fsp_plan *plan, size_t *buf1_offset, int *dims);

void fsp_plan_destroy(fsp_plan *plan);

/*
 * fsp_solve without a workspace, for callers that cannot allocate device
 * memory when they solve: code running while a host framework owns the
 * allocator (plugins, callbacks, pooled applications that forbid library
 * allocations), real-time loops whose memory is fixed at start-up, and paths
 * that must not call cudaMalloc because it can synchronise the device.  This
 * is a calling convention of this library; the paper has no counterpart.
 *
 * Same arguments, layouts and results as fsp_solve.  The scratch is one
 * static device array of FSP_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits; the call allocates nothing (no
 * cudaMalloc, no cudaFree, no allocating library routine).  The plan itself is
 * created beforehand with fsp_plan_create (that call allocates, once per
 * geometry).  A grid whose workspace (fsp_plan_workspace_bytes) exceeds the
 * scratch returns FSP_ERR_WORKSPACE (3D cubes up to 128^3 fit).
 *
 * Set-up: the first call on a device, with that device current, looks up
 * the scratch address on that device (cudaGetSymbolAddress) and keeps it;
 * make that first call before any stream capture.  The address belongs to the
 * device's CUDA context: after cudaDeviceReset the next call looks it up
 * again, so after a reset, too, call once outside any capture first.
 * Every call on a device shares the one scratch array and it keeps the last
 * call's contents (each solve writes every scratch element it later reads, so
 * nothing needs clearing).  Calls that overlap on the GPU (different streams,
 * or different plans at once) race on the scratch: serialise them.  The
 * status is also left in fsp_last_error(), as for every other entry point.
 */
#define FSP_NOALLOC_SCRATCH_BYTES (80u * 1024u * 1024u)
int fsp_solve_noalloc(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FSP_H */
