// fsp_api.cu -- plan objects and the C ABI declared in include/fsp.h.
#include "fsp_internal.h"
#include "fsp_passes.cuh"

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

using namespace fsp;

static thread_local int g_last_error = FSP_OK;

static int set_err(int e)
{
    g_last_error = e;
    return e;
}

int fsp::record_error(int s) { return set_err(s); }

extern "C" int fsp_last_error(void) { return g_last_error; }

extern "C" const char *fsp_error_string(int s)
{
    switch (s) {
    case FSP_OK: return "ok";
    case FSP_ERR_INVALID: return "invalid argument";
    case FSP_ERR_UNSUPPORTED_SIZE: return "unsupported grid size";
    case FSP_ERR_CUDA: return "CUDA runtime error";
    case FSP_ERR_NOMEM: return "out of memory";
    case FSP_ERR_WORKSPACE: return "workspace missing or too small";
    case FSP_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
    }
}

// ----------------------------------------------------------- geometry rules

static bool smooth235(long long m)
{
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

// Oversampled VGF grid per axis: the inverse transform on M points of spacing h
// periodises the kernel with period M h; the 2n convolution reads offsets up to
// n h, so M h >= n h + L keeps the copies away.  At least 4 n (paper Sec. 2,
// last paragraph), smallest even 2^a 3^b 5^c.
static int oversample(int n, double h, double L)
{
    long long need = std::max<long long>(4LL * n, n + (long long)std::ceil(L / h) + 2);
    if (need % 2) ++need;
    while (!smooth235(need)) need += 2;
    return (int)need;
}

// HE G(0) replacements (paper Sec. 1 and the variants named in Sec. 3).
static double he_g0(int dim, const double *h, int method)
{
    const double pi = 3.14159265358979323846;
    if (method == FSP_HE) return dim == 3 ? 1.0 : 1.0 / (2.0 * pi);
    double hmin = h[0];
    for (int a = 1; a < dim; ++a) hmin = std::min(hmin, h[a]);
    if (method == FSP_HE_NEARBY) return dim == 3 ? 1.0 / (4.0 * pi * hmin) : -std::log(hmin) / (2.0 * pi);
    // cell average of G over [-h/2, h/2]^d
    if (dim == 3) {
        // int_box 1/r = sum over faces (divergence of r/r = 2/r); per face the
        // integral of 1/sqrt(a^2 + y^2 + z^2) over [0,b]x[0,c] is J(a; b, c).
        auto J = [](double a, double b, double c) {
            double R = std::sqrt(a * a + b * b + c * c);
            return b * std::log((c + R) / std::sqrt(a * a + b * b)) + c * std::log((b + R) / std::sqrt(a * a + c * c)) -
                   a * std::atan(b * c / (a * R));
        };
        double a = 0.5 * h[0], b = 0.5 * h[1], c = 0.5 * h[2];
        double I = 4.0 * (a * J(a, b, c) + b * J(b, a, c) + c * J(c, a, b));
        return I / (4.0 * pi * h[0] * h[1] * h[2]);
    }
    auto F = [](double x, double y) {
        double r = std::sqrt(x * x + y * y);
        return x * y * std::log(r) - 1.5 * x * y + 0.5 * x * x * std::atan(y / x) + 0.5 * y * y * std::atan(x / y);
    };
    double I = 4.0 * F(0.5 * h[0], 0.5 * h[1]);   // int_cell ln r
    return -I / (2.0 * pi * h[0] * h[1]);
}

// ------------------------------------------------------------------- plans

static std::mutex g_prep_mutex;

static void plan_free(Plan &p)
{
    cudaFree(p.tw0);
    if (p.tw1 != p.tw0) cudaFree(p.tw1);
    if (p.tw2 != p.tw0 && p.tw2 != p.tw1) cudaFree(p.tw2);
    cudaFree(p.K);
    cudaFree(p.K64);
    cudaFree(p.status);
    for (int a = 0; a < 3; ++a) cudaFree(p.dtw[a]);
}

extern "C" fsp_plan *fsp_plan_create_ex(int nx, int ny, int nz, double hx, double hy, double hz, int method,
                                        int dtype, double lambda, double g0, int flags)
{
    const int dim = nz == 0 ? 2 : 3;
    if (nx <= 0 || ny <= 0 || nz < 0 || !(hx > 0) || !(hy > 0) || (dim == 3 && !(hz > 0)) || method < FSP_HE ||
        method > FSP_HE_CELLAVG || (dtype != FSP_F32 && dtype != FSP_F64) || (flags & ~FSP_PLAN_DIRECT)) {
        set_err(FSP_ERR_INVALID);
        return nullptr;
    }
    fsp_plan *handle = inject_fault("alloc") ? nullptr : new (std::nothrow) fsp_plan();
    if (!handle) {
        set_err(FSP_ERR_NOMEM);
        return nullptr;
    }
    Plan &p = handle->p;
    std::memset(&p, 0, sizeof(p));
    p.dim = dim;
    p.n[0] = nx;
    p.n[1] = ny;
    p.n[2] = nz;
    p.h[0] = hx;
    p.h[1] = hy;
    p.h[2] = dim == 3 ? hz : 0.0;
    p.method = method;
    if (dim == 3) {
        p.n0 = nx; p.n1 = ny; p.n2 = nz; p.rows1 = 2 * ny; p.three_d = 1;
    } else {
        p.n0 = nx; p.n1 = 1; p.n2 = ny; p.rows1 = 1; p.three_d = 0;
    }
    const double pi = 3.14159265358979323846;
    const double hh0 = hx, hh2 = dim == 3 ? hz : hy;
    p.k0s = (float)(2.0 * pi / (2.0 * p.n0 * hh0));
    p.k1s = dim == 3 ? (float)(2.0 * pi / (2.0 * ny * hy)) : 0.f;
    p.k2s = (float)(2.0 * pi / (2.0 * p.n2 * hh2));
    p.kd[0] = 2.0 * pi / (2.0 * p.n0 * hh0);
    p.kd[1] = dim == 3 ? 2.0 * pi / (2.0 * ny * hy) : 0.0;
    p.kd[2] = 2.0 * pi / (2.0 * p.n2 * hh2);
    p.dtype = dtype;
    // the column tiles of the first and last passes take 32 reals (16 complex)
    // of the contiguous axis at a time
    const bool fast = supported_axis0(2 * p.n0) && supported_axis2(2 * p.n2) && (p.n2 % 32 == 0) &&
                      (dim == 2 || (supported_axis1(2 * p.n1) && 2 * p.n0 <= 1024 && 2 * p.n2 <= 1024));
    p.direct = dtype == FSP_F64 || (flags & FSP_PLAN_DIRECT) || !fast;
    if (p.direct && (p.n0 > DIRECT_MAX_N || p.n2 > DIRECT_MAX_N || (dim == 3 && p.n1 > DIRECT_MAX_N))) {
        delete handle;
        set_err(FSP_ERR_UNSUPPORTED_SIZE);
        return nullptr;
    }
    if (method == FSP_VGF) {
        double diag = 0.0;
        for (int a = 0; a < dim; ++a) diag += (p.n[a] * p.h[a]) * (p.n[a] * p.h[a]);
        p.L = (lambda > 0 ? lambda : 1.0) * std::sqrt(diag);
        for (int a = 0; a < dim; ++a) p.M[a] = oversample(p.n[a], p.h[a], p.L);
    } else {
        p.g0 = std::isnan(g0) ? he_g0(dim, p.h, method) : g0;
    }
    if (cudaGetDevice(&p.device) != cudaSuccess) {
        delete handle;
        set_err(FSP_ERR_CUDA);
        return nullptr;
    }
    if (!p.direct) {
        std::lock_guard<std::mutex> lk(g_prep_mutex);
        int e = prepare_axis0(2 * p.n0) | prepare_axis2(2 * p.n2) | (dim == 3 ? prepare_axis1(2 * p.n1) : 0);
        if (e) {
            delete handle;
            set_err(FSP_ERR_CUDA);
            return nullptr;
        }
    }
    int rc = FSP_OK;
    const int N0 = 2 * p.n0, N1 = 2 * p.n1, N2 = 2 * p.n2;
    if (p.direct) {
        const int Ns[3] = {N0, dim == 3 ? N1 : 0, N2};
        for (int a = 0; a < 3 && rc == FSP_OK; ++a)
            if (Ns[a] && cudaMalloc(&p.dtw[a], sizeof(double2) * Ns[a]) != cudaSuccess) rc = FSP_ERR_NOMEM;
    } else if (cudaMalloc(&p.tw0, sizeof(float2) * twiddle_entries(N0)) != cudaSuccess) {
        rc = FSP_ERR_NOMEM;
    }
    if (rc == FSP_OK && !p.direct) {
        if (dim == 3 && N1 != N0) {
            if (cudaMalloc(&p.tw1, sizeof(float2) * twiddle_entries(N1)) != cudaSuccess) rc = FSP_ERR_NOMEM;
        } else {
            p.tw1 = p.tw0;
        }
    }
    if (rc == FSP_OK && !p.direct) {
        if (N2 == N0) p.tw2 = p.tw0;
        else if (dim == 3 && N2 == N1) p.tw2 = p.tw1;
        else if (cudaMalloc(&p.tw2, sizeof(float2) * twiddle_entries(N2)) != cudaSuccess) rc = FSP_ERR_NOMEM;
    }
    p.K_count = (size_t)(p.n[0] + 1) * (p.n[1] + 1) * (dim == 3 ? (p.n[2] + 1) : 1);
    if (rc == FSP_OK && cudaMalloc(&p.K, sizeof(float) * p.K_count) != cudaSuccess) rc = FSP_ERR_NOMEM;
    if (rc == FSP_OK && dtype == FSP_F64 && cudaMalloc(&p.K64, sizeof(double) * p.K_count) != cudaSuccess)
        rc = FSP_ERR_NOMEM;
    if (rc == FSP_OK && cudaMalloc(&p.status, sizeof(int)) != cudaSuccess) rc = FSP_ERR_NOMEM;
    if (rc == FSP_OK && cudaMemset(p.status, 0, sizeof(int)) != cudaSuccess) rc = FSP_ERR_CUDA;
    cudaStream_t st = nullptr;
    if (rc == FSP_OK && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc == FSP_OK && p.direct) {
        for (int a = 0; a < 3 && rc == FSP_OK; ++a)
            if (p.dtw[a] && make_direct_twiddles(p.dtw[a], a == 0 ? N0 : a == 1 ? N1 : N2, st)) rc = FSP_ERR_CUDA;
    } else if (rc == FSP_OK) {
        auto fill = [&](float2 *t, int n) {
            return make_twiddles(t, n, st) || make_twiddles_aux(t, n, st) || make_twiddles_gall(t, n, st);
        };
        if (fill(p.tw0, N0)) rc = FSP_ERR_CUDA;
        if (rc == FSP_OK && p.tw1 != p.tw0 && fill(p.tw1, N1)) rc = FSP_ERR_CUDA;
        if (rc == FSP_OK && p.tw2 != p.tw0 && p.tw2 != p.tw1 && fill(p.tw2, N2)) rc = FSP_ERR_CUDA;
    }
    if (rc == FSP_OK) rc = build_kernel_spectrum(&p, st);
    if (st) cudaStreamDestroy(st);
    if (rc != FSP_OK) {
        plan_free(p);
        delete handle;
        set_err(rc);
        return nullptr;
    }
    p.buf_elems = (size_t)(p.n0 + 1) * p.rows1 * p.n2;
    set_err(FSP_OK);
    return handle;
}

extern "C" fsp_plan *fsp_plan_create(int nx, int ny, int nz, double hx, double hy, double hz, int method, int dtype)
{
    return fsp_plan_create_ex(nx, ny, nz, hx, hy, hz, method, dtype, 1.0, NAN, 0);
}

extern "C" void fsp_plan_destroy(fsp_plan *plan)
{
    if (!plan) return;
    plan_free(plan->p);
    delete plan;
}

extern "C" int fsp_plan_geometry(const fsp_plan *plan, int *dim, int *n, double *h, double *L, int *M)
{
    if (!plan) return set_err(FSP_ERR_INVALID);
    const Plan &p = plan->p;
    if (dim) *dim = p.dim;
    for (int a = 0; a < 3; ++a) {
        if (n) n[a] = p.n[a];
        if (h) h[a] = p.h[a];
        if (M) M[a] = p.M[a];
    }
    if (L) *L = p.L;
    return set_err(FSP_OK);
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Workspace of one solve: the two intermediate buffers (buf0, buf1) of the
// FFT passes, or the direct-sum path's regions.  A 2D solve without E (and a
// 2D adjoint without g_E) never touches buf1; in 3D the first pass writes
// buf1 whatever the outputs.
static size_t per_solve_bytes(const Plan &p, bool with_E)
{
    if (p.direct) return direct_workspace_bytes(p);
    return (p.three_d || with_E ? 2 : 1) * align_up(p.buf_elems * sizeof(float2), 256);
}

extern "C" size_t fsp_plan_workspace_bytes(const fsp_plan *plan, int with_E, int batch)
{
    if (!plan || batch < 1) return 0;
    return per_solve_bytes(plan->p, with_E != 0) * (size_t)batch;
}

extern "C" int fsp_plan_set_workspace(fsp_plan *plan, void *dev_ptr, size_t bytes)
{
    if (!plan || !dev_ptr || ((uintptr_t)dev_ptr % 256) != 0) return set_err(FSP_ERR_INVALID);
    if (bytes < per_solve_bytes(plan->p, false)) return set_err(FSP_ERR_WORKSPACE);
    plan->p.ws = dev_ptr;
    plan->p.ws_bytes = bytes;
    return set_err(FSP_OK);
}

extern "C" int fsp_plan_set_pass_events(fsp_plan *plan, void *const *events, int count)
{
    if (!plan || count < 0) return set_err(FSP_ERR_INVALID);
    Plan &p = plan->p;
    if (!events || count == 0) {
        p.n_pass_ev = 0;
        return set_err(FSP_OK);
    }
    const int need = p.three_d ? 6 : 4;
    if (p.direct || count < need || count > 8) return set_err(FSP_ERR_INVALID);   // direct plans have no passes
    for (int i = 0; i < count; ++i) {
        if (!events[i]) return set_err(FSP_ERR_INVALID);
        p.pass_ev[i] = (cudaEvent_t)events[i];
    }
    p.n_pass_ev = count;
    return set_err(FSP_OK);
}

extern "C" int fsp_plan_set_plane_group(fsp_plan *plan, int planes)
{
    if (!plan || planes < 0) return set_err(FSP_ERR_INVALID);
    plan->p.plane_group = planes;
    return set_err(FSP_OK);
}

extern "C" int fsp_plan_device_status(fsp_plan *plan, int clear)
{
    if (!plan || !plan->p.status) return set_err(FSP_ERR_INVALID);
    int v = 0;
    if (cudaMemcpy(&v, plan->p.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return set_err(FSP_ERR_CUDA);
    if (clear && v && cudaMemset(plan->p.status, 0, sizeof(int)) != cudaSuccess) return set_err(FSP_ERR_CUDA);
    return set_err(v);
}

extern "C" int fsp_plan_kernel_spectrum(const fsp_plan *plan, void *host_out, size_t bytes)
{
    if (!plan || !host_out) return set_err(FSP_ERR_INVALID);
    if (bytes < plan->p.K_count * sizeof(float)) return set_err(FSP_ERR_INVALID);
    if (cudaMemcpy(host_out, plan->p.K, plan->p.K_count * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return set_err(FSP_ERR_CUDA);
    return set_err(FSP_OK);
}

// ------------------------------------------------------------------- solves

static bool aligned16(const void *p) { return ((uintptr_t)p % 16) == 0; }

static PassArgs base_args(const Plan &p, void *ws)
{
    PassArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n0 = p.n0;
    a.n1 = p.n1;
    a.n2 = p.n2;
    a.rows1 = p.rows1;
    a.three_d = p.three_d;
    a.k0s = p.k0s;
    a.k1s = p.k1s;
    a.k2s = p.k2s;
    a.tw0 = p.tw0;
    a.tw1 = p.tw1;
    a.tw2 = p.tw2;
    a.K = p.K;
    a.status = p.status;
    a.kx0 = 0;
    a.kxn = p.n0 + 1;
    a.buf0 = reinterpret_cast<float2 *>(ws);
    a.buf1 = reinterpret_cast<float2 *>(reinterpret_cast<char *>(ws) + align_up(p.buf_elems * sizeof(float2), 256));
    return a;
}

static size_t cells(const Plan &p) { return (size_t)p.n0 * p.n1 * p.n2; }

namespace fsp {

static inline void mark(const Plan &p, int i, cudaStream_t st)
{
    if (p.n_pass_ev > i) cudaEventRecord(p.pass_ev[i], st);
}

static PassArgs fwd_args(const Plan &p, void *ws, const float *rho, float *phi, float *E)
{
    PassArgs a = base_args(p, ws);
    const size_t c = cells(p);
    a.in[0] = rho;
    a.out[0] = phi;
    if (E) {
        a.out[1] = E;
        a.out[2] = E + c;
        a.out[3] = p.three_d ? E + 2 * c : nullptr;
    }
    return a;
}

// Plane groups (3D): P2, P3 and P4 run group by group over the k0 planes, so
// that a group's intermediates can stay in L2 between the three passes.  Only
// where those passes are the single-solve kernels that take a plane range
// (TMA column tiles, warp-per-line middle pass: 2 n1, 2 n2 <= 512).
static bool plane_groups_apply(const Plan &p)
{
    return p.three_d && p.plane_group > 0 && p.plane_group < p.n0 + 1 && 2 * p.n1 <= 512 && 2 * p.n2 <= 512 &&
           !(tuned_variant(PASS_P2F, 2 * p.n1) & 4) && !(tuned_variant(PASS_P4F, 2 * p.n1) & 4);
}

// The ungrouped forward schedule, passes 1 .. last of the plan's pass list
// (3D: P1 .. P5; 2D: P1, P3, P5), with the pass events of the plan.
static int run_plain_passes(const Plan &p, const PassArgs &a, int withE, int last, cudaStream_t st)
{
    const int N0 = 2 * p.n0, N1 = 2 * p.n1, N2 = 2 * p.n2;
    int e = 0, m = 0, k = 0;   // k: passes run so far
    mark(p, m++, st);
    {
        Range r("P1 axis 0 pad + R2C");
        e = launch_axis0(PASS_P1F, N0, &a, 1, tuned_variant(PASS_P1F, N0), st);
        ++k;
    }
    mark(p, m++, st);
    if (!e && p.three_d && k < last) {
        Range r("P2 axis 1 forward");
        e = launch_axis1(PASS_P2F, N1, &a, 1, 0, tuned_variant(PASS_P2F, N1), st);
        ++k;
        mark(p, m++, st);
    }
    if (!e && k < last) {
        Range r("P3 axis 2 forward, kernel product, inverse");
        e = launch_axis2(PASS_P3F, N2, &a, 1, withE, tuned_variant(PASS_P3F, N2), st);
        ++k;
        mark(p, m++, st);
    }
    if (!e && p.three_d && k < last) {
        Range r("P4 axis 1 inverse + crop");
        e = launch_axis1(PASS_P4F, N1, &a, 1, withE, tuned_variant(PASS_P4F, N1), st);
        ++k;
        mark(p, m++, st);
    }
    if (!e && k < last) {
        Range r("P5 axis 0 C2R + crop");
        e = launch_axis0(PASS_P5F, N0, &a, 1, tuned_variant(PASS_P5F, N0), st);
        mark(p, m++, st);
    }
    return e ? FSP_ERR_CUDA : FSP_OK;
}

// Forward pipeline for one plan on its workspace `ws`.
int run_forward(const Plan &p, void *ws, const float *rho, float *phi, float *E, cudaStream_t st)
{
    Range range(p.direct ? "fsp solve (direct sums)" : "fsp solve");
    if (p.direct) return run_direct_forward(p, ws, rho, phi, E, st);   // buffers in the plan's precision
    PassArgs a = fwd_args(p, ws, rho, phi, E);
    const int withE = E != nullptr;
    const int N0 = 2 * p.n0, N1 = 2 * p.n1, N2 = 2 * p.n2;
    int e = 0, m = 0;
    if (plane_groups_apply(p)) {
        // pass events: before P1, after P1, then after the grouped P2-P4, after P5
        mark(p, m++, st);
        e = launch_axis0(PASS_P1F, N0, &a, 1, tuned_variant(PASS_P1F, N0), st);
        mark(p, m++, st);
        for (int k = 0; k <= p.n0 && !e; k += p.plane_group) {
            PassArgs g = a;
            g.kx0 = k;
            g.kxn = std::min(p.plane_group, p.n0 + 1 - k);
            e = launch_axis1(PASS_P2F, N1, &g, 1, 0, tuned_variant(PASS_P2F, N1), st);
            if (!e) e = launch_axis2(PASS_P3F, N2, &g, 1, withE, tuned_variant(PASS_P3F, N2), st);
            if (!e) e = launch_axis1(PASS_P4F, N1, &g, 1, withE, tuned_variant(PASS_P4F, N1), st);
        }
        mark(p, m++, st);
        mark(p, m++, st);
        mark(p, m++, st);
        if (!e) e = launch_axis0(PASS_P5F, N0, &a, 1, tuned_variant(PASS_P5F, N0), st);
        mark(p, m++, st);
        return e ? FSP_ERR_CUDA : FSP_OK;
    }
    return run_plain_passes(p, a, withE, p.three_d ? 5 : 3, st);
}

int run_adjoint(const Plan &p, void *ws, const float *g_phi, const float *g_E, float *g_rho, cudaStream_t st)
{
    Range range("fsp adjoint");
    if (p.direct) return run_direct_adjoint(p, ws, g_phi, g_E, g_rho, st);
    if (!g_E) return run_forward(p, ws, g_phi, g_rho, nullptr, st);   // A is symmetric
    PassArgs a = base_args(p, ws);
    const size_t c = cells(p);
    a.in[0] = g_phi;
    a.in[1] = g_E;
    a.in[2] = g_E + c;
    a.in[3] = p.three_d ? g_E + 2 * c : nullptr;
    const int N0 = 2 * p.n0, N1 = 2 * p.n1, N2 = 2 * p.n2;
    int m = 0;
    mark(p, m++, st);
    int e = launch_axis0(PASS_P1A, N0, &a, 1, 0, st);
    mark(p, m++, st);
    if (!e && p.three_d) {
        e = launch_axis1(PASS_P2A, N1, &a, 1, 1, 0, st);
        mark(p, m++, st);
    }
    if (!e) e = launch_axis2(PASS_P3A, N2, &a, 1, 1, tuned_variant(PASS_P3A, N2), st);
    mark(p, m++, st);
    if (!e && p.three_d) {
        e = launch_axis1(PASS_P4F, N1, &a, 1, 0, tuned_variant(PASS_P4F, N1), st);
        mark(p, m++, st);
    }
    if (!e) {
        PassArgs b = a;
        b.out[0] = g_rho;
        b.out[1] = b.out[2] = b.out[3] = nullptr;
        e = launch_axis0(PASS_P5F, N0, &b, 1, tuned_variant(PASS_P5F, N0), st);
    }
    mark(p, m++, st);
    return e ? FSP_ERR_CUDA : FSP_OK;
}

// One pass over many items: the items sharing a padded length go in one launch.
// Launches of the same stage (pass) are independent of each other.
struct PassLaunch {
    int kind, axis, N, flag, stage;
    std::vector<PassArgs> items;
};

static void group_pass(std::vector<PassLaunch> &out, int kind, int axis, int flag, const std::vector<PassArgs> &items,
                       const std::vector<int> &Ns, const std::vector<int> &use, int stage)
{
    std::vector<int> seen;
    for (size_t i = 0; i < items.size(); ++i) {
        if (!use[i] || std::find(seen.begin(), seen.end(), Ns[i]) != seen.end()) continue;
        seen.push_back(Ns[i]);
        PassLaunch L{kind, axis, Ns[i], flag, stage, {}};
        for (size_t k = i; k < items.size(); ++k)
            if (use[k] && Ns[k] == Ns[i]) L.items.push_back(items[k]);
        out.push_back(std::move(L));
    }
}

// Launch plan of a forward batch: P1 over all items, then P2 (3D items), P3,
// P4 (3D items), P5, each split by padded length only.
static std::vector<PassLaunch> batch_launches(const std::vector<const Plan *> &plans, const std::vector<PassArgs> &items,
                                              int withE)
{
    const size_t n = plans.size();
    std::vector<int> N0(n), N1(n), N2(n), all(n, 1), is3(n);
    for (size_t i = 0; i < n; ++i) {
        N0[i] = 2 * plans[i]->n0;
        N1[i] = 2 * plans[i]->n1;
        N2[i] = 2 * plans[i]->n2;
        is3[i] = plans[i]->three_d;
    }
    std::vector<PassLaunch> L;
    group_pass(L, PASS_P1F, 0, 0, items, N0, all, 0);
    group_pass(L, PASS_P2F, 1, 0, items, N1, is3, 1);
    group_pass(L, PASS_P3F, 2, withE, items, N2, all, 2);
    group_pass(L, PASS_P4F, 1, withE, items, N1, is3, 3);
    group_pass(L, PASS_P5F, 0, 0, items, N0, all, 4);
    return L;
}

// Batched launches keep the default variants: the tuning table is timed on
// single solves (whose column passes are the TMA-staged tiles) and does not
// carry over to the batched kernels.
static int launch_one(const PassLaunch &x, cudaStream_t st)
{
    const int n = (int)x.items.size();
    const int var = n == 1 ? tuned_variant(x.kind, x.N) : 0;
    const int e = x.axis == 0 ? launch_axis0(x.kind, x.N, x.items.data(), n, var, st)
                  : x.axis == 1 ? launch_axis1(x.kind, x.N, x.items.data(), n, x.flag, var, st)
                                : launch_axis2(x.kind, x.N, x.items.data(), n, x.flag, var, st);
    return e ? FSP_ERR_CUDA : FSP_OK;
}

// Streams and events that let the launches of one stage run side by side:
// the first launch of a stage goes on the caller's stream, the k-th on aux[k-1],
// forked from and joined back into the caller's stream by events (in a
// captured graph, parallel branches).
struct Fork {
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
};

static int run_launches(const std::vector<PassLaunch> &L, cudaStream_t st, const Fork *fk = nullptr)
{
    size_t i = 0;
    while (i < L.size()) {
        size_t end = i + 1;
        while (end < L.size() && L[end].stage == L[i].stage) ++end;
        const size_t width = end - i;
        if (!fk || width == 1 || fk->aux.size() + 1 < width) {
            for (; i < end; ++i)
                if (launch_one(L[i], st)) return FSP_ERR_CUDA;
            continue;
        }
        if (cudaEventRecord(fk->fork, st) != cudaSuccess) return FSP_ERR_CUDA;
        for (size_t k = 1; k < width; ++k) {
            cudaStream_t s = fk->aux[k - 1];
            if (cudaStreamWaitEvent(s, fk->fork, 0) != cudaSuccess || launch_one(L[i + k], s) ||
                cudaEventRecord(fk->join[k - 1], s) != cudaSuccess)
                return FSP_ERR_CUDA;
        }
        if (launch_one(L[i], st)) return FSP_ERR_CUDA;
        for (size_t k = 1; k < width; ++k)
            if (cudaStreamWaitEvent(st, fk->join[k - 1], 0) != cudaSuccess) return FSP_ERR_CUDA;
        i = end;
    }
    return FSP_OK;
}

} // namespace fsp

extern "C" int fsp_solve(fsp_plan *plan, const void *rho, void *phi, void *E, void *cuda_stream)
{
    if (!plan || !rho || (!phi && !E)) return set_err(FSP_ERR_INVALID);
    if (!aligned16(rho) || (phi && !aligned16(phi)) || (E && !aligned16(E))) return set_err(FSP_ERR_INVALID);
    const Plan &p = plan->p;
    if (!p.ws || p.ws_bytes < per_solve_bytes(p, E != nullptr)) return set_err(FSP_ERR_WORKSPACE);
    return set_err(run_forward(p, p.ws, (const float *)rho, (float *)phi, (float *)E, (cudaStream_t)cuda_stream));
}

// Test hooks: the first passes of a forward solve, and where their results sit.
extern "C" int fsp_plan_run_passes(fsp_plan *plan, const void *rho, int passes, int with_E, void *cuda_stream)
{
    if (!plan || !rho || !aligned16(rho)) return set_err(FSP_ERR_INVALID);
    const Plan &p = plan->p;
    if (p.direct || passes < 1 || passes >= (p.three_d ? 5 : 3)) return set_err(FSP_ERR_INVALID);
    if (!p.ws || p.ws_bytes < per_solve_bytes(p, with_E != 0)) return set_err(FSP_ERR_WORKSPACE);
    const PassArgs a = fwd_args(p, p.ws, (const float *)rho, nullptr, nullptr);
    return set_err(run_plain_passes(p, a, with_E != 0, passes, (cudaStream_t)cuda_stream));
}

extern "C" int fsp_plan_workspace_layout(const fsp_plan *plan, size_t *buf1_offset, int *dims)
{
    if (!plan || !buf1_offset || !dims || plan->p.direct) return set_err(FSP_ERR_INVALID);
    const Plan &p = plan->p;
    *buf1_offset = align_up(p.buf_elems * sizeof(float2), 256);
    dims[0] = p.n0 + 1;
    dims[1] = p.rows1;
    dims[2] = p.n2;
    return set_err(FSP_OK);
}

extern "C" int fsp_solve_adjoint(fsp_plan *plan, const void *g_phi, const void *g_E, void *g_rho, void *cuda_stream)
{
    if (!plan || !g_rho || (!g_phi && !g_E)) return set_err(FSP_ERR_INVALID);
    if ((g_phi && !aligned16(g_phi)) || (g_E && !aligned16(g_E)) || !aligned16(g_rho)) return set_err(FSP_ERR_INVALID);
    const Plan &p = plan->p;
    if (!p.ws || p.ws_bytes < per_solve_bytes(p, g_E != nullptr)) return set_err(FSP_ERR_WORKSPACE);
    return set_err(run_adjoint(p, p.ws, (const float *)g_phi, (const float *)g_E, (float *)g_rho,
                               (cudaStream_t)cuda_stream));
}

// ----------------------------------------------------------------- batches

// Direct-path items of a batch run one after another after the fast launches.
struct DirectJob {
    const Plan *p;
    const void *rho;
    void *phi, *E;
};

struct fsp_batch {
    std::vector<PassLaunch> launches;
    std::vector<DirectJob> direct;
    Fork fork;   // prebuilt batches run the launches of a stage side by side
    ~fsp_batch()
    {
        for (cudaStream_t s : fork.aux) cudaStreamDestroy(s);
        for (cudaEvent_t e : fork.join) cudaEventDestroy(e);
        if (fork.fork) cudaEventDestroy(fork.fork);
    }
};

// Streams for the widest stage of a prebuilt batch (set-up, not a solve).
static int make_fork(fsp_batch &b)
{
    size_t widest = 1;
    for (size_t i = 0; i < b.launches.size();) {
        size_t end = i + 1;
        while (end < b.launches.size() && b.launches[end].stage == b.launches[i].stage) ++end;
        widest = std::max(widest, end - i);
        i = end;
    }
    if (widest == 1) return FSP_OK;
    if (cudaEventCreateWithFlags(&b.fork.fork, cudaEventDisableTiming) != cudaSuccess) return FSP_ERR_CUDA;
    for (size_t k = 1; k < widest; ++k) {
        cudaStream_t s = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return FSP_ERR_CUDA;
        b.fork.aux.push_back(s);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return FSP_ERR_CUDA;
        b.fork.join.push_back(e);
    }
    return FSP_OK;
}

static int check_batch(fsp_plan *const *plans, int count, const void *const *rho, void *const *phi, void *const *E)
{
    if (!plans || count < 1 || !rho || (!phi && !E)) return FSP_ERR_INVALID;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !rho[i] || !aligned16(rho[i])) return FSP_ERR_INVALID;
        if (!(phi && phi[i]) && !(E && E[i])) return FSP_ERR_INVALID;
        if (E && !E[i]) return FSP_ERR_INVALID;   // with_E must hold for every item
        if ((phi && phi[i] && !aligned16(phi[i])) || (E && E[i] && !aligned16(E[i]))) return FSP_ERR_INVALID;
        const Plan &p = plans[i]->p;
        if (!p.ws || p.ws_bytes < per_solve_bytes(p, E != nullptr)) return FSP_ERR_WORKSPACE;
        for (int k = 0; k < i; ++k)
            if (plans[k] == plans[i]) return FSP_ERR_INVALID;
    }
    return FSP_OK;
}

static void plan_batch(fsp_batch &b, fsp_plan *const *plans, int count, const void *const *rho, void *const *phi,
                       void *const *E)
{
    std::vector<const Plan *> ps;
    std::vector<PassArgs> items;
    for (int i = 0; i < count; ++i) {
        const Plan &p = plans[i]->p;
        if (p.direct) {
            b.direct.push_back({&p, rho[i], phi ? phi[i] : nullptr, E ? E[i] : nullptr});
            continue;
        }
        ps.push_back(&p);
        items.push_back(fwd_args(p, p.ws, (const float *)rho[i], phi ? (float *)phi[i] : nullptr,
                                 E ? (float *)E[i] : nullptr));
    }
    if (!items.empty()) b.launches = batch_launches(ps, items, E != nullptr);
}

static int run_batch(const fsp_batch &b, cudaStream_t st)
{
    Range range("fsp batch");
    int rc = run_launches(b.launches, st, b.fork.aux.empty() ? nullptr : &b.fork);
    for (size_t i = 0; i < b.direct.size() && rc == FSP_OK; ++i) {
        const DirectJob &d = b.direct[i];
        rc = run_direct_forward(*d.p, d.p->ws, d.rho, d.phi, d.E, st);
    }
    return rc;
}

extern "C" int fsp_solve_batched(fsp_plan *const *plans, int count, const void *const *rho, void *const *phi,
                                 void *const *E, void *cuda_stream)
{
    int rc = check_batch(plans, count, rho, phi, E);
    if (rc) return set_err(rc);
    fsp_batch b;
    plan_batch(b, plans, count, rho, phi, E);
    return set_err(run_batch(b, (cudaStream_t)cuda_stream));
}

extern "C" fsp_batch *fsp_batch_create(fsp_plan *const *plans, int count, const void *const *rho, void *const *phi,
                                       void *const *E)
{
    int rc = check_batch(plans, count, rho, phi, E);
    if (rc) {
        set_err(rc);
        return nullptr;
    }
    fsp_batch *b = inject_fault("alloc") ? nullptr : new (std::nothrow) fsp_batch();
    if (!b) {
        set_err(FSP_ERR_NOMEM);
        return nullptr;
    }
    plan_batch(*b, plans, count, rho, phi, E);
    rc = make_fork(*b);
    if (rc) {
        delete b;
        set_err(rc);
        return nullptr;
    }
    set_err(FSP_OK);
    return b;
}

extern "C" int fsp_batch_solve(fsp_batch *b, void *cuda_stream)
{
    if (!b) return set_err(FSP_ERR_INVALID);
    return set_err(run_batch(*b, (cudaStream_t)cuda_stream));
}

extern "C" void fsp_batch_destroy(fsp_batch *b) { delete b; }

// Kernels one fsp_batch_solve launches: the solve is captured once on a
// private stream into a graph whose kernel nodes are counted (nothing runs).
extern "C" int fsp_batch_kernel_count(fsp_batch *b, int *count)
{
    if (!b || !count) return set_err(FSP_ERR_INVALID);
    cudaStream_t s = nullptr;
    cudaGraph_t g = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return set_err(FSP_ERR_CUDA);
    int rc = FSP_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc == FSP_OK) {
        const int r = run_batch(*b, s);
        if (cudaStreamEndCapture(s, &g) != cudaSuccess || r != FSP_OK) rc = r != FSP_OK ? r : FSP_ERR_CUDA;
    }
    size_t n = 0;
    if (rc == FSP_OK && cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) rc = FSP_ERR_CUDA;
    std::vector<cudaGraphNode_t> nodes(n);
    if (rc == FSP_OK && n && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) rc = FSP_ERR_CUDA;
    int k = 0;
    for (size_t i = 0; i < n && rc == FSP_OK; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) rc = FSP_ERR_CUDA;
        else if (t == cudaGraphNodeTypeKernel) ++k;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(s);
    if (rc == FSP_OK) *count = k;
    return set_err(rc);
}
