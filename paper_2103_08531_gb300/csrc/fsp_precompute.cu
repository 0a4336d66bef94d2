// fsp_precompute.cu -- once-per-geometry kernel spectrum in FP64 on the device.
//
// The hot path multiplies by K(k) = prod(h)/prod(2n) * DFT_2n(g)(k), the kernel
// g being real and even, so K is real and even in every index and only the
// octant k_a in [0, n_a] is stored (FP32).
//
// HE (paper Sec. 1): g_j = G(|j h|) for j != 0 and g_0 = G(0) replacement.  By
// evenness DFT_2n(g)(k) = sum_{j in octant} prod_a c_{j_a} cos(pi k_a j_a / n_a) g_j,
// c = 1 at j = 0 and j = n (the unpaired offset -n carries g(n)), 2 otherwise.
//
// VGF (paper Sec. 2, last paragraph): g is the inverse DFT on an oversampled
// grid of M_a points, spacing h_a, of F{G^L}(k_m) (Eqs. GLFourier2D/3D),
// restricted to offsets |j_a| <= n_a:
//     g_j = (1/prod(M h)) sum_{m in octant} prod_a w_{m_a} cos(2 pi m_a j_a / M_a) Ghat_m,
// w = 1 at m = 0 and m = M/2, 2 otherwise (F{G^L} is even).  Both sums are
// separable, so per axis the two cosine sums fold into one matrix
//     P_a[k][m] = sum_j c_j w_m cos(pi k j / n_a) cos(2 pi m j / M_a)
// and K = (1 / prod(2 n_a M_a)) (P_0 x P_1 x P_2) Ghat: three contractions over
// the oversampled octant instead of an FFT of the whole (M_a)^d grid.  Axes are
// contracted in order of decreasing shrink ratio (M_a/2+1)/(n_a+1).
//
// Each P entry is evaluated in closed form, not as an (n+1)-term sum: with the
// weights c the j-sum runs over j in [-n, n) (the term at -n equals the one at
// n), the product of cosines splits into cos((a+b) j) + cos((a-b) j), and
//     sum_{j=-n}^{n-1} cos(j t) = sin(n t) cot(t / 2)      (2n where t = 0 mod 2 pi).
// With a = pi k / n and b = 2 pi m / M the angles are pi r / (n M) for the
// integers r = k M +- 2 m n, so every sine is taken of an argument reduced
// exactly in integer arithmetic.
#include "fsp_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace fsp {

// --------------------------------------------------------------- twiddles

__global__ void k_twiddles(float2 *tw, int N)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);   // FP64 angle, rounded once
    tw[m] = make_float2((float)c, (float)-s);
}

int make_twiddles(float2 *tw, int N, cudaStream_t st)
{
    k_twiddles<<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// FP64 table for the direct-sum path: (cos, sin) of 2 pi m / N.
__global__ void k_direct_twiddles(double2 *tw, int N)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)N, &s, &c);
    tw[m] = make_double2(c, s);
}

int make_direct_twiddles(double2 *tw, int N, cudaStream_t st)
{
    k_direct_twiddles<<<(N + 255) / 256, 256, 0, st>>>(tw, N);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ---------------------------------------------------------- axis matrices

// cos(pi a / b) for integers, argument reduced exactly first.
__device__ __forceinline__ double cospi_ratio(long long a, long long b)
{
    long long r = a % (2 * b);
    return cospi((double)r / (double)b);
}

// Q[k][j] = c_j cos(pi k j / n), k, j in [0, n]
__global__ void k_matrix_he(double *Q, int n)
{
    int k = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n || k > n) return;
    double c = (j == 0 || j == n) ? 1.0 : 2.0;
    Q[(size_t)k * (n + 1) + j] = c * cospi_ratio((long long)k * j, n);
}

// sin(pi a / b) for integers, b > 0: a reduced exactly to [0, b/2] first, so
// the double argument of sinpi lies in [0, 1/2] and keeps its relative accuracy.
__device__ __forceinline__ double sinpi_ratio(long long a, long long b)
{
    long long r = a % (2 * b);
    if (r < 0) r += 2 * b;
    double sgn = 1.0;
    if (r >= b) {           // sin(pi + x) = -sin(x)
        r -= b;
        sgn = -1.0;
    }
    if (2 * r > b) r = b - r;   // sin(pi - x) = sin(x)
    return sgn * sinpi((double)r / (double)b);
}

// sum_{j=-n}^{n-1} cos(pi r j / (n M)) = sin(pi r / M) cot(pi r / (2 n M)),
// and 2n where r is a multiple of 2 n M; the cosine of the cotangent is taken
// as sin(pi (n M - r) / (2 n M)).
__device__ __forceinline__ double cos_sum_sym(long long r, long long n, long long M)
{
    const long long D = n * M;
    if (r % (2 * D) == 0) return 2.0 * (double)n;
    return sinpi_ratio(r, M) * sinpi_ratio(D - r, 2 * D) / sinpi_ratio(r, 2 * D);
}

// P[k][m] = w_m sum_j c_j cos(pi k j / n) cos(2 pi m j / M), k in [0,n], m in [0, M/2]
__global__ void k_matrix_vgf(double *P, int n, int M)
{
    int k = blockIdx.y, m = blockIdx.x * blockDim.x + threadIdx.x;
    int mh = M / 2 + 1;
    if (m >= mh || k > n) return;
    const long long a = (long long)k * M, b = 2LL * m * n;
    const double s = 0.5 * (cos_sum_sym(a + b, n, M) + cos_sum_sym(a - b, n, M));
    double w = (m == 0 || 2 * m == M) ? 1.0 : 2.0;
    P[(size_t)k * mh + m] = w * s;
}

// ----------------------------------------------------- values on the octants

struct Axis3 {
    int d;
    int ext[3];      // extents of the octant array
    double step[3];  // spacing of the sampled coordinate (h_a or 2 pi / (M_a h_a))
};

// F{G^L}(|k|) of Eqs. GLFourier3D / GLFourier2D with the k -> 0 limits.
__device__ double ghat_truncated(int d, double L, double k)
{
    if (d == 3) {
        if (k == 0.0) return 0.5 * L * L;
        double s = sin(0.5 * L * k) / k;
        return 2.0 * s * s;
    }
    double x = L * k;
    if (x < 1e-3) {
        double x2 = x * x;
        return L * L * (0.25 - x2 / 64.0) - L * log(L) * L * (0.5 - x2 / 16.0);
    }
    return (1.0 - j0(x)) / (k * k) - L * log(L) * j1(x) / k;
}

__global__ void k_fill_vgf(double *out, Axis3 ax, double L)
{
    size_t total = (size_t)ax.ext[0] * ax.ext[1] * (ax.d == 3 ? ax.ext[2] : 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        size_t rem = i;
        double k2 = 0.0;
        for (int a = ax.d - 1; a >= 0; --a) {
            int m = (int)(rem % ax.ext[a]);
            rem /= ax.ext[a];
            double k = ax.step[a] * m;
            k2 += k * k;
        }
        out[i] = ghat_truncated(ax.d, L, sqrt(k2));
    }
}

__global__ void k_fill_he(double *out, Axis3 ax, double g0)
{
    size_t total = (size_t)ax.ext[0] * ax.ext[1] * (ax.d == 3 ? ax.ext[2] : 1);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        size_t rem = i;
        double r2 = 0.0;
        for (int a = ax.d - 1; a >= 0; --a) {
            int j = (int)(rem % ax.ext[a]);
            rem /= ax.ext[a];
            double x = ax.step[a] * j;
            r2 += x * x;
        }
        double g;
        if (r2 == 0.0) g = g0;
        else if (ax.d == 3) g = 1.0 / (4.0 * M_PI * sqrt(r2));
        else g = -0.5 * log(r2) / (2.0 * M_PI);
        out[i] = g;
    }
}

// ------------------------------------------------------- strided FP64 GEMM
// C(b, r, c) = sum_m A(b, r, m) B(b, m, c), element (i, j, k) of X at
// X[i sX0 + j sX1 + k sX2].  64 x 64 tiles, 16 x 16 threads, 4 x 4 per thread.

struct GemmDesc {
    const double *A;
    const double *B;
    double *C;
    long long sA0, sA1, sA2, sB0, sB1, sB2, sC0, sC1, sC2;
    int R, Cc, Mm;
};

__global__ void __launch_bounds__(256) k_gemm64(GemmDesc g)
{
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int b = blockIdx.z;
    const int r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int m0 = 0; m0 < g.Mm; m0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int rr = e / 16, mm = e % 16;
            int r = r0 + rr, m = m0 + mm;
            As[mm][rr] = (r < g.R && m < g.Mm) ? g.A[b * g.sA0 + r * g.sA1 + m * g.sA2] : 0.0;
            int cc = e % 64, mb = e / 64;
            int c = c0 + cc, m2 = m0 + mb;
            Bs[mb][cc] = (c < g.Cc && m2 < g.Mm) ? g.B[b * g.sB0 + m2 * g.sB1 + c * g.sB2] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int mm = 0; mm < 16; ++mm) {
            double a[4], bb[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[mm][ty + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i) bb[i] = Bs[mm][tx + 16 * i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[i][k] = fma(a[i], bb[k], acc[i][k]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int r = r0 + ty + 16 * i, c = c0 + tx + 16 * k;
            if (r < g.R && c < g.Cc) g.C[b * g.sC0 + r * g.sC1 + c * g.sC2] = acc[i][k];
        }
}

static int gemm(const GemmDesc &g, int batch, cudaStream_t st)
{
    dim3 grid((g.Cc + 63) / 64, (g.R + 63) / 64, batch);
    k_gemm64<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// Contract axis `ax` of the d-dim array `in` (extents ext) with Mat[p][m]
// (p < pout, m < ext[ax]): out has extents ext with ext[ax] -> pout.
static int contract_axis(const double *in, double *out, const double *Mat, int d, const int *ext, int ax, int pout,
                         cudaStream_t st)
{
    long long O = 1, I = 1;
    for (int a = 0; a < ax; ++a) O *= ext[a];
    for (int a = ax + 1; a < d; ++a) I *= ext[a];
    const int Min = ext[ax];
    GemmDesc g{};
    if (I == 1) {
        // out[o][p] = sum_m in[o][m] Mat[p][m]
        g.A = in; g.sA0 = 0; g.sA1 = Min; g.sA2 = 1;
        g.B = Mat; g.sB0 = 0; g.sB1 = 1; g.sB2 = Min;
        g.C = out; g.sC0 = 0; g.sC1 = pout; g.sC2 = 1;
        g.R = (int)O; g.Cc = pout; g.Mm = Min;
        return gemm(g, 1, st);
    }
    // out[o][p][i] = sum_m Mat[p][m] in[o][m][i], batched over o
    g.A = Mat; g.sA0 = 0; g.sA1 = Min; g.sA2 = 1;
    g.B = in; g.sB0 = (long long)Min * I; g.sB1 = I; g.sB2 = 1;
    g.C = out; g.sC0 = (long long)pout * I; g.sC1 = I; g.sC2 = 1;
    g.R = pout; g.Cc = (int)I; g.Mm = Min;
    // grid.z is limited to 65535: split the batch if needed
    for (long long o0 = 0; o0 < O; o0 += 65535) {
        int nb = (int)std::min<long long>(65535, O - o0);
        GemmDesc gg = g;
        gg.B = in + o0 * g.sB0;
        gg.C = out + o0 * g.sC0;
        if (gemm(gg, nb, st)) return -1;
    }
    return 0;
}

__global__ void k_scale_to_f32(const double *src, float *dst, size_t n, double s)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (float)(src[i] * s);
}

__global__ void k_scale_f64(const double *src, double *dst, size_t n, double s)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i] * s;
}

// ------------------------------------------------------------------ driver

// Builds the FP32 octant K into plan->K (device), and the FP64 one into
// plan->K64 when that is allocated.  Returns an fsp_status.
int build_kernel_spectrum(Plan *p, cudaStream_t st)
{
    const int d = p->dim;
    int n[3], M[3] = {0, 0, 0};
    double h[3];
    for (int a = 0; a < d; ++a) {
        n[a] = p->n[a];
        h[a] = p->h[a];
        M[a] = p->M[a];
    }
    const bool vgf = p->method == FSP_VGF;
    int ext[3];
    Axis3 ax{};
    ax.d = d;
    double scale = 1.0;
    for (int a = 0; a < d; ++a) {
        ext[a] = vgf ? M[a] / 2 + 1 : n[a] + 1;
        ax.ext[a] = ext[a];
        ax.step[a] = vgf ? 2.0 * M_PI / (M[a] * h[a]) : h[a];
        scale *= vgf ? 1.0 / (2.0 * n[a] * (double)M[a]) : h[a] / (2.0 * n[a]);
    }
    size_t cur = 1, maxsz = 1;
    for (int a = 0; a < d; ++a) cur *= ext[a];
    maxsz = cur;
    // contraction order: largest shrink first
    int order[3] = {0, 1, 2};
    std::sort(order, order + d, [&](int x, int y) {
        return (double)ext[x] / (n[x] + 1) > (double)ext[y] / (n[y] + 1);
    });
    {
        int e2[3] = {ext[0], ext[1], ext[2]};
        size_t s = cur;
        for (int i = 0; i < d; ++i) {
            int a = order[i];
            s = s / e2[a] * (n[a] + 1);
            e2[a] = n[a] + 1;
            maxsz = std::max(maxsz, s);
        }
    }
    double *bufA = nullptr, *bufB = nullptr, *mats[3] = {nullptr, nullptr, nullptr};
    int rc = FSP_OK;
    if (cudaMalloc(&bufA, maxsz * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&bufB, maxsz * sizeof(double)) != cudaSuccess)
        rc = FSP_ERR_NOMEM;
    for (int a = 0; a < d && rc == FSP_OK; ++a) {
        size_t msz = (size_t)(n[a] + 1) * ext[a];
        if (cudaMalloc(&mats[a], msz * sizeof(double)) != cudaSuccess) {
            rc = FSP_ERR_NOMEM;
            break;
        }
        dim3 grid((ext[a] + 127) / 128, n[a] + 1);
        if (vgf) k_matrix_vgf<<<grid, 128, 0, st>>>(mats[a], n[a], M[a]);
        else k_matrix_he<<<grid, 128, 0, st>>>(mats[a], n[a]);
    }
    if (rc == FSP_OK) {
        if (vgf) k_fill_vgf<<<4096, 256, 0, st>>>(bufA, ax, p->L);
        else k_fill_he<<<4096, 256, 0, st>>>(bufA, ax, p->g0);
        int e[3] = {ext[0], ext[1], ext[2]};
        double *src = bufA, *dst = bufB;
        for (int i = 0; i < d && rc == FSP_OK; ++i) {
            int a = order[i];
            if (contract_axis(src, dst, mats[a], d, e, a, n[a] + 1, st)) rc = FSP_ERR_CUDA;
            e[a] = n[a] + 1;
            std::swap(src, dst);
        }
        if (rc == FSP_OK) {
            size_t oct = 1;
            for (int a = 0; a < d; ++a) oct *= (size_t)(n[a] + 1);
            k_scale_to_f32<<<1024, 256, 0, st>>>(src, p->K, oct, scale);
            if (p->K64) k_scale_f64<<<1024, 256, 0, st>>>(src, p->K64, oct, scale);
        }
    }
    if (rc == FSP_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = FSP_ERR_CUDA;
    if (rc == FSP_OK && cudaGetLastError() != cudaSuccess) rc = FSP_ERR_CUDA;
    cudaFree(bufA);
    cudaFree(bufB);
    for (int a = 0; a < 3; ++a) cudaFree(mats[a]);
    return rc;
}

} // namespace fsp
