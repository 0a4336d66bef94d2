// fsp_fd.cu -- E = -grad(phi) by centred finite differences (the variant the
// paper compares with Fourier differentiation for HE, Sec. 3): interior points
// use (phi[i+1] - phi[i-1]) / (2 h); the first and last cells of each axis use
// the second-order one-sided differences (-3 phi0 + 4 phi1 - phi2) / (2 h) and
// (3 phi[n-1] - 4 phi[n-2] + phi[n-3]) / (2 h).  A memory-bound stencil: phi
// is read once from DRAM (its neighbour rows come from L2) and the field is
// written once.  FP32 grids whose contiguous axis is a multiple of 4 take the
// vector kernel: each thread owns 4 consecutive cells of a row (float4 loads
// and stores), 32-bit indices; other grids take the scalar kernel.
#include "fsp_internal.h"

#include <algorithm>
#include <cstdint>

namespace {

template <class R>
__device__ __forceinline__ R deriv(const R *__restrict__ phi, size_t c, int i, int n, size_t stride, R inv2h)
{
    if (n < 3) return R(0);
    if (i == 0) return (R(-3) * phi[c] + R(4) * phi[c + stride] - phi[c + 2 * stride]) * inv2h;
    if (i == n - 1) return (R(3) * phi[c] - R(4) * phi[c - stride] + phi[c - 2 * stride]) * inv2h;
    return (phi[c + stride] - phi[c - stride]) * inv2h;
}

template <class R>
__global__ void k_fd_gradient(const R *__restrict__ phi, R *__restrict__ E, int n0, int n1, int n2, int dim, R i0,
                              R i1, R i2)
{
    const size_t cells = (size_t)n0 * n1 * n2;
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < cells; c += (size_t)gridDim.x * blockDim.x) {
        const int z = (int)(c % n2);
        const size_t xy = c / n2;
        const int y = (int)(xy % n1), x = (int)(xy / n1);
        E[c] = -deriv(phi, c, x, n0, (size_t)n1 * n2, i0);
        if (dim == 3) {
            E[cells + c] = -deriv(phi, c, y, n1, (size_t)n2, i1);
            E[2 * cells + c] = -deriv(phi, c, z, n2, 1, i2);
        } else {
            E[cells + c] = -deriv(phi, c, z, n2, 1, i2);
        }
    }
}

// One-sided or centred difference at position i of an axis of n cells for the
// four cells held in c (the same expressions as deriv(), lane by lane); m1,
// p1 are the neighbours at -1 and +1, m2 and p2 at -2 and +2 (read only at
// the faces).
__device__ __forceinline__ float fd1(float m2, float m1, float c, float p1, float p2, int i, int n, float inv2h)
{
    if (n < 3) return 0.f;
    if (i == 0) return (-3.f * c + 4.f * p1 - p2) * inv2h;
    if (i == n - 1) return (3.f * c - 4.f * m1 + m2) * inv2h;
    return (p1 - m1) * inv2h;
}

__device__ __forceinline__ float4 ld4(const float *p, unsigned i) { return __ldg(reinterpret_cast<const float4 *>(p) + i); }

// Derivative along an outer axis (stride in float4 units) of the 4 cells at
// float4 index q of position i of n.
__device__ __forceinline__ float4 outer4(const float *__restrict__ phi, unsigned q, unsigned s, int i, int n, float4 c,
                                         float inv2h)
{
    if (n < 3) return make_float4(0.f, 0.f, 0.f, 0.f);
    float4 m1 = c, p1 = c, m2 = c, p2 = c;
    if (i > 0) m1 = ld4(phi, q - s);
    if (i < n - 1) p1 = ld4(phi, q + s);
    if (i == 0) p2 = ld4(phi, q + 2 * s);
    if (i == n - 1) m2 = ld4(phi, q - 2 * s);
    return make_float4(-fd1(m2.x, m1.x, c.x, p1.x, p2.x, i, n, inv2h), -fd1(m2.y, m1.y, c.y, p1.y, p2.y, i, n, inv2h),
                       -fd1(m2.z, m1.z, c.z, p1.z, p2.z, i, n, inv2h), -fd1(m2.w, m1.w, c.w, p1.w, p2.w, i, n, inv2h));
}

// FP32, n2 % 4 == 0: thread = 4 consecutive cells of one (x, y) row.
__global__ void k_fd_gradient4(const float *__restrict__ phi, float *__restrict__ E, int n0, int n1, int n2, int dim,
                               float i0, float i1, float i2)
{
    const unsigned nq = (unsigned)n2 / 4, rows = (unsigned)n0 * (unsigned)n1, total = rows * nq;
    const size_t cells = (size_t)rows * n2;
    float4 *E0 = reinterpret_cast<float4 *>(E);
    float4 *E1 = reinterpret_cast<float4 *>(E + cells);
    float4 *E2 = reinterpret_cast<float4 *>(E + 2 * cells);
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const unsigned row = t / nq, qz = t - row * nq;
        const unsigned x = row / (unsigned)n1, y = row - x * (unsigned)n1;
        const float4 c = ld4(phi, t);
        E0[t] = outer4(phi, t, (unsigned)n1 * nq, (int)x, n0, c, i0);
        // along the contiguous axis: the cell before and the one after this float4
        const int z = 4 * (int)qz;
        const float m = qz > 0 ? __ldg(phi + 4 * t - 1) : c.x;
        const float p = qz + 1 < nq ? __ldg(phi + 4 * t + 4) : c.w;
        float4 ez;
        ez.x = -fd1(0.f, m, c.x, c.y, c.z, z, n2, i2);
        ez.y = -fd1(c.x, c.x, c.y, c.z, c.w, z + 1, n2, i2);   // z + 1 is a face only if n2 == 2 (excluded: n2 % 4 == 0)
        ez.z = -fd1(c.y, c.y, c.z, c.w, p, z + 2, n2, i2);
        ez.w = -fd1(c.y, c.z, c.w, p, 0.f, z + 3, n2, i2);
        if (dim == 3) {
            E1[t] = outer4(phi, t, nq, (int)y, n1, c, i1);
            E2[t] = ez;
        } else {
            E1[t] = ez;
        }
    }
}

} // namespace

extern "C" int fsp_gradient_fd(const fsp_plan *plan, const void *phi, void *E, void *cuda_stream)
{
    if (!plan || !phi || !E) return fsp::record_error(FSP_ERR_INVALID);
    if (((uintptr_t)phi % 16) || ((uintptr_t)E % 16)) return fsp::record_error(FSP_ERR_INVALID);
    const fsp::Plan &p = plan->p;
    const double i0 = 0.5 / p.h[0];
    const double i1 = p.dim == 3 ? 0.5 / p.h[1] : 0.0;
    const double i2 = 0.5 / (p.dim == 3 ? p.h[2] : p.h[1]);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (p.dtype == FSP_F32 && p.n2 % 4 == 0) {
        const unsigned total = (unsigned)p.n0 * p.n1 * (p.n2 / 4);
        const int grid = (int)std::min<unsigned>((total + 255) / 256, (unsigned)sms * 8);
        k_fd_gradient4<<<grid, 256, 0, st>>>((const float *)phi, (float *)E, p.n0, p.n1, p.n2, p.dim, (float)i0,
                                             (float)i1, (float)i2);
    } else if (p.dtype == FSP_F64)
        k_fd_gradient<double><<<sms * 8, 256, 0, st>>>((const double *)phi, (double *)E, p.n0, p.n1, p.n2, p.dim, i0,
                                                       i1, i2);
    else
        k_fd_gradient<float><<<sms * 8, 256, 0, st>>>((const float *)phi, (float *)E, p.n0, p.n1, p.n2, p.dim,
                                                      (float)i0, (float)i1, (float)i2);
    return fsp::record_error(cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA);
}
