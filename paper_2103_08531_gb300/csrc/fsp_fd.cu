// fsp_fd.cu -- E = -grad(phi) by centred finite differences (the variant the
// paper compares with Fourier differentiation for HE, Sec. 3): interior points
// use (phi[i+1] - phi[i-1]) / (2 h); the first and last cells of each axis use
// the second-order one-sided differences (-3 phi0 + 4 phi1 - phi2) / (2 h) and
// (3 phi[n-1] - 4 phi[n-2] + phi[n-3]) / (2 h).  A memory-bound stencil: one
// thread per cell along the contiguous axis, neighbours read through L1/L2.
#include "fsp_internal.h"

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

} // namespace

extern "C" int fsp_gradient_fd(const fsp_plan *plan, const void *phi, void *E, void *cuda_stream)
{
    if (!plan || !phi || !E) return FSP_ERR_INVALID;
    if (((uintptr_t)phi % 16) || ((uintptr_t)E % 16)) return FSP_ERR_INVALID;
    const fsp::Plan &p = plan->p;
    const double i0 = 0.5 / p.h[0];
    const double i1 = p.dim == 3 ? 0.5 / p.h[1] : 0.0;
    const double i2 = 0.5 / (p.dim == 3 ? p.h[2] : p.h[1]);
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (p.dtype == FSP_F64)
        k_fd_gradient<double><<<sms * 8, 256, 0, st>>>((const double *)phi, (double *)E, p.n0, p.n1, p.n2, p.dim, i0,
                                                       i1, i2);
    else
        k_fd_gradient<float><<<sms * 8, 256, 0, st>>>((const float *)phi, (float *)E, p.n0, p.n1, p.n2, p.dim,
                                                      (float)i0, (float)i1, (float)i2);
    return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}
