// fsp_axis0.cu -- launchers of the axis-0 passes (P1 real -> half spectrum, P5 back).
#include "fsp_internal.h"
#include "fsp_passes.cuh"

namespace fsp {

#define FSP_AXIS0_SIZES(X) X(64) X(128) X(192) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

int supported_axis0(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS0_SIZES(X)
#undef X
    default: return 0;
    }
}

template <int N>
static int prep()
{
    using C = ColCfg<N>;
    int e = 0;
    e |= cudaFuncSetAttribute(p1_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    e |= cudaFuncSetAttribute(p1_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    e |= cudaFuncSetAttribute(p5_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    return e;
}

int prepare_axis0(int N)
{
    switch (N) {
#define X(n) case n: return prep<n>();
        FSP_AXIS0_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

template <int N>
static int p1f(const PassArgs &a, float2 *dst, cudaStream_t st)
{
    using C = ColCfg<N>;
    dim3 grid((a.n2 / 2 + C::BZ - 1) / C::BZ, a.n1);
    p1_fwd<N><<<grid, C::THREADS, C::SMEM, st>>>(a, dst);
    return (int)cudaGetLastError();
}

template <int N>
static int p1a(const PassArgs &a, cudaStream_t st)
{
    using C = ColCfg<N>;
    dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n1);
    p1_adj<N><<<grid, C::THREADS, C::SMEM, st>>>(a);
    return (int)cudaGetLastError();
}

template <int N>
static int p5f(const PassArgs &a, cudaStream_t st)
{
    using C = ColCfg<N>;
    dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n1);
    p5_fwd<N><<<grid, C::THREADS, C::SMEM, st>>>(a);
    return (int)cudaGetLastError();
}

int launch_p1_fwd(int N, const PassArgs &a, float2 *dst, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p1f<n>(a, dst, st);
        FSP_AXIS0_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_p1_adj(int N, const PassArgs &a, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p1a<n>(a, st);
        FSP_AXIS0_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_p5_fwd(int N, const PassArgs &a, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p5f<n>(a, st);
        FSP_AXIS0_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

} // namespace fsp
