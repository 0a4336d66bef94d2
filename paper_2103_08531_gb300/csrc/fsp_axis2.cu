// fsp_axis2.cu -- launchers of the axis-2 middle pass (P3: forward, kernel multiply, inverse).
#include "fsp_internal.h"
#include "fsp_passes.cuh"

namespace fsp {

#define FSP_AXIS2_SIZES(X) X(64) X(128) X(192) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

int supported_axis2(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS2_SIZES(X)
#undef X
    default: return 0;
    }
}

template <int N>
static int prep()
{
    using C = RowCfg<N>;
    int e = 0;
    e |= cudaFuncSetAttribute(p3_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    e |= cudaFuncSetAttribute(p3_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    return e;
}

int prepare_axis2(int N)
{
    switch (N) {
#define X(n) case n: return prep<n>();
        FSP_AXIS2_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

template <int N>
static int p3f(const PassArgs &a, int withE, cudaStream_t st)
{
    using C = RowCfg<N>;
    const int lines = (a.n0 + 1) * a.rows1;
    p3_fwd<N><<<(lines + C::LPC - 1) / C::LPC, C::THREADS, C::SMEM, st>>>(a, withE);
    return (int)cudaGetLastError();
}

template <int N>
static int p3a(const PassArgs &a, int hasE, cudaStream_t st)
{
    using C = RowCfg<N>;
    const int lines = (a.n0 + 1) * a.rows1;
    p3_adj<N><<<(lines + C::LPC - 1) / C::LPC, C::THREADS, C::SMEM, st>>>(a, hasE);
    return (int)cudaGetLastError();
}

int launch_p3_fwd(int N, const PassArgs &a, int withE, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p3f<n>(a, withE, st);
        FSP_AXIS2_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_p3_adj(int N, const PassArgs &a, int hasE, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p3a<n>(a, hasE, st);
        FSP_AXIS2_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

} // namespace fsp
