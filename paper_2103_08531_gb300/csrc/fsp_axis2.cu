// fsp_axis2.cu -- launchers of the axis-2 middle pass (P3: forward, kernel multiply, inverse).
#include "fsp_internal.h"
#include "fsp_passes.cuh"

#include <algorithm>

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
struct Occ2 {
    static inline int p3 = 0, p3a = 0;
};

template <int N>
static int prep()
{
    int e = 0;
    if constexpr (N <= 512) {
        using C = WarpCfg<N>;
        e |= cudaFuncSetAttribute(p3_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p3_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        int dev = 0, sms = 0, b = 0, ba = 0;
        e |= cudaGetDevice(&dev);
        e |= cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, p3_fwd<N>, C::THREADS, C::SMEM);
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ba, p3_adj<N>, C::THREADS, C::SMEM);
        Occ2<N>::p3 = sms * (b > 0 ? b : 1);
        Occ2<N>::p3a = sms * (ba > 0 ? ba : 1);
    } else {
        using C = RowCfg<N>;
        e |= cudaFuncSetAttribute(p3_fwd_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p3_adj_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
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
    const int lines = (a.n0 + 1) * a.rows1;
    if constexpr (N <= 512) {
        using C = WarpCfg<N>;
        const int ctas = (lines + C::LPW * C::WARPS - 1) / (C::LPW * C::WARPS);
        p3_fwd<N><<<std::min(ctas, Occ2<N>::p3), C::THREADS, C::SMEM, st>>>(a, withE);
    } else {
        using C = RowCfg<N>;
        p3_fwd_blk<N><<<(lines + C::LPC - 1) / C::LPC, C::THREADS, C::SMEM, st>>>(a, withE);
    }
    return (int)cudaGetLastError();
}

template <int N>
static int p3a(const PassArgs &a, int hasE, cudaStream_t st)
{
    const int lines = (a.n0 + 1) * a.rows1;
    if constexpr (N <= 512) {
        using C = WarpCfg<N>;
        const int ctas = (lines + C::LPW * C::WARPS - 1) / (C::LPW * C::WARPS);
        p3_adj<N><<<std::min(ctas, Occ2<N>::p3a), C::THREADS, C::SMEM, st>>>(a, hasE);
    } else {
        using C = RowCfg<N>;
        p3_adj_blk<N><<<(lines + C::LPC - 1) / C::LPC, C::THREADS, C::SMEM, st>>>(a, hasE);
    }
    return (int)cudaGetLastError();
}

int make_twiddles_aux(float2 *tw, int N, cudaStream_t st)
{
    switch (N) {
#define X(n) \
    case n: k_twiddles_aux<n, typename Plan16<n>::R><<<4, 256, 0, st>>>(tw); return (int)cudaGetLastError();
        X(64) X(128) X(192) X(256) X(512)
#undef X
    default: return 0;   // block-mode lengths use the main table only
    }
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
