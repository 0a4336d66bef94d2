// fsp_axis1.cu -- launchers of the axis-1 passes (P2 forward, P4 inverse; 3D only).
#include "fsp_internal.h"
#include "fsp_passes.cuh"

#include <algorithm>

namespace fsp {

#define FSP_AXIS1_SIZES(X) X(64) X(128) X(192) X(256) X(512) X(1024)

int supported_axis1(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS1_SIZES(X)
#undef X
    default: return 0;
    }
}

template <int N>
struct Occ1 {
    static inline int p2 = 0, p4 = 0;
};

template <int N>
static constexpr size_t smem_p2() { return (size_t)(N / 2 * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }
template <int N>
static constexpr size_t smem_p4() { return (size_t)(2 * N * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }

template <int N>
static int prep()
{
    using C = ColCfg<N>;
    int e = 0;
    e |= cudaFuncSetAttribute(p2_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if constexpr (N <= 512) {
        e |= cudaFuncSetAttribute(p2_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p2<N>());
        e |= cudaFuncSetAttribute(p4_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p4<N>());
        int dev = 0, sms = 0, b2 = 0, b4 = 0;
        e |= cudaGetDevice(&dev);
        e |= cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, p2_fwd<N>, TileCfg<N>::THREADS, smem_p2<N>());
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, p4_fwd<N>, TileCfg<N>::THREADS, smem_p4<N>());
        Occ1<N>::p2 = sms * (b2 > 0 ? b2 : 1);
        Occ1<N>::p4 = sms * (b4 > 0 ? b4 : 1);
    } else {
        e |= cudaFuncSetAttribute(p2_fwd_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p4_fwd_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
    return e;
}

int prepare_axis1(int N)
{
    switch (N) {
#define X(n) case n: return prep<n>();
        FSP_AXIS1_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

template <int N>
static int p2f(const PassArgs &a, const float2 *src, float2 *dst, cudaStream_t st)
{
    if constexpr (N <= 512) {
        const int tiles = (a.n0 + 1) * (a.n2 / TileCfg<N>::C);
        p2_fwd<N><<<std::min(tiles, Occ1<N>::p2), TileCfg<N>::THREADS, smem_p2<N>(), st>>>(a, src, dst);
    } else {
        using C = ColCfg<N>;
        dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n0 + 1);
        p2_fwd_blk<N><<<grid, C::THREADS, C::SMEM, st>>>(a, src, dst);
    }
    return (int)cudaGetLastError();
}

template <int N>
static int p2a(const PassArgs &a, int hasE, cudaStream_t st)
{
    using C = ColCfg<N>;
    dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n0 + 1);
    p2_adj<N><<<grid, C::THREADS, C::SMEM, st>>>(a, hasE);
    return (int)cudaGetLastError();
}

template <int N>
static int p4f(const PassArgs &a, int withE, cudaStream_t st)
{
    if constexpr (N <= 512) {
        const int tiles = (a.n0 + 1) * (a.n2 / TileCfg<N>::C);
        p4_fwd<N><<<std::min(tiles, Occ1<N>::p4), TileCfg<N>::THREADS, smem_p4<N>(), st>>>(a, withE);
    } else {
        using C = ColCfg<N>;
        dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n0 + 1);
        p4_fwd_blk<N><<<grid, C::THREADS, C::SMEM, st>>>(a, withE);
    }
    return (int)cudaGetLastError();
}

int launch_p2_fwd(int N, const PassArgs &a, const float2 *src, float2 *dst, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p2f<n>(a, src, dst, st);
        FSP_AXIS1_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_p2_adj(int N, const PassArgs &a, int hasE, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p2a<n>(a, hasE, st);
        FSP_AXIS1_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

int launch_p4_fwd(int N, const PassArgs &a, int withE, cudaStream_t st)
{
    switch (N) {
#define X(n) case n: return p4f<n>(a, withE, st);
        FSP_AXIS1_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

} // namespace fsp
