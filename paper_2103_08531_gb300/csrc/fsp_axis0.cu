// fsp_axis0.cu -- launchers of the axis-0 passes (P1 real -> half spectrum, P5 back).
#include "fsp_internal.h"
#include "fsp_passes.cuh"

#include <algorithm>

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

// Tile kernels (2n <= 512) are persistent: grid = SMs x resident CTAs per SM.
template <int N>
struct Occ0 {
    static inline int p1 = 0, p5 = 0;
};

template <int N>
static constexpr size_t smem_p1() { return (size_t)(N / 2 * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }
template <int N>
static constexpr size_t smem_p5() { return (size_t)(3 * (N / 2 + 1) * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }

template <int N>
static int prep()
{
    using C = ColCfg<N>;
    int e = 0;
    e |= cudaFuncSetAttribute(p1_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if constexpr (N <= 512) {
        e |= cudaFuncSetAttribute(p1_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p1<N>());
        e |= cudaFuncSetAttribute(p5_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p5<N>());
        int dev = 0, sms = 0, b1 = 0, b5 = 0;
        e |= cudaGetDevice(&dev);
        e |= cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, p1_fwd<N>, TileCfg<N>::THREADS, smem_p1<N>());
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b5, p5_fwd<N>, TileCfg<N>::THREADS, smem_p5<N>());
        Occ0<N>::p1 = sms * (b1 > 0 ? b1 : 1);
        Occ0<N>::p5 = sms * (b5 > 0 ? b5 : 1);
    } else {
        e |= cudaFuncSetAttribute(p1_fwd_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p5_fwd_blk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
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
    if constexpr (N <= 512) {
        const int tiles = a.n1 * (a.n2 / (2 * TileCfg<N>::C));
        p1_fwd<N><<<std::min(tiles, Occ0<N>::p1), TileCfg<N>::THREADS, smem_p1<N>(), st>>>(a, dst);
    } else {
        using C = ColCfg<N>;
        dim3 grid((a.n2 / 2 + C::BZ - 1) / C::BZ, a.n1);
        p1_fwd_blk<N><<<grid, C::THREADS, C::SMEM, st>>>(a, dst);
    }
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
    if constexpr (N <= 512) {
        const int tiles = a.n1 * (a.n2 / TileCfg<N>::C);
        p5_fwd<N><<<std::min(tiles, Occ0<N>::p5), TileCfg<N>::THREADS, smem_p5<N>(), st>>>(a);
    } else {
        using C = ColCfg<N>;
        dim3 grid((a.n2 + C::BZ - 1) / C::BZ, a.n1);
        p5_fwd_blk<N><<<grid, C::THREADS, C::SMEM, st>>>(a);
    }
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
