// fsp_axis1.cu -- launchers of the axis-1 passes (P2 forward, P4 inverse; 3D only).
#include "fsp_internal.h"
#include "fsp_launch.cuh"
#include "fsp_tma.cuh"

#include <algorithm>
#include <cstring>
#include <type_traits>

namespace fsp {

#define FSP_AXIS1_SIZES(X) X(32) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

int supported_axis1(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS1_SIZES(X)
#undef X
    default: return 0;
    }
}

template <int N, int EE>
static constexpr size_t smem_p2() { return (size_t)(N / 2 * TileCfg<N, EE>::C + TileCfg<N, EE>::EX) * sizeof(float2); }
template <int N, int EE>
static constexpr size_t smem_p4() { return (size_t)(2 * N * TileCfg<N, EE>::C + TileCfg<N, EE>::EX) * sizeof(float2); }

template <int N, int MAXI, int EE>
struct Occ1 {
    static inline int p2 = 1, p4 = 1;
};

template <int N, int MAXI, int EE>
static int prep_tiles()
{
    int e = 0, b2 = 0, b4 = 0;
    e |= cudaFuncSetAttribute(p2_fwd<N, MAXI, EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p2<N, EE>());
    e |= cudaFuncSetAttribute(p4_fwd<N, MAXI, EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p4<N, EE>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, p2_fwd<N, MAXI, EE>, TileCfg<N, EE>::THREADS, smem_p2<N, EE>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, p4_fwd<N, MAXI, EE>, TileCfg<N, EE>::THREADS, smem_p4<N, EE>());
    Occ1<N, MAXI, EE>::p2 = std::max(1, b2);
    Occ1<N, MAXI, EE>::p4 = std::max(1, b4);
    return e;
}

template <int N>
static constexpr size_t smem_p2a() { return (size_t)((N + N / 2) * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }

template <int N, int MAXI>
struct OccA1 {
    static inline int p2a = 1;
};

template <int N, int MAXI>
static int prep_one()
{
    using C = ColCfg<N>;
    int e = cudaFuncSetAttribute(p2_adj<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if constexpr (N <= 512) {
        if constexpr (MAXI == 1) e |= prep_tiles<N, MAXI, 16>() | prep_tiles<N, MAXI, 8>();
        int b = 0;
        e |= cudaFuncSetAttribute(p2_adj_t<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p2a<N>());
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, p2_adj_t<N, MAXI>, TileCfg<N>::THREADS, smem_p2a<N>());
        OccA1<N, MAXI>::p2a = std::max(1, b);
    } else {
        e |= cudaFuncSetAttribute(p2_fwd_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p4_fwd_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
    return e;
}

// TMA-staged column tiles (2n <= 512), single solves (MAXI = 1) and batches
template <int N, int MAXI, int ALT = 0>
struct TmaOcc1 {
    static inline int p2 = 1, p4 = 1;
};
template <int N>
static constexpr size_t smem_p2_tma() { return TmaTile<N>::smem(1, N / 2); }
template <int N>
static constexpr size_t smem_p4_tma() { return TmaTile<N>::smem(2, N); }

template <int N, int MAXI, int ALT = 0>
static int prep_tma()
{
    int e = 0, b2 = 0, b4 = 0;
    using C = TileCfg<N, 16, ALT>;
    e |= cudaFuncSetAttribute(p2_tma<N, MAXI, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p2_tma<N>());
    e |= cudaFuncSetAttribute(p4_tma<N, MAXI, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p4_tma<N>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, p2_tma<N, MAXI, ALT>, C::THREADS, smem_p2_tma<N>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b4, p4_tma<N, MAXI, ALT>, C::THREADS, smem_p4_tma<N>());
    TmaOcc1<N, MAXI, ALT>::p2 = std::max(1, b2);
    TmaOcc1<N, MAXI, ALT>::p4 = std::max(1, b4);
    return e;
}

template <int N>
static int prep()
{
    int e = prep_one<N, 1>() | prep_one<N, BATCH_MAX>();
    if constexpr (N <= 512) e |= prep_tma<N, 1>() | prep_tma<N, BATCH_MAX>();
    if constexpr (N <= 512 && Plan16B<N>::HAS) e |= prep_tma<N, 1, 1>();
    return e;
}

// (k0, 16-column tile) units over planes [kx0, kx0 + kxn)
template <int N>
static int units_tma1(const PassArgs &a) { return a.kxn * (a.n2 / 16); }

// The TMA-staged P2 / P4 of one launch's items: maps over each item's buf1
// (P2) or buf0 and buf1 (P4) as [(n0 + 1) rows1][n2] complex.  Variant bits:
// 2 = one CTA per SM; 8 = the second radix split (single solves, lengths
// that have one).
template <int N, class Wk>
static int tma_launch1(int kind, const Wk &w, int flag, int var, cudaStream_t st)
{
    constexpr int MAXI = Wk::max_items;
    using C = TileCfg<N, 16>;
    TmaBatch<MAXI> m;
    std::memset(&m, 0, sizeof(m));
    for (int i = 0; i < w.nitems; ++i) {
        const PassArgs &a = w.item[i];
        const unsigned long long dims[2] = {(unsigned long long)a.n2, (unsigned long long)(a.n0 + 1) * a.rows1};
        const unsigned long long str[1] = {(unsigned long long)a.n2 * 8};
        if (kind == PASS_P2F) {
            const unsigned box[2] = {16, N / 2};
            if (encode_tensor_map(&m.m[i][0], a.buf1, 2, 8, dims, str, box)) return (int)cudaErrorInvalidValue;
        } else {
            const unsigned box[2] = {16, N < 256 ? N : 256};
            if (encode_tensor_map(&m.m[i][0], a.buf0, 2, 8, dims, str, box) ||
                encode_tensor_map(&m.m[i][1], a.buf1, 2, 8, dims, str, box))
                return (int)cudaErrorInvalidValue;
        }
    }
    const int total = w.offs[w.nitems];
    const int sms = sm_count();
    auto go = [&](auto alt) {
        constexpr int ALT = decltype(alt)::value;
        using O = TmaOcc1<N, MAXI, ALT>;
        if (kind == PASS_P2F)
            return launch_pdl(p2_tma<N, MAXI, ALT>, std::min(total, sms * ((var & 2) ? 1 : O::p2)), C::THREADS,
                              smem_p2_tma<N>(), st, w, m);
        return launch_pdl(p4_tma<N, MAXI, ALT>, std::min(total, sms * ((var & 2) ? 1 : O::p4)), C::THREADS,
                          smem_p4_tma<N>(), st, w, m, flag);
    };
    if constexpr (MAXI == 1 && Plan16B<N>::HAS)
        if (var & 8) return go(std::integral_constant<int, 1>{});
    return go(std::integral_constant<int, 0>{});
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
static int units_tile(const PassArgs &a)   // (k0, column tile) units
{
    if constexpr (N <= 512) return (a.n0 + 1) * (a.n2 / FSP_TILE_C);
    else return (a.n0 + 1) * ((a.n2 + ColCfg<N>::BZ - 1) / ColCfg<N>::BZ);
}
template <int N>
static int units_blk(const PassArgs &a)
{
    return (a.n0 + 1) * ((a.n2 + ColCfg<N>::BZ - 1) / ColCfg<N>::BZ);
}

// variant bits: 1 = 8 values per thread in the tiles (else 16); 2 = one CTA per SM
template <int N, int EE, class Wk>
static int tile_launch(int kind, const Wk &w, int flag, int var, cudaStream_t st)
{
    constexpr int MAXI = Wk::max_items;
    const int total = w.offs[w.nitems];
    const int sms = sm_count();
    if (kind == PASS_P2F) {
        const int cap = sms * ((var & 2) ? 1 : Occ1<N, MAXI, EE>::p2);
        return launch_pdl(p2_fwd<N, MAXI, EE>, std::min(total, cap), TileCfg<N, EE>::THREADS, smem_p2<N, EE>(), st, w);
    } else {
        const int cap = sms * ((var & 2) ? 1 : Occ1<N, MAXI, EE>::p4);
        return launch_pdl(p4_fwd<N, MAXI, EE>, std::min(total, cap), TileCfg<N, EE>::THREADS, smem_p4<N, EE>(), st, w, flag);
    }
    return (int)cudaGetLastError();
}

template <int N>
static int run(int kind, const PassArgs *items, int n, int flag, int var, cudaStream_t st)
{
    if constexpr (N <= 512) {
        if ((kind == PASS_P2F || kind == PASS_P4F) && !(var & 4)) {
            bool fits = true;
            for (int i = 0; i < n; ++i) fits = fits && items[i].n2 % 16 == 0;
            if (fits)
                return chunked(items, n, units_tma1<N>, [&](auto &w) { return tma_launch1<N>(kind, w, flag, var, st); });
        }
    }
    if (kind == PASS_P2F || kind == PASS_P4F) {
        return chunked(items, n, units_tile<N>, [&](auto &w) {
            constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
            if constexpr (N <= 512) {
                // the cp.async tiles serve single solves only (tuning variant bit 4);
                // batches take the TMA tiles above
                if constexpr (MAXI == 1)
                    return (var & 1) ? tile_launch<N, 8>(kind, w, flag, var, st) : tile_launch<N, 16>(kind, w, flag, var, st);
                else
                    return (int)cudaErrorInvalidValue;
            } else {
                const int total = w.offs[w.nitems];
                if (kind == PASS_P2F) p2_fwd_blk<N, MAXI><<<total, ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w);
                else p4_fwd_blk<N, MAXI><<<total, ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w, flag);
                return (int)cudaGetLastError();
            }
        });
    }
    if (kind == PASS_P2A) {
        if constexpr (N <= 512) {
            if (flag) {   // the tile version handles the three-stream adjoint (hasE)
                return chunked(items, n, units_tile<N>, [&](auto &w) {
                    constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
                    const int total = w.offs[w.nitems];
                    return launch_pdl(p2_adj_t<N, MAXI>, std::min(total, sm_count() * OccA1<N, MAXI>::p2a),
                                      TileCfg<N>::THREADS, smem_p2a<N>(), st, w);
                });
            }
        }
        return chunked(items, n, units_blk<N>, [&](auto &w) {
            constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
            p2_adj<N, MAXI><<<w.offs[w.nitems], ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w, flag);
            return (int)cudaGetLastError();
        });
    }
    return (int)cudaErrorInvalidValue;
}

int launch_axis1(int kind, int N, const PassArgs *items, int n, int flag, int var, cudaStream_t st)
{
    switch (N) {
#define X(v) case v: return run<v>(kind, items, n, flag, var, st);
        FSP_AXIS1_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

} // namespace fsp
