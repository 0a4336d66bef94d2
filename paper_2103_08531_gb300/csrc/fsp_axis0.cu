// fsp_axis0.cu -- launchers of the axis-0 passes (P1 real -> half spectrum, P5 back).
#include "fsp_internal.h"
#include "fsp_launch.cuh"
#include "fsp_long.cuh"
#include "fsp_tma.cuh"

#include <algorithm>
#include <cstring>
#include <type_traits>

namespace fsp {

#define FSP_AXIS0_SIZES(X) \
    X(32) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096) X(6144) X(8192)

int supported_axis0(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS0_SIZES(X)
#undef X
    default: return 0;
    }
}

// 1: 2D first-axis passes with 2 n0 >= 1536 run persistent with a cp.async
// stage (p1_fwd_pst / p5_fwd_pst); 0: one CTA per column group (p1_fwd_blk / p5_fwd_blk).
#ifndef FSP_LONG_STAGED
#define FSP_LONG_STAGED 1
#endif

template <int N, int EE>
static constexpr size_t smem_p1() { return (size_t)(N / 2 * TileCfg<N, EE>::C + TileCfg<N, EE>::EX) * sizeof(float2); }
template <int N, int EE>
static constexpr size_t smem_p5() { return (size_t)(3 * (N / 2 + 1) * TileCfg<N, EE>::C + TileCfg<N, EE>::EX) * sizeof(float2); }

// resident CTAs per SM of the persistent kernels (set by prepare)
template <int N, int MAXI, int EE>
struct Occ0 {
    static inline int p1 = 1, p5 = 1;
};

template <int N, int MAXI, int EE>
static int prep_tiles()
{
    int e = 0, b1 = 0, b5 = 0;
    e |= cudaFuncSetAttribute(p1_fwd<N, MAXI, EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p1<N, EE>());
    e |= cudaFuncSetAttribute(p5_fwd<N, MAXI, EE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p5<N, EE>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, p1_fwd<N, MAXI, EE>, TileCfg<N, EE>::THREADS, smem_p1<N, EE>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b5, p5_fwd<N, MAXI, EE>, TileCfg<N, EE>::THREADS, smem_p5<N, EE>());
    Occ0<N, MAXI, EE>::p1 = std::max(1, b1);
    Occ0<N, MAXI, EE>::p5 = std::max(1, b5);
    return e;
}

template <int N>
static constexpr size_t smem_p1a() { return (size_t)(2 * (N / 2) * TileCfg<N>::C + TileCfg<N>::EX) * sizeof(float2); }

template <int N, int MAXI>
struct OccA0 {
    static inline int p1a = 1;
};

template <int N, int MAXI>
static int prep_one()
{
    using C = ColCfg<N>;
    int e = cudaFuncSetAttribute(p1_adj<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if constexpr (N <= 512) {
        if constexpr (MAXI == 1) e |= prep_tiles<N, MAXI, 16>() | prep_tiles<N, MAXI, 8>();
        int b = 0;
        e |= cudaFuncSetAttribute(p1_adj_t<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p1a<N>());
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, p1_adj_t<N, MAXI>, TileCfg<N>::THREADS, smem_p1a<N>());
        OccA0<N, MAXI>::p1a = std::max(1, b);
    } else {
        e |= cudaFuncSetAttribute(p1_fwd_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        e |= cudaFuncSetAttribute(p5_fwd_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if constexpr (!C::WIDE) {
            const int sm = (int)LongStage<N>::SMEM;
            e |= cudaFuncSetAttribute(p1_fwd_pst<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            e |= cudaFuncSetAttribute(p5_fwd_pst<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        }
    }
    return e;
}

// TMA-staged column tiles (2n <= 512), single solves (MAXI = 1) and batches
template <int N, int MAXI, int ALT = 0>
struct TmaOcc0 {
    static inline int p1 = 1, p5 = 1;
};
template <int N>
static constexpr size_t smem_p1_tma() { return TmaTile<N>::smem(1, N / 2); }
template <int N>
static constexpr size_t smem_p5_tma() { return TmaTile<N>::smem(3, N / 2); }
static_assert(sizeof(Work<BATCH_MAX>) + sizeof(TmaBatch<BATCH_MAX>) + 16 <= 32764, "kernel parameters too large");

template <int N, int MAXI, int ALT = 0>
static int prep_tma()
{
    int e = 0, b1 = 0, b5 = 0;
    using C = TileCfg<N, 16, ALT>;
    e |= cudaFuncSetAttribute(p1_tma<N, MAXI, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p1_tma<N>());
    e |= cudaFuncSetAttribute(p5_tma<N, MAXI, ALT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p5_tma<N>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, p1_tma<N, MAXI, ALT>, C::THREADS, smem_p1_tma<N>());
    e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b5, p5_tma<N, MAXI, ALT>, C::THREADS, smem_p5_tma<N>());
    TmaOcc0<N, MAXI, ALT>::p1 = std::max(1, b1);
    TmaOcc0<N, MAXI, ALT>::p5 = std::max(1, b5);
    return e;
}

static constexpr size_t smem_p5_4s_b() { return TmaTile<512>::smem(1, 512); }

template <int N>
static int prep()
{
    int e = prep_one<N, 1>() | prep_one<N, BATCH_MAX>();
    if constexpr (N <= 512) e |= prep_tma<N, 1>() | prep_tma<N, BATCH_MAX>();
    if constexpr (N <= 512 && Plan16B<N>::HAS) e |= prep_tma<N, 1, 1>();
    if constexpr (N == L4S::N) {
        e |= cudaFuncSetAttribute(p5_4s_a<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P5A::SMEM);
        e |= cudaFuncSetAttribute(p5_4s_a<BATCH_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P5A::SMEM);
        e |= cudaFuncSetAttribute(p5_4s_b<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p5_4s_b());
        e |= cudaFuncSetAttribute(p5_4s_b<BATCH_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p5_4s_b());
    }
    return e;
}

// P5 of 2D solves with 2 n0 = 8192: the four-step through global memory
// (p5_4s_a / p5_4s_b in fsp_long.cuh), in place in buf0 and buf1.  Every item
// 2D with whole 16-column tiles.
static bool fits_p5_4s(const PassArgs *items, int n)
{
    for (int i = 0; i < n; ++i)
        if (items[i].three_d || items[i].n2 % 16) return false;
    return true;
}
static bool wants_e1(const PassArgs &a) { return a.out[2] != nullptr; }
static bool wants_01(const PassArgs &a) { return a.out[0] != nullptr || a.out[1] != nullptr; }
static int blocks_a(const PassArgs &a) { return (257 * (a.n2 / 2) + 255) / 256; }
static int units_a0(const PassArgs &a) { return wants_e1(a) ? blocks_a(a) : 0; }
static int units_a1(const PassArgs &a) { return wants_01(a) ? blocks_a(a) : 0; }
static int units_b0(const PassArgs &a) { return wants_e1(a) ? 8 * (a.n2 / 16) : 0; }
static int units_b1(const PassArgs &a) { return wants_01(a) ? 2 * 8 * (a.n2 / 16) : 0; }

template <class Wk>
static int launch_p5_4s_b(const Wk &w, int mode, cudaStream_t st)
{
    constexpr int MAXI = Wk::max_items;
    TmaBatch<MAXI> m;
    std::memset(&m, 0, sizeof(m));
    for (int i = 0; i < w.nitems; ++i) {
        const PassArgs &a = w.item[i];
        const unsigned long long dims[2] = {(unsigned long long)a.n2, (unsigned long long)a.n0 + 1};
        const unsigned long long str[1] = {(unsigned long long)a.n2 * 8};
        const unsigned box[2] = {16, 256};
        if ((a.buf0 && encode_tensor_map(&m.m[i][0], a.buf0, 2, 8, dims, str, box)) ||
            (a.buf1 && encode_tensor_map(&m.m[i][1], a.buf1, 2, 8, dims, str, box)))
            return (int)cudaErrorInvalidValue;
    }
    const int total = w.offs[w.nitems];
    return launch_pdl(p5_4s_b<MAXI>, std::min(total, sm_count()), TileCfg<512, 16>::THREADS, smem_p5_4s_b(), st, w,
                      m, mode);
}

static int run_p5_4s(const PassArgs *items, int n, cudaStream_t st)
{
    auto step_a = [&](int mode) {
        return chunked(items, n, mode ? units_a1 : units_a0, [&](auto &w) {
            constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
            const int total = w.offs[w.nitems];
            if (total == 0) return 0;
            return launch_pdl(p5_4s_a<MAXI>, std::min(total, sm_count()), P5A::THREADS, P5A::SMEM, st, w, mode);
        });
    };
    auto step_b = [&](int mode) {
        return chunked(items, n, mode ? units_b1 : units_b0, [&](auto &w) {
            if (w.offs[w.nitems] == 0) return 0;
            return launch_p5_4s_b(w, mode, st);
        });
    };
    // E1 first: its set lives in buf1, which the E0 set overwrites afterwards
    int e = step_a(0);
    if (!e) e = step_b(0);
    if (!e) e = step_a(1);
    if (!e) e = step_b(1);
    return e;
}

template <int N>
static int units_p1_tma(const PassArgs &a) { return a.n1 * (a.n2 / 32); }
template <int N>
static int units_p5_tma(const PassArgs &a) { return a.n1 * (a.n2 / 16); }

// The TMA-staged P1 / P5 of one launch's items: tensor maps of every item
// built here from its own buffers.  Variant bits: 2 = one CTA per SM; 8 = the
// second radix split (single solves, lengths that have one).
template <int N, class Wk>
static int tma_launch0(int kind, const Wk &w, int var, cudaStream_t st)
{
    constexpr int MAXI = Wk::max_items;
    using C = TileCfg<N, 16>;
    TmaBatch<MAXI> m;
    std::memset(&m, 0, sizeof(m));
    for (int i = 0; i < w.nitems; ++i) {
        const PassArgs &a = w.item[i];
        if (kind == PASS_P1F) {
            const unsigned long long dims[3] = {(unsigned long long)a.n2, (unsigned long long)a.n1,
                                                (unsigned long long)a.n0};
            const unsigned long long str[2] = {(unsigned long long)a.n2 * 4, (unsigned long long)a.n1 * a.n2 * 4};
            const unsigned box[3] = {32, 1, N / 2};
            if (encode_tensor_map(&m.m[i][0], a.in[0], 3, 4, dims, str, box)) return (int)cudaErrorInvalidValue;
        } else {
            const unsigned long long dims[3] = {(unsigned long long)a.n2, (unsigned long long)a.rows1,
                                                (unsigned long long)a.n0 + 1};
            const unsigned long long str[2] = {(unsigned long long)a.n2 * 8, (unsigned long long)a.rows1 * a.n2 * 8};
            const unsigned box[3] = {16, 1, N / 2};
            if (encode_tensor_map(&m.m[i][0], a.buf0, 3, 8, dims, str, box) ||
                encode_tensor_map(&m.m[i][1], a.buf1, 3, 8, dims, str, box))
                return (int)cudaErrorInvalidValue;
        }
    }
    const int total = w.offs[w.nitems];
    const int sms = sm_count();
    auto go = [&](auto alt) {
        constexpr int ALT = decltype(alt)::value;
        using O = TmaOcc0<N, MAXI, ALT>;
        if (kind == PASS_P1F)
            return launch_pdl(p1_tma<N, MAXI, ALT>, std::min(total, sms * ((var & 2) ? 1 : O::p1)), C::THREADS,
                              smem_p1_tma<N>(), st, w, m);
        return launch_pdl(p5_tma<N, MAXI, ALT>, std::min(total, sms * ((var & 2) ? 1 : O::p5)), C::THREADS,
                          smem_p5_tma<N>(), st, w, m);
    };
    if constexpr (MAXI == 1 && Plan16B<N>::HAS)
        if (var & 8) return go(std::integral_constant<int, 1>{});
    return go(std::integral_constant<int, 0>{});
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
static int units_p1f(const PassArgs &a)
{
    if constexpr (N <= 512) return a.n1 * (a.n2 / (2 * FSP_TILE_C));
    else return a.n1 * ((a.n2 / 2 + ColCfg<N>::BZ - 1) / ColCfg<N>::BZ);
}
template <int N>
static int units_col(const PassArgs &a)   // (y, column tile) units of P1-adjoint and the block P5
{
    return a.n1 * ((a.n2 + ColCfg<N>::BZ - 1) / ColCfg<N>::BZ);
}
template <int N>
static int units_p5f(const PassArgs &a)
{
    if constexpr (N <= 512) return a.n1 * (a.n2 / FSP_TILE_C);
    else return units_col<N>(a);
}

// Persistent staged long columns (2D, BZ < 16): every item 2D with whole column groups.
template <int N>
static bool staged_fits(int kind, const PassArgs *items, int n)
{
    constexpr int BZ = ColCfg<N>::BZ;
    for (int i = 0; i < n; ++i) {
        const int cols = kind == PASS_P1F ? items[i].n2 / 2 : items[i].n2;
        if (items[i].three_d || cols % BZ) return false;
    }
    return true;
}

// variant bits: 1 = 8 values per thread in the tiles (else 16); 2 = one CTA per SM
template <int N, int EE, class Wk>
static int tile_launch(int kind, const Wk &w, int var, cudaStream_t st)
{
    constexpr int MAXI = Wk::max_items;
    const int total = w.offs[w.nitems];
    const int sms = sm_count();
    if (kind == PASS_P1F) {
        const int cap = sms * ((var & 2) ? 1 : Occ0<N, MAXI, EE>::p1);
        return launch_pdl(p1_fwd<N, MAXI, EE>, std::min(total, cap), TileCfg<N, EE>::THREADS, smem_p1<N, EE>(), st, w);
    } else {
        const int cap = sms * ((var & 2) ? 1 : Occ0<N, MAXI, EE>::p5);
        return launch_pdl(p5_fwd<N, MAXI, EE>, std::min(total, cap), TileCfg<N, EE>::THREADS, smem_p5<N, EE>(), st, w);
    }
    return (int)cudaGetLastError();
}

template <int N>
static int run(int kind, const PassArgs *items, int n, int var, cudaStream_t st)
{
    if constexpr (N <= 512) {
        if ((kind == PASS_P1F || kind == PASS_P5F) && !(var & 4)) {
            bool fits = true;   // the TMA tiles take 32 reals (16 complex) of the contiguous axis at a time
            for (int i = 0; i < n; ++i) fits = fits && items[i].n2 % 32 == 0;
            if (fits)
                return chunked(items, n, kind == PASS_P1F ? units_p1_tma<N> : units_p5_tma<N>,
                               [&](auto &w) { return tma_launch0<N>(kind, w, var, st); });
        }
    }
    if constexpr (N == L4S::N) {   // variant bit 4: the staged block-synchronous columns instead
        if (kind == PASS_P5F && !(var & 4) && fits_p5_4s(items, n)) return run_p5_4s(items, n, st);
    }
    if (kind == PASS_P1F || kind == PASS_P5F) {
        return chunked(items, n, kind == PASS_P1F ? units_p1f<N> : units_p5f<N>, [&](auto &w) {
            constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
            if constexpr (N <= 512) {
                // the cp.async tiles serve single solves only (tuning variant bit 4);
                // batches take the TMA tiles above
                if constexpr (MAXI == 1)
                    return (var & 1) ? tile_launch<N, 8>(kind, w, var, st) : tile_launch<N, 16>(kind, w, var, st);
                else
                    return (int)cudaErrorInvalidValue;
            } else {
                const int total = w.offs[w.nitems];
                if constexpr (!ColCfg<N>::WIDE) {
                    if (FSP_LONG_STAGED && staged_fits<N>(kind, w.item, w.nitems)) {
                        const int grid = std::min(total, sm_count());
                        if (kind == PASS_P1F)
                            return launch_pdl_if(kLongPdl<N>, p1_fwd_pst<N, MAXI>, grid, ColCfg<N>::THREADS, LongStage<N>::SMEM, st, w);
                        return launch_pdl_if(kLongPdl<N>, p5_fwd_pst<N, MAXI>, grid, ColCfg<N>::THREADS, LongStage<N>::SMEM, st, w);
                    }
                }
                if (kind == PASS_P1F) p1_fwd_blk<N, MAXI><<<total, ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w);
                else p5_fwd_blk<N, MAXI><<<total, ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w);
                return (int)cudaGetLastError();
            }
        });
    }
    if (kind == PASS_P1A) {
        if constexpr (N <= 512) {
            return chunked(items, n, units_p5f<N>, [&](auto &w) {   // (y, C-column tile) units
                constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
                const int total = w.offs[w.nitems];
                return launch_pdl(p1_adj_t<N, MAXI>, std::min(total, sm_count() * OccA0<N, MAXI>::p1a),
                                  TileCfg<N>::THREADS, smem_p1a<N>(), st, w);
            });
        } else {
            return chunked(items, n, units_col<N>, [&](auto &w) {
                constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
                p1_adj<N, MAXI><<<w.offs[w.nitems], ColCfg<N>::THREADS, ColCfg<N>::SMEM, st>>>(w);
                return (int)cudaGetLastError();
            });
        }
    }
    return (int)cudaErrorInvalidValue;
}

int launch_axis0(int kind, int N, const PassArgs *items, int n, int var, cudaStream_t st)
{
    switch (N) {
#define X(v) case v: return run<v>(kind, items, n, var, st);
        FSP_AXIS0_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

} // namespace fsp
