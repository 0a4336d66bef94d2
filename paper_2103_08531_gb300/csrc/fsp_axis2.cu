// fsp_axis2.cu -- launchers of the axis-2 middle pass (P3: forward, kernel multiply, inverse).
#include "fsp_internal.h"
#include "fsp_launch.cuh"
#include "fsp_long.cuh"

#include <algorithm>
#include <type_traits>

namespace fsp {

#define FSP_AXIS2_SIZES(X) \
    X(64) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(3072) X(4096) X(6144) X(8192)

int supported_axis2(int N)
{
    switch (N) {
#define X(n) case n: return 1;
        FSP_AXIS2_SIZES(X)
#undef X
    default: return 0;
    }
}

// A single forward solve takes p3_fwd1 (arguments by value) unless this is 0.
#ifndef FSP_P3_ONE
#define FSP_P3_ONE 1
#endif

template <int N, int MAXI>
struct Occ2 {
    static inline int p3 = 1, p3a = 1, p3one = 1, p3oneB = 1, wide = 1, half = 1;
};

// Lines of 768 to 2048 points: the multi-warp-per-line middle pass
// (p3_fwd_wide) unless variant bit 4 asks for the block kernel.
template <int N>
constexpr bool kWide = N == 768 || N == 1024 || N == 1536 || N == 2048;

template <int N, int MAXI>
static int prep_one()
{
    int e = 0;
    if constexpr (N <= 512) {
        using C = WarpCfg<N>;
        e |= cudaFuncSetAttribute(p3_fwd<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if constexpr (MAXI == 1) {
            e |= cudaFuncSetAttribute(p3_fwd1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
            int b1 = 0;
            e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, p3_fwd1<N>, C::THREADS, C::SMEM);
            Occ2<N, MAXI>::p3one = std::max(1, b1);
            if constexpr (Plan16B<N>::HAS) {
                using CB = WarpCfg<N, 1>;
                e |= cudaFuncSetAttribute(p3_fwd1<N, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CB::SMEM);
                e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, p3_fwd1<N, 1>, CB::THREADS, CB::SMEM);
                Occ2<N, MAXI>::p3oneB = std::max(1, b1);
            }
        }
        e |= cudaFuncSetAttribute(p3_adj<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        int b = 0, ba = 0;
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, p3_fwd<N, MAXI>, C::THREADS, C::SMEM);
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ba, p3_adj<N, MAXI>, C::THREADS, C::SMEM);
        Occ2<N, MAXI>::p3 = std::max(1, b);
        Occ2<N, MAXI>::p3a = std::max(1, ba);
    } else {
        using C = RowCfg<N>;
        e |= cudaFuncSetAttribute(p3_fwd_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_STAGED);
        int b = 0;
        e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, p3_fwd_blk<N, MAXI>, C::THREADS, C::SMEM_STAGED);
        Occ2<N, MAXI>::p3 = std::max(1, b);
        e |= cudaFuncSetAttribute(p3_adj_blk<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if constexpr (N == L4S::N)
            e |= cudaFuncSetAttribute(p3_fwd_4s<MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L4S::P3_SMEM);
        if constexpr (kWide<N>) {
            using W = WideCfg<N>;
            int bw = 0;
            e |= cudaFuncSetAttribute(p3_fwd_wide<N, MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)W::SMEM);
            e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bw, p3_fwd_wide<N, MAXI>, W::THREADS, W::SMEM);
            Occ2<N, MAXI>::wide = std::max(1, bw);
        }
        if constexpr (N == HalfCfg::N && MAXI == 1) {   // single solves only (batches keep the defaults)
            int bh = 0;
            e |= cudaFuncSetAttribute(p3_fwd_2h<MAXI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HalfCfg::SMEM);
            e |= cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bh, p3_fwd_2h<MAXI>, HalfCfg::THREADS, HalfCfg::SMEM);
            Occ2<N, MAXI>::half = std::max(1, bh);
        }
    }
    return e;
}

template <int N>
static int prep()
{
    return prep_one<N, 1>() | prep_one<N, BATCH_MAX>();
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
static int units_p3(const PassArgs &a)
{
    const int lines = a.kxn * a.rows1;   // kxn = n0 + 1 except in plane-grouped single solves (p3_fwd1)
    if constexpr (N <= 512) return (lines + WarpCfg<N>::LPW - 1) / WarpCfg<N>::LPW;   // warp-level units
    else return (lines + RowCfg<N>::LPC - 1) / RowCfg<N>::LPC;
}

template <int N>
static int units_wide(const PassArgs &a)
{
    if constexpr (kWide<N>) return ((a.n0 + 1) * a.rows1 + WideCfg<N>::LPC - 1) / WideCfg<N>::LPC;
    else return 0;
}

template <int N>
static int run(int kind, const PassArgs *items, int n, int flag, int var, cudaStream_t st)
{
    const int cap_sm = sm_count();
    if constexpr (N == HalfCfg::N) {   // variant bit 8 (single solves): the line as two 512-point halves
        if (kind == PASS_P3F && (var & 8) && !(var & 4) && n == 1) {
            Work<1> w = make_work<1>(items, 1, units_wide<N>);
            const int grid = std::min(w.offs[1], cap_sm * ((var & 2) ? 1 : Occ2<N, 1>::half));
            return launch_pdl_if(kLongPdl<N>, p3_fwd_2h<1>, grid, HalfCfg::THREADS, HalfCfg::SMEM, st, w, flag);
        }
    }
    if constexpr (kWide<N>) {
        if (kind == PASS_P3F && !(var & 4)) {
            return chunked(items, n, units_wide<N>, [&](auto &w) {
                constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
                const int total = w.offs[w.nitems];
                const int grid = std::min(total, cap_sm * ((var & 2) ? 1 : Occ2<N, MAXI>::wide));
                return launch_pdl_if(kLongPdl<N>, p3_fwd_wide<N, MAXI>, grid, WideCfg<N>::THREADS, WideCfg<N>::SMEM,
                                     st, w, flag);
            });
        }
    }
    return chunked(items, n, units_p3<N>, [&](auto &w) {
        constexpr int MAXI = std::decay_t<decltype(w)>::max_items;
        const int total = w.offs[w.nitems];
        if constexpr (N <= 512) {
            using C = WarpCfg<N>;
            const int ctas = (total + C::WARPS - 1) / C::WARPS;
            // variant bit 2: one CTA per SM (else as many as fit); bit 8 (single
            // solves): the second radix split of the length
            const bool one = (var & 2) != 0;
            constexpr int AB = Plan16B<N>::HAS ? 1 : 0;   // (keeps the branch below well-formed for every N)
            if constexpr (AB && MAXI == 1 && FSP_P3_ONE) {
                using CB = WarpCfg<N, AB>;
                if (kind == PASS_P3F && (var & 8))
                    return launch_pdl(p3_fwd1<N, AB>, std::min((total + CB::WARPS - 1) / CB::WARPS,
                                                              cap_sm * (one ? 1 : Occ2<N, MAXI>::p3oneB)),
                                      CB::THREADS, CB::SMEM, st, w.item[0], flag);
            }
            if (kind == PASS_P3F && MAXI == 1 && FSP_P3_ONE)
                return launch_pdl(p3_fwd1<N>, std::min(ctas, cap_sm * (one ? 1 : Occ2<N, MAXI>::p3one)), C::THREADS,
                                  C::SMEM, st, w.item[0], flag);
            else if (kind == PASS_P3F)
                return launch_pdl(p3_fwd<N, MAXI>, std::min(ctas, cap_sm * (one ? 1 : Occ2<N, MAXI>::p3)), C::THREADS,
                                  C::SMEM, st, w, flag);
            else
                return launch_pdl(p3_adj<N, MAXI>, std::min(ctas, cap_sm * (one ? 1 : Occ2<N, MAXI>::p3a)), C::THREADS,
                                  C::SMEM, st, w, flag);
        } else {
            using C = RowCfg<N>;
            // 8192-point lines: the four-step pass unless variant bit 4 asks for the block kernel
            if constexpr (N == L4S::N) {
                if (kind == PASS_P3F && !(var & 4))
                    return launch_pdl_if(kLongPdl<N>, p3_fwd_4s<MAXI>, std::min(total, cap_sm), L4S::THREADS,
                                         L4S::P3_SMEM, st, w, flag);
            }
            if (kind == PASS_P3F)
                return launch_pdl_if(kLongPdl<N>, p3_fwd_blk<N, MAXI>, std::min(total, cap_sm * ((var & 2) ? 1 : Occ2<N, MAXI>::p3)),
                                  C::THREADS, C::SMEM_STAGED, st, w, flag);
            else p3_adj_blk<N, MAXI><<<total, C::THREADS, C::SMEM, st>>>(w, flag);
        }
        return (int)cudaGetLastError();
    });
}

int has_radix_plan_b(int N)
{
    switch (N) {
#define X(n) case n: return Plan16B<n>::HAS ? 1 : 0;
        FSP_AXIS2_SIZES(X)
#undef X
    default: return 0;
    }
}

int launch_axis2(int kind, int N, const PassArgs *items, int n, int flag, int var, cudaStream_t st)
{
    if (kind != PASS_P3F && kind != PASS_P3A) return (int)cudaErrorInvalidValue;
    switch (N) {
#define X(v) case v: return run<v>(kind, items, n, flag, var, st);
        FSP_AXIS2_SIZES(X)
#undef X
    default: return (int)cudaErrorInvalidValue;
    }
}

// Gathered blocks of every pass (TW_GALL layout) after the N-entry table, for
// the long-line lengths; count of those entries, 0 for other lengths.
int twiddle_gall_entries(int N)
{
    switch (N) {
#define X(n) case n: return AuxEndAll<1, 0, typename Plan1D<n>::R>::value;
        X(768) X(1024) X(1536) X(2048) X(4096) X(8192)
#undef X
    default: return 0;
    }
}

int make_twiddles_gall(float2 *tw, int N, cudaStream_t st)
{
    switch (N) {
#define X(n) \
    case n: k_twiddles_gall<n, typename Plan1D<n>::R><<<(n + 255) / 256, 256, 0, st>>>(tw); return (int)cudaGetLastError();
        X(768) X(1024) X(1536) X(2048) X(4096) X(8192)
#undef X
    default: return 0;
    }
}

// Gathered blocks of Plan16<N> after the N-entry table, then those of
// Plan16B<N> where the length has a second radix split.
template <int N>
static int fill_aux(float2 *tw, cudaStream_t st)
{
    k_twiddles_aux<N, typename Plan16<N>::R><<<4, 256, 0, st>>>(tw);
    if constexpr (Plan16B<N>::HAS) {
        static_assert(AuxEnd<1, AuxOff<N, 1>::value, typename Plan16B<N>::R>::value <= TW_AUX,
                      "both plans' gathered blocks must fit the table's spare entries");
        k_twiddles_aux<N, typename Plan16B<N>::R, AuxOff<N, 1>::value><<<4, 256, 0, st>>>(tw);
    }
    return (int)cudaGetLastError();
}

int make_twiddles_aux(float2 *tw, int N, cudaStream_t st)
{
    switch (N) {
#define X(n) \
    case n: return fill_aux<n>(tw, st);
        X(32) X(64) X(96) X(128) X(192) X(256) X(384) X(512)
#undef X
    default: return 0;   // block-mode lengths use the main table only
    }
}

} // namespace fsp
