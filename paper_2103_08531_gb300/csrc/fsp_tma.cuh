// fsp_tma.cuh -- tensor-memory-access (TMA) staging for the column passes.
//
// The column passes (P1, P2, P4, P5) move tiles of 16 consecutive axis-2
// columns (one 128-byte row segment per line position) between HBM and the
// SM.  Here one thread per CTA issues the tile loads as bulk tensor copies
// (cp.async.bulk.tensor) that land in shared memory in the 128-byte swizzled
// layout and signal an mbarrier with their byte count; the other threads only
// wait on that barrier.  The tile's columns are then transformed by four
// independent groups of threads, four columns each, which synchronise among
// themselves only (a named barrier per group, or the warp when a group is one
// warp), so the groups of a CTA and the loads of the next tile overlap
// instead of running in lock step.
//
// Shared-memory layouts (float2 = one complex value, or two reals in P1):
//   stage: the TMA box as delivered, row r (line position) at r * 128 bytes,
//          the 16-byte chunk of columns (2c, 2c+1) at chunk c ^ (r & 7);
//          every box starts on a 1024-byte boundary.
//   group exchange buffer: position p of the group's column cl at
//          4 * sw(p) + cl, sw(p) = (p & ~3) | ((p ^ (p >> 2) ^ (p >> 4)) & 3):
//          the four positions a half-warp touches in every Stockham exchange
//          of the radix plans used here fall in four different 32-byte bank
//          groups (checked exhaustively for 2n = 64 ... 512 on the host).
//
// Every wait is bounded: a wait that has not seen its barrier phase complete
// after kWaitNs nanoseconds records FSP_ERR_TIMEOUT in the solve's status
// word and the CTA leaves its loop.
#pragma once

#include "../../include/fsp.h"
#include "fsp_passes.cuh"

#include <cuda.h>
#include <stdint.h>

namespace fsp {

// Tensor maps passed by value as __grid_constant__ kernel parameters.
struct TmaMaps {
    CUtensorMap m[2];
};

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make the initialised barrier visible to the async proxy (the TMA unit).
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arrive once and add `bytes` to the transactions the current phase waits for.
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete, at most kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > kWaitNs) return false;
    return true;
}
// Order this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies into shared memory (async proxy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
                     "r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// OR of `pred` over the `count` threads of named barrier `id` (a multiple of 32 threads).
__device__ __forceinline__ bool bar_or(int id, int count, bool pred)
{
    unsigned r;
    asm volatile("{\n\t.reg .pred p, q;\n\t"
                 "setp.ne.u32 p, %1, 0;\n\t"
                 "bar.red.or.pred q, %2, %3, p;\n\t"
                 "selp.u32 %0, 1, 0, q;\n\t}"
                 : "=r"(r)
                 : "r"((unsigned)pred), "r"(id), "r"(count)
                 : "memory");
    return r != 0;
}

// Element (row, col) of a 16-column stage in the 128-byte swizzled layout.
__device__ __forceinline__ int sw128(int row, int col) { return row * 16 + ((((col >> 1) ^ row) & 7) << 1) + (col & 1); }

// Exchange buffer of one group of four columns (see the file comment).
struct GroupView {
    float2 *base;   // group buffer + column
    __device__ __forceinline__ float2 &at(int p) const
    {
        return base[((p & ~3) | ((p ^ (p >> 2) ^ (p >> 4)) & 3)) << 2];
    }
};

// Geometry of the group-tiled passes at padded length N.
template <int N>
struct GroupCfg {
    static constexpr int E = Plan16<N>::E;
    static constexpr int T = N / E;                    // threads per column
    static constexpr int C = 16;                       // columns per tile
    static constexpr int GC = 4;                       // columns per group
    static constexpr int GT = GC * T;                  // threads per group
    static constexpr int GROUPS = C / GC;
    static constexpr int THREADS = GT * GROUPS;
    static constexpr int WARPS = THREADS / 32;
    static_assert(GT % 32 == 0, "a group is a whole number of warps");
    static constexpr int SYNC = GT == 32 ? SYNC_WARP : SYNC_GROUP0 + GT / 32;
    using RAD = typename Plan16<N>::R;
    static constexpr int TWS = AuxEnd<1, N, RAD>::value;   // main table + gathered blocks
    static constexpr int EXG = N * GC;                       // float2 per group exchange buffer
    static constexpr int BOX = N / 2 < 256 ? N / 2 : 256;     // rows per TMA box for a half line
};

// Record a device-side failure in the solve's status word (first one wins).
__device__ __forceinline__ void record_status(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// The shared-memory plan of a group-tiled kernel: `stages` stage buffers of
// `rows` rows each (1024-byte aligned), the group exchange buffers, the
// twiddle copy, the barrier and the reader count.
template <int N>
struct GroupSmem {
    using C = GroupCfg<N>;
    static constexpr size_t stage_bytes(int rows) { return ((size_t)rows * 128 + 1023) / 1024 * 1024; }
    static constexpr size_t bytes(int stages, int rows)
    {
        return 1024 /* alignment slack */ + stages * stage_bytes(rows) + (size_t)C::GROUPS * C::EXG * sizeof(float2) +
               (size_t)C::TWS * sizeof(float2) + 16;
    }
};

struct GroupPtrs {
    float2 *stage[3];
    float2 *ex, *tw;
    uint64_t *bar;
    int *taken;
};

template <int N>
__device__ __forceinline__ GroupPtrs group_smem(unsigned char *raw, int stages, int rows)
{
    using C = GroupCfg<N>;
    GroupPtrs p;
    // align the shared-space offset (the address the TMA unit and the swizzle see)
    const unsigned off = smem_u32(raw);
    const uintptr_t a = reinterpret_cast<uintptr_t>(raw) + (((off + 1023u) & ~1023u) - off);
    unsigned char *b = reinterpret_cast<unsigned char *>(a);
    for (int s = 0; s < 3; ++s) {
        p.stage[s] = reinterpret_cast<float2 *>(b);
        if (s < stages) b += GroupSmem<N>::stage_bytes(rows);
    }
    p.ex = reinterpret_cast<float2 *>(b);
    b += (size_t)C::GROUPS * C::EXG * sizeof(float2);
    p.tw = reinterpret_cast<float2 *>(b);
    b += (size_t)C::TWS * sizeof(float2);
    p.bar = reinterpret_cast<uint64_t *>(b);
    p.taken = reinterpret_cast<int *>(b + 8);
    return p;
}

// Common prologue: twiddle copy, barrier init (thread 0), block barrier.
template <int N>
__device__ __forceinline__ void group_prologue(const GroupPtrs &s, const float2 *gtw)
{
    using C = GroupCfg<N>;
    for (int i = threadIdx.x; i < C::TWS; i += C::THREADS) s.tw[i] = gtw[i];
    if (threadIdx.x == 0) {
        mbar_init(s.bar, 1);
        *s.taken = 0;
        mbar_init_fence();
    }
    __syncthreads();
}

// Called by every warp once it has read the current stage into registers: the
// last warp to do so releases the stage and calls issue() for the next tile.
template <int N, class Issue>
__device__ __forceinline__ void group_release(const GroupPtrs &s, Issue &&issue)
{
    using C = GroupCfg<N>;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        __threadfence_block();
        if (atomicAdd(s.taken, 1) == C::WARPS - 1) {
            atomicExch(s.taken, 0);
            __threadfence_block();
            fence_proxy_async();
            issue();
        }
    }
}

// Bounded wait on the stage barrier, agreed on by the whole group: returns
// false (for every thread of the group) if any of its threads timed out.
template <int N>
__device__ __forceinline__ bool group_wait(const GroupPtrs &s, unsigned parity, int *status)
{
    using C = GroupCfg<N>;
    const bool ok = mbar_wait(s.bar, parity);
    bool fail;
    if constexpr (C::GT == 32) fail = __any_sync(0xffffffffu, !ok);
    else fail = bar_or(1 + (int)threadIdx.x / C::GT, C::GT, !ok);
    if (fail && (threadIdx.x % C::GT) == 0) record_status(status, FSP_ERR_TIMEOUT);
    return !fail;
}

// ------------------------------------------------------------------ kernels
//
// Each kernel is persistent over tiles (grid <= tiles) and mirrors the
// arithmetic of its cp.async counterpart in fsp_passes.cuh (p1_fwd, p2_fwd,
// p4_fwd, p5_fwd): only the staging, the thread-to-column mapping and the
// synchronisation differ.  Thread mapping: group g = tid / GT owns columns
// 4 g .. 4 g + 3 of the tile; inside it, column cl = t % 4 and line thread
// j = t / 4 (t = tid % GT), so a half-warp covers four line positions of
// four adjacent columns (32 bytes of each of four stage rows).

template <int N>
struct GroupThread {
    using C = GroupCfg<N>;
    int g, cl, j, col;
    __device__ __forceinline__ GroupThread()
    {
        const int tid = threadIdx.x;
        g = tid / C::GT;
        const int t = tid % C::GT;
        cl = t % C::GC;
        j = t / C::GC;
        col = C::GC * g + cl;
    }
};

template <int N, int E, bool INV, bool PRUNE_IN>
__device__ __forceinline__ void group_fft(float2 (&v)[E], int j, const float2 *tw, const GroupView &sm)
{
    using C = GroupCfg<N>;
    line_fft<N, E, INV, PRUNE_IN, typename C::RAD, GroupView, C::SYNC, TW_SMEM>(v, j, tw, sm);
}

// P1: rho column pairs (z, z + 1) of a tile of 32 reals -> half spectrum in k0,
// rows 0 .. n1 - 1 of buf1 (3D) or buf0 (2D).  Unit: (y, tile).  Map 0: rho as
// [n0][n1][n2] floats, box 32 x 1 x N/2.
template <int N>
__global__ void __launch_bounds__(GroupCfg<N>::THREADS, 2) p1_tma(const __grid_constant__ PassArgs a,
                                                                  const __grid_constant__ TmaMaps maps)
{
    using C = GroupCfg<N>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const GroupPtrs s = group_smem<N>(smem_raw, 1, NH);
    group_prologue<N>(s, a.tw0);
    const GroupThread<N> th;
    const int zt = a.n2 / 32, units = a.n1 * zt;
    auto issue = [&](int w) {
        mbar_expect_tx(s.bar, NH * 128);
        tma_load_3d(s.stage[0], &maps.m[0], (w % zt) * 32, w / zt, 0, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (threadIdx.x == 0 && w < units) issue(w);
    const GroupView sm{s.ex + th.g * C::EXG + th.cl};
    float2 *__restrict__ dst = a.three_d ? a.buf1 : a.buf0;
    for (unsigned ph = 0; w < units; w += gridDim.x, ph ^= 1) {
        if (!group_wait<N>(s, ph, a.status)) break;
        const int y = w / zt, z0 = (w % zt) * 32 + 2 * th.col;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? s.stage[0][sw128(th.j + r * T, th.col)] : make_float2(0.f, 0.f);
        const int wn = w + gridDim.x;
        group_release<N>(s, [&] {
            if (wn < units) issue(wn);
        });
        group_fft<N, E, false, true>(v, th.j, s.tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) sm.at(th.j + r * T) = v[r];
        lsync<C::SYNC>();
#pragma unroll
        for (int r = 0; r <= E / 2; ++r) {
            const int k = th.j + r * T;
            if (k <= NH) {
                const float2 q = v[r];
                const float2 m = sm.at(k == 0 ? 0 : N - k);
                float4 o;
                o.x = 0.5f * (q.x + m.x);
                o.y = 0.5f * (q.y - m.y);
                o.z = 0.5f * (q.y + m.y);
                o.w = -0.5f * (q.x - m.x);
                *reinterpret_cast<float4 *>(dst + iidx(a, k, y, z0)) = o;
            }
        }
    }
}

// P2: buf1 rows 0 .. n1 - 1 -> forward axis 1 -> buf0 rows 0 .. 2 n1 - 1.
// Unit: (k0, tile).  Map 0: buf1 as [(n0 + 1) rows1][n2] complex, box 16 x N/2.
template <int N>
__global__ void __launch_bounds__(GroupCfg<N>::THREADS, 2) p2_tma(const __grid_constant__ PassArgs a,
                                                                  const __grid_constant__ TmaMaps maps)
{
    using C = GroupCfg<N>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const GroupPtrs s = group_smem<N>(smem_raw, 1, NH);
    group_prologue<N>(s, a.tw1);
    const GroupThread<N> th;
    const int zt = a.n2 / 16, units = (a.n0 + 1) * zt;
    auto issue = [&](int w) {
        mbar_expect_tx(s.bar, NH * 128);
        tma_load_2d(s.stage[0], &maps.m[0], (w % zt) * 16, (w / zt) * a.rows1, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (threadIdx.x == 0 && w < units) issue(w);
    const GroupView sm{s.ex + th.g * C::EXG + th.cl};
    for (unsigned ph = 0; w < units; w += gridDim.x, ph ^= 1) {
        if (!group_wait<N>(s, ph, a.status)) break;
        const int kx = w / zt, z = (w % zt) * 16 + th.col;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? s.stage[0][sw128(th.j + r * T, th.col)] : make_float2(0.f, 0.f);
        const int wn = w + gridDim.x;
        group_release<N>(s, [&] {
            if (wn < units) issue(wn);
        });
        group_fft<N, E, false, true>(v, th.j, s.tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf0[iidx(a, kx, th.j + r * T, z)] = v[r];
    }
}

// P4: buf0 (phi stream, 2 n1 rows) -> rows [0, n1) phi, rows [n1, 2 n1) -i k1 phi;
// buf1 (E2 stream) -> rows [0, n1).  Unit: (k0, tile).  Maps 0 and 1: buf0 and
// buf1 as [(n0 + 1) rows1][n2] complex, box 16 x min(N, 256).
template <int N>
__global__ void __launch_bounds__(GroupCfg<N>::THREADS, 1) p4_tma(const __grid_constant__ PassArgs a,
                                                                  const __grid_constant__ TmaMaps maps, int withE)
{
    using C = GroupCfg<N>;
    constexpr int E = C::E, T = C::T;
    constexpr int BOXR = N < 256 ? N : 256, NB = N / BOXR;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const GroupPtrs s = group_smem<N>(smem_raw, 2, N);
    group_prologue<N>(s, a.tw1);
    const GroupThread<N> th;
    const int zt = a.n2 / 16, units = (a.n0 + 1) * zt;
    auto issue = [&](int w) {
        mbar_expect_tx(s.bar, (withE ? 2 : 1) * N * 128);
        const int x = (w % zt) * 16, y = (w / zt) * a.rows1;
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            tma_load_2d(s.stage[0] + b * BOXR * 16, &maps.m[0], x, y + b * BOXR, s.bar);
            if (withE) tma_load_2d(s.stage[1] + b * BOXR * 16, &maps.m[1], x, y + b * BOXR, s.bar);
        }
    };
    pdl_wait();
    int w = blockIdx.x;
    if (threadIdx.x == 0 && w < units) issue(w);
    const GroupView sm{s.ex + th.g * C::EXG + th.cl};
    const int n1 = a.n1;
    for (unsigned ph = 0; w < units; w += gridDim.x, ph ^= 1) {
        if (!group_wait<N>(s, ph, a.status)) break;
        const int kx = w / zt, z = (w % zt) * 16 + th.col;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = s.stage[0][sw128(th.j + r * T, th.col)];
            q[r] = withE ? s.stage[1][sw128(th.j + r * T, th.col)] : make_float2(0.f, 0.f);
        }
        const int wn = w + gridDim.x;
        group_release<N>(s, [&] {
            if (wn < units) issue(wn);
        });
        if (withE) {
            group_fft<N, E, true, false>(q, th.j, s.tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf1[iidx(a, kx, th.j + r * T, z)] = q[r];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float kk = wave(th.j + r * T, n1, a.k1s);
                q[r] = make_float2(kk * v[r].y, -kk * v[r].x);
            }
            group_fft<N, E, true, false>(q, th.j, s.tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, n1 + th.j + r * T, z)] = q[r];
        }
        group_fft<N, E, true, false>(v, th.j, s.tw, sm);
#pragma unroll
        for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, th.j + r * T, z)] = v[r];
    }
}

// P5: half spectra in k0 -> real outputs.  Unit: (y, tile).  Maps 0 and 1:
// buf0 and buf1 as [n0 + 1][rows1][n2] complex, box 16 x 1 x N/2 (rows
// k0 < n0); the Nyquist row k0 = n0 comes from global memory directly.
// Stages: 0 the phi stream (buf0 row y), 1 the E1 stream (buf0 row n1 + y in
// 3D, buf1 row y in 2D), 2 the E2 stream (buf1 row y, 3D).
template <int N>
__global__ void __launch_bounds__(GroupCfg<N>::THREADS, 1) p5_tma(const __grid_constant__ PassArgs a,
                                                                  const __grid_constant__ TmaMaps maps)
{
    using C = GroupCfg<N>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const GroupPtrs s = group_smem<N>(smem_raw, 3, NH);
    group_prologue<N>(s, a.tw0);
    const GroupThread<N> th;
    float *phi = a.out[0], *e0 = a.out[1], *e1 = a.out[2], *e2 = a.out[3];
    const bool first = phi || e0, second = e1 != nullptr, three = second && a.three_d;
    const int zt = a.n2 / 16, units = a.n1 * zt;
    auto issue = [&](int w) {
        mbar_expect_tx(s.bar, ((first ? 1 : 0) + (second ? 1 : 0) + (three ? 1 : 0)) * NH * 128);
        const int x = (w % zt) * 16, y = w / zt;
        if (first) tma_load_3d(s.stage[0], &maps.m[0], x, y, 0, s.bar);
        if (second) {
            if (a.three_d) tma_load_3d(s.stage[1], &maps.m[0], x, a.n1 + y, 0, s.bar);
            else tma_load_3d(s.stage[1], &maps.m[1], x, y, 0, s.bar);
        }
        if (three) tma_load_3d(s.stage[2], &maps.m[1], x, y, 0, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (threadIdx.x == 0 && w < units) issue(w);
    const GroupView sm{s.ex + th.g * C::EXG + th.cl};
    for (unsigned ph = 0; w < units; w += gridDim.x, ph ^= 1) {
        const int y = w / zt, z = (w % zt) * 16 + th.col;
        // the Nyquist row (k0 = n0) of each stream, read directly
        float2 pN = make_float2(0.f, 0.f), YN = pN, ZN = pN;
        constexpr int jN = NH % T;
        if (th.j == jN) {
            if (first) pN = a.buf0[iidx(a, NH, y, z)];
            if (second) YN = a.three_d ? a.buf0[iidx(a, NH, a.n1 + y, z)] : a.buf1[iidx(a, NH, y, z)];
            if (three) ZN = a.buf1[iidx(a, NH, y, z)];
        }
        if (!group_wait<N>(s, ph, a.status)) break;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = th.j + r * T;
            const int src = k <= NH ? k : N - k;
            const bool nyq = (r == NH / T) && th.j == jN;   // src == NH only there
            float2 p = make_float2(0.f, 0.f), Y = p, Z = p;
            if (first) p = nyq ? pN : s.stage[0][sw128(src < NH ? src : 0, th.col)];
            if (second) Y = nyq ? YN : s.stage[1][sw128(src < NH ? src : 0, th.col)];
            if (three) Z = nyq ? ZN : s.stage[2][sw128(src < NH ? src : 0, th.col)];
            if (k > NH) {
                p.y = -p.y;
                Y.y = -Y.y;
                Z.y = -Z.y;
            }
            if (e0) p = (1.f + wave(k, NH, a.k0s)) * p;   // W = P + i (-i k0 P)
            v[r] = p;
            q[r] = make_float2(Y.x - Z.y, Y.y + Z.x);        // Y + i Z
        }
        const int wn = w + gridDim.x;
        group_release<N>(s, [&] {
            if (wn < units) issue(wn);
        });
        if (first) {
            group_fft<N, E, true, false>(v, th.j, s.tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, th.j + r * T, y, z);
                if (phi) phi[g] = v[r].x;
                if (e0) e0[g] = v[r].y;
            }
        }
        if (second) {
            group_fft<N, E, true, false>(q, th.j, s.tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, th.j + r * T, y, z);
                e1[g] = q[r].x;
                if (a.three_d) e2[g] = q[r].y;
            }
        }
    }
}

} // namespace fsp
