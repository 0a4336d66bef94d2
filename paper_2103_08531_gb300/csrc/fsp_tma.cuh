// fsp_tma.cuh -- tensor-memory-access (TMA) staging for the column passes.
//
// The column passes (P1, P2, P4, P5) move tiles of 16 consecutive axis-2
// columns (one 128-byte row segment per line position) between HBM and the
// SM.  Here one thread per CTA issues each tile's loads as bulk tensor copies
// (cp.async.bulk.tensor) that land in shared memory in the 128-byte swizzled
// layout and signal an mbarrier with their byte count, instead of every
// thread copying 16-byte pieces; the next tile is in flight while the current
// one is transformed.
//
// Shared-memory layout of a stage (float2 = one complex value, or two reals
// in P1): the TMA box as delivered, row r (line position) at r * 128 bytes,
// the 16-byte chunk of columns (2c, 2c+1) at chunk c ^ (r & 7); every box
// starts on a 1024-byte boundary.  A half-warp reads one row (its 16 lanes
// are the 16 columns), so the swizzle only permutes the chunks of that row:
// no bank conflicts.
//
// Every wait is bounded: a wait that has not seen its barrier phase complete
// after kWaitNs nanoseconds records FSP_ERR_TIMEOUT in the solve's status
// word, and the CTA (agreeing through its block barrier) leaves its loop.
#pragma once

#include "../../include/fsp.h"
#include "fsp_passes.cuh"

#include <cuda.h>
#include <stdint.h>

namespace fsp {

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
// Wait for the phase with the given parity to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned long long limit_ns = kWaitNs)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() - t0 > limit_ns) return false;
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

// Element (row, col) of a 16-column stage in the 128-byte swizzled layout.
__device__ __forceinline__ int sw128(int row, int col) { return row * 16 + ((((col >> 1) ^ row) & 7) << 1) + (col & 1); }


// Record a device-side failure in the solve's status word (first one wins).
__device__ __forceinline__ void record_status(int *status, int code)
{
    if (status) atomicCAS(status, 0, code);
}

// Shared memory of a TMA-staged tile kernel: alignment slack, `stages` stage
// buffers of `rows` 128-byte rows (each rounded up to 1024 bytes), the tile
// exchange buffer with the twiddle copy after it (TileCfg::EX), the barrier.
template <int N>
struct TmaTile {
    using C = TileCfg<N, 16>;
    static constexpr size_t stage_bytes(int rows) { return ((size_t)rows * 128 + 1023) / 1024 * 1024; }
    static constexpr size_t smem(int stages, int rows)
    {
        return 1024 + stages * stage_bytes(rows) + (size_t)C::EX * sizeof(float2) + 16;
    }
};

struct TmaSmem {
    float2 *stage[3];
    float2 *ex;
    uint64_t *bar;
};

template <int N>
__device__ __forceinline__ TmaSmem tma_smem(unsigned char *raw, int stages, int rows)
{
    // align the shared-space offset (what the TMA unit and the swizzle see)
    const unsigned off = smem_u32(raw);
    unsigned char *b = raw + (((off + 1023u) & ~1023u) - off);
    TmaSmem s;
    for (int i = 0; i < 3; ++i) {
        s.stage[i] = reinterpret_cast<float2 *>(b);
        if (i < stages) b += TmaTile<N>::stage_bytes(rows);
    }
    s.ex = reinterpret_cast<float2 *>(b);
    s.bar = reinterpret_cast<uint64_t *>(b + (size_t)TileCfg<N, 16>::EX * sizeof(float2));
    return s;
}

// Barrier set-up by thread 0; the caller's next block barrier publishes it.
__device__ __forceinline__ void tma_bar_setup(uint64_t *bar)
{
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
}

// After the stage has been read into registers: true (for every thread) if
// any thread's wait timed out; then thread 0 records it and waits once more,
// bounded, for the copies that may still be in flight.
__device__ __forceinline__ bool tma_tile_failed(bool ok, uint64_t *bar, unsigned parity, int *status)
{
    if (!__syncthreads_or(!ok)) return false;
    if (threadIdx.x == 0) {
        record_status(status, FSP_ERR_TIMEOUT);
        mbar_wait(bar, parity);
    }
    return true;
}

// ------------------------------------------------------------------ kernels
//
// Persistent over tiles (grid <= tiles) of up to MAXI independent solves (a
// Work list, as the other batched passes; MAXI = 1 for one solve), each item
// with its own tensor maps.  Each kernel mirrors the arithmetic and the
// thread mapping of its cp.async counterpart in fsp_passes.cuh (p1_fwd,
// p2_fwd, p4_fwd, p5_fwd: column = tid % 16, line thread j = tid / 16,
// block-synchronous transforms through the [position][16] exchange buffer);
// only the staging differs.  After the block barrier that ends the reads of a
// stage, thread 0 issues the next tile's copies into it.  ALT = 1 transforms
// with the second radix split of the length (Plan16B, tuned variant bit 8).

template <int MAXI>
struct TmaBatch {
    CUtensorMap m[MAXI][2];
};

// P1: rho column pairs (z, z + 1) of a tile of 32 reals -> half spectrum in
// k0, rows 0 .. n1 - 1 of buf1 (3D) or buf0 (2D).  Unit: (y, tile).  Map 0:
// rho as [n0][n1][n2] floats, box 32 x 1 x N/2.
template <int N, int MAXI, int ALT = 0>
__global__ void __launch_bounds__(TileCfg<N, 16>::THREADS) p1_tma(const __grid_constant__ Work<MAXI> W,
                                                                  const __grid_constant__ TmaBatch<MAXI> maps)
{
    using C = TileCfg<N, 16, ALT>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const TmaSmem s = tma_smem<N>(smem_raw, 1, NH);
    const int tid = threadIdx.x, col = tid % 16, j = tid / 16;
    const int nw = W.count();
    tma_bar_setup(s.bar);
    const float2 *tw = C::twiddles(s.ex, W.item[0].tw0);   // (its block barrier also publishes the mbarrier)
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int zt = b.n2 / 32;
        mbar_expect_tx(s.bar, NH * 128);
        tma_load_3d(s.stage[0], &maps.m[it_ub][0], (ub % zt) * 32, ub / zt, 0, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (tid == 0 && w < nw) issue(w);
    const ColView sm{s.ex + col, 16};
    for (unsigned ph = 0; w < nw; w += gridDim.x, ph ^= 1) {
        const bool ok = mbar_wait(s.bar, ph);
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / 32;
        const int y = u / zt, z0 = (u % zt) * 32 + 2 * col;
        float2 *__restrict__ dst = a.three_d ? a.buf1 : a.buf0;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? s.stage[0][sw128(j + r * T, col)] : make_float2(0.f, 0.f);
        if (tma_tile_failed(ok, s.bar, ph, a.status)) break;
        if (tid == 0 && w + (int)gridDim.x < nw) {
            fence_proxy_async();
            issue(w + gridDim.x);
        }
        tile_fft<N, E, false, true, RAD>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) sm.at(j + r * T) = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r <= E / 2; ++r) {
            const int k = j + r * T;
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
        __syncthreads();   // the exchange buffer is reused by the next tile
    }
}

// P2: buf1 rows 0 .. n1 - 1 -> forward axis 1 -> buf0 rows 0 .. 2 n1 - 1.
// Unit: (k0, tile) over planes [kx0, kx0 + kxn).  Map 0: buf1 as
// [(n0 + 1) rows1][n2] complex, box 16 x N/2.
template <int N, int MAXI, int ALT = 0>
__global__ void __launch_bounds__(TileCfg<N, 16>::THREADS) p2_tma(const __grid_constant__ Work<MAXI> W,
                                                                  const __grid_constant__ TmaBatch<MAXI> maps)
{
    using C = TileCfg<N, 16, ALT>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const TmaSmem s = tma_smem<N>(smem_raw, 1, NH);
    const int tid = threadIdx.x, col = tid % 16, j = tid / 16;
    const int nw = W.count();
    tma_bar_setup(s.bar);
    const float2 *tw = C::twiddles(s.ex, W.item[0].tw1);
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int zt = b.n2 / 16;
        mbar_expect_tx(s.bar, NH * 128);
        tma_load_2d(s.stage[0], &maps.m[it_ub][0], (ub % zt) * 16, (b.kx0 + ub / zt) * b.rows1, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (tid == 0 && w < nw) issue(w);
    const ColView sm{s.ex + col, 16};
    for (unsigned ph = 0; w < nw; w += gridDim.x, ph ^= 1) {
        const bool ok = mbar_wait(s.bar, ph);
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / 16;
        const int kx = a.kx0 + u / zt, z = (u % zt) * 16 + col;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? s.stage[0][sw128(j + r * T, col)] : make_float2(0.f, 0.f);
        if (tma_tile_failed(ok, s.bar, ph, a.status)) break;
        if (tid == 0 && w + (int)gridDim.x < nw) {
            fence_proxy_async();
            issue(w + gridDim.x);
        }
        tile_fft<N, E, false, true, RAD>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
    }
}

// P4: buf0 (phi stream, 2 n1 rows) -> rows [0, n1) phi, rows [n1, 2 n1) -i k1 phi;
// buf1 (E2 stream) -> rows [0, n1).  Unit: (k0, tile) over planes [kx0, kx0 + kxn).
// Maps 0 and 1: buf0 and buf1 as [(n0 + 1) rows1][n2] complex, box 16 x min(N, 256).
template <int N, int MAXI, int ALT = 0>
__global__ void __launch_bounds__(TileCfg<N, 16>::THREADS) p4_tma(const __grid_constant__ Work<MAXI> W,
                                                                  const __grid_constant__ TmaBatch<MAXI> maps, int withE)
{
    using C = TileCfg<N, 16, ALT>;
    constexpr int E = C::E, T = C::T;
    constexpr int BOXR = N < 256 ? N : 256, NB = N / BOXR;
    using RAD = typename C::RAD;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const TmaSmem s = tma_smem<N>(smem_raw, 2, N);
    const int tid = threadIdx.x, col = tid % 16, j = tid / 16;
    const int nw = W.count();
    tma_bar_setup(s.bar);
    const float2 *tw = C::twiddles(s.ex, W.item[0].tw1);
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int zt = b.n2 / 16;
        mbar_expect_tx(s.bar, (withE ? 2 : 1) * N * 128);
        const int x = (ub % zt) * 16, y = (b.kx0 + ub / zt) * b.rows1;
#pragma unroll
        for (int bx = 0; bx < NB; ++bx) {
            tma_load_2d(s.stage[0] + bx * BOXR * 16, &maps.m[it_ub][0], x, y + bx * BOXR, s.bar);
            if (withE) tma_load_2d(s.stage[1] + bx * BOXR * 16, &maps.m[it_ub][1], x, y + bx * BOXR, s.bar);
        }
    };
    pdl_wait();
    int w = blockIdx.x;
    if (tid == 0 && w < nw) issue(w);
    const ColView sm{s.ex + col, 16};
    for (unsigned ph = 0; w < nw; w += gridDim.x, ph ^= 1) {
        const bool ok = mbar_wait(s.bar, ph);
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / 16, n1 = a.n1;
        const int kx = a.kx0 + u / zt, z = (u % zt) * 16 + col;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = s.stage[0][sw128(j + r * T, col)];
            q[r] = withE ? s.stage[1][sw128(j + r * T, col)] : make_float2(0.f, 0.f);
        }
        if (tma_tile_failed(ok, s.bar, ph, a.status)) break;
        if (tid == 0 && w + (int)gridDim.x < nw) {
            fence_proxy_async();
            issue(w + gridDim.x);
        }
        if (withE) {
            tile_fft<N, E, true, false, RAD>(q, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf1[iidx(a, kx, j + r * T, z)] = q[r];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float kk = wave(j + r * T, n1, a.k1s);
                q[r] = make_float2(kk * v[r].y, -kk * v[r].x);
            }
            tile_fft<N, E, true, false, RAD>(q, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, n1 + j + r * T, z)] = q[r];
        }
        tile_fft<N, E, true, false, RAD>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
    }
}

// P5: half spectra in k0 -> real outputs.  Unit: (y, tile).  Maps 0 and 1:
// buf0 and buf1 as [n0 + 1][rows1][n2] complex, box 16 x 1 x N/2 (rows
// k0 < n0); the Nyquist row k0 = n0 is read from global memory directly.
// Stages: 0 the phi stream (buf0 row y), 1 the E1 stream (buf0 row n1 + y in
// 3D, buf1 row y in 2D), 2 the E2 stream (buf1 row y, 3D).  Which streams an
// item has follows its outputs.
template <int N, int MAXI, int ALT = 0>
__global__ void __launch_bounds__(TileCfg<N, 16>::THREADS) p5_tma(const __grid_constant__ Work<MAXI> W,
                                                                  const __grid_constant__ TmaBatch<MAXI> maps)
{
    using C = TileCfg<N, 16, ALT>;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const TmaSmem s = tma_smem<N>(smem_raw, 3, NH);
    const int tid = threadIdx.x, col = tid % 16, j = tid / 16;
    const int nw = W.count();
    tma_bar_setup(s.bar);
    const float2 *tw = C::twiddles(s.ex, W.item[0].tw0);
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const bool first = b.out[0] || b.out[1], second = b.out[2] != nullptr, three = second && b.three_d;
        const int zt = b.n2 / 16;
        mbar_expect_tx(s.bar, ((first ? 1 : 0) + (second ? 1 : 0) + (three ? 1 : 0)) * NH * 128);
        const int x = (ub % zt) * 16, y = ub / zt;
        if (first) tma_load_3d(s.stage[0], &maps.m[it_ub][0], x, y, 0, s.bar);
        if (second) {
            if (b.three_d) tma_load_3d(s.stage[1], &maps.m[it_ub][0], x, b.n1 + y, 0, s.bar);
            else tma_load_3d(s.stage[1], &maps.m[it_ub][1], x, y, 0, s.bar);
        }
        if (three) tma_load_3d(s.stage[2], &maps.m[it_ub][1], x, y, 0, s.bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (tid == 0 && w < nw) issue(w);
    const ColView sm{s.ex + col, 16};
    constexpr int jN = NH % T, rN = NH / T;   // the thread and register holding k = NH
    for (unsigned ph = 0; w < nw; w += gridDim.x, ph ^= 1) {
        FSP_UNIT(W, w, a, u);
        float *phi = a.out[0], *e0 = a.out[1], *e1 = a.out[2], *e2 = a.out[3];
        const bool first = phi || e0, second = e1 != nullptr, three = second && a.three_d;
        const int zt = a.n2 / 16;
        const int y = u / zt, z = (u % zt) * 16 + col;
        // the Nyquist row (k0 = n0) of each stream, read directly
        float2 pN = make_float2(0.f, 0.f), YN = pN, ZN = pN;
        if (j == jN) {
            if (first) pN = a.buf0[iidx(a, NH, y, z)];
            if (second) YN = a.three_d ? a.buf0[iidx(a, NH, a.n1 + y, z)] : a.buf1[iidx(a, NH, y, z)];
            if (three) ZN = a.buf1[iidx(a, NH, y, z)];
        }
        const bool ok = mbar_wait(s.bar, ph);
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int src = k <= NH ? k : N - k;
            const bool nyq = r == rN && j == jN;   // src == NH only there
            const int row = src < NH ? src : 0;
            float2 p = make_float2(0.f, 0.f), Y = p, Z = p;
            if (first) p = nyq ? pN : s.stage[0][sw128(row, col)];
            if (second) Y = nyq ? YN : s.stage[1][sw128(row, col)];
            if (three) Z = nyq ? ZN : s.stage[2][sw128(row, col)];
            if (k > NH) {
                p.y = -p.y;
                Y.y = -Y.y;
                Z.y = -Z.y;
            }
            if (e0) p = (1.f + wave(k, NH, a.k0s)) * p;   // W = P + i (-i k0 P)
            v[r] = p;
            q[r] = make_float2(Y.x - Z.y, Y.y + Z.x);        // Y + i Z
        }
        if (tma_tile_failed(ok, s.bar, ph, a.status)) break;
        if (tid == 0 && w + (int)gridDim.x < nw) {
            fence_proxy_async();
            issue(w + gridDim.x);
        }
        if (first) {
            tile_fft<N, E, true, false, RAD>(v, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, j + r * T, y, z);
                if (phi) phi[g] = v[r].x;
                if (e0) e0[g] = v[r].y;
            }
        }
        if (second) {
            tile_fft<N, E, true, false, RAD>(q, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, j + r * T, y, z);
                e1[g] = q[r].x;
                if (a.three_d) e2[g] = q[r].y;
            }
        }
    }
}

} // namespace fsp
