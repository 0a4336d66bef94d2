// fsp_long.cuh -- 8192-point lines of the 2D solve (2n = 8192, a 4096^2 grid)
// as four-step splits, 8192 = 16 x 512: inside one CTA for the middle pass,
// through global memory for the C2R columns.
//
// Forward (n = 512 n1 + n2, k = k1 + 16 k2):
//   X[k1 + 16 k2] = sum_n2 W_512^(n2 k2) W_8192^(n2 k1) sum_n1 x[512 n1 + n2] W_16^(n1 k1)
// Step A: thread t = n2 of the 512 takes the 16-point DFT over n1 (half of the
// inputs are the implied zero padding, Sec. 2) and multiplies output k1 by
// W_8192^(t k1); the results form 16 rows of 512.  Step B: warp k1 transforms
// its row (512 points, warp-synchronous, the engine of the 3D middle pass) and
// holds X[k1 + 16 k2] at k2 = lane + 32 r.  The inverse runs the two steps in
// the other order; cropping to the first half of the line is then the first
// half of the 16-point outputs (n1 < 8).
//
// Against one block-synchronous 8192-point transform (four radix passes,
// three exchanges of the whole line through shared memory, two block barriers
// each) a line needs two block barriers per transform, and the 512-point
// parts run on 16 independent warps.  The C2R columns (axis 0) cannot hold
// more than two such columns per CTA, so they take the split through global
// memory instead (p5_4s_a / p5_4s_b below), where every access is a whole
// row segment of 16 or 32 columns.
#pragma once

#include "fsp_tma.cuh"

namespace fsp {

// 1D bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global memory into shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 4-byte asynchronous copy global -> shared (through L1).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem_dst)), "l"(gmem_src) : "memory");
}

struct L4S {
    static constexpr int N = 8192, N1 = 16, N2 = 512, NH = N / 2;
    static constexpr int THREADS = 512;
    using RAD = typename Plan16<N2>::R;                 // 16 16 2, one warp per 512-point row
    static constexpr int RL = RowSpan<N2, 4>::value;    // row span (one padding slot per 16)
    static constexpr int TWS = AuxEnd<1, N2, RAD>::value;   // 512-point table + gathered block
    static constexpr int KSL = N2 + 2;                  // transposed kernel row stride (floats)
    // shared memory, in bytes (every region a multiple of 16)
    static constexpr size_t ROWS = (size_t)N1 * RL * 8;       // 16 exchange rows
    static constexpr size_t LINE = (size_t)N * 8;             // one full line of complex values
    static constexpr size_t TWB = (size_t)TWS * 8;
    static constexpr size_t KSB = ((size_t)N1 * KSL * 4 + 15) / 16 * 16;
    // middle pass: rows, saved E spectrum (a line), stage (half a line), 512-point table, kernel row, barrier
    static constexpr size_t P3_SMEM = ROWS + LINE + LINE / 2 + TWB + KSB + 16;
};

// Per-thread twiddle bases W_8192^(s t) for s = 1, 2, 4, 8 (exact table
// entries), from which every W_8192^(t k1), k1 < 16, is a product of at most
// three.
struct TwBase {
    float2 w1, w2, w4, w8;
};
__device__ __forceinline__ TwBase tw_base(const float2 *__restrict__ tw8192, int t)
{
    return TwBase{__ldg(tw8192 + t), __ldg(tw8192 + 2 * t), __ldg(tw8192 + 4 * t), __ldg(tw8192 + 8 * t)};
}
// u[k] *= W^(t k) (conjugate for the inverse), k = 1 .. 15.
template <bool INV>
__device__ __forceinline__ void twiddle16(float2 (&u)[16], const TwBase &b)
{
    const float2 w3 = cmul(b.w1, b.w2), w5 = cmul(b.w4, b.w1), w6 = cmul(b.w4, b.w2), w7 = cmul(b.w4, w3);
    const float2 w[16] = {make_float2(1.f, 0.f), b.w1, b.w2, w3, b.w4, w5, w6, w7, b.w8, cmul(b.w8, b.w1),
                          cmul(b.w8, b.w2), cmul(b.w8, w3), cmul(b.w8, b.w4), cmul(b.w8, w5), cmul(b.w8, w6),
                          cmul(b.w8, w7)};
#pragma unroll
    for (int k = 1; k < 16; ++k) u[k] = cmul_dir<INV>(u[k], w[k]);
}

// The 512-point table in the TW_SMEM layout (W_512^m, then the gathered block
// of the second radix-16 pass, W_512^(2 r k)), copied from the 8192-point
// table (W_512^m = W_8192^(16 m): the same FP64 angle, the same rounding).
__device__ __forceinline__ void tw512_from_8192(float2 *stw, const float2 *__restrict__ tw8192)
{
    for (int i = threadIdx.x; i < L4S::TWS; i += blockDim.x) {
        int m;
        if (i < 512) m = 16 * i;
        else m = 32 * ((i - 512) / 16) * ((i - 512) % 16);
        stw[i] = __ldg(tw8192 + m);
    }
}

// Middle pass (axis 2) of 2D solves with 2 n2 = 8192: forward transform of a
// line, times the kernel spectrum, inverse to the phi stream (buf0) and,
// with withE, -i k2 times the product inverse to the E2 stream (buf1).
// Persistent over lines; the next line's input (n2 complex, contiguous) is
// bulk-copied into the stage while the current line is transformed.
template <int MAXI>
__global__ void __launch_bounds__(L4S::THREADS, 1) p3_fwd_4s(const __grid_constant__ Work<MAXI> W, int withE)
{
    using S = L4S;
    constexpr int N = S::N, NH = S::NH, N2 = S::N2;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    float2 *rows = reinterpret_cast<float2 *>(smem_raw);
    float2 *save = reinterpret_cast<float2 *>(smem_raw + S::ROWS);
    float2 *stage = reinterpret_cast<float2 *>(smem_raw + S::ROWS + S::LINE);
    float2 *stw = reinterpret_cast<float2 *>(smem_raw + S::ROWS + S::LINE + S::LINE / 2);
    float *Ks = reinterpret_cast<float *>(smem_raw + S::ROWS + S::LINE + S::LINE / 2 + S::TWB);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + S::ROWS + S::LINE + S::LINE / 2 + S::TWB + S::KSB);
    const int t = threadIdx.x, wp = t >> 5, j = t & 31;
    const int nw = W.count();
    const float2 *tw8192 = W.item[0].tw2;   // every item of the launch has 2 n2 = 8192
    tw512_from_8192(stw, tw8192);
    if (t == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    const TwBase tb = tw_base(tw8192, t);
    __syncthreads();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        mbar_expect_tx(bar, NH * 8);
        bulk_load(stage, b.buf0 + (size_t)(b.kx0 * b.rows1 + ub) * NH, NH * 8, bar);
    };
    pdl_wait();
    int w = blockIdx.x;
    if (t == 0 && w < nw) issue(w);
    // the kernel row of a unit's line, transposed to [k mod 16][k / 16] over
    // the whole line, copied asynchronously (each thread waits for its own
    // copies before the block barrier that ends step A)
    auto fetch_k = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int line = b.kx0 * b.rows1 + ub;
        const float *Kr = krow(b, line / b.rows1, line % b.rows1);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int k = t + N2 * i;
            cp_async4(Ks + (k & 15) * S::KSL + (k >> 4), Kr + (k <= NH ? k : N - k));
        }
        cp_async_commit();
    };
    if (w < nw) fetch_k(w);
    RowView<4> row{rows + wp * S::RL};
    for (unsigned ph = 0; w < nw; w += gridDim.x, ph ^= 1) {
        FSP_UNIT(W, w, a, u);
        const int line = a.kx0 * a.rows1 + u;
        const bool ok = mbar_wait(bar, ph);
        // step A: 16-point DFTs over n1 (inputs n1 >= 8 are the padding)
        float2 x[16];
#pragma unroll
        for (int n1 = 0; n1 < 16; ++n1) x[n1] = n1 < 8 ? stage[t + N2 * n1] : make_float2(0.f, 0.f);
        dft_half_in<16, false>(x);
        twiddle16<false>(x, tb);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) rows[k1 * S::RL + t + (t >> 4)] = x[k1];
        cp_async_wait_all();
        if (__syncthreads_or(!ok)) {   // the rows and the kernel row are complete, the stage is read
            if (t == 0) {
                record_status(a.status, FSP_ERR_TIMEOUT);
                mbar_wait(bar, ph);
            }
            break;
        }
        if (t == 0 && w + (int)gridDim.x < nw) {
            fence_proxy_async();
            issue(w + gridDim.x);
        }
        // step B: warp k1 = wp transforms its row; X[k1 + 16 k2] at k2 = j + 32 r
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = row.at(j + 32 * r);
        line_fft<N2, 16, false, false, S::RAD, RowView<4>, SYNC_WARP, TW_SMEM>(v, j, stw, row);
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const int k2 = j + 32 * r;
            v[r] = Ks[wp * S::KSL + k2] * v[r];
            if (withE) {
                const float kk = wave(wp + 16 * k2, NH, a.k2s);
                save[wp * N2 + k2] = make_float2(kk * v[r].y, -kk * v[r].x);   // -i k2 (K rho^)
            }
        }
        // inverse, phi stream: step B then step A, first half of the line kept
        float2 *L0 = a.buf0 + (size_t)line * NH;
        line_fft<N2, 16, true, false, S::RAD, RowView<4>, SYNC_WARP, TW_SMEM>(v, j, stw, row);
#pragma unroll
        for (int r = 0; r < 16; ++r) row.at(j + 32 * r) = v[r];
        __syncthreads();   // every warp is past its kernel product: the next line's kernel row may land
        if (w + (int)gridDim.x < nw) fetch_k(w + gridDim.x);
#pragma unroll
        for (int k1 = 0; k1 < 16; ++k1) x[k1] = rows[k1 * S::RL + t + (t >> 4)];
        twiddle16<true>(x, tb);
        dft<16, true>(x);
#pragma unroll
        for (int n1 = 0; n1 < 8; ++n1) L0[t + N2 * n1] = x[n1];
        if (withE) {
            __syncthreads();   // the rows are read
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = save[wp * N2 + j + 32 * r];
            line_fft<N2, 16, true, false, S::RAD, RowView<4>, SYNC_WARP, TW_SMEM>(v, j, stw, row);
#pragma unroll
            for (int r = 0; r < 16; ++r) row.at(j + 32 * r) = v[r];
            __syncthreads();
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) x[k1] = rows[k1 * S::RL + t + (t >> 4)];
            twiddle16<true>(x, tb);
            dft<16, true>(x);
            float2 *L1 = a.buf1 + (size_t)line * NH;
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1) L1[t + N2 * n1] = x[n1];
        }
        __syncthreads();   // rows, save and the kernel row are free for the next line
    }
}

// ------------------------------------------------ C2R columns through HBM
//
// The first-axis inverse of 2D solves with 2 n0 = 8192 as a four-step split
// through global memory, k = 512 k1 + k2 and n = n1 + 16 n2:
//   x[n1 + 16 n2] = sum_k2 W_512^(-n2 k2) W_8192^(-n1 k2) sum_k1 X[512 k1 + k2] W_16^(-n1 k1).
// Two columns z0 = 2p, z0 + 1 with half spectra A, B (rows k0 <= NH of a
// buffer) are packed as A + i B, each extended by conjugate symmetry; the
// inverse of the pack is a(z0) + i b(z0 + 1).
// Step 1 (p5_4s_a): the 16-point inverses over k1 with the twiddles
// W_8192^(-n1 k2).  For k2 = t and k2 = 512 - t the inputs are the same 16
// rows (512 a + t, a < 8, and their mirrors 512 b - t, b = 1 .. 8), so one
// thread takes both and writes Y[n1][k2] back into those rows: Y[n1][k2] of
// the pair goes to row 512 (n1 mod 8) + k2, column z0 + (n1 >= 8).  Every
// (row, pair) slot is read and written by one thread only; row NH is read
// (t = 0) and not written.
// Step 2 (p5_4s_b): for fixed n1 = 8 h + a the 512 values Y[n1][k2] are rows
// 512 a .. 512 a + 511 of column 2p + h: a tile pass of 512-point inverses
// over 16 columns, first half kept (n2 < 256), Re -> the field at z0, Im ->
// at z0 + 1.
// Sets: mode 0 takes buf1 (the E1 stream) in place; mode 1 takes buf0 and
// writes the phi set in place (when phi is wanted) and the -i k0 (A + i B)
// set, E0, into buf1 at the same places.  Mode 0 and its step 2 therefore run
// before mode 1.  No workspace beyond buf0 and buf1.

// Step 1.  Unit: a block of 256 threads over (t in [0, 256], pair), pairs
// fastest; mode 0 or 1 for the whole launch.  Persistent; a thread's 16 input
// rows of its next unit are copied (cp.async, 16 bytes each) into its own
// slots of a two-buffer shared stage while the current unit is transformed:
// the in-place stores of a unit never touch the rows of another unit.
struct P5A {
    static constexpr int THREADS = 256;
    static constexpr size_t SMEM = (size_t)2 * 16 * THREADS * sizeof(float4);   // [buffer][row][thread]
};

template <int MAXI>
__global__ void __launch_bounds__(P5A::THREADS) p5_4s_a(const __grid_constant__ Work<MAXI> W, int mode)
{
    constexpr int N = L4S::N, NH = L4S::NH, TH = P5A::THREADS;
    extern __shared__ float4 stg[];
    pdl_trigger();
    pdl_wait();
    const int nw = W.count();
    const int tid = threadIdx.x;
    // rows of unit w for this thread: 512 i + t (slot i) and 512 (i + 1) - t (slot 8 + i)
    auto issue = [&](int w, int bsel) {
        FSP_UNIT(W, w, b, ub);
        const int pairs = b.n2 / 2;
        const int idx = ub * TH + tid;
        if (idx >= 257 * pairs) return;
        const int t = idx / pairs, p = idx % pairs;
        const float4 *col = reinterpret_cast<const float4 *>((mode ? b.buf0 : b.buf1) + 2 * p);
        const size_t ld = (size_t)b.n2 / 2;
        float4 *s = stg + (size_t)bsel * 16 * TH + tid;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            cp_async16(s + i * TH, col + (size_t)(512 * i + t) * ld);
            cp_async16(s + (8 + i) * TH, col + (size_t)(512 * (i + 1) - t) * ld);
        }
    };
    int bsel = 0;
    if ((int)blockIdx.x < nw) issue(blockIdx.x, 0);
    cp_async_commit();
    for (int w = blockIdx.x; w < nw; w += gridDim.x, bsel ^= 1) {
        cp_async_wait_all();
        FSP_UNIT(W, w, a, u);
        const int pairs = a.n2 / 2;
        const int idx = u * TH + tid;
        const bool active = idx < 257 * pairs;
        float4 R[8], M[8];   // rows 512 a + t and 512 b - t (b = a + 1)
        const float4 *s = stg + (size_t)bsel * 16 * TH + tid;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            R[i] = s[i * TH];
            M[i] = s[(8 + i) * TH];
        }
        // the other buffer was read in the previous iteration, whose stores used it
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x, bsel ^ 1);
        cp_async_commit();
        if (!active) continue;
        const int t = idx / pairs, p = idx % pairs;
        float2 *buf = mode ? a.buf0 : a.buf1;
        const bool want0 = mode ? a.out[0] != nullptr : true;   // the set written in place
        const bool want1 = mode && a.out[1] != nullptr;          // -i k0 set into buf1
        const size_t ld = (size_t)a.n2 / 2;   // row stride in float4
        const float2 *tw = a.tw0;   // the 8192-point table
        // one k2 = tt of the pair of offsets; sel 0: tt = t, 1: tt = 512 - t
        auto one = [&](int tt, int sel, bool withk, float2 *dst) {
            float2 x[16];
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                const int k = 512 * k1 + tt;
                float4 q;
                bool cj;
                if (sel == 0) {   // k1 < 8: row 512 k1 + t; else the mirror row 512 (16 - k1) - t
                    q = k1 < 8 ? R[k1] : M[15 - k1];
                    cj = k > NH;
                } else {          // k1 < 8: row 512 (k1 + 1) - t; else the mirror row 512 (15 - k1) + t
                    q = k1 < 8 ? M[k1] : R[15 - k1];
                    cj = k1 >= 8;
                }
                if (cj) {
                    q.y = -q.y;
                    q.w = -q.w;
                }
                float2 v = make_float2(q.x - q.w, q.y + q.z);   // A + i B
                if (withk) {
                    const float kk = wave(k, NH, a.k0s);
                    v = make_float2(kk * v.y, -kk * v.x);          // -i k0 (A + i B)
                }
                x[k1] = v;
            }
            dft<16, true>(x);
            twiddle16<true>(x, tw_base(tw, tt));
            float4 *o = reinterpret_cast<float4 *>(dst + 2 * p);
#pragma unroll
            for (int n1 = 0; n1 < 8; ++n1)
                o[(size_t)(512 * n1 + tt) * ld] = make_float4(x[n1].x, x[n1].y, x[n1 + 8].x, x[n1 + 8].y);
        };
        const bool two = t != 0 && t != 256;
        // every input of this unit is in registers, so the in-place stores cannot overwrite one
        if (want1) {
            one(t, 0, true, a.buf1);
            if (two) one(512 - t, 1, true, a.buf1);
        }
        if (want0) {
            one(t, 0, false, buf);
            if (two) one(512 - t, 1, false, buf);
        }
    }
    cp_async_wait_all();
}

// Step 2.  Unit: (set, a < 8, tile of 16 columns); mode 0: one set, buf1 ->
// E1; mode 1: set 0 buf0 -> phi, set 1 buf1 -> E0 (a set nobody asked for is
// skipped).  Maps 0 and 1: buf0 and buf1 as [n0 + 1][n2] complex, box 16 x
// 256, 128-byte swizzle; the column tile engine of the 512-point passes.
template <int MAXI>
__global__ void __launch_bounds__(TileCfg<512, 16>::THREADS) p5_4s_b(const __grid_constant__ Work<MAXI> W,
                                                                     const __grid_constant__ TmaBatch<MAXI> maps,
                                                                     int mode)
{
    constexpr int N = 512;
    using C = TileCfg<N, 16>;
    constexpr int E = C::E, T = C::T;
    using RAD = typename C::RAD;
    extern __shared__ unsigned char smem_raw[];
    pdl_trigger();
    const TmaSmem s = tma_smem<N>(smem_raw, 1, N);
    const int tid = threadIdx.x, col = tid % 16, j = tid / 16;
    const int nw = W.count();
    tma_bar_setup(s.bar);
    // the 512-point table, W_512^m = W_8192^(16 m), where the tile engine keeps its copy
    float2 *stw = s.ex + N * 16;
    for (int i = tid; i < N; i += C::THREADS) stw[i] = __ldg(W.item[0].tw0 + 16 * i);
    __syncthreads();
    auto field = [&](const PassArgs &b, int set) -> float * { return mode == 0 ? b.out[2] : b.out[set]; };
    auto next_active = [&](int w) -> int {
        for (; w < nw; w += gridDim.x) {
            FSP_UNIT(W, w, b, ub);
            if (field(b, ub / (8 * (b.n2 / 16)))) break;
        }
        return w;
    };
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int zt = b.n2 / 16, set = ub / (8 * zt), r = ub % (8 * zt);
        const CUtensorMap *m = &maps.m[it_ub][(mode == 0 || set == 1) ? 1 : 0];
        mbar_expect_tx(s.bar, N * 128);
        tma_load_2d(s.stage[0], m, (r % zt) * 16, 512 * (r / zt), s.bar);
        tma_load_2d(s.stage[0] + 256 * 16, m, (r % zt) * 16, 512 * (r / zt) + 256, s.bar);
    };
    pdl_wait();
    int w = next_active(blockIdx.x);
    if (tid == 0 && w < nw) issue(w);
    const ColView sm{s.ex + col, 16};
    for (unsigned ph = 0; w < nw; ph ^= 1) {
        const bool ok = mbar_wait(s.bar, ph);
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / 16, set = u / (8 * zt), r = u % (8 * zt);
        const int n1 = 8 * (col & 1) + r / zt, pcol = ((r % zt) * 16 + col) >> 1;
        float *out = field(a, set);
        float2 v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = s.stage[0][sw128(j + q * T, col)];
        if (tma_tile_failed(ok, s.bar, ph, a.status)) break;
        const int wn = next_active(w + gridDim.x);
        if (tid == 0 && wn < nw) {
            fence_proxy_async();
            issue(wn);
        }
        tile_fft<N, E, true, false, RAD>(v, j, stw, sm);
#pragma unroll
        for (int q = 0; q < E / 2; ++q)
            *reinterpret_cast<float2 *>(out + gidx(a, n1 + 16 * (j + q * T), 0, 2 * pcol)) = v[q];
        w = wn;
    }
}

} // namespace fsp
