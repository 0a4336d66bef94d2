// fsp_passes.cuh -- the five passes of the padded FFT convolution.
//
// Grid: n0 x n1 x n2 cells, axis 2 contiguous (a 2D problem is n0 x 1 x n2 with
// no middle-axis passes).  Every pass works on whole padded lines (length 2 n_a)
// that never touch memory: the zero half of the input is never loaded (pruned
// first pass) and only the n_a cropped outputs are stored.
//
// Forward pipeline (paper Sec. 1 HE formula; Sec. 2 VGF uses the same steps with
// its kernel; E by Fourier differentiation, paper Sec. 3):
//   P1  axis 0, real -> half spectrum (k0 in [0, n0]); two real columns of axis 2
//       packed as one complex column, separated with the conjugate symmetry.
//   P2  axis 1 forward (3D only).
//   P3  axis 2 forward, times the kernel spectrum K(k) (and -i k2 K for E2),
//       axis 2 inverse -- the middle pass, one or two output streams.
//   P4  axis 1 inverse (3D only); the phi stream also yields -i k1 phi.
//   P5  axis 0 half spectrum -> real, phi stream -> (phi, E0) through the
//       packing W = (1 + k0) P, the (E1, E2) streams -> (E1, E2) through
//       W = Y + i Z.
// Adjoint pipeline: the same passes with the streams merged instead of split:
// the gradient spectrum is K (G_phi + sum_a i k_a G_Ea).
//
// Intermediate layout: complex [n0 + 1][rows1][n2], rows1 = 2 n1 in 3D, 1 in 2D.
#pragma once

#include "fsp_fft.cuh"
#include <stdint.h>
#include <type_traits>

namespace fsp {

struct PassArgs {
    int n0, n1, n2;   // cells per axis (n1 = 1 for 2D)
    int rows1;        // middle rows of the intermediate layout: 2 n1 (3D) or 1 (2D)
    int three_d;      // 1: axis 1 is transformed
    float k0s, k1s, k2s;   // 2 pi / (2 n_a h_a)
    const float2 *tw0, *tw1, *tw2;
    const float *K;   // [n0 + 1][n1 + 1 (3D) or 1][n2 + 1]
    float2 *buf0, *buf1;
    const float *in[4];
    float *out[4];
    int *status;      // device status word of the solve (0 = fine; set by bounded waits that gave up)
    int kx0, kxn;     // planes k0 in [kx0, kx0 + kxn) for the plane-grouped passes (p2_tma, p3_fwd1,
                      // p4_tma); every other pass covers all n0 + 1 planes
};

// FSP_DEBUG_BOUNDS (a debug build, see build.py): every intermediate and grid
// index is checked against its buffer's extent; an index outside it records
// FSP_ERR_INVALID in the solve's status word (fsp_plan_device_status) and the
// access goes to element 0 instead, so a bad index is reported without a
// fault.  Release builds compile the plain index arithmetic.
#ifdef FSP_DEBUG_BOUNDS
__device__ __forceinline__ size_t checked_index(const PassArgs &a, bool ok, size_t i)
{
    if (ok) return i;
    if (a.status) atomicCAS(a.status, 0, 1 /* FSP_ERR_INVALID */);
    return 0;
}
#endif
__device__ __forceinline__ size_t iidx(const PassArgs &a, int k0, int row, int z)
{
    const size_t i = ((size_t)k0 * a.rows1 + row) * a.n2 + z;
#ifdef FSP_DEBUG_BOUNDS
    return checked_index(a, k0 >= 0 && k0 <= a.n0 && row >= 0 && row < a.rows1 && z >= 0 && z < a.n2, i);
#else
    return i;
#endif
}
__device__ __forceinline__ size_t gidx(const PassArgs &a, int x, int y, int z)
{
    const size_t i = ((size_t)x * a.n1 + y) * a.n2 + z;
#ifdef FSP_DEBUG_BOUNDS
    return checked_index(a, x >= 0 && x < a.n0 && y >= 0 && y < a.n1 && z >= 0 && z < a.n2, i);
#else
    return i;
#endif
}

// Signed wavenumber index of position k on a padded axis of n cells: m in
// [-n, n), with the unpaired m = -n mapped to 0.
__device__ __forceinline__ float wave(int k, int n, float s)
{
    int m = k < n ? k : (k == n ? 0 : k - 2 * n);
    return s * (float)m;
}

// A launch's work: up to MAXI independent problems (items), item i owning
// work units [offs[i], offs[i+1]).  Passed by value as a __grid_constant__
// kernel parameter, so a batch of solves needs no device-side scratch.
template <int MAXI>
struct Work {
    static constexpr int max_items = MAXI;
    PassArgs item[MAXI];
    int offs[MAXI + 1];
    int nitems;
    __device__ __forceinline__ int count() const { return offs[nitems]; }
    // item owning unit w: the last i with offs[i] <= w
    __device__ __forceinline__ int find(int w) const
    {
        if constexpr (MAXI == 1) {
            return 0;
        } else {
            int lo = 0, hi = nitems - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (offs[mid] <= w) lo = mid;
                else hi = mid - 1;
            }
            return lo;
        }
    }
};
constexpr int BATCH_MAX = 32;   // items per batched launch

// Programmatic dependent launch.  The forward passes are launched with the
// programmatic stream-serialization attribute, so a pass's CTAs may be
// scheduled while the previous pass is still finishing.  Each such pass
// releases its own dependents at once (pdl_trigger) and waits for the
// previous grid to complete, with its writes visible, before it touches
// global memory (pdl_wait).  Both are no-ops for a launch without the
// attribute.
#ifndef FSP_PDL
#define FSP_PDL 1
#endif
__device__ __forceinline__ void pdl_trigger()
{
#if FSP_PDL
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}
__device__ __forceinline__ void pdl_wait()
{
#if FSP_PDL
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

#define FSP_UNIT(W, w, a, u)                  \
    const int it_##u = (W).find(w);           \
    const PassArgs &a = (W).item[it_##u];     \
    const int u = (w) - (W).offs[it_##u]

// Block-synchronous column tiles (lengths above 512, and the adjoint entry
// passes).  With 16 columns the exchange buffer is row-major [pos][col] (a
// half-warp covers one 128-byte row: conflict-free); narrower tiles, forced by
// long lines, store each column contiguously with one padding slot per 16
// positions, which keeps their Stockham exchanges conflict-free too.
template <int N>
struct ColCfg {
    static constexpr int E = Plan1D<N>::E;
    static constexpr int T = N / E;
    static constexpr int BZ = (T * 16 <= 1024) ? 16 : (1024 / T);
    static constexpr int THREADS = T * BZ;
    static constexpr bool WIDE = BZ >= 16;
    // Per-column span when !WIDE: at least RowSpan (one padding slot per 16
    // positions), rounded up to SPAN = 16 / BZ (mod 16) so that the BZ columns a
    // half-warp touches sit 32 / BZ banks apart and their exchanges do not
    // collide (the columns are interleaved across lanes: tid -> (tid % BZ, tid / BZ)).
    static constexpr int SPAN = (RowSpan<N, 4>::value + 15 - (16 / BZ) % 16) / 16 * 16 + (16 / BZ) % 16;
    static constexpr size_t SMEM = (size_t)(WIDE ? N * BZ : SPAN * BZ) * sizeof(float2);
    using View = typename std::conditional<WIDE, ColView, RowView<4>>::type;
    static __device__ __forceinline__ View view(float2 *smem, int col)
    {
        if constexpr (WIDE) return ColView{smem + col, BZ};
        else return RowView<4>{smem + col * SPAN};
    }
};

// Twiddle source of the long-line forward middle pass, per length as measured:
// the all-pass gathered table (a warp's consecutive k read consecutive entries)
// at 2n = 2048 and 8192, power products (TW_POW) at 1024 and 4096, where the
// gathered loads were slower.  A value here forces one source.
#ifndef FSP_ROW_TW
#define FSP_ROW_TW -1
#endif
template <int N>
constexpr int kRowTw = FSP_ROW_TW >= 0 ? FSP_ROW_TW : ((N == 2048 || N == 8192) ? TW_GALL : TW_POW);

template <int N>
struct RowCfg {
    static constexpr int E = Plan1D<N>::E;
    static constexpr int T = N / E;
    static constexpr int LPC = (T >= 256) ? 1 : (256 / T);
    static constexpr int THREADS = T * LPC;
    static constexpr int PAD = 4;
    static constexpr int SPAN = RowSpan<N, PAD>::value;
    static constexpr size_t SMEM = (size_t)SPAN * LPC * sizeof(float2);
    // 512-thread lines (2 n >= 4096) keep the product spectrum in shared memory
    // instead of a second register array (the registers would spill)
    static constexpr bool SAVE = T >= 256;
    // cp.async stage after the exchange lines, rounded up to a 16-byte boundary
    static constexpr int STAGE_OFF = (SPAN * LPC + 1) / 2 * 2;   // in float2
    static_assert((STAGE_OFF * sizeof(float2)) % 16 == 0, "cp.async stage must be 16-byte aligned");
    static constexpr size_t SMEM_STAGED = (size_t)STAGE_OFF * sizeof(float2) + (size_t)LPC * (N / 2) * sizeof(float2) +
                                          (SAVE ? (size_t)LPC * N * sizeof(float2) : 0);
};

// ----------------------------------------------------------------- P1 (axis 0)

// Forward: rho columns (z, z+1) packed as re/im; output rows 0..n1-1 of buf_out.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p1_fwd_blk(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 / 2 + BZ - 1) / BZ;
    const int y = u / xt;
    const int z0 = 2 * ((u % xt) * BZ + col);
    const bool act = z0 < a.n2;
    const float *rho = a.in[0];
    float2 *__restrict__ dst = a.three_d ? a.buf1 : a.buf0;
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        v[r] = make_float2(0.f, 0.f);
        if (r < E / 2 && act) v[r] = __ldg(reinterpret_cast<const float2 *>(rho + gidx(a, j + r * T, y, z0)));
    }
    const auto sm = C::view(smem, col);
    line_fft<N, E, false, true, RAD>(v, j, a.tw0, sm);
#pragma unroll
    for (int r = 0; r < E; ++r) sm.at(j + r * T) = v[r];
    __syncthreads();
    constexpr int NH = N / 2;
#pragma unroll
    for (int r = 0; r <= E / 2; ++r) {
        const int k = j + r * T;
        if (k <= NH && act) {
            const float2 w = v[r];
            const float2 m = sm.at(k == 0 ? 0 : N - k);
            float4 o;
            o.x = 0.5f * (w.x + m.x);
            o.y = 0.5f * (w.y - m.y);
            o.z = 0.5f * (w.y + m.y);
            o.w = -0.5f * (w.x - m.x);
            *reinterpret_cast<float4 *>(dst + iidx(a, k, y, z0)) = o;
        }
    }
}

// Adjoint: per column z, W1 = g_phi + i g_E0, W2 = g_E1 + i g_E2 (3D) or g_E1 (2D).
// Outputs U = F g_phi + i k0 F g_E0 -> buf0 row y; F g_E1 -> buf0 row n1 + y (3D)
// or buf1 row y (2D); F g_E2 -> buf1 row y (3D).
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p1_adj(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 + BZ - 1) / BZ;
    const int y = u / xt;
    const int z = (u % xt) * BZ + col;
    const bool act = z < a.n2;
    const float *gp = a.in[0], *g0 = a.in[1], *g1 = a.in[2], *g2 = a.in[3];
    const bool hasE = g0 != nullptr;
    const auto sm = C::view(smem, col);
    constexpr int NH = N / 2;
    for (int pass = 0; pass < (hasE ? 2 : 1); ++pass) {
        const float *re = pass == 0 ? gp : g1;
        const float *im = pass == 0 ? g0 : (a.three_d ? g2 : nullptr);
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = make_float2(0.f, 0.f);
            if (r < E / 2 && act) {
                const size_t g = gidx(a, j + r * T, y, z);
                v[r].x = re ? __ldg(re + g) : 0.f;
                v[r].y = im ? __ldg(im + g) : 0.f;
            }
        }
        line_fft<N, E, false, true, RAD>(v, j, a.tw0, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) sm.at(j + r * T) = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r <= E / 2; ++r) {
            const int k = j + r * T;
            if (k <= NH && act) {
                const float2 w = v[r];
                const float2 m = sm.at(k == 0 ? 0 : N - k);
                const float2 A = make_float2(0.5f * (w.x + m.x), 0.5f * (w.y - m.y));   // F re
                const float2 B = make_float2(0.5f * (w.y + m.y), -0.5f * (w.x - m.x));  // F im
                if (pass == 0) {
                    const float kk = wave(k, NH, a.k0s);
                    // U = A + i k0 B
                    a.buf0[iidx(a, k, y, z)] = make_float2(A.x - kk * B.y, A.y + kk * B.x);
                } else if (a.three_d) {
                    a.buf0[iidx(a, k, a.n1 + y, z)] = A;
                    a.buf1[iidx(a, k, y, z)] = B;
                } else {
                    a.buf1[iidx(a, k, y, z)] = A;
                }
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------- P2 (axis 1)

// Forward: src rows 0..n1-1 -> dst rows 0..2n1-1.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p2_fwd_blk(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 + BZ - 1) / BZ;
    const int kx = u / xt;
    const int z = (u % xt) * BZ + col;
    const bool act = z < a.n2;
    const float2 *__restrict__ src = a.buf1;
    float2 *__restrict__ dst = a.buf0;
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        v[r] = make_float2(0.f, 0.f);
        if (r < E / 2 && act) v[r] = src[iidx(a, kx, j + r * T, z)];
    }
    line_fft<N, E, false, true, RAD>(v, j, a.tw1, C::view(smem, col));
    if (act) {
#pragma unroll
        for (int r = 0; r < E; ++r) dst[iidx(a, kx, j + r * T, z)] = v[r];
    }
}

// Adjoint: buf0 rows [0,n1) = U, rows [n1,2n1) = F g_E1 (if E), buf1 rows [0,n1) = F g_E2.
// buf0 <- F1 U + i k1 F1 (F g_E1) (all rows); buf1 <- F1 (F g_E2) (all rows).
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p2_adj(const __grid_constant__ Work<MAXI> W, int hasE)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 + BZ - 1) / BZ;
    const int kx = u / xt;
    const int z = (u % xt) * BZ + col;
    const bool act = z < a.n2;
    const int n1 = a.n1;
    const auto sm = C::view(smem, col);
    float2 v[E], w[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        v[r] = make_float2(0.f, 0.f);
        w[r] = make_float2(0.f, 0.f);
        if (r < E / 2 && act) {
            v[r] = a.buf0[iidx(a, kx, j + r * T, z)];
            if (hasE) w[r] = a.buf0[iidx(a, kx, n1 + j + r * T, z)];
        }
    }
    line_fft<N, E, false, true, RAD>(v, j, a.tw1, sm);
    if (hasE) {
        line_fft<N, E, false, true, RAD>(w, j, a.tw1, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float kk = wave(j + r * T, n1, a.k1s);
            v[r] = make_float2(v[r].x - kk * w[r].y, v[r].y + kk * w[r].x);
        }
    }
    if (act) {
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
    }
    if (hasE) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            w[r] = make_float2(0.f, 0.f);
            if (r < E / 2 && act) w[r] = a.buf1[iidx(a, kx, j + r * T, z)];
        }
        line_fft<N, E, false, true, RAD>(w, j, a.tw1, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E; ++r) a.buf1[iidx(a, kx, j + r * T, z)] = w[r];
        }
    }
}

// ------------------------------------------------------------ P3 (axis 2, middle)

__device__ __forceinline__ const float *krow(const PassArgs &a, int kx, int row)
{
    if (a.three_d) {
        const int n1 = a.n1;
        const int kyf = row <= n1 ? row : 2 * n1 - row;
        return a.K + ((size_t)kx * (n1 + 1) + kyf) * (a.n2 + 1);
    }
    return a.K + (size_t)kx * (a.n2 + 1);
}

// Forward: line of buf0 -> F2 -> x K -> inverse -> buf0 (phi stream), and
// -i k2 K -> inverse -> buf1 (E2 stream) when withE.
// Long lines (2 n2 >= 1024): LPC lines per CTA, persistent over line groups;
// the next group's pruned input (LPC x n2 contiguous complex) is copied into
// shared memory with cp.async while the current group is transformed.
template <int N, int MAXI>
__global__ void __launch_bounds__(RowCfg<N>::THREADS) p3_fwd_blk(const __grid_constant__ Work<MAXI> W, int withE)
{
    using C = RowCfg<N>;
    constexpr int E = C::E, T = C::T, LPC = C::LPC, NH = N / 2;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *stage = smem + C::STAGE_OFF;   // LPC x NH complex, 16-byte aligned
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const int nw = W.count();
    RowView<C::PAD> sm{smem + li * C::SPAN};
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int lines = (b.n0 + 1) * b.rows1;
        const int first = ub * LPC;
        const int cnt = min(LPC, lines - first);
        const float2 *src = b.buf0 + (size_t)first * b.n2;   // cnt contiguous lines
        const int chunks = cnt * NH / 2;                      // 16-byte chunks
        for (int c = threadIdx.x; c < chunks; c += C::THREADS) cp_async16(stage + 2 * c, src + 2 * c);
    };
    int w = blockIdx.x;
    pdl_wait();
    if (w < nw) issue(w);
    cp_async_commit();
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int lines = (a.n0 + 1) * a.rows1;
        const int line = u * LPC + li;
        const bool act = line < lines;
        const int lc = act ? line : 0;
        const int kx = lc / a.rows1, row = lc % a.rows1;
        constexpr int n2 = N / 2;   // every item of a length-N launch has n2 = N / 2
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = (r < E / 2 && act) ? stage[li * NH + j + r * T] : make_float2(0.f, 0.f);
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
        line_fft<N, E, false, true, RAD, RowView<C::PAD>, SYNC_BLOCK, kRowTw<N>>(v, j, a.tw2, sm);
        const float *Kr = krow(a, kx, row);
        if constexpr (C::SAVE) {
            float2 *sv = stage + LPC * NH + li * N;   // product spectrum of this line
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int k = j + r * T;
                const int kf = k <= n2 ? k : N - k;
                v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
                sv[k] = v[r];
            }
            line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_BLOCK, kRowTw<N>>(v, j, a.tw2, sm);
            if (act) {
                float2 *L0 = a.buf0 + (size_t)lc * n2;
#pragma unroll
                for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
            }
            if (withE) {
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const int k = j + r * T;
                    const float kk = wave(k, n2, a.k2s);
                    const float2 sk = sv[k];
                    v[r] = make_float2(kk * sk.y, -kk * sk.x);   // -i k2 (K rho^)
                }
                line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_BLOCK, kRowTw<N>>(v, j, a.tw2, sm);
                if (act) {
                    float2 *L1 = a.buf1 + (size_t)lc * n2;
#pragma unroll
                    for (int r = 0; r < E / 2; ++r) L1[j + r * T] = v[r];
                }
            }
        } else {
            float2 q[E];
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const int k = j + r * T;
                const int kf = k <= n2 ? k : N - k;
                const float kv = act ? __ldg(Kr + kf) : 0.f;
                v[r] = kv * v[r];
                const float kk = wave(k, n2, a.k2s);
                q[r] = make_float2(kk * v[r].y, -kk * v[r].x);   // -i k2 (K rho^)
            }
            line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_BLOCK, kRowTw<N>>(v, j, a.tw2, sm);
            if (act) {
                float2 *L0 = a.buf0 + (size_t)lc * n2;
#pragma unroll
                for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
            }
            if (withE) {
                line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_BLOCK, kRowTw<N>>(q, j, a.tw2, sm);
                if (act) {
                    float2 *L1 = a.buf1 + (size_t)lc * n2;
#pragma unroll
                    for (int r = 0; r < E / 2; ++r) L1[j + r * T] = q[r];
                }
            }
        }
    }
    cp_async_wait_all();
}

// Adjoint: buf0 line V (and buf1 line Z when hasE) -> K (F2 V + i k2 F2 Z) -> inverse -> buf0.
template <int N, int MAXI>
__global__ void __launch_bounds__(RowCfg<N>::THREADS) p3_adj_blk(const __grid_constant__ Work<MAXI> W, int hasE)
{
    using C = RowCfg<N>;
    constexpr int E = C::E, T = C::T, LPC = C::LPC;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int lines = (a.n0 + 1) * a.rows1;
    const int line = u * LPC + li;
    const bool act = line < lines;
    const int lc = act ? line : 0;
    const int kx = lc / a.rows1, row = lc % a.rows1;
    const int n2 = a.n2;
    float2 *L0 = a.buf0 + (size_t)lc * n2;
    float2 *L1 = a.buf1 + (size_t)lc * n2;
    RowView<C::PAD> sm{smem + li * C::SPAN};
    float2 v[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        v[r] = make_float2(0.f, 0.f);
        if (r < E / 2 && act) v[r] = L0[j + r * T];
    }
    line_fft<N, E, false, true, RAD>(v, j, a.tw2, sm);
    if (hasE) {
        float2 w[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            w[r] = make_float2(0.f, 0.f);
            if (r < E / 2 && act) w[r] = L1[j + r * T];
        }
        line_fft<N, E, false, true, RAD>(w, j, a.tw2, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float kk = wave(j + r * T, n2, a.k2s);
            v[r] = make_float2(v[r].x - kk * w[r].y, v[r].y + kk * w[r].x);
        }
    }
    const float *Kr = krow(a, kx, row);
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int k = j + r * T;
        const int kf = k <= n2 ? k : N - k;
        v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
    }
    line_fft<N, E, true, false, RAD>(v, j, a.tw2, sm);
    if (act) {
#pragma unroll
        for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
    }
}

// ----------------------------------------------------------------- P4 (axis 1)

// Forward: buf0 (phi stream, all rows) -> inverse -> rows [0,n1); with E also
// -i k1 phi -> rows [n1,2n1) of buf0 and buf1 (E2 stream) -> rows [0,n1) of buf1.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p4_fwd_blk(const __grid_constant__ Work<MAXI> W, int withE)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 + BZ - 1) / BZ;
    const int kx = u / xt;
    const int z = (u % xt) * BZ + col;
    const bool act = z < a.n2;
    const int zc = act ? z : 0;
    const int n1 = a.n1;
    const auto sm = C::view(smem, col);
    float2 v[E], q[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        v[r] = a.buf0[iidx(a, kx, j + r * T, zc)];
        const float kk = wave(j + r * T, n1, a.k1s);
        q[r] = make_float2(kk * v[r].y, -kk * v[r].x);
    }
    line_fft<N, E, true, false, RAD>(v, j, a.tw1, sm);
    if (act) {
#pragma unroll
        for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
    }
    if (withE) {
        line_fft<N, E, true, false, RAD>(q, j, a.tw1, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf0[iidx(a, kx, n1 + j + r * T, z)] = q[r];
        }
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = a.buf1[iidx(a, kx, j + r * T, zc)];
        line_fft<N, E, true, false, RAD>(v, j, a.tw1, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) a.buf1[iidx(a, kx, j + r * T, z)] = v[r];
        }
    }
}

// ----------------------------------------------------------------- P5 (axis 0)

// Forward: phi stream (buf0 rows [0,n1)) -> (phi, E0) via W = (1 + k0) P; E1/E2
// streams -> (E1, E2) via W = Y + i Z (3D: Y = buf0 rows n1 + y, Z = buf1 rows
// y; 2D: Y = buf1 row 0, Z absent).  Adjoint uses mode phi-only.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p5_fwd_blk(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    FSP_UNIT(W, blockIdx.x, a, u);
    const int xt = (a.n2 + BZ - 1) / BZ;
    const int y = u / xt;
    const int z = (u % xt) * BZ + col;
    const bool act = z < a.n2;
    const int zc = act ? z : 0;
    constexpr int NH = N / 2;
    float *phi = a.out[0], *e0 = a.out[1], *e1 = a.out[2], *e2 = a.out[3];
    const auto sm = C::view(smem, col);
    if (phi || e0) {
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int src = k <= NH ? k : N - k;
            float2 p = a.buf0[iidx(a, src, y, zc)];
            if (k > NH) p.y = -p.y;
            if (e0) {
                const float kk = wave(k, NH, a.k0s);
                p = (1.f + kk) * p;   // W = P + i (-i k0 P): Re -> phi, Im -> E0
            }
            v[r] = p;
        }
        line_fft<N, E, true, false, RAD>(v, j, a.tw0, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, j + r * T, y, z);
                if (phi) phi[g] = v[r].x;
                if (e0) e0[g] = v[r].y;
            }
        }
    }
    if (e1) {
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int src = k <= NH ? k : N - k;
            float2 Y, Z = make_float2(0.f, 0.f);
            if (a.three_d) {
                Y = a.buf0[iidx(a, src, a.n1 + y, zc)];
                Z = a.buf1[iidx(a, src, y, zc)];
            } else {
                Y = a.buf1[iidx(a, src, y, zc)];
            }
            if (k > NH) {
                Y.y = -Y.y;
                Z.y = -Z.y;
            }
            v[r] = make_float2(Y.x - Z.y, Y.y + Z.x);   // Y + i Z
        }
        line_fft<N, E, true, false, RAD>(v, j, a.tw0, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const size_t g = gidx(a, j + r * T, y, z);
                e1[g] = v[r].x;
                if (a.three_d) e2[g] = v[r].y;
            }
        }
    }
}

// ------------------------------- persistent staged passes for long columns
//
// 2D problems with 2 n0 >= 1536 hold only BZ = 2..8 columns of the first axis
// per CTA, one CTA per SM.  These persistent versions copy the next column
// group's input rows into a shared-memory stage with cp.async while the
// current group is transformed, so the (narrow, row-strided) loads overlap
// the FFT instead of stalling it.  Layout: exchange buffer (ColCfg), then the
// stage [rows][BZ] on a 16-byte boundary.
// Twiddle source of the staged long-column passes: by default the all-pass
// gathered table at 2n = 8192 and power products below (measured: the gathered
// loads win at 4096^2 and lose at 1024^2); a value here forces one source.
#ifndef FSP_COL_TW
#define FSP_COL_TW -1
#endif
template <int N>
constexpr int kColTw = FSP_COL_TW >= 0 ? FSP_COL_TW : (N >= 8192 ? TW_GALL : TW_POW);

template <int N>
struct LongStage {
    using C = ColCfg<N>;
    static constexpr int OFF = (C::SPAN * C::BZ + 1) / 2 * 2;   // float2
    static constexpr int ROWS = N / 2 + 1;
    static constexpr int TWOFF = OFF + ROWS * C::BZ;             // quarter table (TW_QSMEM)
    static constexpr int TWQ = FSP_COL_TW == TW_QSMEM ? N / 4 : 0;
    static constexpr size_t SMEM = (size_t)(TWOFF + TWQ) * sizeof(float2);
    static_assert(!C::WIDE, "staged long columns are for BZ < 16");
    // Every thread of the block calls this once, before its first transform.
    static __device__ __forceinline__ const float2 *twiddles(float2 *smem, const float2 *gtw)
    {
        if constexpr (TWQ > 0) {
            float2 *t = smem + TWOFF;
            for (int i = threadIdx.x; i < TWQ; i += C::THREADS) t[i] = gtw[i];
            __syncthreads();
            return t;
        } else {
            return gtw;
        }
    }
    // cp.async rows [0, rows) of BZ complex columns (row r at src + r * ld) into stage
    static __device__ __forceinline__ void copy(float2 *stage, const float2 *src, size_t ld, int rows)
    {
        constexpr int CH = C::BZ / 2;   // 16-byte chunks per row
        for (int c = threadIdx.x; c < rows * CH; c += C::THREADS) {
            const int r = c / CH, q = c % CH;
            cp_async16(stage + r * C::BZ + 2 * q, src + (size_t)r * ld + 2 * q);
        }
    }
};

// P1 (2D, 2 n0 >= 1536), persistent.  Unit: a group of BZ packed column pairs.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p1_fwd_pst(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    using S = LongStage<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ, NH = N / 2;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *stage = smem + S::OFF;   // [NH][BZ] packed pairs
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    const int nw = W.count();
    const float2 *tw = S::twiddles(smem, W.item[0].tw0);   // the table depends on N only
    auto issue = [&](int w) {
        FSP_UNIT(W, w, b, ub);
        const int z0 = 2 * BZ * ub;   // first real column
        S::copy(stage, reinterpret_cast<const float2 *>(b.in[0] + z0), b.n2 / 2, NH);
    };
    int w = blockIdx.x;
    pdl_wait();
    if (w < nw) issue(w);
    cp_async_commit();
    const auto sm = C::view(smem, col);
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int z0 = 2 * (BZ * u + col);
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? stage[(j + r * T) * BZ + col] : make_float2(0.f, 0.f);
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
        line_fft<N, E, false, true, RAD, typename C::View, SYNC_BLOCK, kColTw<N>>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) sm.at(j + r * T) = v[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r <= E / 2; ++r) {
            const int k = j + r * T;
            if (k <= NH) {
                const float2 x = v[r];
                const float2 m = sm.at(k == 0 ? 0 : N - k);
                float4 o;
                o.x = 0.5f * (x.x + m.x);
                o.y = 0.5f * (x.y - m.y);
                o.z = 0.5f * (x.y + m.y);
                o.w = -0.5f * (x.x - m.x);
                *reinterpret_cast<float4 *>(a.buf0 + iidx(a, k, 0, z0)) = o;
            }
        }
        __syncthreads();   // the exchange buffer is reused by the next group
    }
    cp_async_wait_all();
}

// P5 (2D, 2 n0 >= 1536), persistent over (column group, stream) jobs: stream 0
// is buf0 -> (phi, E0) by W = (1 + k0) P, stream 1 is buf1 -> E1.  The next
// job's rows are staged while the current job is transformed.
template <int N, int MAXI>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) p5_fwd_pst(const __grid_constant__ Work<MAXI> W)
{
    using C = ColCfg<N>;
    using S = LongStage<N>;
    constexpr int E = C::E, T = C::T, BZ = C::BZ, NH = N / 2;
    using RAD = typename Plan1D<N>::R;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *stage = smem + S::OFF;   // [NH + 1][BZ]
    const int col = threadIdx.x % BZ, j = threadIdx.x / BZ;
    const int nw = W.count();
    const float2 *tw = S::twiddles(smem, W.item[0].tw0);   // the table depends on N only
    // job t: unit blockIdx.x + (t / 2) gridDim.x, stream t % 2; next active job from t
    auto next = [&](int t) -> int {
        for (;; ++t) {
            const int w = blockIdx.x + (t >> 1) * (int)gridDim.x;
            if (w >= nw) return -1;
            FSP_UNIT(W, w, b, ub);
            if ((t & 1) ? b.out[2] != nullptr : (b.out[0] != nullptr || b.out[1] != nullptr)) return t;
        }
    };
    auto issue = [&](int t) {
        FSP_UNIT(W, blockIdx.x + (t >> 1) * (int)gridDim.x, b, ub);
        const float2 *src = ((t & 1) ? b.buf1 : b.buf0) + BZ * ub;
        S::copy(stage, src, b.n2, NH + 1);
    };
    int t = next(0);
    pdl_wait();
    if (t >= 0) issue(t);
    cp_async_commit();
    const auto sm = C::view(smem, col);
    while (t >= 0) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, blockIdx.x + (t >> 1) * (int)gridDim.x, a, u);
        const int z = BZ * u + col;
        const bool s1 = (t & 1) != 0;
        float *oa = s1 ? a.out[2] : a.out[0];
        float *ob = s1 ? nullptr : a.out[1];
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int src = k <= NH ? k : N - k;
            float2 p = stage[src * BZ + col];
            if (k > NH) p.y = -p.y;
            if (ob) p = (1.f + wave(k, NH, a.k0s)) * p;   // W = P + i (-i k0 P): Re -> phi, Im -> E0
            v[r] = p;
        }
        __syncthreads();
        const int tn = next(t + 1);
        if (tn >= 0) issue(tn);
        cp_async_commit();
        line_fft<N, E, true, false, RAD, typename C::View, SYNC_BLOCK, kColTw<N>>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E / 2; ++r) {
            const size_t g = gidx(a, j + r * T, 0, z);
            if (oa) oa[g] = v[r].x;
            if (ob) ob[g] = v[r].y;
        }
        t = tn;
    }
    cp_async_wait_all();
}



// =====================================================================
// Persistent, cp.async-staged column passes (2 n <= 512) and warp-per-line
// middle pass.  A column tile is 16 consecutive axis-2 columns by the whole
// line; T = N / E threads per column (E = 16 values per thread), lanes
// across columns so every global row access is 128 B or wider.  The CTA
// loops over tiles; the next tile is copied into shared memory with cp.async
// while the current one is transformed, so loads overlap the arithmetic.
// =====================================================================

#ifndef FSP_TILE_C
#define FSP_TILE_C 16
#endif
template <int N, int EE, int ALT = 0>
struct TilePlan {
    static constexpr int E = Plan16<N>::E;
    using R = typename Plan16<N>::R;
};
template <int N>
struct TilePlan<N, 8, 0> {
    static constexpr int E = Plan1D<N>::E;
    using R = typename Plan1D<N>::R;
};
template <int N>
struct TilePlan<N, 16, 1> {
    static constexpr int E = Plan16B<N>::E;
    using R = typename Plan16B<N>::R;
};

// Twiddle source of the column tiles: a copy of the table in shared memory
// (TW_STABLE) or the global table through the read-only cache (TW_TABLE).
#ifndef FSP_TILE_TW
#define FSP_TILE_TW TW_STABLE
#endif

// EE = 16: 16 values per thread (Plan16, or Plan16B with ALT = 1); EE = 8:
// Plan1D (8 per thread, 12 for 192).
template <int N, int EE = 16, int ALT = 0>
struct TileCfg {
    static constexpr int E = TilePlan<N, EE, ALT>::E;
    static constexpr int T = N / E;
    static constexpr int C = FSP_TILE_C;           // columns per tile (complex)
    static constexpr int THREADS = T * C;
    using RAD = typename TilePlan<N, EE, ALT>::R;
    static constexpr int TWS = FSP_TILE_TW == TW_STABLE ? N : 0;
    // exchange buffer (N x C), then the twiddle copy; the last region of
    // every tile kernel's shared memory, in float2
    static constexpr int EX = N * C + TWS;
    // Every thread calls this once, before its first transform.
    static __device__ __forceinline__ const float2 *twiddles(float2 *ex, const float2 *gtw)
    {
        if constexpr (TWS > 0) {
            float2 *stw = ex + N * C;
            for (int i = threadIdx.x; i < TWS; i += THREADS) stw[i] = gtw[i];
            __syncthreads();
            return stw;
        } else {
            return gtw;
        }
    }
};

// Column-tile transform: block-synchronous, twiddles from FSP_TILE_TW.
template <int N, int E, bool INV, bool PRUNE_IN, class RAD>
__device__ __forceinline__ void tile_fft(float2 (&v)[E], int j, const float2 *__restrict__ tw, const ColView &sm)
{
    line_fft<N, E, INV, PRUNE_IN, RAD, ColView, SYNC_BLOCK, FSP_TILE_TW>(v, j, tw, sm);
}

// Rows [0, nrows) of C complex (8 C bytes) each into dst (row r at dst + C r).
template <int C>
__device__ __forceinline__ void issue_rows(float2 *dst, const void *src, size_t row_bytes_stride, int nrows, int tid,
                                           int nthr)
{
    constexpr int CH = C / 2;   // 16-byte chunks per row
    const char *s = reinterpret_cast<const char *>(src);
    for (int c = tid; c < nrows * CH; c += nthr) {
        const int r = c / CH, part = c % CH;
        cp_async16(dst + r * C + part * 2, s + (size_t)r * row_bytes_stride + part * 16);
    }
}

// P1: rho pairs (z, z+1) -> half spectrum in k0, output rows 0..n1-1 of buf1
// (3D) or buf0 (2D).  Unit: (y, tile of 2C reals of axis 2).
template <int N, int MAXI, int EE>
__global__ void __launch_bounds__(TileCfg<N, EE>::THREADS) p1_fwd(const __grid_constant__ Work<MAXI> W)
{
    using C = TileCfg<N, EE>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *stage = smem, *ex = smem + NH * CC;
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / (2 * CC);
        const int y = u / zt, z0 = (u % zt) * (2 * CC);
        issue_rows<CC>(stage, a.in[0] + gidx(a, 0, y, z0), (size_t)a.n1 * a.n2 * sizeof(float), NH, tid, C::THREADS);
    };
    int w = blockIdx.x;
    pdl_wait();   // the previous pass's output (and its reads of our outputs) are complete
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw0);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / (2 * CC);
        const int y = u / zt, z0 = (u % zt) * (2 * CC) + 2 * col;
        float2 *__restrict__ dst = a.three_d ? a.buf1 : a.buf0;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? stage[(j + r * T) * CC + col] : make_float2(0.f, 0.f);
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
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
    }
    cp_async_wait_all();
}

// P2: buf1 rows 0..n1-1 -> forward axis 1 -> buf0 rows 0..2n1-1.  Unit: (k0, tile of C columns).
template <int N, int MAXI, int EE>
__global__ void __launch_bounds__(TileCfg<N, EE>::THREADS) p2_fwd(const __grid_constant__ Work<MAXI> W)
{
    using C = TileCfg<N, EE>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *stage = smem, *ex = smem + NH * CC;
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z0 = (u % zt) * CC;
        issue_rows<CC>(stage, a.buf1 + iidx(a, kx, 0, z0), (size_t)a.n2 * sizeof(float2), NH, tid, C::THREADS);
    };
    int w = blockIdx.x;
    pdl_wait();   // the previous pass's output (and its reads of our outputs) are complete
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw1);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z = (u % zt) * CC + col;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? stage[(j + r * T) * CC + col] : make_float2(0.f, 0.f);
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
        tile_fft<N, E, false, true, RAD>(v, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
    }
    cp_async_wait_all();
}

// P4: buf0 (phi stream, 2 n1 rows) -> rows [0,n1) phi, rows [n1,2n1) -i k1 phi;
// buf1 (E2 stream) -> rows [0,n1).  Unit: (k0, tile of C columns).
template <int N, int MAXI, int EE>
__global__ void __launch_bounds__(TileCfg<N, EE>::THREADS) p4_fwd(const __grid_constant__ Work<MAXI> W, int withE)
{
    using C = TileCfg<N, EE>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *st0 = smem, *st1 = smem + N * CC, *ex = smem + 2 * N * CC;
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z0 = (u % zt) * CC;
        const size_t rs = (size_t)a.n2 * sizeof(float2);
        issue_rows<CC>(st0, a.buf0 + iidx(a, kx, 0, z0), rs, N, tid, C::THREADS);
        if (withE) issue_rows<CC>(st1, a.buf1 + iidx(a, kx, 0, z0), rs, N, tid, C::THREADS);
    };
    int w = blockIdx.x;
    pdl_wait();   // the previous pass's output (and its reads of our outputs) are complete
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw1);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z = (u % zt) * CC + col;
        const int n1 = a.n1;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = st0[(j + r * T) * CC + col];
            q[r] = withE ? st1[(j + r * T) * CC + col] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
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
    cp_async_wait_all();
}

// P5: half spectra in k0 -> real outputs (see the header comment).  Unit: (y, tile of C columns).
template <int N, int MAXI, int EE>
__global__ void __launch_bounds__(TileCfg<N, EE>::THREADS) p5_fwd(const __grid_constant__ Work<MAXI> W)
{
    using C = TileCfg<N, EE>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T, NH = N / 2, ROWS = N / 2 + 1;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *sA = smem, *sB = smem + ROWS * CC, *sC = smem + 2 * ROWS * CC, *ex = smem + 3 * ROWS * CC;
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int y = u / zt, z0 = (u % zt) * CC;
        const size_t rs = (size_t)a.rows1 * a.n2 * sizeof(float2);
        if (a.out[0] || a.out[1]) issue_rows<CC>(sA, a.buf0 + iidx(a, 0, y, z0), rs, ROWS, tid, C::THREADS);
        if (a.out[2]) {
            if (a.three_d) {
                issue_rows<CC>(sB, a.buf0 + iidx(a, 0, a.n1 + y, z0), rs, ROWS, tid, C::THREADS);
                issue_rows<CC>(sC, a.buf1 + iidx(a, 0, y, z0), rs, ROWS, tid, C::THREADS);
            } else {
                issue_rows<CC>(sB, a.buf1 + iidx(a, 0, y, z0), rs, ROWS, tid, C::THREADS);
            }
        }
    };
    int w = blockIdx.x;
    pdl_wait();   // the previous pass's output (and its reads of our outputs) are complete
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw0);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int y = u / zt, z = (u % zt) * CC + col;
        float *phi = a.out[0], *e0 = a.out[1], *e1 = a.out[2], *e2 = a.out[3];
        const bool first = phi || e0, second = e1 != nullptr;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int src = k <= NH ? k : N - k;
            float2 p = make_float2(0.f, 0.f), Y = p, Z = p;
            if (first) p = sA[src * CC + col];
            if (second) {
                Y = sB[src * CC + col];
                if (a.three_d) Z = sC[src * CC + col];
            }
            if (k > NH) {
                p.y = -p.y;
                Y.y = -Y.y;
                Z.y = -Z.y;
            }
            if (e0) p = (1.f + wave(k, NH, a.k0s)) * p;   // W = P + i (-i k0 P)
            v[r] = p;
            q[r] = make_float2(Y.x - Z.y, Y.y + Z.x);        // Y + i Z
        }
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
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
    cp_async_wait_all();
}

// Adjoint P1 (persistent tiles): per column z, W1 = g_phi + i g_E0 and
// W2 = g_E1 + i g_E2 (3D) or g_E1 (2D); outputs U = F g_phi + i k0 F g_E0 ->
// buf0 row y; F g_E1 -> buf0 row n1 + y (3D) / buf1 row y (2D); F g_E2 ->
// buf1 row y (3D).  Unit: (y, tile of C columns).  Stage: the four inputs,
// n0 rows x C floats each.
template <int N, int MAXI>
__global__ void __launch_bounds__(TileCfg<N>::THREADS) p1_adj_t(const __grid_constant__ Work<MAXI> W)
{
    using C = TileCfg<N>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float *stage = reinterpret_cast<float *>(smem);            // [4][NH][CC] floats
    float2 *ex = smem + 2 * NH * CC;                            // after 4 * NH * CC floats
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int y = u / zt, z0 = (u % zt) * CC;
        const size_t rs = (size_t)a.n1 * a.n2 * sizeof(float);
        for (int s = 0; s < 4; ++s)
            if (a.in[s])
                issue_rows<CC / 2>(reinterpret_cast<float2 *>(stage + s * NH * CC), a.in[s] + gidx(a, 0, y, z0), rs, NH,
                                   tid, C::THREADS);
    };
    int w = blockIdx.x;
    pdl_wait();
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw0);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int y = u / zt, z = (u % zt) * CC + col;
        const bool has[4] = {a.in[0] != nullptr, a.in[1] != nullptr, a.in[2] != nullptr, a.in[3] != nullptr};
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = make_float2(0.f, 0.f);
            q[r] = make_float2(0.f, 0.f);
            if (r < E / 2) {
                const int o = (j + r * T) * CC + col;
                v[r].x = has[0] ? stage[o] : 0.f;
                v[r].y = has[1] ? stage[NH * CC + o] : 0.f;
                q[r].x = has[2] ? stage[2 * NH * CC + o] : 0.f;
                q[r].y = (has[3] && a.three_d) ? stage[3 * NH * CC + o] : 0.f;
            }
        }
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 1) {
#pragma unroll
                for (int r = 0; r < E; ++r) v[r] = q[r];
            }
            tile_fft<N, E, false, true, RAD>(v, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E; ++r) sm.at(j + r * T) = v[r];
            __syncthreads();
#pragma unroll
            for (int r = 0; r <= E / 2; ++r) {
                const int k = j + r * T;
                if (k <= NH) {
                    const float2 c = v[r];
                    const float2 m = sm.at(k == 0 ? 0 : N - k);
                    const float2 A = make_float2(0.5f * (c.x + m.x), 0.5f * (c.y - m.y));   // F re
                    const float2 B = make_float2(0.5f * (c.y + m.y), -0.5f * (c.x - m.x));  // F im
                    if (pass == 0) {
                        const float kk = wave(k, NH, a.k0s);
                        a.buf0[iidx(a, k, y, z)] = make_float2(A.x - kk * B.y, A.y + kk * B.x);   // A + i k0 B
                    } else if (a.three_d) {
                        a.buf0[iidx(a, k, a.n1 + y, z)] = A;
                        a.buf1[iidx(a, k, y, z)] = B;
                    } else {
                        a.buf1[iidx(a, k, y, z)] = A;
                    }
                }
            }
            __syncthreads();
        }
    }
    cp_async_wait_all();
}

// Adjoint P2 (persistent tiles): buf0 rows [0,n1) = U, [n1,2n1) = F g_E1,
// buf1 rows [0,n1) = F g_E2 -> buf0 <- F1 U + i k1 F1(F g_E1), buf1 <- F1(F g_E2).
// Unit: (k0, tile of C columns).
template <int N, int MAXI>
__global__ void __launch_bounds__(TileCfg<N>::THREADS) p2_adj_t(const __grid_constant__ Work<MAXI> W)
{
    using C = TileCfg<N>;
    constexpr int CC = C::C;
    constexpr int E = C::E, T = C::T, NH = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    float2 *st0 = smem, *st1 = smem + N * CC, *ex = smem + (N + NH) * CC;
    const int tid = threadIdx.x, col = tid % CC, j = tid / CC;
    const int nw = W.count();
    auto issue = [&](int w) {
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z0 = (u % zt) * CC;
        const size_t rs = (size_t)a.n2 * sizeof(float2);
        issue_rows<CC>(st0, a.buf0 + iidx(a, kx, 0, z0), rs, N, tid, C::THREADS);
        issue_rows<CC>(st1, a.buf1 + iidx(a, kx, 0, z0), rs, NH, tid, C::THREADS);
    };
    int w = blockIdx.x;
    pdl_wait();
    if (w < nw) issue(w);
    cp_async_commit();
    ColView sm{ex + col, CC};
    const float2 *tw = C::twiddles(ex, W.item[0].tw1);   // the table depends on N only
    for (; w < nw; w += gridDim.x) {
        cp_async_wait_all();
        __syncthreads();
        FSP_UNIT(W, w, a, u);
        const int zt = a.n2 / CC;
        const int kx = u / zt, z = (u % zt) * CC + col;
        const int n1 = a.n1;
        float2 v[E], q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            v[r] = r < E / 2 ? st0[(j + r * T) * CC + col] : make_float2(0.f, 0.f);
            q[r] = r < E / 2 ? st0[(NH + j + r * T) * CC + col] : make_float2(0.f, 0.f);
        }
        tile_fft<N, E, false, true, RAD>(v, j, tw, sm);
        tile_fft<N, E, false, true, RAD>(q, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const float kk = wave(j + r * T, n1, a.k1s);
            v[r] = make_float2(v[r].x - kk * q[r].y, v[r].y + kk * q[r].x);
            q[r] = r < E / 2 ? st1[(j + r * T) * CC + col] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (w + (int)gridDim.x < nw) issue(w + gridDim.x);
        cp_async_commit();
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf0[iidx(a, kx, j + r * T, z)] = v[r];
        tile_fft<N, E, false, true, RAD>(q, j, tw, sm);
#pragma unroll
        for (int r = 0; r < E; ++r) a.buf1[iidx(a, kx, j + r * T, z)] = q[r];
    }
    cp_async_wait_all();
}

// ------------------------------------------------- warp-per-line middle pass

#ifndef FSP_P3_TW
#define FSP_P3_TW TW_SMEM
#endif

// Optional minimum resident blocks for the middle pass.  Leave unset: a
// bound of 1 lets the compiler take far more registers (measured slower).
#ifdef FSP_P3_MINB
#define FSP_P3_BOUNDS(t) __launch_bounds__(t, FSP_P3_MINB)
#else
#define FSP_P3_BOUNDS(t) __launch_bounds__(t)
#endif
// ALT = 1: the second radix split (Plan16B; tuned variant bit 8), whose
// gathered twiddle blocks follow those of the first in the same table.
template <int N, int ALT = 0>
using P3Plan = typename PlanSel<N, ALT>::type;

template <int N, int ALT = 0>
struct WarpCfg {
    static constexpr int E = P3Plan<N, ALT>::E;
    static constexpr int T = N / E;
    static constexpr int LPW = 32 / T;     // lines per warp
    static constexpr int WARPS = 4;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int PAD = 4;
    static constexpr int SPAN = RowSpan<N, PAD>::value;
    using RAD = typename P3Plan<N, ALT>::R;
    static constexpr int OFF = AuxOff<N, ALT>::value;   // the plan's gathered blocks after the table
    static constexpr int RL = SPAN;             // shared memory per line (exchange buffer)
    // TW_SMEM: the twiddle table (main part and gathered blocks) after the lines
    static constexpr int TWOFF = RL * LPW * WARPS;
    static constexpr int TWS = FSP_P3_TW == TW_SMEM ? AuxEnd<1, N + OFF, RAD>::value : 0;
    static constexpr size_t SMEM = (size_t)(TWOFF + TWS) * sizeof(float2);
    // With TW_SMEM: copy the table into shared memory (every thread of the
    // block calls this once, before its first transform) and return the copy.
    static __device__ __forceinline__ const float2 *twiddles(float2 *smem, const float2 *gtw)
    {
        if constexpr (TWS > 0) {
            float2 *stw = smem + TWOFF;
            for (int i = threadIdx.x; i < TWS; i += THREADS) stw[i] = gtw[i];
            __syncthreads();
            return stw;
        } else {
            return gtw;
        }
    }
};

// Forward middle pass, one warp per line (or per 32/T lines), persistent over
// lines with the next line's input prefetched into registers.  Unit: a group
// of LPW lines of one item (warp-level).
template <int N, int MAXI>
__global__ void FSP_P3_BOUNDS(WarpCfg<N>::THREADS) p3_fwd(const __grid_constant__ Work<MAXI> W,
                                                                           int withE)
{
    using C = WarpCfg<N>;
    constexpr int E = C::E, T = C::T, LPW = C::LPW;
    constexpr int n2 = N / 2;   // every item of a length-N launch has n2 = N / 2
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int li = lane / T, j = lane % T;
    // (the single-item bound is computed from the geometry: the register
    // allocation of this kernel is sensitive to where the bound comes from)
    const int nw = MAXI == 1 ? ((W.item[0].n0 + 1) * W.item[0].rows1 + LPW - 1) / LPW : W.count();
    const int gstride = gridDim.x * C::WARPS;
    RowView<C::PAD> sm{smem + (warp * LPW + li) * C::RL};
    const float2 *tw = C::twiddles(smem, W.item[0].tw2);   // the table depends on N only
    pdl_wait();
    int g = blockIdx.x * C::WARPS + warp;
    float2 pv[E / 2];
    auto fetch = [&](int gg) {
        const int it = W.find(gg < nw ? gg : 0);
        const PassArgs &b = W.item[it];
        const int bline = (gg - W.offs[it]) * LPW + li;
        const bool bact = gg < nw && bline < (b.n0 + 1) * b.rows1;
        const float2 *L = b.buf0 + (size_t)(bact ? bline : 0) * n2;
#pragma unroll
        for (int r = 0; r < E / 2; ++r)
            if (bact) pv[r] = L[j + r * T];
    };
#pragma unroll
    for (int r = 0; r < E / 2; ++r) pv[r] = make_float2(0.f, 0.f);
    fetch(g);
    for (; g < nw; g += gstride) {
        FSP_UNIT(W, g, a, u);
        const int lines = (a.n0 + 1) * a.rows1;
        const int line = u * LPW + li;
        const bool act = line < lines;
        const int lc = act ? line : 0;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? pv[r] : make_float2(0.f, 0.f);
        fetch(g + gstride);
        const int kx = lc / a.rows1, row = lc % a.rows1;
        line_fft<N, E, false, true, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(v, j, tw, sm);
        const float *Kr = krow(a, kx, row);
        float2 q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int kf = k <= n2 ? k : N - k;
            v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
            const float kk = wave(k, n2, a.k2s);
            q[r] = make_float2(kk * v[r].y, -kk * v[r].x);
        }
        line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(v, j, tw, sm);
        if (act) {
            float2 *L0 = a.buf0 + (size_t)lc * n2;
#pragma unroll
            for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
        }
        if (withE) {
            line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(q, j, tw, sm);
            if (act) {
                float2 *L1 = a.buf1 + (size_t)lc * n2;
#pragma unroll
                for (int r = 0; r < E / 2; ++r) L1[j + r * T] = q[r];
            }
        }
    }
}

// Single-solve forward middle pass (the arguments by value; same arithmetic
// as p3_fwd below, kept separate because its register allocation is smaller).
template <int N, int ALT = 0>
__global__ void FSP_P3_BOUNDS(WarpCfg<N>::THREADS) p3_fwd1(PassArgs a, int withE)
{
    using C = WarpCfg<N, ALT>;
    constexpr int E = C::E, T = C::T, LPW = C::LPW;
    // the launcher runs length N on lines of n2 = N / 2 cells; a compile-time
    // n2 turns the wavenumber and kernel-octant index arithmetic into constants
    constexpr int n2 = N / 2;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int li = lane / T, j = lane % T;
    const int lines = a.kxn * a.rows1;       // lines of planes [kx0, kx0 + kxn)
    const int line0 = a.kx0 * a.rows1;
    // line -> (k0, row): shifts when rows1 (2 n1, or 1 in 2D) is a power of two
    const bool pow2 = (a.rows1 & (a.rows1 - 1)) == 0;
    const int rsh = __ffs(a.rows1) - 1;
    const int groups = (lines + LPW - 1) / LPW;
    const int gstride = gridDim.x * C::WARPS;
    RowView<C::PAD> sm{smem + (warp * LPW + li) * C::RL};
    const float2 *tw = C::twiddles(smem, a.tw2);
    pdl_wait();
    int g = blockIdx.x * C::WARPS + warp;
    float2 pv[E / 2];   // the next line's pruned input, prefetched into registers
    auto fetch = [&](int gg) {
        const int line = gg * LPW + li;
        const bool act = gg < groups && line < lines;
        const float2 *L = a.buf0 + (size_t)(line0 + (act ? line : 0)) * n2;
#pragma unroll
        for (int r = 0; r < E / 2; ++r)
            if (act) pv[r] = L[j + r * T];
    };
#pragma unroll
    for (int r = 0; r < E / 2; ++r) pv[r] = make_float2(0.f, 0.f);
    fetch(g);
    for (; g < groups; g += gstride) {
        const int line = g * LPW + li;
        const bool act = line < lines;
        const int lc = line0 + (act ? line : 0);   // absolute line index
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? pv[r] : make_float2(0.f, 0.f);
        fetch(g + gstride);
        const int kx = pow2 ? lc >> rsh : lc / a.rows1;
        const int row = pow2 ? lc & (a.rows1 - 1) : lc % a.rows1;
        line_fft<N, E, false, true, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW, C::OFF>(v, j, tw, sm);
        const float *Kr = krow(a, kx, row);
        float2 u[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int kf = k <= n2 ? k : N - k;
            v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
            const float kk = wave(k, n2, a.k2s);
            u[r] = make_float2(kk * v[r].y, -kk * v[r].x);   // -i k2 (K rho^)
        }
        line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW, C::OFF>(v, j, tw, sm);
        if (act) {
            float2 *L0 = a.buf0 + (size_t)lc * n2;
#pragma unroll
            for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
        }
        if (withE) {
            line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW, C::OFF>(u, j, tw, sm);
            if (act) {
                float2 *L1 = a.buf1 + (size_t)lc * n2;
#pragma unroll
                for (int r = 0; r < E / 2; ++r) L1[j + r * T] = u[r];
            }
        }
    }
}

// Forward middle pass for 768- to 2048-point lines (2 n2 = 768, 1024, 1536, 2048):
// 16 values per thread, a line spread over N / 512 warps that synchronise
// among themselves only (a named barrier per line), four warps per CTA,
// persistent over line groups with the next line's input prefetched into
// registers, as the warp-per-line pass does for shorter lines.  Twiddles: the
// all-pass gathered blocks copied into shared memory (consecutive lanes read
// consecutive entries in every pass).  Exchange lines padded one slot per 16
// (conflict-free for these radix plans: bank simulation on the host).
// Resident CTAs the register allocation of p3_fwd_wide is sized for (3: 168
// registers, 12 warps per SM; 4: 128 registers with a small spill, 16 warps).
#ifndef FSP_WIDE_MINB
#define FSP_WIDE_MINB 3
#endif
template <int N>
struct WideCfg {
    static constexpr int E = Plan1D<N>::E;
    using RAD = typename Plan1D<N>::R;
    static constexpr int T = N / E;
    static_assert(T % 32 == 0 && T <= 128, "a line is one to four whole warps");
    static constexpr int WPL = T / 32;            // warps per line
    static constexpr int WARPS = 4;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int LPC = WARPS / WPL;       // lines per CTA
    static constexpr int PAD = 4;
    static constexpr int SPAN = RowSpan<N, PAD>::value;
    static constexpr int TWG = AuxEndAll<1, 0, RAD>::value;   // gathered twiddle entries
    static constexpr size_t SMEM = (size_t)(LPC * SPAN + TWG) * sizeof(float2);
    static constexpr int SYNC = LPC == 1 ? SYNC_BLOCK : SYNC_LINE0 + WPL;
};

template <int N, int MAXI>
__global__ void __launch_bounds__(WideCfg<N>::THREADS, FSP_WIDE_MINB) p3_fwd_wide(const __grid_constant__ Work<MAXI> W, int withE)
{
    using C = WideCfg<N>;
    constexpr int E = C::E, T = C::T, LPC = C::LPC;
    constexpr int n2 = N / 2;   // every item of a length-N launch has n2 = N / 2
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    const int li = threadIdx.x / T, j = threadIdx.x % T;
    const int nw = W.count();
    RowView<C::PAD> sm{smem + li * C::SPAN};
    float2 *stw = smem + LPC * C::SPAN;
    {
        const float2 *gtw = W.item[0].tw2 + N;   // the gathered blocks follow the N-entry table
        for (int i = threadIdx.x; i < C::TWG; i += C::THREADS) stw[i] = gtw[i];
    }
    __syncthreads();
    pdl_wait();
    float2 pv[E / 2];   // the next line's pruned input
    auto fetch = [&](int gg) {
        const int it = W.find(gg < nw ? gg : 0);
        const PassArgs &b = W.item[it];
        const int bline = (gg - W.offs[it]) * LPC + li;
        const bool bact = gg < nw && bline < (b.n0 + 1) * b.rows1;
        const float2 *L = b.buf0 + (size_t)(bact ? bline : 0) * n2;
#pragma unroll
        for (int r = 0; r < E / 2; ++r)
            if (bact) pv[r] = L[j + r * T];
    };
#pragma unroll
    for (int r = 0; r < E / 2; ++r) pv[r] = make_float2(0.f, 0.f);
    int g = blockIdx.x;
    fetch(g);
    for (; g < nw; g += gridDim.x) {
        FSP_UNIT(W, g, a, u);
        const int lines = (a.n0 + 1) * a.rows1;
        const int line = u * LPC + li;
        const bool act = line < lines;
        const int lc = act ? line : 0;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = r < E / 2 ? pv[r] : make_float2(0.f, 0.f);
        fetch(g + gridDim.x);
        const int kx = lc / a.rows1, row = lc % a.rows1;
        line_fft<N, E, false, true, RAD, RowView<C::PAD>, C::SYNC, TW_GSMEM>(v, j, stw, sm);
        const float *Kr = krow(a, kx, row);
        float2 q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int kf = k <= n2 ? k : N - k;
            v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
            const float kk = wave(k, n2, a.k2s);
            q[r] = make_float2(kk * v[r].y, -kk * v[r].x);   // -i k2 (K rho^)
        }
        line_fft<N, E, true, false, RAD, RowView<C::PAD>, C::SYNC, TW_GSMEM>(v, j, stw, sm);
        if (act) {
            float2 *L0 = a.buf0 + (size_t)lc * n2;
#pragma unroll
            for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
        }
        if (withE) {
            line_fft<N, E, true, false, RAD, RowView<C::PAD>, C::SYNC, TW_GSMEM>(q, j, stw, sm);
            if (act) {
                float2 *L1 = a.buf1 + (size_t)lc * n2;
#pragma unroll
                for (int r = 0; r < E / 2; ++r) L1[j + r * T] = q[r];
            }
        }
    }
}

// Forward middle pass for 1024-point lines as two 512-point halves: the split
// k = 2 k2 + k1, n = n2 + 512 n1 with one radix-2 step.  The input is zero for
// n >= 512, so that step is a twiddle only:
//   X[2 k2 + k1] = DFT_512( x[n2] W_1024^(n2 k1) )[k2],
// and warp k1 of a line transforms its half of the spectrum alone, warp-
// synchronously, with the 512-point engine of the middle pass (16 values per
// lane, shuffle exchange before the closing radix-2 pass).  After the product
// with the kernel octant (and -i k2 for E), the inverse halves A_k1 = IDFT_512
// of X[2 k2 + k1] give the cropped output
//   x[n] = A_0[n] + W_1024^(-n) A_1[n],  n < 512,
// one exchange of half a line between the two warps through shared memory
// (warp 0 finishes n < 256, warp 1 the rest).  The 512-point table (main part
// and gathered blocks) is read out of the 1024-point table, W_512^m = W_1024^2m
// (the same FP64 angle, so the same FP32 values).  Two lines per CTA of four
// warps, persistent over line pairs, the next line's input prefetched into
// registers.  Tuned variant bit 8 at 2n = 1024.
struct HalfCfg {
    static constexpr int N = 1024, H = 512, E = 16;
    using RAD = Plan16<512>::R;
    static constexpr int WARPS = 4, THREADS = 32 * WARPS, LPC = 2;
    static constexpr int PAD = 4;
    static constexpr int SPAN = RowSpan<H, PAD>::value;     // per-warp exchange line
    static constexpr int TW = AuxEnd<1, H, RAD>::value;      // 512-point table with its gathered blocks
    static constexpr int XB = WARPS * SPAN;                   // combine buffers: [line][stream][H]
    static constexpr int TWO = XB + LPC * 2 * H;              // the 512-point table
    static constexpr int W1O = TWO + TW;                      // W_1024^n, n < 512
    static constexpr size_t SMEM = (size_t)(W1O + H) * sizeof(float2);
    static_assert(TW == H + 256, "the table fill below follows the 16 x 16 x 2 plan");
};

template <int MAXI>
__global__ void __launch_bounds__(HalfCfg::THREADS) p3_fwd_2h(const __grid_constant__ Work<MAXI> W, int withE)
{
    using C = HalfCfg;
    constexpr int E = C::E, H = C::H, N = C::N, LPC = C::LPC;
    constexpr int n2 = H;   // cells per line
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    const int warp = threadIdx.x / 32, j = threadIdx.x % 32;
    const int li = warp / 2, half = warp % 2;
    const int nw = W.count();
    RowView<C::PAD> sm{smem + warp * C::SPAN};
    float2 *cb = smem + C::XB + li * 2 * H;   // this line's combine buffers (phi, E)
    float2 *stw = smem + C::TWO;
    float2 *w1 = smem + C::W1O;
    {
        const float2 *g = W.item[0].tw2;   // the 1024-point table (every item of the launch has 2 n2 = 1024)
        for (int i = threadIdx.x; i < H; i += C::THREADS) {
            stw[i] = g[2 * i];
            w1[i] = g[i];
        }
        // gathered block of the second pass (NS = 16, R = 16): [r][k] = W_512^(2 r k)
        for (int i = threadIdx.x; i < 256; i += C::THREADS) stw[H + i] = g[(4 * (i / 16) * (i % 16)) % N];
    }
    __syncthreads();
    pdl_wait();
    float2 pv[E];   // the next line's input (n < 512)
    auto fetch = [&](int gg) {
        const int it = W.find(gg < nw ? gg : 0);
        const PassArgs &b = W.item[it];
        const int bline = (gg - W.offs[it]) * LPC + li;
        const bool bact = gg < nw && bline < (b.n0 + 1) * b.rows1;
        const float2 *L = b.buf0 + (size_t)(bact ? bline : 0) * n2;
#pragma unroll
        for (int r = 0; r < E; ++r)
            if (bact) pv[r] = L[j + 32 * r];
    };
#pragma unroll
    for (int r = 0; r < E; ++r) pv[r] = make_float2(0.f, 0.f);
    // the two warps of a line meet at named barrier 1 + li
    auto line_sync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + li), "n"(64) : "memory"); };
    // cropped output of an inverse half: x[n] = A_0[n] + W^(-n) A_1[n], n < 512
    auto combine = [&](float2 (&x)[E], float2 *buf, float2 *dst, bool act) {
        if (half == 0) {
#pragma unroll
            for (int r = E / 2; r < E; ++r) buf[j + 32 * r] = x[r];
        } else {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) buf[j + 32 * r] = cmul_dir<true>(x[r], w1[j + 32 * r]);
        }
        line_sync();
        if (half == 0) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const float2 o = x[r] + buf[j + 32 * r];
                if (act) dst[j + 32 * r] = o;
            }
        } else {
#pragma unroll
            for (int r = E / 2; r < E; ++r) {
                const float2 o = buf[j + 32 * r] + cmul_dir<true>(x[r], w1[j + 32 * r]);
                if (act) dst[j + 32 * r] = o;
            }
        }
    };
    int g = blockIdx.x;
    fetch(g);
    for (; g < nw; g += gridDim.x) {
        FSP_UNIT(W, g, a, u);
        const int lines = (a.n0 + 1) * a.rows1;
        const int line = u * LPC + li;
        const bool act = line < lines;
        const int lc = act ? line : 0;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = half ? cmul(pv[r], w1[j + 32 * r]) : pv[r];
        fetch(g + gridDim.x);
        const int kx = lc / a.rows1, row = lc % a.rows1;
        line_fft<H, E, false, false, RAD, RowView<C::PAD>, SYNC_WARP, TW_SMEM>(v, j, stw, sm);
        const float *Kr = krow(a, kx, row);
        float2 q[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = 2 * (j + 32 * r) + half;
            const int kf = k <= n2 ? k : N - k;
            v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
            const float kk = wave(k, n2, a.k2s);
            q[r] = make_float2(kk * v[r].y, -kk * v[r].x);   // -i k2 (K rho^)
        }
        line_fft<H, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, TW_SMEM>(v, j, stw, sm);
        combine(v, cb, a.buf0 + (size_t)lc * n2, act);
        if (withE) {
            line_fft<H, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, TW_SMEM>(q, j, stw, sm);
            combine(q, cb + H, a.buf1 + (size_t)lc * n2, act);
        }
        // the next line's combines write these buffers only after both warps
        // have passed the barrier of the other stream (or of this one, without E)
        if (!withE) line_sync();
    }
}

// Adjoint middle pass, warp per line group.
template <int N, int MAXI>
__global__ void __launch_bounds__(WarpCfg<N>::THREADS) p3_adj(const __grid_constant__ Work<MAXI> W, int hasE)
{
    using C = WarpCfg<N>;
    constexpr int E = C::E, T = C::T, LPW = C::LPW;
    using RAD = typename C::RAD;
    extern __shared__ float2 smem[];
    pdl_trigger();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int li = lane / T, j = lane % T;
    const int nw = W.count();
    constexpr int n2 = N / 2;   // every item of a length-N launch has n2 = N / 2
    RowView<C::PAD> sm{smem + (warp * LPW + li) * C::RL};
    const float2 *tw = C::twiddles(smem, W.item[0].tw2);   // the table depends on N only
    pdl_wait();
    for (int g = blockIdx.x * C::WARPS + warp; g < nw; g += gridDim.x * C::WARPS) {
        FSP_UNIT(W, g, a, u);
        const int lines = (a.n0 + 1) * a.rows1;
        const int line = u * LPW + li;
        const bool act = line < lines;
        const int lc = act ? line : 0;
        float2 *L0 = a.buf0 + (size_t)lc * n2;
        float2 *L1 = a.buf1 + (size_t)lc * n2;
        float2 v[E];
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = (r < E / 2 && act) ? L0[j + r * T] : make_float2(0.f, 0.f);
        line_fft<N, E, false, true, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(v, j, tw, sm);
        if (hasE) {
            float2 q[E];
#pragma unroll
            for (int r = 0; r < E; ++r) q[r] = (r < E / 2 && act) ? L1[j + r * T] : make_float2(0.f, 0.f);
            line_fft<N, E, false, true, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(q, j, tw, sm);
#pragma unroll
            for (int r = 0; r < E; ++r) {
                const float kk = wave(j + r * T, n2, a.k2s);
                v[r] = make_float2(v[r].x - kk * q[r].y, v[r].y + kk * q[r].x);
            }
        }
        const int kx = lc / a.rows1, row = lc % a.rows1;
        const float *Kr = krow(a, kx, row);
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int k = j + r * T;
            const int kf = k <= n2 ? k : N - k;
            v[r] = (act ? __ldg(Kr + kf) : 0.f) * v[r];
        }
        line_fft<N, E, true, false, RAD, RowView<C::PAD>, SYNC_WARP, FSP_P3_TW>(v, j, tw, sm);
        if (act) {
#pragma unroll
            for (int r = 0; r < E / 2; ++r) L0[j + r * T] = v[r];
        }
    }
}

// Launch a pass with the programmatic stream-serialization attribute when
// pdl (see pdl_trigger / pdl_wait); the kernel must call pdl_wait before its
// first global-memory access.
template <class Kern, class... Args>
inline int launch_pdl_if(bool pdl, Kern kern, int grid, int threads, size_t smem, cudaStream_t st, const Args &...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = FSP_PDL && pdl;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return (int)cudaLaunchKernelEx(&cfg, kern, args...);
}

template <class Kern, class... Args>
inline int launch_pdl(Kern kern, int grid, int threads, size_t smem, cudaStream_t st, const Args &...args)
{
    return launch_pdl_if(true, kern, grid, threads, smem, st, args...);
}

// Long lines (2n >= 2048) gain from the early scheduling while a pass is short
// (2n = 2048: 1024^2 solves -11%) and lose once it is long (2n = 8192: 4096^2
// +1.2%, measured), so their launches use it below 2n = 8192 only.
template <int N>
constexpr bool kLongPdl = N < 8192;

} // namespace fsp
