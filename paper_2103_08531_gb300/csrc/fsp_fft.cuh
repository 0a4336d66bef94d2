// fsp_fft.cuh -- register-resident FFT engine for the padded convolution.
//
// One line of N complex values is spread over T = N / E threads, thread j holding
// the E values at positions j + r T (r < E).  The transform is a Stockham
// decimation-in-time sequence of radix-R passes (R in {2, 3, 4, 8, 16}); in pass s
// (NS = product of the earlier radices) butterfly b = j + q T (q < E / R) takes
// x[b + r N / R], multiplies by W^(r (b mod NS) N / (NS R)), does an R-point DFT
// and sends output u to position (b / NS) NS R + (b mod NS) + u NS.  Between
// passes the values go through shared memory; after the last pass every output
// lands back in the register it came from, in natural order (position j + r T).
//
// "Pruned" input: when positions >= N/2 are known to be zero (the zero padding of
// the convolution, paper Sec. 1), the first pass loads and combines only the
// lower half: each butterfly has R/2 nonzero inputs, and its R-point DFT is done
// as two R/2-point DFTs.  Output pruning needs no code: callers store only the
// outputs that survive the crop and the compiler drops the rest.
//
// Twiddles come from a table W_N^m = exp(-2 pi i m / N), m < N, rounded to FP32
// from FP64 angles at plan creation; the inverse transform uses the conjugate.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>

namespace fsp {

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward direction) or +i (inverse direction)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by exp(-/+ 2 pi i / 8)
template <bool INV>
__device__ __forceinline__ float2 w8_1(float2 a)
{
    const float c = 0.70710678118654752f;
    return INV ? make_float2(c * (a.x - a.y), c * (a.x + a.y)) : make_float2(c * (a.x + a.y), c * (a.y - a.x));
}
// multiply by exp(-/+ 2 pi i 3 / 8)
template <bool INV>
__device__ __forceinline__ float2 w8_3(float2 a)
{
    const float c = 0.70710678118654752f;
    return INV ? make_float2(-c * (a.x + a.y), c * (a.x - a.y)) : make_float2(c * (a.y - a.x), -c * (a.x + a.y));
}
template <bool INV>
__device__ __forceinline__ float2 cmul_dir(float2 a, float2 w)
{
    return INV ? cmulc(a, w) : cmul(a, w);
}

// ---------------------------------------------------------------- butterflies
// In place, natural order in and out: X_u = sum_r v_r exp(-/+ 2 pi i r u / R).

template <bool INV>
__device__ __forceinline__ void dft2(float2 &a, float2 &b)
{
    float2 t = a;
    a = t + b;
    b = t - b;
}

template <bool INV>
__device__ __forceinline__ void dft3(float2 &a, float2 &b, float2 &c)
{
    const float s3 = 0.86602540378443865f;
    float2 t1 = b + c;
    float2 t2 = a - 0.5f * t1;
    float2 t3 = s3 * (b - c);
    a = a + t1;
    b = t2 + rot<INV>(t3);
    c = t2 - rot<INV>(t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    float2 s0 = a0 + a2, d0 = a0 - a2, s1 = a1 + a3, d1 = rot<INV>(a1 - a3);
    a0 = s0 + s1;
    a2 = s0 - s1;
    a1 = d0 + d1;
    a3 = d0 - d1;
}

template <bool INV>
__device__ __forceinline__ void dft8(float2 *v)
{
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = w8_1<INV>(o1);
    o2 = rot<INV>(o2);
    o3 = w8_3<INV>(o3);
    v[0] = e0 + o0;
    v[4] = e0 - o0;
    v[1] = e1 + o1;
    v[5] = e1 - o1;
    v[2] = e2 + o2;
    v[6] = e2 - o2;
    v[3] = e3 + o3;
    v[7] = e3 - o3;
}

// exp(-/+ 2 pi i u / 16), u = 1..7 (cos, sin of u pi / 8)
template <bool INV>
__device__ __forceinline__ float2 w16(float2 a, int u)
{
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, c2 = 0.70710678118654752f;
    float2 w;
    switch (u) {
    case 1: w = make_float2(c1, -s1); break;
    case 2: w = make_float2(c2, -c2); break;
    case 3: w = make_float2(s1, -c1); break;
    case 4: w = make_float2(0.f, -1.f); break;
    case 5: w = make_float2(-s1, -c1); break;
    case 6: w = make_float2(-c2, -c2); break;
    default: w = make_float2(-c1, -s1); break;
    }
    if (u == 4) return rot<INV>(a);
    return cmul_dir<INV>(a, w);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2 *v)
{
    float2 e[8], o[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        e[i] = v[2 * i];
        o[i] = v[2 * i + 1];
    }
    dft8<INV>(e);
    dft8<INV>(o);
#pragma unroll
    for (int u = 1; u < 8; ++u) o[u] = w16<INV>(o[u], u);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        v[u] = e[u] + o[u];
        v[u + 8] = e[u] - o[u];
    }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *v)
{
    if constexpr (R == 2) dft2<INV>(v[0], v[1]);
    else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 16) dft16<INV>(v);
    else static_assert(R == 2, "unsupported radix");
}

// R-point DFT of v[0..R/2) followed by R/2 zeros:
// X_{2u} = DFT_{R/2}(v)_u,  X_{2u+1} = DFT_{R/2}(v_r w_R^r)_u.
template <int R, bool INV>
__device__ __forceinline__ void dft_half_in(float2 *v)
{
    if constexpr (R == 2) {
        v[1] = v[0];
    } else if constexpr (R == 4) {
        float2 a = v[0], b = v[1];
        float2 bb = rot<INV>(b);
        v[0] = a + b;
        v[2] = a - b;
        v[1] = a + bb;
        v[3] = a - bb;
    } else if constexpr (R == 8) {
        float2 a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
        float2 b0 = a0, b1 = w8_1<INV>(a1), b2 = rot<INV>(a2), b3 = w8_3<INV>(a3);
        dft4<INV>(a0, a1, a2, a3);
        dft4<INV>(b0, b1, b2, b3);
        v[0] = a0;
        v[2] = a1;
        v[4] = a2;
        v[6] = a3;
        v[1] = b0;
        v[3] = b1;
        v[5] = b2;
        v[7] = b3;
    } else if constexpr (R == 16) {
        float2 a[8], b[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            a[r] = v[r];
            b[r] = (r == 0) ? v[0] : w16<INV>(v[r], r);
        }
        dft8<INV>(a);
        dft8<INV>(b);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            v[2 * u] = a[u];
            v[2 * u + 1] = b[u];
        }
    } else {
        static_assert(R % 2 == 0, "a pruned first pass needs an even radix");
    }
}

// ------------------------------------------------------------ shared memory views

// Column tile: position p of column c at base[p * ld + c].
struct ColView {
    float2 *base;
    int ld;
    __device__ __forceinline__ float2 &at(int p) const { return base[p * ld]; }
};

// Contiguous line with one padding slot every 2^PAD positions (bank spreading).
template <int PAD>
struct RowView {
    float2 *base;
    __device__ __forceinline__ float2 &at(int p) const { return base[p + (p >> PAD)]; }
};

template <int N, int PAD>
struct RowSpan {
    static constexpr int value = N + (N >> PAD) + 1;
};

// ------------------------------------------------------------------ cp.async

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------- passes

// Sync group of a transform: the whole block, one warp, or (SYNC_LINE0 + w) the
// w warps of one line, with named barrier 1 + threadIdx.x / (32 w).
enum { SYNC_BLOCK = 0, SYNC_WARP = 1, SYNC_LINE0 = 64 };
// Twiddle sources: TW_TABLE loads each W^(r m) from the table (cheap when the
// lanes of a warp share m, as in column tiles); TW_POW loads W^m, W^2m, W^4m,
// W^8m and forms the other powers by products (lanes with distinct m).
// TW_GATHER (lanes own consecutive j): passes with NS < 32 read a small table
// laid out [r][k] after the main one (tw + N + OFF), so a warp's loads are
// contiguous; later passes read the main table, already contiguous in k.
// TW_SMEM: as TW_GATHER, but the caller has copied the whole table (main
// part and gathered blocks) into shared memory and passes that copy.
// TW_STABLE: as TW_TABLE, from a copy of the main table in shared memory.
// TW_QSMEM: a shared-memory copy of the first quarter of the table only
// (N a multiple of 4): W^(m + N/4) = -i W^m, so W^m is the entry m mod N/4
// turned by (-i)^(m div N/4).
// TW_GALL: gathered blocks [r][k] for every pass with NS > 1 (not only NS < 32),
// read from global memory: a warp's 16-32 consecutive k read consecutive
// entries (the long-line passes, whose tables do not fit in shared memory).
// TW_GSMEM: the TW_GALL blocks copied into shared memory, passed without the
// main table in front (entry [pass][r][k] at tw + OFF + r NS + k).
enum { TW_TABLE = 0, TW_POW = 1, TW_GATHER = 2, TW_SMEM = 3, TW_STABLE = 4, TW_QSMEM = 5, TW_GALL = 7, TW_GSMEM = 8 };

// W_N^m (m < N) from the quarter table.
template <int N>
__device__ __forceinline__ float2 qtw(const float2 *tq, int m)
{
    constexpr int Q = N / 4;
    const int qd = m / Q;
    const float2 t = tq[m - qd * Q];
    float2 r = (qd & 1) ? make_float2(t.y, -t.x) : t;   // times -i
    if (qd & 2) r = make_float2(-r.x, -r.y);             // times -1
    return r;
}

template <int TW>
__device__ __forceinline__ float2 ldtw(const float2 *p)
{
    if constexpr (TW == TW_SMEM || TW == TW_STABLE || TW == TW_GSMEM) return *p;
    else return __ldg(p);
}

template <int SYNC>
__device__ __forceinline__ void lsync()
{
    if constexpr (SYNC == SYNC_WARP) {
        __syncwarp();
    } else if constexpr (SYNC > SYNC_LINE0) {
        constexpr int LT = 32 * (SYNC - SYNC_LINE0);
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / LT), "n"(LT) : "memory");
    } else {
        __syncthreads();
    }
}

// u[r] *= W^(r m) (conjugated for the inverse), r = 1 .. R-1.
template <int R, bool INV, int TW>
__device__ __forceinline__ void twiddle(float2 *u, const float2 *__restrict__ tw, int m)
{
    if constexpr (TW == TW_TABLE || TW == TW_SMEM || TW == TW_STABLE || R <= 3) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], ldtw<TW>(tw + r * m));
    } else {
        float2 w[R];
        w[1] = __ldg(tw + m);
        w[2] = __ldg(tw + 2 * m);
        w[3] = cmul(w[1], w[2]);
        if constexpr (R >= 8) {
            w[4] = __ldg(tw + 4 * m);
            w[5] = cmul(w[1], w[4]);
            w[6] = cmul(w[2], w[4]);
            w[7] = cmul(w[3], w[4]);
        }
        if constexpr (R >= 16) {
            w[8] = __ldg(tw + 8 * m);
#pragma unroll
            for (int r = 9; r < 16; ++r) w[r] = cmul(w[8], w[r - 8]);
        }
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], w[r]);
    }
}

template <int... RS>
struct Radices {};

template <int N, int E, bool INV, int NS, class RAD, int SYNC, int TW, int OFF = 0>
struct Passes;

template <int N, int E, bool INV, int NS, int SYNC, int TW, int OFF>
struct Passes<N, E, INV, NS, Radices<>, SYNC, TW, OFF> {
    template <bool PRUNE, class View>
    static __device__ __forceinline__ void run(float2 (&)[E], int, const float2 *__restrict__, const View &)
    {
    }
};

// Offset of the gathered twiddle block of the pass after one with (NS, R).
template <int NS, int R, int OFF>
struct NextOff {
    static constexpr int value = OFF + ((NS > 1 && NS < 32) ? R * NS : 0);
};
// The same in the TW_GALL layout (a block for every pass with NS > 1).
template <int NS, int R, int OFF>
struct NextOffAll {
    static constexpr int value = OFF + (NS > 1 ? R * NS : 0);
};
template <int TW, int NS, int R, int OFF>
struct NextOffT {
    static constexpr int value =
        (TW == TW_GALL || TW == TW_GSMEM) ? NextOffAll<NS, R, OFF>::value : NextOff<NS, R, OFF>::value;
};

// Twiddles of butterfly column k (= b mod NS) in a pass with (NS, R); OFF is
// the pass's gathered block in the TW_GATHER / TW_SMEM layouts.
template <int N, int R, bool INV, int NS, int TW, int OFF>
__device__ __forceinline__ void pass_twiddles(float2 *u, const float2 *__restrict__ tw, int k)
{
    if constexpr (TW == TW_GALL) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], __ldg(tw + N + OFF + r * NS + k));
    } else if constexpr (TW == TW_GSMEM) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], tw[OFF + r * NS + k]);
    } else if constexpr (TW == TW_QSMEM) {
        static_assert(N % 4 == 0, "the quarter table needs N divisible by 4");
        const int m = k * (N / (NS * R));
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], qtw<N>(tw, r * m));
    } else if constexpr ((TW == TW_GATHER || TW == TW_SMEM) && NS < 32) {
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul_dir<INV>(u[r], ldtw<TW>(tw + N + OFF + r * NS + k));
    } else {
        twiddle<R, INV, TW == TW_GATHER ? TW_TABLE : TW>(u, tw, k * (N / (NS * R)));
    }
}

// End of the gathered blocks of a radix plan (entries after the main table).
template <int NS, int OFF, class RAD>
struct AuxEnd;
template <int NS, int OFF>
struct AuxEnd<NS, OFF, Radices<>> {
    static constexpr int value = OFF;
};
template <int NS, int OFF, int R, int... RS>
struct AuxEnd<NS, OFF, Radices<R, RS...>> {
    static constexpr int value = AuxEnd<NS * R, NextOff<NS, R, OFF>::value, Radices<RS...>>::value;
};

// Shuffle exchange before a closing radix-2 pass.  With 32 threads per line
// (lane = j), one butterfly per thread (E = R) and NS R = N / 2, thread j's R
// outputs sit at positions h N/2 + (j mod 16) + 16 u (h = j / 16): the next
// pass needs positions j + 32 r, which are thread j's outputs u = h + 2 i and
// the outputs u = (1 - h) + 2 i of lane j ^ 16.  So the exchange is a swap of
// half the registers between lane pairs: E/2 shuffles instead of a trip
// through shared memory.
#ifndef FSP_SHFL_PAIR
#define FSP_SHFL_PAIR 1
#endif
#ifndef FSP_HALF_XCH
#define FSP_HALF_XCH 1
#endif
template <int... RS>
struct IsClosingRadix2 : std::false_type {};
template <>
struct IsClosingRadix2<2> : std::true_type {};

template <int E>
__device__ __forceinline__ void pair_exchange(float2 (&v)[E], const float2 *u, int j)
{
    const bool hi = (j & 16) != 0;
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
        const float2 keep = hi ? u[2 * i + 1] : u[2 * i];
        const float2 send = hi ? u[2 * i] : u[2 * i + 1];
        float2 recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 16);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 16);
        v[i] = hi ? recv : keep;
        v[E / 2 + i] = hi ? keep : recv;
    }
}

// Does the pass with (NS, radices RAD) take the block-synchronous half exchange?
template <int N, int E, int NS, int SYNC, class RAD>
struct IsHalfPass : std::false_type {};
template <int N, int E, int NS, int SYNC, int R, int... RS>
struct IsHalfPass<N, E, NS, SYNC, Radices<R, RS...>>
    : std::integral_constant<bool, FSP_HALF_XCH && SYNC == SYNC_BLOCK && N / E == 32 && E == R && 2 * NS * R == N &&
                                       IsClosingRadix2<RS...>::value> {};

template <int N, int E, bool INV, int NS, int R, int... RS, int SYNC, int TW, int OFF>
struct Passes<N, E, INV, NS, Radices<R, RS...>, SYNC, TW, OFF> {
    template <bool PRUNE, class View>
    static __device__ __forceinline__ void run(float2 (&v)[E], int j, const float2 *__restrict__ tw, const View &sm)
    {
        constexpr int T = N / E;
        constexpr int Q = E / R;
        constexpr bool LAST = sizeof...(RS) == 0;
        constexpr bool PAIR = FSP_SHFL_PAIR && SYNC == SYNC_WARP && T == 32 && Q == 1 && 2 * NS * R == N &&
                              IsClosingRadix2<RS...>::value;
        // Block-synchronous form of the same lane-pair swap: only the half of
        // the outputs that changes thread goes through shared memory.  The
        // branches are warp-uniform in column tiles (j = tid / columns).
        // Its stores go to positions the storing thread itself read in the
        // previous exchange (p = j mod 32), so that exchange needs no closing
        // barrier before them.
        constexpr bool HALF = IsHalfPass<N, E, NS, SYNC, Radices<R, RS...>>::value;
        constexpr bool NEXT_HALF = IsHalfPass<N, E, NS * R, SYNC, Radices<RS...>>::value;
        static_assert(E % R == 0, "E must be a multiple of every radix");
        if constexpr (HALF) {
            const int k = j % NS;
            float2 u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[r];
            pass_twiddles<N, R, INV, NS, TW, OFF>(u, tw, k);
            dft<R, INV>(u);
            const bool hi = (j & 16) != 0;
            // output u of thread j sits at position hi N/2 + (j mod 16) + 16 u;
            // thread j parks what its partner j ^ 16 needs at j + 32 i (hi) or
            // j + N/2 + 32 i (lo), slots that only thread j read before
            if (hi) {
#pragma unroll
                for (int i = 0; i < E / 2; ++i) sm.at(j + 32 * i) = u[2 * i];
            } else {
#pragma unroll
                for (int i = 0; i < E / 2; ++i) sm.at(j + N / 2 + 32 * i) = u[2 * i + 1];
            }
            lsync<SYNC>();
            if (hi) {
#pragma unroll
                for (int i = 0; i < E / 2; ++i) {
                    v[i] = sm.at((j & 15) + N / 2 + 32 * i);
                    v[E / 2 + i] = u[2 * i + 1];
                }
            } else {
#pragma unroll
                for (int i = 0; i < E / 2; ++i) {
                    v[i] = u[2 * i];
                    v[E / 2 + i] = sm.at(j + 16 + 32 * i);
                }
            }
            lsync<SYNC>();
            Passes<N, E, INV, NS * R, Radices<RS...>, SYNC, TW, NextOffT<TW, NS, R, OFF>::value>::template run<false>(v, j, tw,
                                                                                                         sm);
            return;
        }
        if constexpr (PAIR) {
            const int k = j % NS;
            float2 u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[r];
            pass_twiddles<N, R, INV, NS, TW, OFF>(u, tw, k);
            dft<R, INV>(u);
            pair_exchange<E>(v, u, j);
            Passes<N, E, INV, NS * R, Radices<RS...>, SYNC, TW, NextOffT<TW, NS, R, OFF>::value>::template run<false>(v, j, tw,
                                                                                                         sm);
            return;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int b = j + q * T;
            const int k = b % NS;
            float2 u[R];
#pragma unroll
            for (int r = 0; r < R; ++r) u[r] = v[q + r * Q];
            if constexpr (NS > 1) pass_twiddles<N, R, INV, NS, TW, OFF>(u, tw, k);
            if constexpr (PRUNE && NS == 1) dft_half_in<R, INV>(u);
            else dft<R, INV>(u);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[q + r * Q] = u[r];
            } else {
                const int base = (b / NS) * NS * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) sm.at(base + r * NS) = u[r];
            }
        }
        if constexpr (!LAST) {
            lsync<SYNC>();
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = sm.at(j + r * T);
            if constexpr (!NEXT_HALF) lsync<SYNC>();
            Passes<N, E, INV, NS * R, Radices<RS...>, SYNC, TW, NextOffT<TW, NS, R, OFF>::value>::template run<false>(v, j, tw,
                                                                                                         sm);
        }
    }
};

// Whole-line transform.  Precondition: every thread of the sync group (block
// or warp) calls it and nobody still reads the shared buffer.  On return the
// shared buffer is free again.
// OFF: where the plan's gathered twiddle blocks start after the N-entry table
// (TW_GATHER / TW_SMEM; 0 for the first plan of a length).
template <int N, int E, bool INV, bool PRUNE_IN, class RAD, class View, int SYNC = SYNC_BLOCK, int TW = TW_TABLE,
          int OFF = 0>
__device__ __forceinline__ void line_fft(float2 (&v)[E], int j, const float2 *__restrict__ tw, const View &sm)
{
    Passes<N, E, INV, 1, RAD, SYNC, TW, OFF>::template run<PRUNE_IN>(v, j, tw, sm);
}

// Gathered twiddle blocks for a radix plan: for every pass with 1 < NS < 32,
// entry [r][k] (r < R, k < NS) = W_N^(r k N / (NS R)), FP64 angle rounded once.
template <int N, int NS, int OFF, class RAD>
struct AuxFill {
    static __device__ void run(float2 *, int) {}
};
template <int N, int NS, int OFF, int R, int... RS>
struct AuxFill<N, NS, OFF, Radices<R, RS...>> {
    static __device__ void run(float2 *aux, int i)
    {
        if constexpr (NS > 1 && NS < 32) {
            if (i < R * NS) {
                const int r = i / NS, k = i % NS;
                const long long e = (long long)r * k * (N / (NS * R));
                double sn, cs;
                sincospi(2.0 * (double)(e % N) / (double)N, &sn, &cs);
                aux[OFF + i] = make_float2((float)cs, (float)-sn);
            }
        }
        AuxFill<N, NS * R, NextOff<NS, R, OFF>::value, Radices<RS...>>::run(aux, i);
    }
};
// The TW_GALL layout: a block [r][k] for every pass with NS > 1.
template <int N, int NS, int OFF, class RAD>
struct AuxFillAll {
    static __device__ void run(float2 *, int) {}
};
template <int N, int NS, int OFF, int R, int... RS>
struct AuxFillAll<N, NS, OFF, Radices<R, RS...>> {
    static __device__ void run(float2 *aux, int i)
    {
        if constexpr (NS > 1) {
            if (i < R * NS) {
                const int r = i / NS, k = i % NS;
                const long long e = (long long)r * k * (N / (NS * R));
                double sn, cs;
                sincospi(2.0 * (double)(e % N) / (double)N, &sn, &cs);
                aux[OFF + i] = make_float2((float)cs, (float)-sn);
            }
        }
        AuxFillAll<N, NS * R, NextOffAll<NS, R, OFF>::value, Radices<RS...>>::run(aux, i);
    }
};
template <int NS, int OFF, class RAD>
struct AuxEndAll;
template <int NS, int OFF>
struct AuxEndAll<NS, OFF, Radices<>> {
    static constexpr int value = OFF;
};
template <int NS, int OFF, int R, int... RS>
struct AuxEndAll<NS, OFF, Radices<R, RS...>> {
    static constexpr int value = AuxEndAll<NS * R, NextOffAll<NS, R, OFF>::value, Radices<RS...>>::value;
};
template <int N, class RAD>
__global__ void k_twiddles_gall(float2 *tw)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
        AuxFillAll<N, 1, 0, RAD>::run(tw + N, i);
}

template <int N, class RAD, int OFF = 0>
__global__ void k_twiddles_aux(float2 *tw)
{
    AuxFill<N, 1, OFF, RAD>::run(tw + N, blockIdx.x * blockDim.x + threadIdx.x);
}

// Radix plans per padded length for block-synchronous tiles (E values per thread).
template <int N>
struct Plan1D;
template <> struct Plan1D<32> { static constexpr int E = 8; using R = Radices<8, 4>; };
template <> struct Plan1D<64> { static constexpr int E = 8; using R = Radices<8, 8>; };
template <> struct Plan1D<96> { static constexpr int E = 12; using R = Radices<4, 4, 2, 3>; };
template <> struct Plan1D<128> { static constexpr int E = 8; using R = Radices<8, 8, 2>; };
template <> struct Plan1D<192> { static constexpr int E = 12; using R = Radices<4, 4, 4, 3>; };
template <> struct Plan1D<256> { static constexpr int E = 8; using R = Radices<8, 8, 4>; };
template <> struct Plan1D<384> { static constexpr int E = 12; using R = Radices<4, 4, 4, 2, 3>; };
template <> struct Plan1D<512> { static constexpr int E = 8; using R = Radices<8, 8, 8>; };
template <> struct Plan1D<768> { static constexpr int E = 12; using R = Radices<4, 4, 4, 4, 3>; };
template <> struct Plan1D<1024> { static constexpr int E = 16; using R = Radices<16, 8, 8>; };
template <> struct Plan1D<1536> { static constexpr int E = 12; using R = Radices<4, 4, 4, 4, 2, 3>; };
template <> struct Plan1D<2048> { static constexpr int E = 16; using R = Radices<16, 16, 8>; };
template <> struct Plan1D<3072> { static constexpr int E = 12; using R = Radices<4, 4, 4, 4, 4, 3>; };
template <> struct Plan1D<4096> { static constexpr int E = 16; using R = Radices<16, 16, 16>; };
template <> struct Plan1D<6144> { static constexpr int E = 12; using R = Radices<4, 4, 4, 4, 4, 2, 3>; };
template <> struct Plan1D<8192> { static constexpr int E = 16; using R = Radices<16, 8, 8, 8>; };

// Radix plans for 16-values-per-thread work (one warp or less per line).
template <int N>
struct Plan16;
template <> struct Plan16<32> { static constexpr int E = 8; using R = Radices<8, 4>; };
template <> struct Plan16<64> { static constexpr int E = 8; using R = Radices<8, 8>; };
template <> struct Plan16<96> { static constexpr int E = 12; using R = Radices<4, 4, 2, 3>; };
template <> struct Plan16<128> { static constexpr int E = 16; using R = Radices<16, 8>; };
template <> struct Plan16<192> { static constexpr int E = 12; using R = Radices<4, 4, 4, 3>; };
template <> struct Plan16<256> { static constexpr int E = 16; using R = Radices<16, 16>; };
template <> struct Plan16<384> { static constexpr int E = 12; using R = Radices<4, 4, 4, 2, 3>; };
template <> struct Plan16<512> { static constexpr int E = 16; using R = Radices<16, 16, 2>; };

// A second radix split of the same lengths with the same values per thread,
// the alternative a tuned launch variant can pick (variant bit 8): radix 8
// first, so the pruned first pass and every exchange move other strides.
template <int N>
struct Plan16B {
    static constexpr bool HAS = false;
};
template <> struct Plan16B<128> { static constexpr bool HAS = true; static constexpr int E = 16; using R = Radices<8, 16>; };
template <> struct Plan16B<256> { static constexpr bool HAS = true; static constexpr int E = 16; using R = Radices<8, 8, 4>; };
template <> struct Plan16B<512> { static constexpr bool HAS = true; static constexpr int E = 16; using R = Radices<8, 8, 8>; };

// The plan of a length: ALT = 0 Plan16, ALT = 1 Plan16B.
template <int N, int ALT>
struct PlanSel {
    using type = Plan16<N>;
};
template <int N>
struct PlanSel<N, 1> {
    using type = Plan16B<N>;
};

// Gathered twiddle blocks of Plan16B<N> start where those of Plan16<N> end
// (offsets after the N-entry table; the first plan's blocks start at 0).
template <int N, int ALT>
struct AuxOff {
    static constexpr int value = ALT ? AuxEnd<1, 0, typename Plan16<N>::R>::value : 0;
};


} // namespace fsp
