// fsp_direct.cu -- the direct-sum DFT path: any grid size, FP32 or FP64.
//
// The fast passes cover padded lengths 2 n of the forms listed in fsp.h, in
// FP32.  The paper's convergence studies (Sec. 3: N = 10 ... 100 cells per
// axis, so 2 N with large prime factors) and FP64 solves need other sizes and
// another precision; plans for them run this path.  It computes the same
// pruned convolution as the fast passes (paper Sec. 1, Eq. "eq:convolution";
// Fourier differentiation, Sec. 3):
//
//   G1  X   = DFT_x(rho padded)            kx in [0, n0]    (half spectrum)
//   G2  Y   = DFT_y(X padded)              ky in [0, 2 n1)  (3D only)
//   G3  per (kx, ky) line: S = K DFT_z(Y padded); Phi = IDFT_z(S),
//       Ez = IDFT_z(-i kz S), both cropped to z < n2
//   G4  IDFT_y of Phi, of -i ky Phi and of Ez, cropped to y < n1 (3D only)
//   G5  real inverse along x from the half spectra (Hermitian extension),
//       cropped to x < n0: phi, E_x (times -i kx), E_y, E_z
//
// with every 1D transform taken by its definition, X_k = sum_j x_j
// exp(-/+ 2 pi i j k / N): one output per thread, O(N) work per output.  K is
// the plan's kernel octant (prod(h) / prod(2n) folded in), in the plan's
// precision.  Twiddles are cos / sin of 2 pi m / N from FP64 angles, rounded
// to the working precision.
#include "fsp_internal.h"

#include <algorithm>
#include <cstdint>

namespace fsp {

namespace {

template <class R>
struct alignas(2 * sizeof(R)) Cx {
    R re, im;
};

template <class R>
__device__ __forceinline__ Cx<R> twid(const double2 *tw, long long m, bool inv)
{
    const double2 t = tw[m];
    return Cx<R>{(R)t.x, inv ? (R)t.y : (R)-t.y};
}

template <class R>
__device__ __forceinline__ void madd(Cx<R> &acc, Cx<R> x, Cx<R> w)
{
    acc.re += x.re * w.re - x.im * w.im;
    acc.im += x.re * w.im + x.im * w.re;
}

// Signed wavenumber of index k on a padded axis of 2 n points, zero at the
// unpaired index n (Fourier differentiation with the Nyquist entry zero).
__device__ __forceinline__ double wavenum(long long k, long long n, double s)
{
    const long long m = k < n ? k : (k == n ? 0 : k - 2 * n);
    return s * (double)m;
}

template <class R>
__device__ __forceinline__ Cx<R> times_minus_i(Cx<R> x, R kk)
{
    return Cx<R>{kk * x.im, -kk * x.re};
}

// out(o, k, i) = sum_{j < J} m(j) in(o, j, i) W^(+-k j), W = exp(2 pi i / N),
// i contiguous; m(j) = -i k(j) when mult, else 1.
struct DftArgs {
    const void *in;
    void *out;
    long long O, J, K, I;
    long long in_o, in_j, out_o, out_k;
    int N;
    const double2 *tw;
    int mult;
    double ks;
    int real_in;
};

template <class R, bool INV>
__global__ void k_direct_dft(DftArgs a)
{
    const long long total = a.O * a.K * a.I;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx % a.I, t = idx / a.I;
        const long long k = t % a.K, o = t / a.K;
        Cx<R> acc{0, 0};
        long long m = 0;   // k j mod N
        const long long base = o * a.in_o + i;
        for (long long j = 0; j < a.J; ++j) {
            Cx<R> x;
            if (a.real_in) x = Cx<R>{static_cast<const R *>(a.in)[base + j * a.in_j], (R)0};
            else x = static_cast<const Cx<R> *>(a.in)[base + j * a.in_j];
            if (a.mult) x = times_minus_i(x, (R)wavenum(j, a.N / 2, a.ks));
            madd(acc, x, twid<R>(a.tw, m, INV));
            m += k;
            if (m >= a.N) m -= a.N;
        }
        static_cast<Cx<R> *>(a.out)[o * a.out_o + k * a.out_k + i] = acc;
    }
}

// G3: one block per (kx, ky) line of the y-transformed half spectrum.
struct MidArgs {
    const void *in;      // [lines][n2]
    void *phi;           // [lines][n2]
    void *ez;            // [lines][n2] or null
    long long lines;
    int rows;            // ky rows per kx: 2 n1 (3D) or 1 (2D)
    int n1, n2, N2, three_d;
    const double2 *tw;   // N2 entries
    const void *K;       // kernel octant, working precision
    double k2s;
};

template <class R>
__global__ void k_direct_mid(MidArgs a)
{
    extern __shared__ unsigned char raw[];
    Cx<R> *L = reinterpret_cast<Cx<R> *>(raw);   // input line, n2
    Cx<R> *S = L + a.n2;                          // product spectrum, N2
    const R *K = static_cast<const R *>(a.K);
    for (long long line = blockIdx.x; line < a.lines; line += gridDim.x) {
        const Cx<R> *src = static_cast<const Cx<R> *>(a.in) + line * a.n2;
        for (int z = threadIdx.x; z < a.n2; z += blockDim.x) L[z] = src[z];
        __syncthreads();
        const long long kx = line / a.rows, row = line % a.rows;
        const long long kyf = row <= a.n1 ? row : 2LL * a.n1 - row;
        const R *Kr = K + (a.three_d ? (kx * (a.n1 + 1) + kyf) * (a.n2 + 1) : kx * (a.n2 + 1));
        for (int kz = threadIdx.x; kz < a.N2; kz += blockDim.x) {
            Cx<R> acc{0, 0};
            long long m = 0;
            for (int z = 0; z < a.n2; ++z) {
                madd(acc, L[z], twid<R>(a.tw, m, false));
                m += kz;
                if (m >= a.N2) m -= a.N2;
            }
            const R kv = Kr[kz <= a.n2 ? kz : a.N2 - kz];
            S[kz] = Cx<R>{kv * acc.re, kv * acc.im};
        }
        __syncthreads();
        for (int z = threadIdx.x; z < a.n2; z += blockDim.x) {
            Cx<R> p{0, 0}, e{0, 0};
            long long m = 0;
            for (int kz = 0; kz < a.N2; ++kz) {
                const Cx<R> w = twid<R>(a.tw, m, true);
                madd(p, S[kz], w);
                if (a.ez) madd(e, times_minus_i(S[kz], (R)wavenum(kz, a.n2, a.k2s)), w);
                m += z;
                if (m >= a.N2) m -= a.N2;
            }
            static_cast<Cx<R> *>(a.phi)[line * a.n2 + z] = p;
            if (a.ez) static_cast<Cx<R> *>(a.ez)[line * a.n2 + z] = e;
        }
        __syncthreads();
    }
}

// G5: real outputs out[c][x][i] (x < n0) from half spectra in[c][kx][i]
// (kx <= n0) by the Hermitian extension F(2 n0 - k) = conj F(k):
//   f(x) = Re F(0) + Re(F(n0) (-1)^x) + 2 sum_{0<k<n0} Re(F(k) W^(k x)).
// multx[c]: F = -i kx H (E_x from the potential's spectrum).  The output is
// sign[c] f, stored, or added to the output when acc[c] (the adjoint sums).
struct C2rArgs {
    const void *in[4];
    void *out[4];
    int multx[4];
    int acc[4];
    double sign[4];
    long long I;
    int n0, N0;
    const double2 *tw;
    double k0s;
};

template <class R>
__global__ void k_direct_c2r(C2rArgs a)
{
    const long long total = (long long)a.n0 * a.I;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long i = idx % a.I, x = idx / a.I;
        for (int c = 0; c < 4; ++c) {
            if (!a.out[c]) continue;
            const Cx<R> *H = static_cast<const Cx<R> *>(a.in[c]);
            R f = 0;
            long long m = 0;
            for (int k = 0; k <= a.n0; ++k) {
                Cx<R> F = H[(long long)k * a.I + i];
                if (a.multx[c]) F = times_minus_i(F, (R)wavenum(k, a.n0, a.k0s));
                const Cx<R> w = twid<R>(a.tw, m, true);
                const R re = F.re * w.re - F.im * w.im;
                f += (k == 0 || k == a.n0) ? re : 2 * re;
                m += x;
                if (m >= a.N0) m -= a.N0;
            }
            R *o = static_cast<R *>(a.out[c]) + x * a.I + i;
            if (a.acc[c]) *o += (R)a.sign[c] * f;
            else *o = (R)a.sign[c] * f;
        }
    }
}

int grid_for(long long work, int threads)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const long long blocks = (work + threads - 1) / threads;
    return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sms * 16));
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace regions (complex elements): A, then B.
void regions(const Plan &p, long long &ea, long long &eb)
{
    const long long h0 = p.n0 + 1;
    if (p.three_d) {
        ea = h0 * p.n2 * std::max<long long>(p.n1, 4LL * p.n1);
        eb = h0 * p.n2 * 3LL * p.n1;
    } else {
        ea = h0 * p.n2;
        eb = 2 * h0 * p.n2;
    }
}

} // namespace

size_t direct_workspace_bytes(const Plan &p)
{
    long long ea, eb;
    regions(p, ea, eb);
    const size_t c = p.dtype == FSP_F64 ? sizeof(double2) : sizeof(float2);
    return align256((size_t)ea * c) + align256((size_t)eb * c);
}

namespace {

template <class R>
int launch_dft(const DftArgs &a, bool inv, cudaStream_t st)
{
    const int g = grid_for(a.O * a.K * a.I, 256);
    if (inv) k_direct_dft<R, true><<<g, 256, 0, st>>>(a);
    else k_direct_dft<R, false><<<g, 256, 0, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// The forward pipeline G1..G5 (see the file comment).  out: phi, E0, E1, E2
// (null to skip; E2 only in 3D); acc / sign: accumulate instead of store.
template <class R>
int direct_pipeline(const Plan &p, void *ws, const void *rho, void *const out[4], const int acc[4],
                    const double sign[4], cudaStream_t st)
{
    using C = Cx<R>;
    long long ea, eb;
    regions(p, ea, eb);
    C *A = static_cast<C *>(ws);
    C *B = reinterpret_cast<C *>(static_cast<char *>(ws) + align256((size_t)ea * sizeof(C)));
    const long long n0 = p.n0, n1 = p.n1, n2 = p.n2, h0 = n0 + 1;
    const bool wantZ = p.three_d ? out[3] != nullptr : out[2] != nullptr;   // the axis-2 component
    const void *K = p.dtype == FSP_F64 ? (const void *)p.K64 : (const void *)p.K;
    // G1: x, real input, kx in [0, n0]  ->  A [h0][n1][n2]
    {
        DftArgs a{};
        a.in = rho;
        a.out = A;
        a.O = 1; a.J = n0; a.K = h0; a.I = n1 * n2;
        a.in_o = 0; a.in_j = n1 * n2; a.out_o = 0; a.out_k = n1 * n2;
        a.N = 2 * p.n0; a.tw = p.dtw[0]; a.real_in = 1;
        if (launch_dft<R>(a, false, st)) return FSP_ERR_CUDA;
    }
    const C *mid_in = A;
    C *phi_s = B, *ez_s = B + h0 * n2 * (p.three_d ? 2 * n1 : 1);
    if (p.three_d) {
        // G2: y forward  A [h0][n1][n2]  ->  B [h0][2 n1][n2]
        DftArgs a{};
        a.in = A; a.out = B;
        a.O = h0; a.J = n1; a.K = 2 * n1; a.I = n2;
        a.in_o = n1 * n2; a.in_j = n2; a.out_o = 2 * n1 * n2; a.out_k = n2;
        a.N = 2 * p.n1; a.tw = p.dtw[1];
        if (launch_dft<R>(a, false, st)) return FSP_ERR_CUDA;
        mid_in = B;
        phi_s = A;
        ez_s = A + h0 * 2 * n1 * n2;
    }
    // G3: z forward, times K, inverse(s)
    {
        MidArgs m{};
        m.in = mid_in; m.phi = phi_s; m.ez = wantZ ? ez_s : nullptr;
        m.rows = p.three_d ? 2 * p.n1 : 1;
        m.lines = h0 * m.rows;
        m.n1 = p.n1; m.n2 = p.n2; m.N2 = 2 * p.n2; m.three_d = p.three_d;
        m.tw = p.dtw[2]; m.K = K; m.k2s = p.kd[2];
        const size_t smem = (size_t)(m.n2 + m.N2) * sizeof(C);
        k_direct_mid<R><<<grid_for(m.lines * 256, 256), 256, smem, st>>>(m);
        if (cudaGetLastError() != cudaSuccess) return FSP_ERR_CUDA;
    }
    const C *hphi = phi_s, *hy = nullptr, *hz = wantZ ? ez_s : nullptr;
    if (p.three_d) {
        // G4: y inverse with crop: Phi, -i ky Phi, Ez  ->  B [3][h0][n1][n2]
        const long long S1 = h0 * n1 * n2;
        DftArgs a{};
        a.O = h0; a.J = 2 * n1; a.K = n1; a.I = n2;
        a.in_o = 2 * n1 * n2; a.in_j = n2; a.out_o = n1 * n2; a.out_k = n2;
        a.N = 2 * p.n1; a.tw = p.dtw[1]; a.ks = p.kd[1];
        a.in = phi_s; a.out = B;
        if (launch_dft<R>(a, true, st)) return FSP_ERR_CUDA;
        if (out[2]) {
            a.out = B + S1; a.mult = 1;
            if (launch_dft<R>(a, true, st)) return FSP_ERR_CUDA;
            a.mult = 0;
            hy = B + S1;
        }
        if (wantZ) {
            a.in = ez_s; a.out = B + 2 * S1;
            if (launch_dft<R>(a, true, st)) return FSP_ERR_CUDA;
            hz = B + 2 * S1;
        }
        hphi = B;
    }
    // G5: real inverse along x
    C2rArgs c{};
    c.I = n1 * n2; c.n0 = p.n0; c.N0 = 2 * p.n0; c.tw = p.dtw[0]; c.k0s = p.kd[0];
    c.in[0] = hphi; c.out[0] = out[0];
    c.in[1] = hphi; c.out[1] = out[1]; c.multx[1] = 1;
    if (p.three_d) {
        c.in[2] = hy; c.out[2] = out[2];
        c.in[3] = hz; c.out[3] = out[3];
    } else {
        c.in[2] = hz; c.out[2] = out[2];
    }
    for (int i = 0; i < 4; ++i) {
        c.acc[i] = acc[i];
        c.sign[i] = sign[i];
    }
    k_direct_c2r<R><<<grid_for(n0 * c.I, 256), 256, 0, st>>>(c);
    return cudaGetLastError() == cudaSuccess ? FSP_OK : FSP_ERR_CUDA;
}

template <class R>
int direct_forward_t(const Plan &p, void *ws, const void *rho, void *phi, void *E, cudaStream_t st)
{
    const size_t c = (size_t)p.n0 * p.n1 * p.n2;
    R *e = static_cast<R *>(E);
    void *out[4] = {phi, e ? (void *)e : nullptr, e ? (void *)(e + c) : nullptr,
                    (e && p.three_d) ? (void *)(e + 2 * c) : nullptr};
    const int acc[4] = {0, 0, 0, 0};
    const double sign[4] = {1, 1, 1, 1};
    return direct_pipeline<R>(p, ws, rho, out, acc, sign, st);
}

// g_rho = A g_phi - sum_a B_a g_E[a]: A g is the potential of the solve of g,
// B_a g its a-th field component, so one pipeline per input term.
template <class R>
int direct_adjoint_t(const Plan &p, void *ws, const void *g_phi, const void *g_E, void *g_rho, cudaStream_t st)
{
    const size_t c = (size_t)p.n0 * p.n1 * p.n2;
    const int comps = p.three_d ? 3 : 2;
    bool first = true;
    if (g_phi) {
        void *out[4] = {g_rho, nullptr, nullptr, nullptr};
        const int acc[4] = {0, 0, 0, 0};
        const double sign[4] = {1, 1, 1, 1};
        int rc = direct_pipeline<R>(p, ws, g_phi, out, acc, sign, st);
        if (rc) return rc;
        first = false;
    }
    if (g_E) {
        for (int a = 0; a < comps; ++a) {
            void *out[4] = {nullptr, nullptr, nullptr, nullptr};
            int acc[4] = {0, 0, 0, 0};
            const double sign[4] = {-1, -1, -1, -1};
            out[1 + a] = g_rho;
            acc[1 + a] = first ? 0 : 1;
            int rc = direct_pipeline<R>(p, ws, static_cast<const R *>(g_E) + a * c, out, acc, sign, st);
            if (rc) return rc;
            first = false;
        }
    }
    return FSP_OK;
}

} // namespace

int run_direct_forward(const Plan &p, void *ws, const void *rho, void *phi, void *E, cudaStream_t st)
{
    return p.dtype == FSP_F64 ? direct_forward_t<double>(p, ws, rho, phi, E, st)
                              : direct_forward_t<float>(p, ws, rho, phi, E, st);
}

int run_direct_adjoint(const Plan &p, void *ws, const void *g_phi, const void *g_E, void *g_rho, cudaStream_t st)
{
    return p.dtype == FSP_F64 ? direct_adjoint_t<double>(p, ws, g_phi, g_E, g_rho, st)
                              : direct_adjoint_t<float>(p, ws, g_phi, g_E, g_rho, st);
}

} // namespace fsp
