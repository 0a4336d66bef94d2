/*
 * fsp_oracle.c -- plain FP64 CPU oracle for the free-space Poisson solvers of
 * Hockney-Eastwood (HE) and Vico-Greengard-Ferrando (VGF).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the solver package links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA path.  Everything is double precision and written for reading, not for
 * speed: a recursive mixed-radix FFT with a naive DFT for prime lengths,
 * explicit sums for the kernels, explicit loops for the convolution.
 *
 * Problem (paper Sec. 1, Eq. "eq:Poisson" and "eq:convolution"):
 *     Laplacian(phi) = -rho,  phi = rho * G,  E = -grad(phi),
 *     G(r) = 1/(4 pi r) in 3D,  G(r) = -ln(r)/(2 pi) in 2D.
 *
 * Grid: n[a] cell-centred points per axis with spacing h[a].  Arrays are
 * row-major [n0][n1][n2] (3D) or [n0][n1] (2D), the last axis contiguous.
 * The padded grid has 2 n[a] points per axis; a kernel array "g2n" holds the
 * real-space Green's function on it at offsets j[a] in [-n[a], n[a]), stored
 * wrapped (offset j lives at index j mod 2n[a]).
 *
 * Discrete method shared by HE and VGF (paper Sec. 1, the HE formula; Sec. 2,
 * last paragraph: "the only difference ... is the Green's function"):
 *     phi = prod(h) * IDFT_2n( DFT_2n(rho padded) * DFT_2n(g) ) cropped,
 *     E_a = prod(h) * IDFT_2n( -i k_a DFT_2n(rho padded) DFT_2n(g) ) cropped,
 * IDFT including 1/prod(2n), k_a = 2 pi m / (2 n_a h_a), m in [-n_a, n_a),
 * the unpaired Nyquist index m = -n_a given k_a = 0 (Fourier differentiation,
 * paper Sec. 3, two-dimensional example).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_NOMEM 4

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------ threads */

int orc_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
    return omp_get_max_threads();
#else
    (void)t;
    return 1;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- FFT */

/* exp(sign * 2 pi i e / n), with e reduced modulo n first. */
static cplx unit_root(long long e, long long n, int sign)
{
    e %= n;
    if (e < 0) e += n;
    double ang = TWO_PI * (double)e / (double)n;
    return cos(ang) + (double)sign * sin(ang) * I;
}

/* Definition of the DFT:  y[k] = sum_t x[t*stride] exp(sign 2 pi i k t / n). */
static void dft_definition(int n, const cplx *x, long stride, cplx *y, int sign)
{
    for (int k = 0; k < n; ++k) {
        cplx acc = 0.0;
        for (int t = 0; t < n; ++t) acc += x[(long)t * stride] * unit_root((long long)k * t, n, sign);
        y[k] = acc;
    }
}

static int smallest_factor(int n)
{
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

/*
 * Recursive mixed-radix decimation in time.  With n = p m and the p
 * interleaved subsequences x_q[t] = x[q + p t] (q < p, t < m):
 *     X[k + m s] = sum_q  W^{q (k + m s)}  X_q[k],   W = exp(sign 2 pi i / n).
 * "root" is a table of exp(sign 2 pi i e / N) for the top-level length N and
 * "scale" = N / n maps this level's exponents into it.  "work" must hold 2n
 * values: the p sub-transforms go to work[0..n), deeper levels use work + n.
 * Prime lengths fall back to the definition.
 */
static void fft_rec(int n, const cplx *x, long stride, cplx *y, int sign, const cplx *root, long scale,
                    long ntop, cplx *work)
{
    if (n == 1) {
        y[0] = x[0];
        return;
    }
    int p = smallest_factor(n);
    if (p == n) {
        dft_definition(n, x, stride, y, sign);
        return;
    }
    int m = n / p;
    for (int q = 0; q < p; ++q) fft_rec(m, x + q * stride, stride * p, work + (long)q * m, sign, root, scale * p, ntop, work + n);
    for (int s = 0; s < p; ++s) {
        for (int k = 0; k < m; ++k) {
            long kk = k + (long)m * s;
            cplx acc = 0.0;
            for (int q = 0; q < p; ++q) acc += work[(long)q * m + k] * root[((long)q * kk % n) * scale % ntop];
            y[kk] = acc;
        }
    }
}

static cplx *root_table(int n, int sign)
{
    cplx *root = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!root) return NULL;
    for (int e = 0; e < n; ++e) root[e] = unit_root(e, n, sign);
    return root;
}

/* In-place 1D FFT of n complex values (interleaved re, im), unnormalised. */
int orc_fft1d(int n, double *re_im, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return ORC_ERR_ARG;
    cplx *root = root_table(n, sign);
    cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n * 3);
    if (!root || !buf) {
        free(root);
        free(buf);
        return ORC_ERR_NOMEM;
    }
    cplx *in = (cplx *)re_im;
    memcpy(buf, in, sizeof(cplx) * (size_t)n);
    fft_rec(n, buf, 1, in, sign, root, 1, n, buf + n);
    free(root);
    free(buf);
    return ORC_OK;
}

/* The DFT by its definition, for checking the FFT. */
int orc_dft1d_definition(int n, const double *in_re_im, double *out_re_im, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1)) return ORC_ERR_ARG;
    dft_definition(n, (const cplx *)in_re_im, 1, (cplx *)out_re_im, sign);
    return ORC_OK;
}

/*
 * Transform a d-dimensional complex array (row-major, shape dims[0..d)) along
 * one axis, line by line (the multi-dimensional DFT is the product of the 1D
 * ones along each axis).
 */
static int fft_axis(cplx *a, int d, const int *dims, int axis, int sign)
{
    long stride = 1;
    for (int b = axis + 1; b < d; ++b) stride *= dims[b];
    long outer = 1;
    for (int b = 0; b < axis; ++b) outer *= dims[b];
    int n = dims[axis];
    long lines = outer * stride;
    cplx *root = root_table(n, sign);
    if (!root) return ORC_ERR_NOMEM;
    int fail = 0;
#pragma omp parallel
    {
        cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)n * 4);
        if (!buf) {
#pragma omp atomic write
            fail = 1;
        } else {
#pragma omp for schedule(static)
            for (long line = 0; line < lines; ++line) {
                long o = line / stride, i = line % stride;
                cplx *base = a + o * stride * n + i;
                for (int t = 0; t < n; ++t) buf[t] = base[(long)t * stride];
                fft_rec(n, buf, 1, buf + n, sign, root, 1, n, buf + 2 * n);
                for (int t = 0; t < n; ++t) base[(long)t * stride] = buf[n + t];
            }
            free(buf);
        }
    }
    free(root);
    return fail ? ORC_ERR_NOMEM : ORC_OK;
}

static int fft_nd(cplx *a, int d, const int *dims, int sign)
{
    for (int axis = 0; axis < d; ++axis) {
        int rc = fft_axis(a, d, dims, axis, sign);
        if (rc) return rc;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ helpers */

static int check_dims(int d, const int *n)
{
    if (d != 2 && d != 3) return 0;
    for (int a = 0; a < d; ++a)
        if (n[a] < 1) return 0;
    return 1;
}

static long count(int d, const int *dims)
{
    long c = 1;
    for (int a = 0; a < d; ++a) c *= dims[a];
    return c;
}

/* Signed offset of wrapped index i on a periodic axis of length 2n: [-n, n). */
static int wrapped_offset(int i, int n)
{
    return i < n ? i : i - 2 * n;
}

/* ------------------------------------------------------- Green's functions */

/* Free-space Green's function of eq:convolution. */
static double green(int d, double r)
{
    if (d == 3) return 1.0 / (4.0 * M_PI * r);
    return -log(r) / (2.0 * M_PI);
}

/*
 * HE kernel (paper Sec. 1): the Green's function sampled at the grid offsets
 * of the padded domain, with the singular value at r = 0 replaced by g0.
 */
int orc_kernel_he(int d, const int *n, const double *h, double g0, double *g2n)
{
    if (!check_dims(d, n) || !h || !g2n) return ORC_ERR_ARG;
    int dims[3];
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    long total = count(d, dims);
    for (long idx = 0; idx < total; ++idx) {
        long rem = idx;
        double r2 = 0.0;
        for (int a = d - 1; a >= 0; --a) {
            int i = (int)(rem % dims[a]);
            rem /= dims[a];
            double x = wrapped_offset(i, n[a]) * h[a];
            r2 += x * x;
        }
        g2n[idx] = (r2 == 0.0) ? g0 : green(d, sqrt(r2));
    }
    return ORC_OK;
}

/*
 * Fourier transform of the truncated kernel G^L (paper Eq. GLFourier2D and
 * GLFourier3D), with its finite value at k = 0:
 *   3D:  2 (sin(L k / 2) / k)^2,                k -> 0:  L^2 / 2
 *   2D:  (1 - J0(L k)) / k^2 - L ln(L) J1(L k) / k,
 *                                               k -> 0:  (L^2/4)(1 - 2 ln L)
 * For L k below 1e-3 the 2D form is evaluated from its Taylor series to avoid
 * the cancellation in 1 - J0.
 */
static double truncated_green_hat(int d, double L, double k)
{
    if (d == 3) {
        if (k == 0.0) return 0.5 * L * L;
        double s = sin(0.5 * L * k) / k;
        return 2.0 * s * s;
    }
    double x = L * k;
    if (x < 1e-3) {
        double x2 = x * x;
        double one_minus_j0_over_k2 = L * L * (0.25 - x2 / 64.0);
        double j1_over_k = L * (0.5 - x2 / 16.0);
        return one_minus_j0_over_k2 - L * log(L) * j1_over_k;
    }
    return (1.0 - j0(x)) / (k * k) - L * log(L) * j1(x) / k;
}

/*
 * VGF kernel (paper Sec. 2, last paragraph): the inverse DFT, on an oversampled
 * grid of M[a] points per axis with spacing h[a], of the samples of F{G^L} at
 * k_a = 2 pi m_a / (M_a h_a), m_a in [-M_a/2, M_a/2), restricted to the offsets
 * j in [-n, n) of the padded grid:
 *     g_j = (1 / prod_a(M_a h_a)) sum_m F{G^L}(k_m) exp(i k_m . j h).
 * F{G^L} depends only on |k|, so it is even in every component; pairing m_a
 * with -m_a turns each axis sum into a cosine sum over m_a in [0, M_a/2] with
 * weight 1 at m_a = 0 and at the unpaired m_a = M_a/2 and weight 2 otherwise.
 * The sum is evaluated one axis at a time (the multi-dimensional inverse DFT
 * is the product of 1D ones), on the non-negative offsets j_a in [0, n_a]; g
 * is even, so the wrapped 2n grid is filled by reflection (the offset -n_a
 * takes the value at +n_a).  M[a] must be even.
 */
static double *cos_table(int n, int M)
{
    /* C[j][m] = w(m) cos(2 pi m j / M), j in [0, n], m in [0, M/2] */
    int mh = M / 2 + 1;
    double *c = (double *)malloc(sizeof(double) * (size_t)(n + 1) * mh);
    if (!c) return NULL;
    for (int j = 0; j <= n; ++j)
        for (int m = 0; m < mh; ++m) {
            double w = (m == 0 || 2 * m == M) ? 1.0 : 2.0;
            c[(long)j * mh + m] = w * creal(unit_root((long long)m * j, M, 1));
        }
    return c;
}

int orc_kernel_vgf(int d, const int *n, const double *h, double L, const int *M, double *g2n)
{
    if (!check_dims(d, n) || !h || !M || !g2n || !(L > 0.0)) return ORC_ERR_ARG;
    for (int a = 0; a < d; ++a)
        if (M[a] < 2 || M[a] % 2) return ORC_ERR_ARG;
    int mh[3] = {1, 1, 1}, nh[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) {
        mh[a] = M[a] / 2 + 1;
        nh[a] = n[a] + 1;
    }
    double *C[3] = {NULL, NULL, NULL};
    for (int a = 0; a < d; ++a) C[a] = cos_table(n[a], M[a]);
    double norm = 1.0;
    for (int a = 0; a < d; ++a) norm *= M[a] * h[a];
    double *oct = NULL; /* g on the non-negative offsets, shape nh */
    int rc = ORC_OK;
    for (int a = 0; a < d; ++a)
        if (!C[a]) rc = ORC_ERR_NOMEM;

    if (rc == ORC_OK && d == 3) {
        /* A[mx][my][jz] = sum_mz C_z[jz][mz] Ghat(mx, my, mz) */
        double *A = (double *)malloc(sizeof(double) * (size_t)mh[0] * mh[1] * nh[2]);
        double *B = (double *)malloc(sizeof(double) * (size_t)mh[0] * nh[1] * nh[2]);
        oct = (double *)malloc(sizeof(double) * (size_t)nh[0] * nh[1] * nh[2]);
        if (!A || !B || !oct) rc = ORC_ERR_NOMEM;
        if (rc == ORC_OK) {
#pragma omp parallel
            {
                double *row = (double *)malloc(sizeof(double) * (size_t)mh[2]);
#pragma omp for schedule(static)
                for (long p = 0; p < (long)mh[0] * mh[1]; ++p) {
                    int mx = (int)(p / mh[1]), my = (int)(p % mh[1]);
                    double kx = TWO_PI * mx / (M[0] * h[0]), ky = TWO_PI * my / (M[1] * h[1]);
                    for (int mz = 0; mz < mh[2]; ++mz) {
                        double kz = TWO_PI * mz / (M[2] * h[2]);
                        row[mz] = truncated_green_hat(3, L, sqrt(kx * kx + ky * ky + kz * kz));
                    }
                    for (int jz = 0; jz < nh[2]; ++jz) {
                        double s = 0.0;
                        for (int mz = 0; mz < mh[2]; ++mz) s += C[2][(long)jz * mh[2] + mz] * row[mz];
                        A[p * nh[2] + jz] = s;
                    }
                }
                free(row);
            }
            /* B[mx][jy][jz] = sum_my C_y[jy][my] A[mx][my][jz] */
#pragma omp parallel for schedule(static)
            for (long p = 0; p < (long)mh[0] * nh[1]; ++p) {
                int mx = (int)(p / nh[1]), jy = (int)(p % nh[1]);
                for (int jz = 0; jz < nh[2]; ++jz) {
                    double s = 0.0;
                    for (int my = 0; my < mh[1]; ++my)
                        s += C[1][(long)jy * mh[1] + my] * A[((long)mx * mh[1] + my) * nh[2] + jz];
                    B[p * nh[2] + jz] = s;
                }
            }
            /* oct[jx][jy][jz] = sum_mx C_x[jx][mx] B[mx][jy][jz] / prod(M h) */
#pragma omp parallel for schedule(static)
            for (long p = 0; p < (long)nh[0] * nh[1]; ++p) {
                int jx = (int)(p / nh[1]), jy = (int)(p % nh[1]);
                for (int jz = 0; jz < nh[2]; ++jz) {
                    double s = 0.0;
                    for (int mx = 0; mx < mh[0]; ++mx)
                        s += C[0][(long)jx * mh[0] + mx] * B[((long)mx * nh[1] + jy) * nh[2] + jz];
                    oct[p * nh[2] + jz] = s / norm;
                }
            }
        }
        free(A);
        free(B);
    } else if (rc == ORC_OK) {
        /* A[mx][jy] = sum_my C_y[jy][my] Ghat(mx, my);  oct = C_x A / prod(M h) */
        double *A = (double *)malloc(sizeof(double) * (size_t)mh[0] * nh[1]);
        oct = (double *)malloc(sizeof(double) * (size_t)nh[0] * nh[1]);
        if (!A || !oct) rc = ORC_ERR_NOMEM;
        if (rc == ORC_OK) {
#pragma omp parallel
            {
                double *row = (double *)malloc(sizeof(double) * (size_t)mh[1]);
#pragma omp for schedule(static)
                for (int mx = 0; mx < mh[0]; ++mx) {
                    double kx = TWO_PI * mx / (M[0] * h[0]);
                    for (int my = 0; my < mh[1]; ++my) {
                        double ky = TWO_PI * my / (M[1] * h[1]);
                        row[my] = truncated_green_hat(2, L, sqrt(kx * kx + ky * ky));
                    }
                    for (int jy = 0; jy < nh[1]; ++jy) {
                        double s = 0.0;
                        for (int my = 0; my < mh[1]; ++my) s += C[1][(long)jy * mh[1] + my] * row[my];
                        A[(long)mx * nh[1] + jy] = s;
                    }
                }
                free(row);
            }
#pragma omp parallel for schedule(static)
            for (int jx = 0; jx < nh[0]; ++jx)
                for (int jy = 0; jy < nh[1]; ++jy) {
                    double s = 0.0;
                    for (int mx = 0; mx < mh[0]; ++mx) s += C[0][(long)jx * mh[0] + mx] * A[(long)mx * nh[1] + jy];
                    oct[(long)jx * nh[1] + jy] = s / norm;
                }
        }
        free(A);
    }
    if (rc == ORC_OK) {
        /* reflect the non-negative offsets onto the wrapped padded grid */
        int dims[3] = {1, 1, 1};
        for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
        long total = count(d, dims);
        for (long idx = 0; idx < total; ++idx) {
            long rem = idx, o = 0, mul = 1;
            for (int a = d - 1; a >= 0; --a) {
                int i = (int)(rem % dims[a]);
                rem /= dims[a];
                o += (long)abs(wrapped_offset(i, n[a])) * mul;
                mul *= nh[a];
            }
            g2n[idx] = oct[o];
        }
    }
    free(oct);
    for (int a = 0; a < d; ++a) free(C[a]);
    return rc;
}

/*
 * The same VGF kernel taken literally as the paper states it: fill the whole
 * oversampled grid with F{G^L}(k_m) (complex array, natural FFT order), take
 * its inverse FFT, divide by prod(M h), and keep the offsets [-n, n).  Costs
 * prod(M) complex values: small grids only.  Used to check orc_kernel_vgf.
 */
int orc_kernel_vgf_fullgrid(int d, const int *n, const double *h, double L, const int *M, double *g2n)
{
    if (!check_dims(d, n) || !h || !M || !g2n || !(L > 0.0)) return ORC_ERR_ARG;
    for (int a = 0; a < d; ++a)
        if (M[a] < 2 * n[a] || M[a] % 2) return ORC_ERR_ARG;
    long total = count(d, M);
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)total);
    if (!a) return ORC_ERR_NOMEM;
    for (long idx = 0; idx < total; ++idx) {
        long rem = idx;
        double k2 = 0.0;
        for (int b = d - 1; b >= 0; --b) {
            int i = (int)(rem % M[b]);
            rem /= M[b];
            int m = i < M[b] / 2 ? i : i - M[b]; /* [-M/2, M/2) */
            double k = TWO_PI * m / (M[b] * h[b]);
            k2 += k * k;
        }
        a[idx] = truncated_green_hat(d, L, sqrt(k2));
    }
    int rc = fft_nd(a, d, M, +1);
    if (rc == ORC_OK) {
        double norm = 1.0;
        for (int b = 0; b < d; ++b) norm *= M[b] * h[b];
        int dims[3] = {1, 1, 1};
        for (int b = 0; b < d; ++b) dims[b] = 2 * n[b];
        long out = count(d, dims);
        for (long idx = 0; idx < out; ++idx) {
            long rem = idx, src = 0, mul = 1;
            for (int b = d - 1; b >= 0; --b) {
                int i = (int)(rem % dims[b]);
                rem /= dims[b];
                int j = wrapped_offset(i, n[b]);
                int im = j >= 0 ? j : j + M[b];
                src += (long)im * mul;
                mul *= M[b];
            }
            g2n[idx] = creal(a[src]) / norm;
        }
    }
    free(a);
    return rc;
}

/* DFT_2n of a real kernel on the padded grid: re and im of the full spectrum. */
int orc_kernel_spectrum(int d, const int *n, const double *g2n, double *re, double *im)
{
    if (!check_dims(d, n) || !g2n || !re || !im) return ORC_ERR_ARG;
    int dims[3];
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    long total = count(d, dims);
    cplx *a = (cplx *)malloc(sizeof(cplx) * (size_t)total);
    if (!a) return ORC_ERR_NOMEM;
    for (long i = 0; i < total; ++i) a[i] = g2n[i];
    int rc = fft_nd(a, d, dims, -1);
    for (long i = 0; rc == ORC_OK && i < total; ++i) {
        re[i] = creal(a[i]);
        im[i] = cimag(a[i]);
    }
    free(a);
    return rc;
}

/* ---------------------------------------------------------------- solves */

/* Wavenumber of index i on the padded axis: 2 pi m / (2 n h), Nyquist -> 0. */
static double wavenumber(int i, int n, double h)
{
    int m = wrapped_offset(i, n);
    if (m == -n) return 0.0;
    return TWO_PI * m / (2.0 * n * h);
}

/* Zero-pad a real [n] array into a complex [2n] array. */
static void pad_into(int d, const int *n, const double *src, cplx *dst)
{
    int dims[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    memset(dst, 0, sizeof(cplx) * (size_t)count(d, dims));
    long total = count(d, n);
    for (long idx = 0; idx < total; ++idx) {
        long rem = idx, o = 0, mul = 1;
        for (int a = d - 1; a >= 0; --a) {
            int i = (int)(rem % n[a]);
            rem /= n[a];
            o += (long)i * mul;
            mul *= dims[a];
        }
        dst[o] = src[idx];
    }
}

/* Real part of the [0, n) corner of a complex [2n] array, times s. */
static void crop_from(int d, const int *n, const cplx *src, double s, double *dst)
{
    int dims[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    long total = count(d, n);
    for (long idx = 0; idx < total; ++idx) {
        long rem = idx, o = 0, mul = 1;
        for (int a = d - 1; a >= 0; --a) {
            int i = (int)(rem % n[a]);
            rem /= n[a];
            o += (long)i * mul;
            mul *= dims[a];
        }
        dst[idx] = creal(src[o]) * s;
    }
}

/* Multi-index of a flat index on the padded grid. */
static void unflatten(int d, const int *dims, long idx, int *out)
{
    for (int a = d - 1; a >= 0; --a) {
        out[a] = (int)(idx % dims[a]);
        idx /= dims[a];
    }
}

/*
 * phi and E by the padded FFT convolution stated at the top of this file.
 * phi: [n] or NULL; E: [d][n] or NULL.
 */
int orc_solve(int d, const int *n, const double *h, const double *g2n, const double *rho, double *phi, double *E)
{
    if (!check_dims(d, n) || !h || !g2n || !rho || (!phi && !E)) return ORC_ERR_ARG;
    int dims[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    long total = count(d, dims);
    long cells = count(d, n);
    cplx *rho_hat = (cplx *)malloc(sizeof(cplx) * (size_t)total);
    cplx *g_hat = (cplx *)malloc(sizeof(cplx) * (size_t)total);
    cplx *work = (cplx *)malloc(sizeof(cplx) * (size_t)total);
    int rc = (rho_hat && g_hat && work) ? ORC_OK : ORC_ERR_NOMEM;
    if (rc == ORC_OK) {
        pad_into(d, n, rho, rho_hat);
        rc = fft_nd(rho_hat, d, dims, -1);
    }
    if (rc == ORC_OK) {
        for (long i = 0; i < total; ++i) g_hat[i] = g2n[i];
        rc = fft_nd(g_hat, d, dims, -1);
    }
    double hprod = 1.0;
    for (int a = 0; a < d; ++a) hprod *= h[a];
    double s = hprod / (double)total; /* prod(h) and the 1/prod(2n) of the IDFT */
    for (int out = -1; rc == ORC_OK && out < d; ++out) {
        if (out < 0 && !phi) continue;
        if (out >= 0 && !E) break;
        for (long i = 0; i < total; ++i) {
            cplx v = rho_hat[i] * g_hat[i];
            if (out >= 0) {
                int mi[3];
                unflatten(d, dims, i, mi);
                v *= -I * wavenumber(mi[out], n[out], h[out]);
            }
            work[i] = v;
        }
        rc = fft_nd(work, d, dims, +1);
        if (rc == ORC_OK) crop_from(d, n, work, s, out < 0 ? phi : E + (long)out * cells);
    }
    free(rho_hat);
    free(g_hat);
    free(work);
    return rc;
}

/*
 * Brute-force discrete convolution: phi_i = prod(h) sum_j rho_j g_{i-j}, the
 * aperiodic convolution the padded FFT computes exactly.  O(cells^2).
 */
int orc_direct_phi(int d, const int *n, const double *h, const double *g2n, const double *rho, double *phi)
{
    if (!check_dims(d, n) || !h || !g2n || !rho || !phi) return ORC_ERR_ARG;
    int dims[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    double hprod = 1.0;
    for (int a = 0; a < d; ++a) hprod *= h[a];
    long cells = count(d, n);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < cells; ++i) {
        int ii[3];
        unflatten(d, n, i, ii);
        double s = 0.0;
        for (long j = 0; j < cells; ++j) {
            int jj[3];
            unflatten(d, n, j, jj);
            long o = 0;
            for (int a = 0; a < d; ++a) {
                int off = ii[a] - jj[a];
                if (off < 0) off += dims[a];
                o = o * dims[a] + off;
            }
            s += rho[j] * g2n[o];
        }
        phi[i] = hprod * s;
    }
    return ORC_OK;
}

/*
 * The same brute-force sum evaluated only at the listed cells (flat indices),
 * for checking large grids at sampled points: O(cells) per point.
 */
int orc_direct_phi_at(int d, const int *n, const double *h, const double *g2n, const double *rho, long npoints,
                      const long *points, double *phi)
{
    if (!check_dims(d, n) || !h || !g2n || !rho || !points || !phi || npoints < 0) return ORC_ERR_ARG;
    int dims[3] = {1, 1, 1};
    for (int a = 0; a < d; ++a) dims[a] = 2 * n[a];
    double hprod = 1.0;
    for (int a = 0; a < d; ++a) hprod *= h[a];
    long cells = count(d, n);
#pragma omp parallel for schedule(dynamic)
    for (long p = 0; p < npoints; ++p) {
        int ii[3];
        unflatten(d, n, points[p], ii);
        double s = 0.0;
        for (long j = 0; j < cells; ++j) {
            if (rho[j] == 0.0) continue;
            int jj[3];
            unflatten(d, n, j, jj);
            long o = 0;
            for (int a = 0; a < d; ++a) {
                int off = ii[a] - jj[a];
                if (off < 0) off += dims[a];
                o = o * dims[a] + off;
            }
            s += rho[j] * g2n[o];
        }
        phi[p] = hprod * s;
    }
    return ORC_OK;
}

/*
 * Adjoint of the solve map rho -> (phi, E):  g_rho = A^T g_phi + sum_a B_a^T g_E[a],
 * with A the phi map and B_a the E_a map.  g is even, so A is symmetric; the
 * Fourier derivative kernel -i k_a g_hat is odd (the Nyquist index carries
 * k = 0), so B_a^T = -B_a.  Hence g_rho = A g_phi - sum_a B_a g_E[a], each
 * term being one forward solve.  g_phi or g_E may be NULL (taken as zero).
 */
int orc_adjoint(int d, const int *n, const double *h, const double *g2n, const double *g_phi, const double *g_E,
                double *g_rho)
{
    if (!check_dims(d, n) || !h || !g2n || !g_rho || (!g_phi && !g_E)) return ORC_ERR_ARG;
    long cells = count(d, n);
    double *tmp_phi = (double *)malloc(sizeof(double) * (size_t)cells);
    double *tmp_E = (double *)malloc(sizeof(double) * (size_t)cells * d);
    int rc = (tmp_phi && tmp_E) ? ORC_OK : ORC_ERR_NOMEM;
    for (long i = 0; i < cells; ++i) g_rho[i] = 0.0;
    if (rc == ORC_OK && g_phi) {
        rc = orc_solve(d, n, h, g2n, g_phi, tmp_phi, NULL);
        for (long i = 0; rc == ORC_OK && i < cells; ++i) g_rho[i] += tmp_phi[i];
    }
    for (int a = 0; rc == ORC_OK && g_E && a < d; ++a) {
        rc = orc_solve(d, n, h, g2n, g_E + (long)a * cells, NULL, tmp_E);
        for (long i = 0; rc == ORC_OK && i < cells; ++i) g_rho[i] -= tmp_E[(long)a * cells + i];
    }
    free(tmp_phi);
    free(tmp_E);
    return rc;
}
