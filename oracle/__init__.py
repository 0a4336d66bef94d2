"""FP64 CPU oracle for the HE and VGF free-space Poisson solvers.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The solver package
never imports it and it imports nothing from the solver package: the two share
no code, header, table or constant generator.  The arithmetic lives in
``fsp_oracle.c`` (plain C, double precision, its own FFT); this module only
marshals numpy arrays into it and holds the two geometry rules the method
needs (the truncation radius L and the oversampled grid M), restated here from
the paper independently of the CUDA path.

Parity status: every function here is pinned by ``tests/test_oracle.py``
against closed forms, brute force, the DFT definition and invariants.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libfsp_oracle.so")
_lib = None

HE, VGF = "he", "vgf"


def build(force: bool = False) -> str:
    """Compile fsp_oracle.c into libfsp_oracle.so with gcc (OpenMP if present)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC", _SRC]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        sig = {
            "orc_set_threads": [ctypes.c_int],
            "orc_get_threads": [],
            "orc_fft1d": [ctypes.c_int, dp, ctypes.c_int],
            "orc_dft1d_definition": [ctypes.c_int, dp, dp, ctypes.c_int],
            "orc_kernel_he": [ctypes.c_int, ip, dp, ctypes.c_double, dp],
            "orc_kernel_vgf": [ctypes.c_int, ip, dp, ctypes.c_double, ip, dp],
            "orc_kernel_vgf_fullgrid": [ctypes.c_int, ip, dp, ctypes.c_double, ip, dp],
            "orc_kernel_spectrum": [ctypes.c_int, ip, dp, dp, dp],
            "orc_solve": [ctypes.c_int, ip, dp, dp, dp, dp, dp],
            "orc_direct_phi": [ctypes.c_int, ip, dp, dp, dp, dp],
            "orc_direct_phi_at": [ctypes.c_int, ip, dp, dp, dp, ctypes.c_long, ctypes.POINTER(ctypes.c_long), dp],
            "orc_adjoint": [ctypes.c_int, ip, dp, dp, dp, dp, dp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ivec(v):
    arr = (ctypes.c_int * 3)(*(list(v) + [0] * (3 - len(v))))
    return arr


def _dvec(v):
    return (ctypes.c_double * 3)(*(list(float(x) for x in v) + [0.0] * (3 - len(v))))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_threads(t: int) -> int:
    return _load().orc_set_threads(int(t))


def threads() -> int:
    return _load().orc_get_threads()


# ----------------------------------------------------------------- FFT

def fft(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Own mixed-radix FFT (unnormalised), exp(sign 2 pi i k t / n)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(_load().orc_fft1d(a.size, _dp(a.view(np.float64)), int(sign)), "fft")
    return a


def dft_definition(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """The DFT evaluated from its definition, O(n^2)."""
    a = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(a)
    _check(_load().orc_dft1d_definition(a.size, _dp(a.view(np.float64)), _dp(out.view(np.float64)), int(sign)),
           "dft")
    return out


# ------------------------------------------------------ geometry rules

def truncation_radius(n, h, lam: float = 1.0) -> float:
    """L for VGF: the box diagonal sqrt(sum (n_a h_a)^2), times lam.

    The windowed kernel G^L equals G for r <= L (paper Sec. 2, eq:windowed), and
    must do so for every pair of grid points; the largest separation between
    two cell centres is sqrt(sum ((n_a - 1) h_a)^2), below the box diagonal.
    """
    return lam * math.sqrt(sum((na * ha) ** 2 for na, ha in zip(n, h)))


def _is_2_3_5_smooth(m: int) -> bool:
    for p in (2, 3, 5):
        while m % p == 0:
            m //= p
    return m == 1


def oversampled_size(n, h, L):
    """M per axis for the VGF precomputation.

    The paper (Sec. 2, last paragraph) oversamples by 4 (a (4N)^d grid) for its
    unit box with L just above sqrt(d).  The inverse DFT on M points of spacing h
    returns the kernel periodised with period M h; the offsets used by the 2n
    convolution reach the box side n h, so copies stay away from them when
    M h >= n h + L.  Reading adopted: M_a is the smallest even 2^a 3^b 5^c that
    is >= max(4 n_a, n_a + ceil(L / h_a) + 2), which is 4 n_a for cubes.
    """
    out = []
    for na, ha in zip(n, h):
        need = max(4 * na, na + int(math.ceil(L / ha)) + 2)
        m = need + (need % 2)
        while not _is_2_3_5_smooth(m):
            m += 2
        out.append(m)
    return out


def he_g0(d: int) -> float:
    """HE value substituted for G(0): 1 in 3D, 1/(2 pi) in 2D (paper Sec. 1 and Sec. 3)."""
    return 1.0 if d == 3 else 1.0 / (2.0 * math.pi)


def he_g0_variant(d: int, h, method: str) -> float:
    """G(0) replacement for the HE variants compared in the paper (Sec. 3).

    'he': the literal value (he_g0); 'he_nearby': G at the smallest spacing;
    'he_cellavg': the mean of G over the cell [-h/2, h/2]^d, by adaptive
    quadrature of the integrable singularity (the integral over the cell is 2^d
    times the integral over the positive corner box).
    """
    if method == "he":
        return he_g0(d)
    hmin = min(h[:d])
    if method == "he_nearby":
        return 1.0 / (4.0 * math.pi * hmin) if d == 3 else -math.log(hmin) / (2.0 * math.pi)
    if method != "he_cellavg":
        raise ValueError(method)
    from scipy import integrate
    half = [0.5 * x for x in h[:d]]
    if d == 3:
        val, _ = integrate.tplquad(lambda z, y, x: 1.0 / math.sqrt(x * x + y * y + z * z),
                                   0, half[0], 0, half[1], 0, half[2], epsabs=1e-14, epsrel=1e-12)
        return 8.0 * val / (4.0 * math.pi * h[0] * h[1] * h[2])
    val, _ = integrate.dblquad(lambda y, x: math.log(math.hypot(x, y)), 0, half[0], 0, half[1],
                               epsabs=1e-14, epsrel=1e-12)
    return -4.0 * val / (2.0 * math.pi * h[0] * h[1])


# ------------------------------------------------------------- kernels

def kernel_he(n, h, g0: float | None = None) -> np.ndarray:
    """HE real-space kernel on the wrapped padded grid, shape 2n."""
    d = len(n)
    g = np.empty([2 * a for a in n], dtype=np.float64)
    _check(_load().orc_kernel_he(d, _ivec(n), _dvec(h), float(he_g0(d) if g0 is None else g0), _dp(g)), "kernel_he")
    return g


def kernel_vgf(n, h, L: float | None = None, M=None, literal: bool = False) -> np.ndarray:
    """VGF real-space kernel on the wrapped padded grid, shape 2n.

    literal=True evaluates it the paper's way on the whole oversampled grid with
    the oracle's FFT (small grids only); the default evaluates the same inverse
    DFT as cosine sums over the non-negative octant.
    """
    d = len(n)
    if L is None:
        L = truncation_radius(n, h)
    if M is None:
        M = oversampled_size(n, h, L)
    g = np.empty([2 * a for a in n], dtype=np.float64)
    fn = _load().orc_kernel_vgf_fullgrid if literal else _load().orc_kernel_vgf
    _check(fn(d, _ivec(n), _dvec(h), float(L), _ivec(M), _dp(g)), "kernel_vgf")
    return g


def kernel(method: str, n, h, **kw) -> np.ndarray:
    if method == HE:
        return kernel_he(n, h, **kw)
    if method == VGF:
        return kernel_vgf(n, h, **kw)
    raise ValueError(method)


def kernel_spectrum(g2n: np.ndarray) -> np.ndarray:
    """DFT of the wrapped padded kernel (complex, full padded grid)."""
    g = np.ascontiguousarray(g2n, dtype=np.float64)
    n = [s // 2 for s in g.shape]
    re = np.empty_like(g)
    im = np.empty_like(g)
    _check(_load().orc_kernel_spectrum(g.ndim, _ivec(n), _dp(g), _dp(re), _dp(im)), "kernel_spectrum")
    return re + 1j * im


def scaled_spectrum_octant(g2n: np.ndarray, h) -> np.ndarray:
    """prod(h)/prod(2n) * Re DFT(g) on indices [0, n_a] per axis.

    This is the real, even multiplier the padded convolution applies in Fourier
    space with every constant factor of the HE formula folded in.
    """
    spec = kernel_spectrum(g2n)
    n = [s // 2 for s in g2n.shape]
    s = float(np.prod(h)) / float(np.prod(g2n.shape))
    sl = tuple(slice(0, a + 1) for a in n)
    return np.ascontiguousarray(spec.real[sl] * s)


# -------------------------------------------------------------- solves

def solve_with_kernel(g2n: np.ndarray, rho: np.ndarray, h, with_phi: bool = True, with_E: bool = True):
    """phi, E from the padded FFT convolution with kernel g2n (FP64)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    d = r.ndim
    n = list(r.shape)
    assert list(g2n.shape) == [2 * a for a in n]
    phi = np.empty_like(r) if with_phi else None
    E = np.empty([d] + n, dtype=np.float64) if with_E else None
    _check(_load().orc_solve(d, _ivec(n), _dvec(h), _dp(np.ascontiguousarray(g2n)), _dp(r), _dp(phi), _dp(E)),
           "solve")
    return phi, E


def solve(method: str, rho: np.ndarray, h, with_phi: bool = True, with_E: bool = True, **kw):
    g = kernel(method, list(rho.shape), h, **kw)
    return solve_with_kernel(g, rho, h, with_phi, with_E)


def direct_phi(g2n: np.ndarray, rho: np.ndarray, h) -> np.ndarray:
    """Brute-force aperiodic convolution prod(h) sum_j rho_j g_{i-j} (tiny grids)."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    out = np.empty_like(r)
    _check(_load().orc_direct_phi(r.ndim, _ivec(r.shape), _dvec(h), _dp(np.ascontiguousarray(g2n)), _dp(r),
                                  _dp(out)), "direct_phi")
    return out


def direct_phi_at(g2n: np.ndarray, rho: np.ndarray, h, flat_points) -> np.ndarray:
    """Brute-force phi at the given flat cell indices only."""
    r = np.ascontiguousarray(rho, dtype=np.float64)
    pts = np.ascontiguousarray(flat_points, dtype=np.int64)
    out = np.empty(pts.size, dtype=np.float64)
    _check(_load().orc_direct_phi_at(r.ndim, _ivec(r.shape), _dvec(h), _dp(np.ascontiguousarray(g2n)), _dp(r),
                                     pts.size, pts.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _dp(out)),
           "direct_phi_at")
    return out


def adjoint_with_kernel(g2n: np.ndarray, g_phi, g_E, h) -> np.ndarray:
    """Adjoint of rho -> (phi, E): g_rho = A g_phi - sum_a B_a g_E[a]."""
    ref = g_phi if g_phi is not None else g_E[0]
    d = ref.ndim
    n = list(ref.shape)
    gp = None if g_phi is None else np.ascontiguousarray(g_phi, dtype=np.float64)
    ge = None if g_E is None else np.ascontiguousarray(g_E, dtype=np.float64)
    out = np.empty(n, dtype=np.float64)
    _check(_load().orc_adjoint(d, _ivec(n), _dvec(h), _dp(np.ascontiguousarray(g2n)), _dp(gp), _dp(ge), _dp(out)),
           "adjoint")
    return out


def fd_gradient(phi: np.ndarray, h) -> np.ndarray:
    """E = -grad(phi) by centred differences, second-order one-sided at the faces.

    The finite-difference field the paper sets beside Fourier differentiation
    for HE (Sec. 3): (phi[i+1] - phi[i-1]) / (2h) inside; at i = 0 the
    difference (-3 phi0 + 4 phi1 - phi2) / (2h) and its mirror at i = n - 1.
    """
    p = np.asarray(phi, dtype=np.float64)
    out = np.empty((p.ndim,) + p.shape)
    for a in range(p.ndim):
        q = np.moveaxis(p, a, 0)
        d = np.empty_like(q)
        d[1:-1] = (q[2:] - q[:-2]) / (2 * h[a])
        d[0] = (-3 * q[0] + 4 * q[1] - q[2]) / (2 * h[a])
        d[-1] = (3 * q[-1] - 4 * q[-2] + q[-3]) / (2 * h[a])
        out[a] = -np.moveaxis(d, 0, a)
    return out
