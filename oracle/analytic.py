"""Closed-form and quadrature potentials of Gaussian charges (FP64, CPU).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Conventions follow the paper's problem statement (Sec. 1): Laplacian(phi) = -rho,
E = -grad(phi), free-space Green's function 1/(4 pi r) in 3D and -ln(r)/(2 pi)
in 2D.  A Gaussian of charge Q, centre c and widths sigma_a is
    rho(x) = Q prod_a exp(-(x_a - c_a)^2 / (2 sigma_a^2)) / sqrt(2 pi sigma_a^2).

* 3D isotropic (paper Sec. 3, three-dimensional example):
      phi = Q erf(r / (sqrt(2) sigma)) / (4 pi r).
* 2D isotropic (paper Sec. 3, two-dimensional example).  The printed formula
  has Ei of a positive argument, which diverges at r = 0; the potential that
  satisfies Laplacian(phi) = -rho with phi ~ -Q ln(r)/(2 pi) far away is
      phi = -(Q / (4 pi)) [E1(r^2 / (2 sigma^2)) + ln(r^2)],  E1(x) = -Ei(-x),
  and that reading is the one used here.
* Anisotropic 3D (no elementary form): the heat-kernel representation
      1/(4 pi r) = int_0^inf (4 pi t)^(-3/2) exp(-r^2 / (4 t)) dt
  convolved with the Gaussian gives
      phi(x) = Q int_0^inf prod_a N(x_a - c_a; sigma_a^2 + 2 t) dt,
      E_a(x) = Q int_0^inf (x_a - c_a) / (sigma_a^2 + 2 t) prod_b N(...) dt,
  with N(y; v) = exp(-y^2 / (2 v)) / sqrt(2 pi v), integrated here over
  t = exp(s) with adaptive quadrature.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special


def phi_gauss3_iso(r, sigma, Q=1.0):
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-8 * sigma
    rs = np.where(small, 1.0, r)
    out[:] = Q * special.erf(rs / (math.sqrt(2.0) * sigma)) / (4.0 * math.pi * rs)
    out[small] = Q * math.sqrt(2.0 / math.pi) / (4.0 * math.pi * sigma)
    return out


def Er_gauss3_iso(r, sigma, Q=1.0):
    """Radial field E_r = -d phi / d r of the isotropic 3D Gaussian."""
    r = np.asarray(r, dtype=np.float64)
    rs = np.where(r < 1e-8 * sigma, 1.0, r)
    a = rs / (math.sqrt(2.0) * sigma)
    val = Q / (4.0 * math.pi * rs ** 2) * (special.erf(a) - 2.0 / math.sqrt(math.pi) * a * np.exp(-a * a))
    return np.where(r < 1e-8 * sigma, 0.0, val)


def phi_gauss2_iso(r, sigma, Q=1.0):
    r = np.asarray(r, dtype=np.float64)
    x = r * r / (2.0 * sigma * sigma)
    small = x < 1e-12
    xs = np.where(small, 1.0, x)
    val = -(Q / (4.0 * math.pi)) * (special.exp1(xs) + np.log(np.where(small, 1.0, r * r)))
    # r -> 0: E1(x) + ln(r^2) -> -gamma + ln(2 sigma^2)
    lim = -(Q / (4.0 * math.pi)) * (-np.euler_gamma + math.log(2.0 * sigma * sigma))
    return np.where(small, lim, val)


def Er_gauss2_iso(r, sigma, Q=1.0):
    r = np.asarray(r, dtype=np.float64)
    rs = np.where(r < 1e-12, 1.0, r)
    val = Q * (-np.expm1(-rs * rs / (2.0 * sigma * sigma))) / (2.0 * math.pi * rs)
    return np.where(r < 1e-12, 0.0, val)


def field_iso(points, centre, sigma, Q, d):
    """phi and E (shape [d, ...]) of one isotropic Gaussian at the given points [..., d]."""
    p = np.asarray(points, dtype=np.float64) - np.asarray(centre, dtype=np.float64)
    r = np.sqrt(np.sum(p * p, axis=-1))
    if d == 3:
        phi = phi_gauss3_iso(r, sigma, Q)
        Er = Er_gauss3_iso(r, sigma, Q)
    else:
        phi = phi_gauss2_iso(r, sigma, Q)
        Er = Er_gauss2_iso(r, sigma, Q)
    rs = np.where(r == 0.0, 1.0, r)
    E = np.stack([Er * p[..., a] / rs for a in range(d)], axis=0)
    return phi, E


def field_aniso3(points, centre, sigmas, Q):
    """phi and E of one anisotropic 3D Gaussian by the heat-kernel integral."""
    p = np.atleast_2d(np.asarray(points, dtype=np.float64) - np.asarray(centre, dtype=np.float64))
    s2 = np.asarray(sigmas, dtype=np.float64) ** 2

    def integrand(s):
        t = math.exp(s)
        v = s2 + 2.0 * t                                   # [3]
        dens = np.prod(np.exp(-p * p / (2.0 * v)) / np.sqrt(2.0 * math.pi * v), axis=-1)  # [P]
        out = np.empty((4, p.shape[0]))
        out[0] = dens
        out[1:] = (p / v).T * dens
        return out * t                                     # dt = t ds

    res, _ = integrate.quad_vec(integrand, -60.0, 80.0, epsabs=1e-14, epsrel=1e-12, limit=2000)
    return Q * res[0], Q * res[1:]


def mixture_field(points, gaussians, d):
    """Sum of the fields of several Gaussians: list of (centre, sigmas, Q)."""
    pts = np.asarray(points, dtype=np.float64)
    phi = np.zeros(pts.shape[:-1])
    E = np.zeros((d,) + pts.shape[:-1])
    for centre, sigmas, Q in gaussians:
        sig = np.atleast_1d(np.asarray(sigmas, dtype=np.float64))
        if np.all(sig == sig[0]):
            ph, e = field_iso(pts, centre, float(sig[0]), Q, d)
        else:
            if d != 3:
                raise NotImplementedError("anisotropic 2D Gaussians are not needed")
            ph, e = field_aniso3(pts.reshape(-1, 3), centre, sig, Q)
            ph = ph.reshape(pts.shape[:-1])
            e = e.reshape((3,) + pts.shape[:-1])
        phi += ph
        E += e
    return phi, E
