"""Seeded synthetic inputs for the free-space Poisson workloads.

This module holds input generation only (grids, Gaussian charge densities and
their parameters) and none of the solver's arithmetic; it is the one module
that both the oracle-side tests and the CUDA-side tests, benchmark and smoke
check import.  The workloads mirror the paper's experiments (Sec. 3: Gaussian
charges with closed-form potentials on a box) at the sizes the GPU path is
measured on.

Grid convention: n_a cell-centred points per axis with spacing h_a on a box
centred at the origin, x_{a,i} = -n_a h_a / 2 + (i + 1/2) h_a.  Arrays are
row-major with the last axis contiguous.  A Gaussian is (centre, sigmas, Q):
    rho(x) = Q prod_a exp(-(x_a - c_a)^2 / (2 sigma_a^2)) / sqrt(2 pi sigma_a^2).
Densities are generated in FP64 and rounded to FP32 once; the oracle is fed the
same rounded values.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def axis_coords(n: int, h: float) -> np.ndarray:
    return -0.5 * n * h + (np.arange(n, dtype=np.float64) + 0.5) * h


def grid_points(shape, h) -> np.ndarray:
    """Cell-centre coordinates, shape [*shape, d]."""
    axes = [axis_coords(n, hh) for n, hh in zip(shape, h)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack(mesh, axis=-1)


def gaussian_density(shape, h, gaussians, dtype=np.float32) -> np.ndarray:
    """Sum of Gaussians sampled at cell centres (separable per Gaussian)."""
    d = len(shape)
    rho = np.zeros(shape, dtype=np.float64)
    for centre, sigmas, Q in gaussians:
        sig = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (d,))
        factors = []
        for a in range(d):
            x = axis_coords(shape[a], h[a]) - centre[a]
            factors.append(np.exp(-x * x / (2.0 * sig[a] ** 2)) / math.sqrt(2.0 * math.pi * sig[a] ** 2))
        term = factors[0]
        for f in factors[1:]:
            term = np.multiply.outer(term, f)
        rho += Q * term
    return rho.astype(dtype) if dtype is not None else rho


def gaussian_bumps(shape, h, gaussians, dtype=np.float32) -> np.ndarray:
    """Sum of unnormalised bumps Q exp(-|x - c|^2 / (2 sigma^2)) (a smooth target field)."""
    d = len(shape)
    out = np.zeros(shape, dtype=np.float64)
    for centre, sigmas, Q in gaussians:
        sig = np.broadcast_to(np.asarray(sigmas, dtype=np.float64), (d,))
        factors = [np.exp(-(axis_coords(shape[a], h[a]) - centre[a]) ** 2 / (2.0 * sig[a] ** 2)) for a in range(d)]
        term = factors[0]
        for f in factors[1:]:
            term = np.multiply.outer(term, f)
        out += Q * term
    return out.astype(dtype) if dtype is not None else out


@dataclass
class Problem:
    """One solve: grid shape, spacings and the Gaussians that make rho."""
    name: str
    shape: tuple
    h: tuple
    gaussians: list = field(default_factory=list)

    @property
    def d(self) -> int:
        return len(self.shape)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    def rho(self, dtype=np.float32) -> np.ndarray:
        return gaussian_density(self.shape, self.h, self.gaussians, dtype)


def random_mixture(rng, count, d, centre_range=0.5, sigma_range=(0.05, 0.15), iso=False):
    gs = []
    for _ in range(count):
        c = rng.uniform(-centre_range, centre_range, size=d)
        if iso:
            s = np.full(d, rng.uniform(*sigma_range))
        else:
            s = rng.uniform(*sigma_range, size=d)
        q = rng.uniform(-1.0, 1.0)
        gs.append((c, s, q))
    return gs


def unit_gaussian_3d(n: int = 32, sigma: float = 0.15, side: float = 2.0) -> Problem:
    """Unit charge, isotropic, at the origin of the cube [-side/2, side/2]^3."""
    h = side / n
    return Problem(f"gauss3_{n}", (n, n, n), (h, h, h), [(np.zeros(3), np.full(3, sigma), 1.0)])


def unit_gaussian_2d(n: int = 64, sigma: float = 0.05, side: float = 1.0) -> Problem:
    h = side / n
    return Problem(f"gauss2_{n}", (n, n), (h, h), [(np.zeros(2), np.full(2, sigma), 1.0)])


def mixture_3d(n: int = 256, count: int = 8, seed: int = 1, side: float = 2.0) -> Problem:
    """Anisotropic 3D mixture: centres U[-0.5,0.5]^3, sigma_a U[0.05,0.15], Q U[-1,1]."""
    rng = np.random.default_rng(seed)
    h = side / n
    return Problem(f"mix3_{n}_s{seed}", (n, n, n), (h, h, h), random_mixture(rng, count, 3))


def mixture_2d(n: int = 4096, count: int = 16, seed: int = 2, side: float = 2.0) -> Problem:
    """Isotropic 2D mixture: sigma U[0.02,0.08], Q U[-1,1] redrawn until |sum Q| > 0.1."""
    rng = np.random.default_rng(seed)
    h = side / n
    while True:
        gs = random_mixture(rng, count, 2, sigma_range=(0.02, 0.08), iso=True)
        if abs(sum(g[2] for g in gs)) > 0.1:
            break
    return Problem(f"mix2_{n}_s{seed}", (n, n), (h, h), gs)


BEAM_SHAPES = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (64, 64, 256), (128, 128, 512)]


def beam_batch(count: int = 64, seed: int = 3, shapes=None, h_range=(0.005, 0.03)) -> list:
    """Independent elongated beam-bunch solves with uneven shapes and spacings.

    Shape uniform from ``shapes``; h_a U[h_range] per axis; one unit Gaussian at
    the box centre with sigma_x = sigma_y = (min xy side)/16 * U[0.75,1.25] and
    sigma_z = sigma_x * U[1,8], clipped to side_z/12.
    """
    rng = np.random.default_rng(seed)
    shapes = BEAM_SHAPES if shapes is None else shapes
    out = []
    for i in range(count):
        shape = tuple(shapes[rng.integers(len(shapes))])
        h = tuple(float(x) for x in rng.uniform(*h_range, size=3))
        sides = [n * hh for n, hh in zip(shape, h)]
        sx = min(sides[0], sides[1]) / 16.0 * rng.uniform(0.75, 1.25)
        sz = min(sx * rng.uniform(1.0, 8.0), sides[2] / 12.0)
        out.append(Problem(f"beam{i}_{shape[0]}x{shape[1]}x{shape[2]}", shape, h,
                           [(np.zeros(3), np.array([sx, sx, sz]), 1.0)]))
    return out


def training_batch(n: int = 128, batch: int = 8, seeds=range(10, 18), target_seed: int = 4, side: float = 2.0):
    """Batch of 4-Gaussian densities and a smooth target field for a loss on phi.

    rho_b: 4-Gaussian mixtures drawn like ``mixture_3d`` (seeds 10..17).
    phi_target: a sum of 8 unnormalised Gaussian bumps (seed 4) scaled to the
    magnitude of a typical potential.
    """
    h = side / n
    probs = [mixture_3d(n, 4, s, side) for s in list(seeds)[:batch]]
    rng = np.random.default_rng(target_seed)
    bumps = random_mixture(rng, 8, 3, sigma_range=(0.1, 0.3))
    target = gaussian_bumps((n, n, n), (h, h, h), bumps) * 0.05
    return probs, target
