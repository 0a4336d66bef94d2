"""The seeded input generators follow the stated recipe (CPU only).

The workloads stand in for the paper's Gaussian-charge experiments (Sec. 3) at
the measured sizes; these checks pin the grid convention, the normalisation and
each workload's parameter distribution, so that a drift in the generator shows
up here rather than as a moved benchmark figure.
"""
import math

import numpy as np

import workloads as W


def test_cell_centred_grid_symmetric_about_origin():
    x = W.axis_coords(8, 0.25)
    assert np.allclose(x, -1.0 + 0.125 + 0.25 * np.arange(8))
    assert abs(x.sum()) < 1e-15 and np.allclose(np.diff(x), 0.25)
    pts = W.grid_points((3, 4), (0.5, 0.1))
    assert pts.shape == (3, 4, 2) and np.allclose(pts[1, :, 0], 0.0) and np.allclose(pts[:, 0, 1], -0.15)


def test_gaussian_is_normalised_and_rounded_once():
    shape, h = (40, 48, 36), (0.05, 0.04, 0.06)
    g = [(np.array([0.1, -0.05, 0.0]), np.array([0.12, 0.1, 0.15]), -0.7)]
    rho64 = W.gaussian_density(shape, h, g, dtype=None)
    assert abs(rho64.sum() * np.prod(h) + 0.7) < 1e-8       # well inside the box: total charge Q
    rho32 = W.gaussian_density(shape, h, g, np.float32)
    assert rho32.dtype == np.float32 and np.array_equal(rho32, rho64.astype(np.float32))


def test_headline_mixture_recipe():
    """8 anisotropic Gaussians, centres U[-0.5,0.5]^3, sigma_a U[0.05,0.15], Q U[-1,1], seed 1, 256^3 on [-1,1]^3."""
    p = W.mixture_3d()
    assert p.shape == (256, 256, 256) and p.h == (2 / 256,) * 3 and len(p.gaussians) == 8
    for c, s, q in p.gaussians:
        assert np.all(np.abs(c) <= 0.5) and np.all((0.05 <= s) & (s <= 0.15)) and -1 <= q <= 1
        assert len(set(np.round(s, 12))) == 3                  # anisotropic
    # the draws do not depend on the grid size, and repeat for the seed
    small = W.mixture_3d(16)
    for (c1, s1, q1), (c2, s2, q2) in zip(p.gaussians, small.gaussians):
        assert np.array_equal(c1, c2) and np.array_equal(s1, s2) and q1 == q2
    other = W.mixture_3d(16, seed=2)
    assert not np.array_equal(other.gaussians[0][0], small.gaussians[0][0])


def test_2d_mixture_recipe():
    """16 isotropic Gaussians, sigma U[0.02,0.08], Q U[-1,1] redrawn until |sum Q| > 0.1, seed 2, 4096^2 on [-1,1]^2."""
    p = W.mixture_2d()
    assert p.shape == (4096, 4096) and p.h == (2 / 4096,) * 2 and len(p.gaussians) == 16
    assert abs(sum(g[2] for g in p.gaussians)) > 0.1
    for c, s, q in p.gaussians:
        assert s[0] == s[1] and 0.02 <= s[0] <= 0.08 and np.all(np.abs(c) <= 0.5) and -1 <= q <= 1


def test_beam_batch_recipe():
    probs = W.beam_batch()
    assert len(probs) == 64
    assert {p.shape for p in probs} == set(W.BEAM_SHAPES)     # every shape class occurs at seed 3
    for p in probs:
        assert all(0.005 <= hh <= 0.03 for hh in p.h)
        (c, s, q), = p.gaussians
        sides = [n * hh for n, hh in zip(p.shape, p.h)]
        base = min(sides[0], sides[1]) / 16
        assert q == 1.0 and np.array_equal(c, np.zeros(3)) and s[0] == s[1]
        assert 0.75 * base <= s[0] <= 1.25 * base
        assert s[2] <= sides[2] / 12 + 1e-15
        assert s[2] >= min(s[0], sides[2] / 12) - 1e-15


def test_training_batch_recipe():
    probs, target = W.training_batch(16, 8)
    assert len(probs) == 8 and all(len(p.gaussians) == 4 for p in probs) and target.shape == (16, 16, 16)
    assert [p.name for p in probs] == [f"mix3_16_s{s}" for s in range(10, 18)]
    assert target.dtype == np.float32 and 0 < np.abs(target).max() < 1.0
    assert math.isfinite(float(target.sum()))
