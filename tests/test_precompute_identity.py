"""The closed form behind the GPU's once-per-geometry VGF axis matrix (CPU only).

Sec. 2 builds the VGF kernel by an inverse DFT on the oversampled grid restricted
to the 2N grid, followed by DFT_2N; per axis the two cosine sums fold into
    P[k][m] = w_m sum_{j=0}^{n} c_j cos(pi k j / n) cos(2 pi m j / M)
(c = 1 at j = 0, n, else 2; w = 1 at m = 0, M/2, else 2).  The device evaluates
each entry as (w_m / 2) [T(k M + 2 m n) + T(k M - 2 m n)], with
T(r) = sum_{j=-n}^{n-1} cos(pi r j / (n M)) = sin(pi r / M) cot(pi r / (2 n M)),
T = 2n where r is a multiple of 2 n M, and every sine argument reduced exactly in
integers.  This test checks that identity, written the way the kernel takes it,
against the (n+1)-term sum summed with math.fsum, on full ranges at small n and
on sampled entries (including the ones next to the singular angles) at the
largest padded lengths.
"""
import math

import numpy as np
import pytest


def _sinpi_ratio(a, b):
    r = a % (2 * b)
    sgn = 1.0
    if r >= b:
        r -= b
        sgn = -1.0
    if 2 * r > b:
        r = b - r
    return sgn * math.sin(math.pi * (r / b))


def _cos_sum_sym(r, n, M):
    D = n * M
    if r % (2 * D) == 0:
        return 2.0 * n
    return _sinpi_ratio(r, M) * _sinpi_ratio(D - r, 2 * D) / _sinpi_ratio(r, 2 * D)


def _entry_closed(k, m, n, M):
    w = 1.0 if (m == 0 or 2 * m == M) else 2.0
    return w * 0.5 * (_cos_sum_sym(k * M + 2 * m * n, n, M) + _cos_sum_sym(k * M - 2 * m * n, n, M))


def _entry_sum(k, m, n, M):
    j = np.arange(n + 1)
    c = np.where((j == 0) | (j == n), 1.0, 2.0)
    a = np.cos(np.pi * ((k * j) % (2 * n)) / n)
    b = np.cos(np.pi * ((2 * m * j) % (2 * M)) / M)
    w = 1.0 if (m == 0 or 2 * m == M) else 2.0
    return w * math.fsum(c * a * b)


@pytest.mark.parametrize("n,M", [(1, 4), (2, 8), (3, 12), (16, 64), (5, 30), (32, 130)])
def test_closed_form_every_entry(n, M):
    worst = max(abs(_entry_closed(k, m, n, M) - _entry_sum(k, m, n, M))
                for k in range(n + 1) for m in range(M // 2 + 1))
    assert worst <= 1e-14 * 2 * n


@pytest.mark.parametrize("n,M", [(128, 512), (256, 1024), (2048, 8192), (4096, 16384), (50, 250)])
def test_closed_form_sampled_and_near_singular(n, M):
    rng = np.random.default_rng(n + M)
    ks = [0, n, n // 2] + [int(x) for x in rng.integers(0, n + 1, 12)]
    ms = [0, M // 2, M // 4] + [int(x) for x in rng.integers(0, M // 2 + 1, 12)]
    pairs = [(k, m) for k in ks for m in ms]
    for k in ks:                       # k M close to 2 m n: the angle near a multiple of 2 pi
        m0 = (k * M) // (2 * n)
        pairs += [(k, mm) for mm in (m0 - 1, m0, m0 + 1) if 0 <= mm <= M // 2]
    worst = max(abs(_entry_closed(k, m, n, M) - _entry_sum(k, m, n, M)) for k, m in pairs)
    assert worst <= 1e-14 * 2 * n


def test_the_unpaired_offset_is_counted_once():
    """Dropping the weight rule (c_n = 2 instead of 1) changes the sum: the symmetric range is [-n, n), not [-n, n]."""
    n, M, k, m = 8, 32, 3, 4     # the term at j = n is cos(3 pi) cos(2 pi) = -1
    j = np.arange(n + 1)
    c_wrong = np.where(j == 0, 1.0, 2.0)
    wrong = 2.0 * math.fsum(c_wrong * np.cos(np.pi * k * j / n) * np.cos(2 * np.pi * m * j / M))
    assert abs(_entry_closed(k, m, n, M) - _entry_sum(k, m, n, M)) < 1e-13
    assert abs(wrong - _entry_sum(k, m, n, M)) > 1e-3
