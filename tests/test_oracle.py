"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper and the mathematics fix:
the DFT definition and numpy's FFT (a library routine), brute-force direct
summation of the discrete aperiodic convolution, the closed-form potentials of
Gaussian charges (paper Sec. 3), the convergence orders the paper states (HE
second order, Sec. 1; VGF spectral, Sec. 2), the truncation invariance behind
eq:PoissonWindowed, linearity, translation and reflection symmetry, the far
field, and the adjoint identity.  A plausible mistake in the oracle (a dropped
factor, a wrong sign or index, a transposed operand) fails at least one.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import analytic as A


def rel_linf(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


# ------------------------------------------------------------------ FFT

@pytest.mark.parametrize("n", list(range(1, 65)) + [96, 100, 128, 192, 210, 512])
def test_fft_matches_definition_and_numpy(oracle_mod, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign in (-1, 1):
        got = oracle_mod.fft(x, sign)
        if n <= 210:
            ref = oracle_mod.dft_definition(x, sign)
            assert np.max(np.abs(got - ref)) <= 1e-13 * n * max(1.0, np.max(np.abs(ref)))
        lib = np.fft.fft(x) if sign == -1 else np.fft.ifft(x) * n
        assert np.max(np.abs(got - lib)) <= 1e-13 * n * np.max(np.abs(lib))


def test_fft_closed_forms(oracle_mod):
    n = 48
    delta = np.zeros(n, complex)
    delta[0] = 1
    assert np.allclose(oracle_mod.fft(delta), np.ones(n), atol=1e-15)
    t = np.arange(n)
    for k0 in (0, 1, 7, 24, 47):
        tone = np.exp(2j * np.pi * k0 * t / n)
        spec = oracle_mod.fft(tone, -1)
        want = np.zeros(n, complex)
        want[k0] = n
        assert np.max(np.abs(spec - want)) < 1e-12


# ---------------------------------------------- convolution vs brute force

@pytest.mark.parametrize("method", ["he", "vgf"])
@pytest.mark.parametrize("shape,h", [((6, 5, 4), (0.3, 0.25, 0.4)), ((7, 7, 7), (0.1, 0.1, 0.1)),
                                     ((12, 9), (0.05, 0.07)), ((16, 16), (1 / 16, 1 / 16))])
def test_fft_convolution_equals_direct_sum(oracle_mod, method, shape, h):
    rng = np.random.default_rng(3)
    rho = rng.standard_normal(shape)
    g = oracle_mod.kernel(method, list(shape), h)
    phi, _ = oracle_mod.solve_with_kernel(g, rho, h, True, False)
    ref = oracle_mod.direct_phi(g, rho, h)
    assert rel_linf(phi, ref) < 1e-13


def test_direct_sum_is_the_written_convolution(oracle_mod):
    """Direct sum checked against a pure-Python double loop on a tiny grid."""
    shape, h = (3, 4), (0.2, 0.3)
    rng = np.random.default_rng(5)
    rho = rng.standard_normal(shape)
    g = oracle_mod.kernel_he(list(shape), h)
    want = np.zeros(shape)
    for i0 in range(3):
        for i1 in range(4):
            s = 0.0
            for j0 in range(3):
                for j1 in range(4):
                    d0, d1 = (i0 - j0) * h[0], (i1 - j1) * h[1]
                    r = math.hypot(d0, d1)
                    gv = 1 / (2 * math.pi) if r == 0 else -math.log(r) / (2 * math.pi)
                    s += rho[j0, j1] * gv
            want[i0, i1] = h[0] * h[1] * s
    assert rel_linf(oracle_mod.direct_phi(g, rho, h), want) < 1e-14


# ------------------------------------------------------------ VGF kernel

@pytest.mark.parametrize("shape,h", [((6, 6, 6), (0.2, 0.2, 0.2)), ((4, 6, 10), (0.3, 0.1, 0.07)),
                                     ((10, 14), (0.1, 0.05)), ((8, 8), (1 / 8, 1 / 8))])
def test_vgf_cosine_sum_equals_literal_oversampled_ifft(oracle_mod, shape, h):
    """Octant cosine sums == the paper's recipe (IFFT on the whole M grid, restrict)."""
    a = oracle_mod.kernel_vgf(list(shape), h)
    b = oracle_mod.kernel_vgf(list(shape), h, literal=True)
    assert rel_linf(a, b) < 1e-13


@pytest.mark.parametrize("method", ["he", "vgf"])
def test_kernel_even_and_spectrum_real(oracle_mod, method):
    shape, h = (6, 8, 10), (0.1, 0.12, 0.07)
    g = oracle_mod.kernel(method, list(shape), h)
    # even under j -> -j on the wrapped grid
    flipped = np.roll(g[::-1, ::-1, ::-1], 1, axis=(0, 1, 2))
    assert np.array_equal(g, flipped)
    spec = oracle_mod.kernel_spectrum(g)
    assert np.max(np.abs(spec.imag)) < 1e-12 * np.max(np.abs(spec.real))


@pytest.mark.parametrize("method", ["he", "vgf"])
def test_kernel_at_minus_n_never_reaches_phi(oracle_mod, method):
    """Sec. 2's restriction keeps j_a in [-n_a, n_a); the plane j_a = -n_a (stored at index n_a)
    is never reached by the cropped convolution phi_i = sum_j rho_j g_(i-j), |i_a - j_a| <= n_a - 1.
    Changing g there leaves phi alone; a restriction shifted by one index would not. E does feel it:
    the spectral derivative (Sec. 4) is a dense circulant on the padded grid, so it reads phi~ at the
    padded points too, and those see the plane."""
    shape, h = (5, 6, 4), (0.11, 0.09, 0.13)
    rho = np.random.default_rng(21).standard_normal(shape)
    g = oracle_mod.kernel(method, list(shape), h)
    p0, E0 = oracle_mod.solve_with_kernel(g, rho, h)
    for a, n in enumerate(shape):
        g2 = g.copy()
        sl = [slice(None)] * 3
        sl[a] = n
        g2[tuple(sl)] += 7.0
        p1, E1 = oracle_mod.solve_with_kernel(g2, rho, h)
        assert np.max(np.abs(p1 - p0)) < 1e-12 * np.max(np.abs(p0))
        assert np.max(np.abs(E1 - E0)) > 1e-3 * np.max(np.abs(E0))
        # one plane inside the restricted window does reach phi
        g3 = g.copy()
        sl[a] = n - 1
        g3[tuple(sl)] += 7.0
        p3, _ = oracle_mod.solve_with_kernel(g3, rho, h)
        assert np.max(np.abs(p3 - p0)) > 1e-3 * np.max(np.abs(p0))


def test_vgf_spectrum_at_k0_limits():
    """The k -> 0 values of F{G^L} (3D L^2/2, 2D (L^2/4)(1 - 2 ln L)) match the limit of the formula."""
    from scipy import special
    L = 2.7
    for k in (1e-3, 1e-4):
        f3 = 2 * (math.sin(L * k / 2) / k) ** 2
        assert abs(f3 - L * L / 2) < 1e-5 * L * L
        x = L * k
        f2 = (1 - special.j0(x)) / k ** 2 - L * math.log(L) * special.j1(x) / k
        assert abs(f2 - (L * L / 4) * (1 - 2 * math.log(L))) < 1e-4


# -------------------------------------------------- closed-form solutions

def _compare_closed_form(oracle_mod, prob, method):
    rho = prob.rho(np.float64)
    phi, E = oracle_mod.solve(method, rho, prob.h)
    pex, Eex = A.mixture_field(W.grid_points(prob.shape, prob.h), prob.gaussians, prob.d)
    return rel_linf(phi, pex), rel_linf(E, Eex), np.max(np.abs(E - Eex))


def test_c1_cube_closed_form(oracle_mod):
    """32^3 on [-1,1]^3, sigma = 0.15: VGF to ~1e-11, HE only ~1e-2."""
    prob = W.unit_gaussian_3d(32, 0.15, 2.0)
    ep, eE, _ = _compare_closed_form(oracle_mod, prob, "vgf")
    assert ep < 1e-9 and eE < 1e-9
    hp, hE, _ = _compare_closed_form(oracle_mod, prob, "he")
    assert 1e-3 < hp < 1e-1 and hE > 1e-3


def test_he_g0_enters_as_a_point_self_term(oracle_mod):
    """HE replaces G(0) by a finite value (paper Sec. 1: 1 in 3D; Sec. 3.1: 1/(2 pi) in 2D).  The
    solve is linear in the kernel and that value sits at offset 0 only, so changing it moves phi by
    (g0 - g0') prod(h) rho at every cell and nowhere else: the literal defaults must show up there
    with exactly those constants."""
    rng = np.random.default_rng(31)
    for n, h, g0 in (((10, 12, 9), (0.1, 0.07, 0.12), 1.0), ((14, 11), (0.09, 0.13), 1.0 / (2.0 * math.pi))):
        rho = rng.standard_normal(n)
        phi_def, _ = oracle_mod.solve_with_kernel(oracle_mod.kernel_he(list(n), h), rho, h, with_E=False)
        phi_zero, _ = oracle_mod.solve_with_kernel(oracle_mod.kernel_he(list(n), h, g0=0.0), rho, h, with_E=False)
        want = g0 * float(np.prod(h)) * rho
        assert np.max(np.abs((phi_def - phi_zero) - want)) <= 1e-12 * np.max(np.abs(want))
        # the same through the method name the GPU path uses
        phi_m, _ = oracle_mod.solve("he", rho, h, with_E=False)
        assert np.max(np.abs(phi_m - phi_def)) <= 1e-13 * np.max(np.abs(phi_def))


def test_paper_3d_example(oracle_mod):
    """Paper Sec. 3, 3D: sigma = 0.05 on [-0.5,0.5]^3; VGF far below HE at N = 32, 64."""
    for n, vgf_tol in ((32, 1e-7), (64, 1e-13)):
        prob = W.unit_gaussian_3d(n, 0.05, 1.0)
        ep, eE, _ = _compare_closed_form(oracle_mod, prob, "vgf")
        hp, _, _ = _compare_closed_form(oracle_mod, prob, "he")
        assert ep < vgf_tol
        assert hp > 1e-3


def test_paper_2d_example(oracle_mod):
    """Paper Sec. 3, 2D: sigma = 0.05 on [-0.5,0.5]^2 with the E1 reading of the potential."""
    prob = W.unit_gaussian_2d(40, 0.05, 1.0)
    ep, _, eEabs = _compare_closed_form(oracle_mod, prob, "vgf")
    assert ep < 1e-11 and eEabs < 1e-8
    prob = W.unit_gaussian_2d(60, 0.05, 1.0)
    ep, _, eEabs = _compare_closed_form(oracle_mod, prob, "vgf")
    assert ep < 1e-13 and eEabs < 1e-12
    hp, _, _ = _compare_closed_form(oracle_mod, prob, "he")
    assert hp > 1e-3


def test_convergence_orders(oracle_mod):
    """HE error falls like h^2 (paper Sec. 1); VGF error falls spectrally (Sec. 2)."""
    errs = {}
    for n in (16, 32, 64):
        prob = W.unit_gaussian_3d(n, 0.05, 1.0)
        errs[("he", n)] = _compare_closed_form(oracle_mod, prob, "he")[0]
        errs[("vgf", n)] = _compare_closed_form(oracle_mod, prob, "vgf")[0]
    slope = math.log2(errs[("he", 32)] / errs[("he", 64)])
    assert 1.5 < slope < 2.5
    assert errs[("vgf", 16)] / errs[("vgf", 32)] > 1e4
    for n in (16, 32, 64):
        assert errs[("vgf", n)] < errs[("he", n)]


def test_anisotropic_quadrature_matches_isotropic_closed_form():
    """The heat-kernel quadrature for anisotropic Gaussians reduces to erf for equal sigmas."""
    pts = np.array([[0.1, 0.2, -0.3], [0.0, 0.0, 0.0], [0.5, -0.5, 0.4]])
    ph, E = A.field_aniso3(pts, np.zeros(3), np.array([0.1, 0.1, 0.1]), 0.7)
    ph2, E2 = A.field_iso(pts, np.zeros(3), 0.1, 0.7, 3)
    assert rel_linf(ph, ph2) < 1e-10 and np.max(np.abs(E - E2)) < 1e-9


def test_anisotropic_mixture_closed_form(oracle_mod):
    """Three anisotropic Gaussians: VGF vs the quadrature potential on sampled points."""
    rng = np.random.default_rng(11)
    gs = W.random_mixture(rng, 3, 3, centre_range=0.3, sigma_range=(0.08, 0.12))
    # 5.8 sigma from every face: the charge the box cuts off is below 1e-8
    prob = W.Problem("aniso", (48, 48, 48), (2 / 48,) * 3, gs)
    rho = prob.rho(np.float64)
    phi, E = oracle_mod.solve("vgf", rho, prob.h)
    pts = W.grid_points(prob.shape, prob.h)
    idx = tuple(rng.integers(0, 48, size=(3, 40)))
    pex, Eex = A.mixture_field(pts[idx], gs, 3)
    assert np.max(np.abs(phi[idx] - pex)) < 1e-7 * np.max(np.abs(phi))
    assert np.max(np.abs(E[(slice(None),) + idx] - Eex)) < 1e-6 * np.max(np.abs(E))


# --------------------------------------------------- geometry and invariants

def test_truncation_invariance(oracle_mod):
    """Any L beyond the box diagonal gives the same potential (eq:PoissonWindowed)."""
    prob = W.unit_gaussian_3d(16, 0.12, 2.0)
    rho = prob.rho(np.float64)
    L1 = oracle_mod.truncation_radius(prob.shape, prob.h, 1.0)
    L2 = oracle_mod.truncation_radius(prob.shape, prob.h, 1.35)
    p1, E1 = oracle_mod.solve("vgf", rho, prob.h, L=L1)
    p2, E2 = oracle_mod.solve("vgf", rho, prob.h, L=L2)
    assert rel_linf(p1, p2) < 1e-5 and rel_linf(E1, E2) < 1e-4
    # far too short a window changes the answer (plants a mistake in the kernel)
    L3 = 0.5 * L1
    p3, _ = oracle_mod.solve("vgf", rho, prob.h, L=L3)
    assert rel_linf(p3, p1) > 1e-2


def test_oversampling_rule_for_elongated_box(oracle_mod):
    """4N oversampling aliases on an elongated box; the M h >= side + L rule does not."""
    prob = W.Problem("long", (12, 12, 48), (1 / 12,) * 3, [(np.zeros(3), np.array([0.08, 0.08, 0.3]), 1.0)])
    rho = prob.rho(np.float64)
    L = oracle_mod.truncation_radius(prob.shape, prob.h)
    M_rule = oracle_mod.oversampled_size(prob.shape, prob.h, L)
    pts = W.grid_points(prob.shape, prob.h)
    pex, _ = A.mixture_field(pts.reshape(-1, 3)[::97], prob.gaussians, 3)
    p_rule, _ = oracle_mod.solve("vgf", rho, prob.h, L=L, M=M_rule, with_E=False)
    p_4n, _ = oracle_mod.solve("vgf", rho, prob.h, L=L, M=[4 * n for n in prob.shape], with_E=False)
    assert M_rule[0] > 4 * 12
    e_rule = np.max(np.abs(p_rule.reshape(-1)[::97] - pex)) / np.max(np.abs(pex))
    e_4n = np.max(np.abs(p_4n.reshape(-1)[::97] - pex)) / np.max(np.abs(pex))
    assert e_rule < 1e-3 and e_4n > 10 * e_rule


def test_oversampled_size_is_4n_for_cubes(oracle_mod):
    for n in (8, 32, 256):
        h = 2.0 / n
        L = oracle_mod.truncation_radius((n, n, n), (h, h, h))
        assert oracle_mod.oversampled_size((n, n, n), (h, h, h), L) == [4 * n] * 3


@pytest.mark.parametrize("method", ["he", "vgf"])
def test_linearity(oracle_mod, method):
    rng = np.random.default_rng(7)
    shape, h = (10, 12, 8), (0.1, 0.09, 0.13)
    r1, r2 = rng.standard_normal(shape), rng.standard_normal(shape)
    g = oracle_mod.kernel(method, list(shape), h)
    p1, E1 = oracle_mod.solve_with_kernel(g, r1, h)
    p2, E2 = oracle_mod.solve_with_kernel(g, r2, h)
    p3, E3 = oracle_mod.solve_with_kernel(g, 2.5 * r1 - 0.75 * r2, h)
    assert rel_linf(p3, 2.5 * p1 - 0.75 * p2) < 1e-13
    assert rel_linf(E3, 2.5 * E1 - 0.75 * E2) < 1e-13


@pytest.mark.parametrize("method", ["he", "vgf"])
def test_translation_by_whole_cells(oracle_mod, method):
    """Shifting a compact rho by whole cells shifts phi exactly where both are in the box."""
    shape, h = (16, 16, 16), (0.1, 0.1, 0.1)
    rng = np.random.default_rng(8)
    rho = np.zeros(shape)
    rho[4:9, 5:10, 3:8] = rng.standard_normal((5, 5, 5))
    s = (3, 2, 4)
    rho_s = np.roll(rho, s, axis=(0, 1, 2))
    g = oracle_mod.kernel(method, list(shape), h)
    p, E = oracle_mod.solve_with_kernel(g, rho, h)
    ps, Es = oracle_mod.solve_with_kernel(g, rho_s, h)
    assert rel_linf(ps[3:, 2:, 4:], p[:-3, :-2, :-4]) < 1e-12
    assert rel_linf(Es[:, 3:, 2:, 4:], E[:, :-3, :-2, :-4]) < 1e-12


@pytest.mark.parametrize("method", ["he", "vgf"])
def test_reflection_symmetry(oracle_mod, method):
    """Reflecting rho along x reflects phi and E_y, E_z and negates E_x (E = -grad phi)."""
    shape, h = (10, 9, 8), (0.1, 0.11, 0.12)
    rho = np.random.default_rng(9).standard_normal(shape)
    g = oracle_mod.kernel(method, list(shape), h)
    p, E = oracle_mod.solve_with_kernel(g, rho, h)
    pr, Er = oracle_mod.solve_with_kernel(g, rho[::-1].copy(), h)
    assert rel_linf(pr, p[::-1]) < 1e-12
    assert rel_linf(Er[0], -E[0][::-1]) < 1e-12
    assert rel_linf(Er[1], E[1][::-1]) < 1e-12


def test_field_is_minus_gradient(oracle_mod):
    """E_x ~ -d phi / dx by centred differences for a smooth rho (sign and axis order)."""
    prob = W.unit_gaussian_3d(48, 0.2, 2.0)
    prob.gaussians = [(np.array([0.1, -0.2, 0.15]), np.array([0.2, 0.25, 0.3]), 1.0)]
    phi, E = oracle_mod.solve("vgf", prob.rho(np.float64), prob.h)
    for a in range(3):
        fd = -(np.roll(phi, -1, axis=a) - np.roll(phi, 1, axis=a)) / (2 * prob.h[a])
        inner = (slice(2, -2),) * 3
        assert rel_linf(fd[inner], E[a][inner]) < 2e-2


def test_far_field(oracle_mod):
    """For a compact charge the potential at the box corners approaches Q/(4 pi r) (3D) and -Q ln r/(2 pi) (2D)."""
    prob = W.unit_gaussian_3d(32, 0.12, 2.0)
    phi, _ = oracle_mod.solve("vgf", prob.rho(np.float64), prob.h, with_E=False)
    q = float(np.sum(prob.rho(np.float64)) * np.prod(prob.h))
    r = math.sqrt(3) * (1 - 0.5 * prob.h[0])
    assert abs(phi[0, 0, 0] - q / (4 * math.pi * r)) < 1e-10
    prob = W.unit_gaussian_2d(64, 0.08, 2.0)
    phi, _ = oracle_mod.solve("vgf", prob.rho(np.float64), prob.h, with_E=False)
    q = float(np.sum(prob.rho(np.float64)) * np.prod(prob.h))
    r = math.sqrt(2) * (1 - 0.5 * prob.h[0])
    assert abs(phi[0, 0] + q * math.log(r) / (2 * math.pi)) < 1e-10


# ----------------------------------------------------------------- adjoint

@pytest.mark.parametrize("method", ["he", "vgf"])
def test_adjoint_matches_explicit_transpose(oracle_mod, method):
    """Build the solve map column by column on a tiny grid; its transpose == orc_adjoint."""
    shape, h = (4, 3, 4), (0.2, 0.3, 0.25)
    cells = int(np.prod(shape))
    g = oracle_mod.kernel(method, list(shape), h)
    cols = []
    for c in range(cells):
        e = np.zeros(cells)
        e[c] = 1.0
        p, E = oracle_mod.solve_with_kernel(g, e.reshape(shape), h)
        cols.append(np.concatenate([p.ravel(), E.ravel()]))
    Mat = np.array(cols).T          # [(1+d) cells, cells]
    rng = np.random.default_rng(12)
    gp = rng.standard_normal(shape)
    gE = rng.standard_normal((3,) + shape)
    want = Mat.T @ np.concatenate([gp.ravel(), gE.ravel()])
    got = oracle_mod.adjoint_with_kernel(g, gp, gE, h)
    assert rel_linf(got.ravel(), want) < 1e-12
    # A is symmetric, each B_a antisymmetric
    A_ = Mat[:cells]
    assert np.max(np.abs(A_ - A_.T)) < 1e-13 * np.max(np.abs(A_))
    for a in range(3):
        B = Mat[cells * (a + 1):cells * (a + 2)]
        assert np.max(np.abs(B + B.T)) < 1e-13 * np.max(np.abs(B))


# ----------------------------------------------------------------- golden

def test_golden_c1_samples(oracle_mod):
    """Oracle values stored by tests/golden/make_golden.py reproduce on this machine,
    and the stored VGF values sit on the erf closed form while HE's do not."""
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "c1_samples.json")
    gold = json.load(open(path))
    prob = W.unit_gaussian_3d(32, 0.15, 2.0)
    rho = prob.rho(np.float32).astype(np.float64)
    idx = tuple(np.array(gold["cells"]).T)
    for method in ("he", "vgf"):
        phi, E = oracle_mod.solve(method, rho, prob.h)
        assert np.max(np.abs(phi[idx] - np.array(gold[method]["phi"]))) < 1e-12
        assert np.max(np.abs(E[(slice(None),) + idx].T - np.array(gold[method]["E"]))) < 1e-12
    cf = np.array(gold["closed_form"]["phi"])
    assert np.max(np.abs(np.array(gold["vgf"]["phi"]) - cf)) < 1e-7 * np.max(np.abs(cf))
    assert np.max(np.abs(np.array(gold["he"]["phi"]) - cf)) > 1e-4 * np.max(np.abs(cf))


def test_direct_sum_at_points_matches_full_direct_sum(oracle_mod):
    shape, h = (6, 7, 8), (0.1, 0.2, 0.15)
    rho = np.random.default_rng(13).standard_normal(shape)
    g = oracle_mod.kernel_vgf(list(shape), h)
    full = oracle_mod.direct_phi(g, rho, h)
    pts = np.array([0, 5, 17, 100, 335])
    assert np.max(np.abs(oracle_mod.direct_phi_at(g, rho, h, pts) - full.ravel()[pts])) < 1e-13 * np.max(np.abs(full))


def test_he_cell_average_constants(oracle_mod):
    """Cell-average G(0): unit cube int 1/|x| = 2.380077..., unit square int ln|x| = -1.061175..."""
    g3 = oracle_mod.he_g0_variant(3, (1.0, 1.0, 1.0), "he_cellavg")
    assert abs(g3 * 4 * math.pi - 2.3800772) < 1e-6
    g2 = oracle_mod.he_g0_variant(2, (1.0, 1.0), "he_cellavg")
    assert abs(-g2 * 2 * math.pi - (-1.0611759)) < 1e-6
    # nearby value is G at the smallest spacing
    assert oracle_mod.he_g0_variant(3, (0.1, 0.2, 0.3), "he_nearby") == pytest.approx(1 / (4 * math.pi * 0.1))
    # cell average scales like 1/h in 3D
    assert oracle_mod.he_g0_variant(3, (0.5, 0.5, 0.5), "he_cellavg") == pytest.approx(2 * g3, rel=1e-9)


def test_fd_gradient_exact_on_quadratics(oracle_mod):
    """Centred and second-order one-sided differences are exact for quadratics (E = -grad phi)."""
    shape, h = (7, 6, 5), (0.3, 0.2, 0.5)
    x, y, z = np.meshgrid(*[np.arange(n) * hh for n, hh in zip(shape, h)], indexing="ij")
    phi = 1.5 * x * x - 0.7 * x * y + 2.0 * z * z + 0.3 * y - z + 4.0
    E = oracle_mod.fd_gradient(phi, h)
    assert np.allclose(E[0], -(3.0 * x - 0.7 * y), atol=1e-12)
    assert np.allclose(E[1], -(-0.7 * x + 0.3), atol=1e-12)
    assert np.allclose(E[2], -(4.0 * z - 1.0), atol=1e-12)
    # cubic terms are not exact: the scheme is second order
    E3 = oracle_mod.fd_gradient(x ** 3, h)
    assert np.max(np.abs(E3[0] + 3 * x ** 2)) > 1e-3


def test_fd_gradient_second_order_for_he(oracle_mod):
    """The paper's HE + finite-difference field converges like h^2 (Sec. 3)."""
    errs = []
    for n in (32, 64):
        prob = W.unit_gaussian_2d(n, 0.05, 1.0)
        phi, _ = oracle_mod.solve("vgf", prob.rho(np.float64), prob.h, with_E=False)
        _, Eex = A.mixture_field(W.grid_points(prob.shape, prob.h), prob.gaussians, 2)
        E = oracle_mod.fd_gradient(phi, prob.h)
        inner = (slice(None), slice(2, -2), slice(2, -2))
        errs.append(np.max(np.abs(E[inner] - Eex[inner])))
    assert 3.0 < errs[0] / errs[1] < 5.0
