"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Every comparison runs both sides on the same seeded FP32 inputs (the oracle
reads them as FP64).  Tolerance: relative L-inf <= 1e-5 for phi and for E
(max |x - x_ref| / max |x_ref|), the accuracy the FP32 pipeline is built to.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import analytic as A

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fsp():
    from paper_2103_08531_gb300 import build
    build.build()
    import paper_2103_08531_gb300 as pkg
    pkg.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return pkg


def rel(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def gpu_solve(fsp, prob, method, with_E=True, **kw):
    rho32 = prob.rho(np.float32)
    plan = fsp.Plan(prob.shape, prob.h, method, **kw)
    phi, E = plan.solve(torch.from_numpy(rho32).cuda(), with_E=with_E)
    torch.cuda.synchronize()
    return plan, rho32, phi.cpu().numpy(), (E.cpu().numpy() if E is not None else None)


SMALL = [
    ("cube32", (32, 32, 32), (2 / 32,) * 3),
    ("aniso", (32, 64, 96), (0.03, 0.02, 0.011)),
    ("flat", (64, 32, 32), (0.01, 0.03, 0.02)),
    ("2d", (64, 128), (0.02, 0.011)),
    ("2d_sq", (256, 256), (1 / 128, 1 / 128)),
]


def _mixture(shape, h, seed, count=3):
    rng = np.random.default_rng(seed)
    side = [n * hh for n, hh in zip(shape, h)]
    gs = []
    for _ in range(count):
        c = np.array([rng.uniform(-0.25, 0.25) * s for s in side])
        sig = np.array([rng.uniform(0.06, 0.12) * s for s in side])
        gs.append((c, sig, rng.uniform(-1, 1)))
    return W.Problem("mix", shape, h, gs)


# ---------------------------------------------------------------- geometry

@pytest.mark.parametrize("name,shape,h", SMALL + [("beam", (64, 64, 256), (0.005, 0.02, 0.03))])
def test_geometry_rules_match_oracle(fsp, oracle_mod, name, shape, h):
    plan = fsp.Plan(shape, h, "vgf")
    g = plan.geometry()
    L = oracle_mod.truncation_radius(shape, h)
    assert g["n"] == list(shape)
    assert abs(g["L"] - L) <= 1e-12 * L
    assert g["M"] == oracle_mod.oversampled_size(shape, h, L)


# ---------------------------------------------------------- kernel spectrum

@pytest.mark.parametrize("method", ["he", "vgf", "he_nearby", "he_cellavg"])
@pytest.mark.parametrize("name,shape,h", SMALL)
def test_kernel_spectrum_parity(fsp, oracle_mod, method, name, shape, h):
    """FP64 device precompute, rounded to FP32, vs the oracle's DFT of its kernel."""
    plan = fsp.Plan(shape, h, method)
    K = plan.kernel_spectrum().astype(np.float64)
    if method == "vgf":
        g = oracle_mod.kernel_vgf(list(shape), h)
    else:
        g = oracle_mod.kernel_he(list(shape), h, g0=oracle_mod.he_g0_variant(len(shape), h, method))
    ref = oracle_mod.scaled_spectrum_octant(g, h)
    assert K.shape == ref.shape
    err = np.abs(K - ref)
    assert np.all(err <= 2 ** -23 * np.abs(ref) + 1e-12 * np.max(np.abs(ref)))


# --------------------------------------------------------------- solves

@pytest.mark.parametrize("method", ["vgf", "he"])
@pytest.mark.parametrize("name,shape,h", SMALL)
def test_solve_parity(fsp, oracle_mod, method, name, shape, h):
    prob = _mixture(shape, h, seed=hash(name) % 1000)
    plan, rho32, phi, E = gpu_solve(fsp, prob, method)
    g = oracle_mod.kernel(method, list(shape), h)
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rho32.astype(np.float64), h)
    assert rel(phi, p_ref) <= TOL
    assert rel(E, E_ref) <= TOL
    for a in range(len(shape)):
        assert rel(E[a], E_ref[a]) <= 4 * TOL


LONG = [
    ("z1024", (32, 32, 512), (0.03, 0.03, 0.004), "vgf"),     # middle pass on 1024-point lines (two warps a line)
    ("z1024he", (64, 32, 512), (0.02, 0.03, 0.004), "he"),
    ("y1024", (96, 512), (0.01, 0.002), "vgf"),                # 2D, 1024-point middle lines
    ("y2048", (64, 1024), (0.01, 0.001), "vgf"),               # 2D, 2048-point middle lines (four warps a line)
    ("y4096", (64, 2048), (0.01, 0.001), "he"),                # 2D, 4096-point middle lines
    ("y8192", (32, 4096), (0.02, 0.0005), "he"),               # 2D, 8192-point middle lines
    ("x4096", (2048, 64), (0.001, 0.01), "he"),                # 2D, 4096-point column tiles (narrow)
    ("x8192", (4096, 32), (0.0005, 0.02), "he"),               # 2D, 8192-point column tiles (narrow)
]


# padded lengths 32, 96, 384 and 768 (2^a 3^b) on the FFT passes, every axis role; 2D also 1536, 3072, 6144
MIXED_LENGTHS = [
    ("n16_48_192", (16, 48, 192), (0.05, 0.03, 0.01), "vgf"),    # 2n = 32, 96, 384
    ("n384_48_64", (384, 48, 64), (0.004, 0.03, 0.02), "he"),    # 2n0 = 768 (block column tiles)
    ("n32_16_384", (32, 16, 384), (0.03, 0.05, 0.004), "vgf"),   # 2n2 = 768 (multi-warp middle lines)
    ("n96_384_96", (96, 384, 96), (0.02, 0.004, 0.02), "vgf"),   # 2n1 = 768, 2n2 = 192
    ("2d_192_384", (192, 384), (0.01, 0.005), "vgf"),            # 2D: 384 columns, 768-point lines
    ("2d_48_96", (48, 96), (0.04, 0.02), "he"),                  # 2D: 96 columns
    ("2d_768_32", (768, 32), (0.002, 0.03), "vgf"),              # 2D: 1536-point columns (staged, radix 3)
    ("2d_32_768", (32, 768), (0.03, 0.002), "he"),               # 2D: 1536-point lines (four warps a line)
    ("2d_1536_32", (1536, 32), (0.001, 0.03), "vgf"),            # 2D: 3072-point columns
    ("2d_32_1536", (32, 1536), (0.03, 0.001), "vgf"),            # 2D: 3072-point lines (block kernel)
    ("2d_3072_32", (3072, 32), (0.0006, 0.03), "he"),            # 2D: 6144-point columns
    ("2d_32_3072", (32, 3072), (0.03, 0.0006), "vgf"),           # 2D: 6144-point lines
]


def _runs_fft_passes(plan):
    """Plans on the direct-sum path refuse pass events; the FFT-pass plans take them."""
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(plan.passes + 1)]
    for e in evs:
        e.record()   # torch creates the CUDA event on its first record
    try:
        plan.set_pass_events(evs)
    except Exception:
        return False
    plan.set_pass_events(None)
    return True


@pytest.mark.parametrize("name,shape,h,method", MIXED_LENGTHS)
def test_solve_parity_more_lengths(fsp, oracle_mod, name, shape, h, method):
    prob = _mixture(shape, h, seed=len(name) + 7)
    plan, rho32, phi, E = gpu_solve(fsp, prob, method)
    assert _runs_fft_passes(plan)
    g = oracle_mod.kernel(method, list(shape), h)
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rho32.astype(np.float64), h)
    assert rel(phi, p_ref) <= TOL
    assert rel(E, E_ref) <= TOL
    # adjoint through the same passes
    rng = np.random.default_rng(3)
    gp = rng.standard_normal(shape)
    gE = rng.standard_normal((len(shape),) + shape)
    g_rho = plan.adjoint(torch.from_numpy(gp.astype(np.float32)).cuda(), torch.from_numpy(gE.astype(np.float32)).cuda())
    ref = oracle_mod.adjoint_with_kernel(g, gp.astype(np.float32).astype(np.float64),
                                         gE.astype(np.float32).astype(np.float64), h)
    assert rel(g_rho.cpu(), ref) <= TOL


@pytest.mark.parametrize("name,shape,h,method", LONG)
def test_solve_parity_long_lines(fsp, oracle_mod, name, shape, h, method):
    """The long-line passes (multi-warp and block-synchronous) for 1024- to 8192-point lines against the oracle."""
    prob = _mixture(shape, h, seed=len(name))
    plan, rho32, phi, E = gpu_solve(fsp, prob, method)
    g = oracle_mod.kernel(method, list(shape), h)
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rho32.astype(np.float64), h)
    assert rel(phi, p_ref) <= TOL
    assert rel(E, E_ref) <= TOL


@pytest.mark.parametrize("name,shape,h", SMALL[:2] + SMALL[3:4])
def test_phi_only_and_E_only(fsp, name, shape, h):
    prob = _mixture(shape, h, seed=5)
    rho = torch.from_numpy(prob.rho(np.float32)).cuda()
    plan = fsp.Plan(shape, h, "vgf")
    phi, E = plan.solve(rho)
    phi1, none = plan.solve(rho, with_E=False)
    none2, E1 = plan.solve(rho, with_phi=False)
    assert none is None and none2 is None
    assert rel(phi1.cpu(), phi.cpu()) <= 1e-6
    assert rel(E1.cpu(), E.cpu()) <= 1e-6


def test_c1_closed_form(fsp):
    """32^3 unit Gaussian (sigma 0.15) on [-1,1]^3: the GPU VGF solve sits on the erf potential."""
    prob = W.unit_gaussian_3d(32, 0.15, 2.0)
    _, _, phi, E = gpu_solve(fsp, prob, "vgf")
    pex, Eex = A.mixture_field(W.grid_points(prob.shape, prob.h), prob.gaussians, 3)
    assert rel(phi, pex) < 3e-6 and rel(E, Eex) < 3e-6
    _, _, phi_he, _ = gpu_solve(fsp, prob, "he")
    assert rel(phi_he, pex) > 1e-3


def test_2d_closed_form(fsp):
    prob = W.unit_gaussian_2d(128, 0.05, 1.0)
    _, _, phi, E = gpu_solve(fsp, prob, "vgf")
    pex, Eex = A.mixture_field(W.grid_points(prob.shape, prob.h), prob.gaussians, 2)
    assert rel(phi, pex) < 3e-6 and rel(E, Eex) < 3e-6


# --------------------------------------------------------------- adjoint

@pytest.mark.parametrize("method", ["vgf", "he"])
@pytest.mark.parametrize("name,shape,h", [SMALL[1], SMALL[3]])
def test_adjoint_parity(fsp, oracle_mod, method, name, shape, h):
    rng = np.random.default_rng(21)
    d = len(shape)
    gp = rng.standard_normal(shape).astype(np.float32)
    gE = rng.standard_normal((d,) + shape).astype(np.float32)
    plan = fsp.Plan(shape, h, method)
    g = oracle_mod.kernel(method, list(shape), h)
    got = plan.adjoint(torch.from_numpy(gp).cuda(), torch.from_numpy(gE).cuda()).cpu().numpy()
    ref = oracle_mod.adjoint_with_kernel(g, gp.astype(np.float64), gE.astype(np.float64), h)
    assert rel(got, ref) <= TOL
    got_e = plan.adjoint(None, torch.from_numpy(gE).cuda()).cpu().numpy()
    ref_e = oracle_mod.adjoint_with_kernel(g, None, gE.astype(np.float64), h)
    assert rel(got_e, ref_e) <= TOL
    got_p = plan.adjoint(torch.from_numpy(gp).cuda(), None).cpu().numpy()
    ref_p = oracle_mod.adjoint_with_kernel(g, gp.astype(np.float64), None, h)
    assert rel(got_p, ref_p) <= TOL


@pytest.mark.parametrize("name,shape,h", [SMALL[0], SMALL[4]])
def test_adjoint_dot_product(fsp, name, shape, h):
    """<(phi, E)(rho), (psi, chi)> == <rho, adjoint(psi, chi)> with the GPU on both sides."""
    rng = np.random.default_rng(22)
    d = len(shape)
    rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    psi = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    chi = torch.from_numpy(rng.standard_normal((d,) + shape).astype(np.float32)).cuda()
    plan = fsp.Plan(shape, h, "vgf")
    phi, E = plan.solve(rho)
    g = plan.adjoint(psi, chi)
    lhs = (phi.double() * psi.double()).sum() + (E.double() * chi.double()).sum()
    rhs = (rho.double() * g.double()).sum()
    scale = (phi.double().abs() * psi.double().abs()).sum() + (E.double().abs() * chi.double().abs()).sum()
    assert abs(float(lhs - rhs)) <= 1e-6 * float(scale)


def test_autograd_matches_fd_and_oracle_gradient(fsp, oracle_mod):
    """loss = sum (phi - phi_t)^2 + 0.1 sum |E|^2: FspSolve backward vs FP64 central differences."""
    n, B = 32, 2
    probs, target = W.training_batch(n, B, seeds=range(10, 10 + B))
    h = probs[0].h
    plan = fsp.Plan((n, n, n), h, "vgf")
    tgt = torch.from_numpy(target).cuda()
    g2n = oracle_mod.kernel_vgf([n, n, n], h)
    rng = np.random.default_rng(5)
    for prob in probs:
        rho32 = prob.rho(np.float32)
        rho = torch.from_numpy(rho32).cuda().requires_grad_(True)
        phi, E = fsp.FspSolve.apply(rho, plan)
        loss = ((phi - tgt) ** 2).sum() + 0.1 * (E ** 2).sum()
        loss.backward()
        grad = rho.grad.cpu().numpy().astype(np.float64)

        r64 = rho32.astype(np.float64)
        t64 = target.astype(np.float64)

        def L(r):
            p, e = oracle_mod.solve_with_kernel(g2n, r, h)
            return np.sum((p - t64) ** 2) + 0.1 * np.sum(e ** 2)

        p0, e0 = oracle_mod.solve_with_kernel(g2n, r64, h)
        ref = oracle_mod.adjoint_with_kernel(g2n, 2 * (p0 - t64), 0.2 * e0, h)
        assert rel(grad, ref) <= 2 * TOL
        eps = 1e-2 * np.max(np.abs(r64))
        for idx in map(tuple, rng.integers(0, n, size=(32, 3))):
            rp, rm = r64.copy(), r64.copy()
            rp[idx] += eps
            rm[idx] -= eps
            fd = (L(rp) - L(rm)) / (2 * eps)
            assert abs(grad[idx] - fd) <= 2 * TOL * np.max(np.abs(ref))


# --------------------------------------------------------------- batches

def test_batched_equals_single(fsp):
    shapes = [((32, 32, 32), (0.02, 0.03, 0.025)), ((64, 32, 32), (0.01, 0.02, 0.03)),
              ((32, 64, 96), (0.03, 0.01, 0.02)), ((32, 32, 128), (0.02, 0.02, 0.005)),
              ((32, 32, 512), (0.02, 0.02, 0.004)), ((64, 32, 512), (0.03, 0.02, 0.004))]
    plans, rhos = [], []
    for i, (s, h) in enumerate(shapes):
        plans.append(fsp.Plan(s, h, "vgf"))
        rhos.append(torch.from_numpy(_mixture(s, h, 40 + i).rho(np.float32)).cuda())
    phis, Es = fsp.solve_batched(plans, rhos)
    batch = fsp.Batch(plans, rhos)
    bphis, bEs = batch.run()
    for p, r, ph, E, bph, bE in zip(plans, rhos, phis, Es, bphis, bEs):
        ph1, E1 = p.solve(r)
        assert torch.equal(ph, ph1) and torch.equal(E, E1)
        assert torch.equal(bph, ph1) and torch.equal(bE, E1)


def test_batched_2d_long_lines_equal_single(fsp, oracle_mod):
    """2D items with 8192-point lines in one batch (the four-step middle pass; the four-step C2R
    columns through buf0 / buf1): the batched launches give the single solves' bits, and those
    match the oracle."""
    shapes = [((32, 4096), (0.02, 0.0005)), ((16, 4096), (0.03, 0.0004)), ((64, 4096), (0.01, 0.0005)),
              ((4096, 32), (0.0005, 0.02)), ((4096, 64), (0.0004, 0.01))]
    plans = [fsp.Plan(s, h, "vgf") for s, h in shapes]
    rhos32 = [_mixture(s, h, 70 + i).rho(np.float32) for i, (s, h) in enumerate(shapes)]
    rhos = [torch.from_numpy(r).cuda() for r in rhos32]
    phis, Es = fsp.solve_batched(plans, rhos)
    for (s, h), p, r, r32, ph, E in zip(shapes, plans, rhos, rhos32, phis, Es):
        ph1, E1 = p.solve(r)
        assert torch.equal(ph, ph1) and torch.equal(E, E1)
    s, h = shapes[0]
    g = oracle_mod.kernel_vgf(list(s), h)
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rhos32[0].astype(np.float64), h)
    assert rel(phis[0].cpu(), p_ref) <= TOL and rel(Es[0].cpu(), E_ref) <= TOL


def test_2d_8192_columns_phi_only_and_E_only(fsp):
    """The four-step C2R columns with only phi (no buf1) or only E (no phi set) requested."""
    shape, h = (4096, 64), (0.0004, 0.01)
    rho = torch.from_numpy(_mixture(shape, h, seed=81).rho(np.float32)).cuda()
    plan = fsp.Plan(shape, h, "vgf")
    phi, E = plan.solve(rho)
    phi1, none = plan.solve(rho, with_E=False)
    none2, E1 = plan.solve(rho, with_phi=False)
    assert none is None and none2 is None
    assert torch.equal(phi1, phi) and torch.equal(E1, E)


def test_batched_many_mixed_items_and_graph(fsp):
    """More items than one launch holds (chunks), 2D and 3D mixed, uneven shapes; graph replay."""
    rng = np.random.default_rng(44)
    specs = []
    shapes3 = [(32, 32, 32), (64, 32, 32), (32, 64, 96), (96, 32, 64), (32, 32, 128), (64, 64, 64)]
    for i in range(40):
        if i % 5 == 4:
            s = (64, 128) if i % 2 else (128, 64)
        else:
            s = shapes3[i % len(shapes3)]
        h = tuple(float(x) for x in rng.uniform(0.01, 0.03, size=len(s)))
        specs.append((s, h))
    plans = [fsp.Plan(s, h, "vgf") for s, h in specs]
    rhos = [torch.from_numpy(_mixture(s, h, 100 + i, count=1).rho(np.float32)).cuda() for i, (s, h) in enumerate(specs)]
    batch = fsp.Batch(plans, rhos)
    g = batch.capture()
    for r in rhos:
        r.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for p, r, ph, E in zip(plans, rhos, batch.phis, batch.Es):
        ph1, E1 = p.solve(r)
        assert torch.equal(ph, ph1) and torch.equal(E, E1)


def test_batch_kernel_count(fsp):
    """fsp_batch_kernel_count reports one launch per (pass, padded length) of the batch, and the
    counting capture leaves the batch usable."""
    specs = [((32, 32, 32), (0.02, 0.02, 0.02)), ((32, 32, 32), (0.03, 0.02, 0.01)),
             ((64, 32, 128), (0.01, 0.02, 0.005))]
    plans = [fsp.Plan(s, h, "vgf") for s, h in specs]
    rhos = [torch.from_numpy(_mixture(s, h, 120 + i, count=1).rho(np.float32)).cuda() for i, (s, h) in enumerate(specs)]
    batch = fsp.Batch(plans, rhos)
    # P1 and P5: 2 n0 in {64, 128}; P2 and P4: 2 n1 = 64; P3: 2 n2 in {64, 256}
    assert batch.kernel_count() == 8
    assert fsp.Batch(plans[:1], rhos[:1]).kernel_count() == 5
    phis, Es = batch.run()
    torch.cuda.synchronize()
    for p, r, ph, E in zip(plans, rhos, phis, Es):
        ph1, E1 = p.solve(r)
        assert torch.equal(ph, ph1) and torch.equal(E, E1)


def test_batched_rejects_repeated_plan(fsp):
    p = fsp.Plan((32, 32, 32), (0.02, 0.02, 0.02), "vgf")
    r = torch.zeros((32, 32, 32), device="cuda")
    with pytest.raises(fsp.FspError):
        fsp.solve_batched([p, p], [r, r])


@pytest.mark.parametrize("name,shape,h", [SMALL[1], SMALL[3], ("z1024", (32, 32, 512), (0.03, 0.03, 0.004))])
def test_fd_gradient_matches_oracle(fsp, oracle_mod, name, shape, h):
    """Centred-difference E from the GPU phi equals the oracle's finite differences of the same phi."""
    prob = _mixture(shape, h, seed=81)
    plan = fsp.Plan(shape, h, "he")
    phi, _ = plan.solve(torch.from_numpy(prob.rho(np.float32)).cuda(), with_E=False)
    E = plan.gradient_fd(phi)
    p64 = phi.cpu().numpy().astype(np.float64)
    ref = oracle_mod.fd_gradient(p64, h)
    got = E.cpu().numpy().astype(np.float64)
    assert rel(got, ref) <= 1e-5
    # Element-wise: the FP32 stencil takes at most six roundings (the product
    # by 3, two sums, the scaling, and 1/2h rounded to FP32), so it errs by at
    # most about 6u (u = 2^-24) times the stencil of |phi|, i.e. the sum of
    # |coefficient * phi| / 2h: the standard bound for a short dot product.
    bound = np.empty_like(ref)
    for a in range(p64.ndim):
        q = np.moveaxis(np.abs(p64), a, 0)
        s = np.empty_like(q)
        s[1:-1] = q[2:] + q[:-2]
        s[0] = 3 * q[0] + 4 * q[1] + q[2]
        s[-1] = 3 * q[-1] + 4 * q[-2] + q[-3]
        bound[a] = np.moveaxis(s, 0, a) / (2 * h[a])
    assert np.all(np.abs(got - ref) <= 6 * 2.0**-24 * bound * (1 + 1e-6) + 1e-30)


def test_host_pipeline_matches_solve(fsp):
    """Overlapped host->device, solve and device->host streams give the same results as plain solves."""
    shape, h = (64, 32, 96), (0.02, 0.03, 0.01)
    plan = fsp.Plan(shape, h, "vgf")
    hosts = [torch.from_numpy(_mixture(shape, h, 70 + i).rho(np.float32)).pin_memory() for i in range(5)]
    phis = [torch.empty(shape).pin_memory() for _ in hosts]
    Es = [torch.empty((3,) + shape).pin_memory() for _ in hosts]
    pipe = fsp.HostPipeline(plan, depth=2)
    pipe.run(hosts, phis, Es)
    torch.cuda.synchronize()
    for r, ph, E in zip(hosts, phis, Es):
        ph1, E1 = plan.solve(r.cuda())
        assert torch.equal(ph, ph1.cpu()) and torch.equal(E, E1.cpu())


@pytest.mark.parametrize("shape,h,dtype,depth,with_phi,with_E", [
    ((128, 96), (0.01, 0.02), "f32", 3, True, False),        # 2D, phi only, three slots
    ((13, 17, 11), (0.05, 0.04, 0.06), "f64", 1, False, True),  # FP64 direct-sum plan, E only, one slot
])
def test_host_pipeline_modes(fsp, shape, h, dtype, depth, with_phi, with_E):
    """The host pipe in other modes: 2D, FP64 plans, one or three slots, phi or E alone, pageable and pinned
    host buffers; each result equals the plain solve's."""
    np_dt, t_dt = (np.float32, torch.float32) if dtype == "f32" else (np.float64, torch.float64)
    plan = fsp.Plan(shape, h, "vgf", dtype=dtype)
    d = len(shape)
    hosts = [torch.from_numpy(_mixture(shape, h, 90 + i).rho(np_dt)) for i in range(4)]
    hosts = [x.pin_memory() if i % 2 else x for i, x in enumerate(hosts)]   # pinned and pageable
    phis = [torch.empty(shape, dtype=t_dt) for _ in hosts] if with_phi else None
    Es = [torch.empty((d,) + shape, dtype=t_dt) for _ in hosts] if with_E else None
    pipe = fsp.HostPipeline(plan, depth=depth, with_phi=with_phi, with_E=with_E)
    pipe.run(hosts, phis, Es)
    torch.cuda.synchronize()
    for i, r in enumerate(hosts):
        ph1, E1 = plan.solve(r.cuda(), with_phi=with_phi, with_E=with_E)
        if with_phi:
            assert torch.equal(phis[i], ph1.cpu())
        if with_E:
            assert torch.equal(Es[i], E1.cpu())
    pipe.close()
    with pytest.raises(ValueError):
        fsp.HostPipeline(plan, depth=2).run(hosts, None, None)   # outputs missing


# --------------------------------------------------------------- autotuner

def _write_cache(path, arch, shape, var_tile, var_p3):
    d = len(shape)
    Ns = {"p1_fwd": 2 * shape[0], "p5_fwd": 2 * shape[0], "p3_fwd": 2 * shape[-1]}
    if d == 3:
        Ns.update({"p2_fwd": 2 * shape[1], "p4_fwd": 2 * shape[1]})
    entries = {f"{k}/{N}": (var_p3 if k == "p3_fwd" else var_tile) for k, N in Ns.items()}
    import json
    with open(path, "w") as f:
        json.dump({arch: entries}, f)


@pytest.mark.parametrize("shape,h", [((64, 64, 32), (0.02, 0.025, 0.03)), ((32, 128, 64), (0.03, 0.01, 0.02)),
                                     ((128, 64), (0.01, 0.02)), ((32, 64, 128), (0.03, 0.02, 0.01)),
                                     ((32, 32, 256), (0.03, 0.02, 0.005)), ((32, 32, 512), (0.03, 0.02, 0.004)),
                                     ((256, 32, 32), (0.004, 0.03, 0.02)), ((32, 256, 32), (0.03, 0.004, 0.02)),
                                     ((32, 4096), (0.02, 0.0005)), ((4096, 32), (0.0005, 0.02))])
def test_every_tuning_variant_is_correct(fsp, oracle_mod, shape, h, tmp_path):
    """Each launch variant the autotuner can pick gives the oracle's answer."""
    cap = torch.cuda.get_device_capability()
    arch = f"sm_{cap[0] * 10 + cap[1]}"
    prob = _mixture(shape, h, seed=61)
    rho32 = prob.rho(np.float32)
    rho = torch.from_numpy(rho32).cuda()
    plan = fsp.Plan(shape, h, "vgf")
    g = oracle_mod.kernel_vgf(list(shape), h)
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rho32.astype(np.float64), h)
    path = str(tmp_path / "tune.json")
    try:
        # column tiles: 0 TMA-staged group tiles, 2 the same one CTA per SM, 4 / 5 the cp.async
        # block tiles with 16 / 8 values per thread, 6 / 7 those one CTA per SM
        # middle pass (bits 2 and, at 2n = 1024 / 2048, 4): the same bits of vt; at 2n = 8192
        # bit 4 takes the block-synchronous line kernel instead of the four-step pass, and for
        # 8192-point columns (P5) the staged block kernel instead of the four-step through HBM;
        # 8 / 10: the second radix split (8 x 16, 8 x 8 x 4, 8 x 8 x 8 at 2n = 128, 256, 512) in
        # the TMA tiles and the middle pass, and 1024-point middle lines as two 512-point
        # halves, alone and one CTA per SM
        for vt, vp in [(0, 0), (2, 2), (4, 4), (5, 4), (6, 6), (7, 6), (8, 8), (10, 10)]:
            _write_cache(path, arch, shape, vt, vp)
            plan.autotune(path, 0)
            assert fsp.tuned_variant("p1_fwd", 2 * shape[0]) == vt
            assert fsp.tuned_variant("p3_fwd", 2 * shape[-1]) == vp
            phi, E = plan.solve(rho)
            assert rel(phi.cpu(), p_ref) <= TOL and rel(E.cpu(), E_ref) <= TOL, (vt, vp)
    finally:
        _write_cache(path, arch, shape, 0, 0)
        plan.autotune(path, 0)


def test_autotune_measures_and_writes_cache(fsp, tmp_path):
    import json
    shape, h = (64, 64, 64), (0.02, 0.02, 0.02)
    plan = fsp.Plan(shape, h, "vgf")
    rho = torch.from_numpy(_mixture(shape, h, seed=62).rho(np.float32)).cuda()
    phi0, E0 = plan.solve(rho)
    path = tmp_path / "tune.json"
    plan.autotune(path, 2)
    data = json.load(open(path))
    (arch, entries), = data.items()
    assert arch.startswith("sm_")
    assert set(entries) == {"p1_fwd/128", "p2_fwd/128", "p3_fwd/128", "p4_fwd/128", "p5_fwd/128"}
    phi1, E1 = plan.solve(rho)
    assert rel(phi1.cpu(), phi0.cpu()) <= TOL and rel(E1.cpu(), E0.cpu()) <= TOL
    # reset the process-wide table for the remaining tests
    for k in entries:
        entries[k] = 0
    json.dump({arch: entries}, open(path, "w"))
    plan.autotune(path, 0)


# ------------------------------------------------------------ plane groups

@pytest.mark.parametrize("shape,h,groups", [((64, 64, 64), (0.02, 0.02, 0.02), (1, 5, 16, 64)),
                                            ((96, 128, 256), (0.01, 0.015, 0.007), (7, 32))])
def test_plane_groups_give_the_same_bits(fsp, shape, h, groups):
    """The middle passes run group by group over the k0 planes: identical results, clean status."""
    plan = fsp.Plan(shape, h, "vgf")
    rho = torch.from_numpy(_mixture(shape, h, seed=91).rho(np.float32)).cuda()
    phi0, E0 = plan.solve(rho)
    phi_only0, _ = plan.solve(rho, with_E=False)
    for g in groups:
        plan.set_plane_group(g)
        phi, E = plan.solve(rho)
        ph1, _ = plan.solve(rho, with_E=False)
        torch.cuda.synchronize()
        assert torch.equal(phi, phi0) and torch.equal(E, E0), g
        assert torch.equal(ph1, phi_only0), g
    plan.set_plane_group(0)
    assert plan.device_status() == 0


# ------------------------------------------------------- bounded device waits

def test_device_wait_gives_up_and_the_context_stays_usable(fsp):
    """A shared-memory barrier wait that can never complete gives up after its limit, records
    FSP_ERR_TIMEOUT and returns; solves on the same context still give the right answer."""
    import time
    lib = fsp.load()
    t = time.perf_counter()
    assert lib.fsp_selftest_wait_timeout(0.05) == 6   # FSP_ERR_TIMEOUT
    assert time.perf_counter() - t < 5.0
    assert lib.fsp_last_error() == 6
    assert lib.fsp_selftest_wait_timeout(0.0) == 1
    shape, h = (32, 32, 32), (2 / 32,) * 3
    plan = fsp.Plan(shape, h, "vgf")
    rho = torch.from_numpy(_mixture(shape, h, seed=3).rho(np.float32)).cuda()
    phi, E = plan.solve(rho)
    phi2, E2 = plan.solve(rho)
    torch.cuda.synchronize()
    assert torch.equal(phi, phi2) and torch.isfinite(E).all()
    assert plan.device_status() == 0


# ------------------------------------------------------------ edge cases

@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("name,shape,h", [SMALL[1], SMALL[3]])
def test_zero_density_gives_zero(fsp, name, shape, h, direct):
    """rho = 0: every output is exactly zero (no stale workspace contents leak in)."""
    plan = fsp.Plan(shape, h, "vgf", direct=direct)
    plan.solve(torch.from_numpy(_mixture(shape, h, 5).rho(np.float32)).cuda())   # dirty the workspace first
    phi, E = plan.solve(torch.zeros(shape, device="cuda"))
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(phi)) == 0 and int(torch.count_nonzero(E)) == 0


@pytest.mark.parametrize("method", ["vgf", "he"])
@pytest.mark.parametrize("name,shape,h,cell", [("cube32", (32, 32, 32), (2 / 32,) * 3, (5, 17, 30)),
                                               ("aniso", (32, 64, 96), (0.03, 0.02, 0.011), (31, 0, 40)),
                                               ("2d", (64, 128), (0.02, 0.011), (10, 127))])
def test_point_charge_reproduces_the_kernel(fsp, oracle_mod, method, name, shape, h, cell):
    """A unit point charge (rho = 1 / prod(h) at one cell) gives phi_i = g(x_i - x_c): the
    oracle's real-space kernel itself, read by offset -- no oracle FFT is involved."""
    rho = np.zeros(shape, dtype=np.float32)
    rho[cell] = 1.0 / np.prod(h)
    phi, _ = fsp.Plan(shape, h, method).solve(torch.from_numpy(rho).cuda(), with_E=False)
    g = oracle_mod.kernel(method, list(shape), h)
    idx = np.ix_(*[(np.arange(n) - c) % (2 * n) for n, c in zip(shape, cell)])
    assert rel(phi.cpu(), g[idx]) <= TOL


@pytest.mark.parametrize("dtype,tol", [("f32", TOL), ("f64", 1e-11)])
@pytest.mark.parametrize("shape,h", [((1, 1, 1), (0.1, 0.2, 0.3)), ((1, 5, 2), (0.1, 0.05, 0.2)),
                                     ((3, 1), (0.1, 0.3)), ((2, 2), (0.2, 0.2))])
def test_degenerate_sizes(fsp, oracle_mod, shape, h, dtype, tol):
    """One or two cells per axis (padded lengths 2 and 4) through the direct-sum path."""
    rng = np.random.default_rng(11)
    np_dt = np.float32 if dtype == "f32" else np.float64
    rho = rng.standard_normal(shape).astype(np_dt)
    phi, E = fsp.Plan(shape, h, "vgf", dtype=dtype).solve(torch.from_numpy(rho).cuda())
    p_ref, E_ref = oracle_mod.solve_with_kernel(oracle_mod.kernel_vgf(list(shape), h), rho.astype(np.float64), h)
    assert rel(phi.cpu(), p_ref) <= tol
    if np.max(np.abs(E_ref)) > 0:
        assert np.max(np.abs(E.cpu().numpy() - E_ref)) <= tol * max(np.max(np.abs(E_ref)), np.max(np.abs(p_ref)))


def test_largest_3d_axes_sampled(fsp, oracle_mod):
    """2n = 1024 on the first two axes (the largest 3D passes: column tiles of 1024 points on
    axes 0 and 1): HE phi at 32 sampled cells against the brute-force sum."""
    shape, h = (512, 512, 32), (1 / 256, 1 / 256, 1 / 16)
    prob = _mixture(shape, h, seed=12)
    _, rho32, phi, E = gpu_solve(fsp, prob, "he")
    g = oracle_mod.kernel_he(list(shape), h)
    pts = np.random.default_rng(13).integers(0, phi.size, size=32)
    ref = oracle_mod.direct_phi_at(g, rho32.astype(np.float64), h, pts)
    assert np.max(np.abs(phi.ravel()[pts] - ref)) <= TOL * np.max(np.abs(phi))
    assert np.all(np.isfinite(E))


# ------------------------------------------------------------ full sizes

def test_full_size_256_vgf_against_oracle(fsp, oracle_mod):
    """The 256^3 FP32 mixture (8 anisotropic Gaussians, seed 1) against the FP64 oracle, every cell."""
    prob = W.mixture_3d(256, 8, 1)
    plan, rho32, phi, E = gpu_solve(fsp, prob, "vgf")
    g = oracle_mod.kernel_vgf(list(prob.shape), prob.h)
    K = plan.kernel_spectrum().astype(np.float64)
    ref_K = oracle_mod.scaled_spectrum_octant(g, prob.h)
    assert np.all(np.abs(K - ref_K) <= 2 ** -23 * np.abs(ref_K) + 1e-12 * np.max(np.abs(ref_K)))
    p_ref, E_ref = oracle_mod.solve_with_kernel(g, rho32.astype(np.float64), prob.h)
    assert rel(phi, p_ref) <= TOL
    assert rel(E, E_ref) <= TOL


def test_full_size_256_he_sampled(fsp, oracle_mod):
    """HE at 256^3: phi at 48 sampled cells against the brute-force sum."""
    prob = W.mixture_3d(256, 8, 1)
    _, rho32, phi, _ = gpu_solve(fsp, prob, "he", with_E=False)
    g = oracle_mod.kernel_he(list(prob.shape), prob.h)
    pts = np.random.default_rng(7).integers(0, phi.size, size=48)
    ref = oracle_mod.direct_phi_at(g, rho32.astype(np.float64), prob.h, pts)
    assert np.max(np.abs(phi.ravel()[pts] - ref)) <= TOL * np.max(np.abs(phi))


def test_full_size_2d_closed_form(fsp):
    """4096^2 mixture of 16 isotropic Gaussians: VGF vs the E1 closed form at every cell."""
    prob = W.mixture_2d(4096, 16, 2)
    _, _, phi, E = gpu_solve(fsp, prob, "vgf")
    pts = W.grid_points(prob.shape, prob.h)
    sl = (slice(None, None, 7), slice(None, None, 5))
    pex, Eex = A.mixture_field(pts[sl], prob.gaussians, 2)
    assert rel(phi[sl], pex) < 2e-5
    assert rel(E[(slice(None),) + sl], Eex) < 2e-5


def test_full_size_linearity_and_translation(fsp):
    """Properties at 256^3 that hold at any size: linearity, whole-cell translation."""
    prob = W.mixture_3d(256, 8, 1)
    plan = fsp.Plan(prob.shape, prob.h, "vgf")
    rho = torch.from_numpy(prob.rho(np.float32)).cuda()
    phi, E = plan.solve(rho)
    phi2, E2 = plan.solve(2.0 * rho)
    assert rel((phi2 / 2).cpu(), phi.cpu()) <= 1e-6
    comp = torch.zeros_like(rho)
    comp[40:120, 60:140, 30:110] = rho[40:120, 60:140, 30:110]
    pa, Ea = plan.solve(comp)
    pb, Eb = plan.solve(torch.roll(comp, shifts=(17, -9, 23), dims=(0, 1, 2)))
    assert rel(pb[17:, :-9, 23:].cpu(), pa[:-17, 9:, :-23].cpu()) <= 2e-6
    assert rel(Eb[:, 17:, :-9, 23:].cpu(), Ea[:, :-17, 9:, :-23].cpu()) <= 2e-6
