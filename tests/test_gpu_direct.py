"""GPU parity of the direct-sum path (any grid size, FP32 or FP64) against the FP64 oracle.

Sizes the FFT passes do not cover -- the paper's convergence studies use
N = 10 ... 100 per axis (Sec. 3), so 2N with factors 11, 13, 17, 19 -- and FP64
plans run the direct-sum path.  Tolerances: FP32 relative L-inf <= 1e-5 (the
pipeline's target); FP64 relative L-inf <= 1e-11: both sides compute the same
discrete convolution in FP64, the direct sums accumulate O(N) terms of
rounding ~1e-16 each, far below it.
"""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import analytic as A

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-11


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


def _mixture(shape, h, seed, count=3):
    rng = np.random.default_rng(seed)
    side = [n * hh for n, hh in zip(shape, h)]
    gs = []
    for _ in range(count):
        c = np.array([rng.uniform(-0.25, 0.25) * s for s in side])
        sig = np.array([rng.uniform(0.06, 0.12) * s for s in side])
        gs.append((c, sig, rng.uniform(-1, 1)))
    return W.Problem("mix", shape, h, gs)


ODD = [
    ("p13x17x11", (13, 17, 11), (0.05, 0.04, 0.06)),    # 2n = 26, 34, 22
    ("p10x19x7", (10, 19, 7), (0.07, 0.03, 0.08)),      # 2n = 20, 38, 14 (odd contiguous n)
    ("2d_p19x23", (19, 23), (0.05, 0.045)),              # 2n = 38, 46
    ("2d_p50x37", (50, 37), (0.02, 0.03)),               # 2n = 100, 74
]


def _oracle(oracle_mod, method, shape, h, rho64):
    g = oracle_mod.kernel(method, list(shape), h)
    return oracle_mod.solve_with_kernel(g, rho64, h)


@pytest.mark.parametrize("dtype,tol", [("f32", TOL32), ("f64", TOL64)])
@pytest.mark.parametrize("method", ["vgf", "he"])
@pytest.mark.parametrize("name,shape,h", ODD)
def test_direct_odd_sizes_match_oracle(fsp, oracle_mod, name, shape, h, method, dtype, tol):
    prob = _mixture(shape, h, seed=91)
    np_dt = np.float32 if dtype == "f32" else np.float64
    rho = prob.rho(np_dt)
    plan = fsp.Plan(shape, h, method, dtype=dtype)
    phi, E = plan.solve(torch.from_numpy(rho).cuda())
    torch.cuda.synchronize()
    assert phi.dtype == plan.dtype and E.dtype == plan.dtype
    p_ref, E_ref = _oracle(oracle_mod, method, shape, h, rho.astype(np.float64))
    assert rel(phi.cpu(), p_ref) <= tol
    assert rel(E.cpu(), E_ref) <= tol


@pytest.mark.parametrize("name,shape,h", [("cube32", (32, 32, 32), (2 / 32,) * 3), ("2d", (64, 128), (0.02, 0.011))])
def test_direct_path_equals_fft_passes(fsp, name, shape, h):
    """The direct sums and the FFT passes compute the same FP32 solve on a covered size."""
    prob = _mixture(shape, h, seed=92)
    rho = torch.from_numpy(prob.rho(np.float32)).cuda()
    p_fast, E_fast = fsp.Plan(shape, h, "vgf").solve(rho)
    p_dir, E_dir = fsp.Plan(shape, h, "vgf", direct=True).solve(rho)
    torch.cuda.synchronize()
    assert rel(p_dir.cpu(), p_fast.cpu()) <= 2e-6
    assert rel(E_dir.cpu(), E_fast.cpu()) <= 2e-6


@pytest.mark.parametrize("name,shape,h", [("cube32", (32, 32, 32), (2 / 32,) * 3), ("2d", (64, 128), (0.02, 0.011))])
def test_f64_on_covered_sizes(fsp, oracle_mod, name, shape, h):
    prob = _mixture(shape, h, seed=93)
    rho = prob.rho(np.float64)
    phi, E = fsp.Plan(shape, h, "vgf", dtype="f64").solve(torch.from_numpy(rho).cuda())
    p_ref, E_ref = _oracle(oracle_mod, "vgf", shape, h, rho)
    assert rel(phi.cpu(), p_ref) <= TOL64
    assert rel(E.cpu(), E_ref) <= TOL64


@pytest.mark.parametrize("dtype,tol", [("f32", TOL32), ("f64", TOL64)])
@pytest.mark.parametrize("name,shape,h", [ODD[0], ODD[2]])
def test_direct_adjoint_matches_oracle(fsp, oracle_mod, name, shape, h, dtype, tol):
    rng = np.random.default_rng(94)
    np_dt = np.float32 if dtype == "f32" else np.float64
    d = len(shape)
    g_phi = rng.standard_normal(shape).astype(np_dt)
    g_E = rng.standard_normal((d,) + shape).astype(np_dt)
    plan = fsp.Plan(shape, h, "vgf", dtype=dtype)
    g = plan.adjoint(torch.from_numpy(g_phi).cuda(), torch.from_numpy(g_E).cuda())
    ref = oracle_mod.adjoint_with_kernel(oracle_mod.kernel_vgf(list(shape), h), g_phi.astype(np.float64),
                                         g_E.astype(np.float64), h)
    assert rel(g.cpu(), ref) <= tol
    # potential-only and field-only adjoints
    g1 = plan.adjoint(torch.from_numpy(g_phi).cuda(), None)
    ref1 = oracle_mod.adjoint_with_kernel(oracle_mod.kernel_vgf(list(shape), h), g_phi.astype(np.float64), None, h)
    assert rel(g1.cpu(), ref1) <= tol
    g2 = plan.adjoint(None, torch.from_numpy(g_E).cuda())
    ref2 = oracle_mod.adjoint_with_kernel(oracle_mod.kernel_vgf(list(shape), h), None, g_E.astype(np.float64), h)
    assert rel(g2.cpu(), ref2) <= tol


def test_f64_adjoint_dot_product_identity(fsp):
    """<(phi, E)(rho), (g_phi, g_E)> = <rho, adjoint(g_phi, g_E)> in FP64 on an odd grid."""
    shape, h = (11, 14, 9), (0.06, 0.05, 0.07)
    rng = np.random.default_rng(95)
    rho = torch.from_numpy(rng.standard_normal(shape)).cuda()
    g_phi = torch.from_numpy(rng.standard_normal(shape)).cuda()
    g_E = torch.from_numpy(rng.standard_normal((3,) + shape)).cuda()
    plan = fsp.Plan(shape, h, "vgf", dtype="f64")
    phi, E = plan.solve(rho)
    lhs = float((phi * g_phi).sum() + (E * g_E).sum())
    rhs = float((rho * plan.adjoint(g_phi, g_E)).sum())
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_direct_batch_mixes_paths(fsp):
    """A batch holding FFT-pass plans and direct-path plans equals their single solves."""
    cases = [((32, 32, 32), (0.03,) * 3, {}), ((13, 17, 11), (0.05, 0.04, 0.06), {}),
             ((64, 32, 32), (0.01, 0.03, 0.02), {}), ((10, 12, 14), (0.05,) * 3, {"direct": True})]
    plans = [fsp.Plan(s, h, "vgf", **kw) for s, h, kw in cases]
    rhos = [torch.from_numpy(_mixture(s, h, 96 + i).rho(np.float32)).cuda() for i, (s, h, _) in enumerate(cases)]
    phis, Es = fsp.solve_batched(plans, rhos)
    b = fsp.Batch(plans, rhos)
    b.capture()
    b.graph.replay()
    torch.cuda.synchronize()
    for p, r, ph, E, ph2, E2 in zip(plans, rhos, phis, Es, b.phis, b.Es):
        ph1, E1 = p.solve(r)
        assert torch.equal(ph, ph1) and torch.equal(E, E1)
        assert torch.equal(ph2, ph1) and torch.equal(E2, E1)


def test_f64_fd_gradient_matches_oracle(fsp, oracle_mod):
    shape, h = (13, 17, 11), (0.05, 0.04, 0.06)
    prob = _mixture(shape, h, seed=97)
    plan = fsp.Plan(shape, h, "he", dtype="f64")
    phi, _ = plan.solve(torch.from_numpy(prob.rho(np.float64)).cuda(), with_E=False)
    E = plan.gradient_fd(phi)
    ref = oracle_mod.fd_gradient(phi.cpu().numpy(), h)
    assert rel(E.cpu(), ref) <= 1e-14


def test_f64_autograd_through_direct_path(fsp):
    shape, h = (9, 10, 11), (0.07, 0.06, 0.05)
    rng = np.random.default_rng(98)
    plan = fsp.Plan(shape, h, "vgf", dtype="f64")
    rho = torch.from_numpy(rng.standard_normal(shape)).cuda().requires_grad_(True)
    w_phi = torch.from_numpy(rng.standard_normal(shape)).cuda()
    w_E = torch.from_numpy(rng.standard_normal((3,) + shape)).cuda()
    phi, E = fsp.FspSolve.apply(rho, plan)
    loss = (phi * w_phi).sum() + (E * w_E).sum()
    loss.backward()
    # the map is linear: the gradient is the adjoint applied to the weights
    ref = plan.adjoint(w_phi, w_E)
    assert torch.allclose(rho.grad, ref, rtol=0, atol=1e-14 * float(ref.abs().max()))


# ------------------------------------------------- the paper's convergence study

def _unit_gaussian_error(fsp, method, n, sigma=0.05, side=1.0):
    """Relative L-inf error of the FP64 GPU phi against the erf potential of a unit Gaussian."""
    prob = W.unit_gaussian_3d(n, sigma, side)
    plan = fsp.Plan(prob.shape, prob.h, method, dtype="f64")
    phi, _ = plan.solve(torch.from_numpy(prob.rho(np.float64)).cuda(), with_E=False)
    pts = W.grid_points(prob.shape, prob.h)
    r = np.sqrt(np.sum(pts * pts, axis=-1))
    return rel(phi.cpu(), A.phi_gauss3_iso(r, sigma))


def test_f64_vgf_converges_spectrally_he_like_h2(fsp):
    """The paper's 3D convergence study on the GPU in FP64 (Sec. 3), at sizes only the direct
    path covers (2n = 24, 48, 96): HE's error falls like h^2 (Sec. 1), VGF's spectrally (Sec. 2)."""
    err = {(m, n): _unit_gaussian_error(fsp, m, n) for m in ("he", "vgf") for n in (12, 24, 48)}
    slope = math.log2(err[("he", 24)] / err[("he", 48)])
    assert 1.5 < slope < 2.5
    assert err[("vgf", 24)] / err[("vgf", 48)] > 1e3
    assert err[("vgf", 48)] < 1e-6
    for n in (12, 24, 48):
        assert err[("vgf", n)] < err[("he", n)]


def test_direct_plan_rejects_pass_events(fsp):
    """Per-pass timing events belong to the FFT passes; a direct-path plan refuses them."""
    plan = fsp.Plan((13, 17, 11), (0.05, 0.04, 0.06), "vgf")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in evs:
        e.record()
    with pytest.raises(fsp.FspError):
        plan.set_pass_events(evs)


_DEBUG_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_2103_08531_gb300 import _lib, build
_lib.load(build.DEBUG_LIB)                      # every call below goes to the bounds-checked build
import paper_2103_08531_gb300 as fsp
import oracle, workloads as W
worst = 0.0
for shape, h in (((32, 64, 96), (0.03, 0.02, 0.011)), ((64, 128), (0.02, 0.011)), ((16, 48, 192), (0.05, 0.03, 0.01)),
                 ((13, 17, 11), (0.05, 0.04, 0.06))):
    prob = W.Problem("d", shape, h, [(np.zeros(len(shape)), np.array([0.1 * n * x for n, x in zip(shape, h)]), 1.0)])
    rho32 = prob.rho(np.float32)
    plan = fsp.Plan(shape, h, "vgf")
    phi, E = plan.solve(torch.from_numpy(rho32).cuda())
    g = plan.adjoint(phi, E)
    torch.cuda.synchronize()
    assert plan.device_status() == 0, shape
    k = oracle.kernel_vgf(list(shape), h)
    p_ref, E_ref = oracle.solve_with_kernel(k, rho32.astype(np.float64), h)
    worst = max(worst, float(np.max(np.abs(phi.cpu().numpy() - p_ref)) / np.max(np.abs(p_ref))))
print("ok", worst)
"""


@pytest.mark.slow
def test_debug_bounds_build_reports_no_bad_index(fsp):
    """The FSP_DEBUG_BOUNDS build (every intermediate and grid index checked against its buffer)
    runs solves and adjoints of 3D, 2D, new-length and direct-path plans with a clean device
    status and the oracle's answer; it runs in a child process that loads only that build."""
    import os
    import subprocess
    import sys
    from paper_2103_08531_gb300 import build
    build.build(debug_bounds=True)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _DEBUG_SCRIPT.format(root=root)], capture_output=True, text=True,
                         timeout=600)
    assert res.returncode == 0, res.stderr[-3000:]
    assert res.stdout.startswith("ok")
    assert float(res.stdout.split()[1]) <= 1e-5
