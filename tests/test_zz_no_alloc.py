"""The workspace-free solve entry point (fsp_solve_noalloc), through the C ABI.

fsp_solve_noalloc exists for callers that cannot allocate device memory when
they solve (code running under a host framework's allocator, fixed-memory
real-time loops, paths that must not call cudaMalloc): it uses a static device
scratch array instead of a caller-provided workspace.  Its results must match
the ordinary entry point, fsp_solve, on consecutive calls that reuse the same
scratch.  This file is collected last so that a failing run stops after every
other test has run; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-5   # relative L-inf, as in the other GPU parity tests


def _rel(x, ref):
    x = x.double().cpu()
    ref = ref.double().cpu()
    return float((x - ref).abs().max() / ref.abs().max())


@pytest.fixture(scope="module")
def fsp():
    from paper_2103_08531_gb300 import build
    build.build()
    import paper_2103_08531_gb300 as pkg
    pkg.load()
    return pkg


def _noalloc(lib, plan, rho, phi, E):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fsp_solve_noalloc(plan.handle, ctypes.c_void_p(rho.data_ptr()),
                                 ctypes.c_void_p(phi.data_ptr()) if phi is not None else None,
                                 ctypes.c_void_p(E.data_ptr()) if E is not None else None, s)


@pytest.mark.parametrize("shape,h", [((64, 96, 32), (0.02, 0.015, 0.03)), ((128, 64), (0.01, 0.02))])
def test_noalloc_matches_fsp_solve_on_consecutive_calls(fsp, shape, h):
    lib = fsp.load()
    plan = fsp.Plan(shape, h, "vgf")
    rng = np.random.default_rng(77)
    d = len(shape)
    for call in range(2):
        rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        phi_ref, E_ref = plan.solve(rho)
        phi = torch.empty_like(rho)
        E = torch.empty((d,) + shape, dtype=torch.float32, device="cuda")
        assert _noalloc(lib, plan, rho, phi, E) == 0
        torch.cuda.synchronize()
        assert _rel(phi, phi_ref) <= TOL, call
        assert _rel(E, E_ref) <= TOL, call
    # phi only, then E only, reuse the same scratch
    phi2 = torch.empty_like(rho)
    assert _noalloc(lib, plan, rho, phi2, None) == 0
    E2 = torch.empty((d,) + shape, dtype=torch.float32, device="cuda")
    assert _noalloc(lib, plan, rho, None, E2) == 0
    torch.cuda.synchronize()
    assert _rel(phi2, phi_ref) <= TOL and _rel(E2, E_ref) <= TOL


def test_noalloc_at_the_documented_limit_128_cubed(fsp):
    # 128^3 is the largest cube whose workspace fits the 80 MiB scratch
    lib = fsp.load()
    shape, h = (128, 128, 128), (2 / 128,) * 3
    plan = fsp.Plan(shape, h, "vgf")
    assert lib.fsp_plan_workspace_bytes(plan.handle, 1, 1) <= 80 * 1024 * 1024
    rng = np.random.default_rng(5)
    for call in range(2):
        rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        phi_ref, E_ref = plan.solve(rho)
        phi = torch.empty_like(rho)
        E = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
        assert _noalloc(lib, plan, rho, phi, E) == 0
        assert lib.fsp_last_error() == 0
        torch.cuda.synchronize()
        assert _rel(phi, phi_ref) <= TOL, call
        assert _rel(E, E_ref) <= TOL, call


def test_noalloc_fp64_direct_plan(fsp):
    # FP64 plans run the direct-sum path; its workspace (in FP64) also lives in the scratch
    lib = fsp.load()
    shape, h = (13, 17, 11), (0.05, 0.04, 0.06)
    plan = fsp.Plan(shape, h, "vgf", dtype="f64")
    rng = np.random.default_rng(6)
    for call in range(2):
        rho = torch.from_numpy(rng.standard_normal(shape)).cuda()
        phi_ref, E_ref = plan.solve(rho)
        phi = torch.empty_like(rho)
        E = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, plan, rho, phi, E) == 0
        torch.cuda.synchronize()
        assert _rel(phi, phi_ref) <= 1e-12, call
        assert _rel(E, E_ref) <= 1e-12, call


def test_noalloc_call_allocates_no_device_memory(fsp):
    lib = fsp.load()
    shape, h = (64, 64, 64), (2 / 64,) * 3
    plan = fsp.Plan(shape, h, "he")
    rho = torch.from_numpy(np.random.default_rng(7).standard_normal(shape).astype(np.float32)).cuda()
    phi = torch.empty_like(rho)
    E = torch.empty((3,) + shape, dtype=torch.float32, device="cuda")
    assert _noalloc(lib, plan, rho, phi, E) == 0   # warm: the scratch address is looked up here
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert _noalloc(lib, plan, rho, phi, E) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_grids_beyond_the_scratch(fsp):
    lib = fsp.load()
    plan = fsp.Plan((256, 256, 256), (2 / 256,) * 3, "vgf")
    need = lib.fsp_plan_workspace_bytes(plan.handle, 1, 1)
    assert need > 80 * 1024 * 1024
    rho = torch.zeros((256, 256, 256), device="cuda")
    phi = torch.empty_like(rho)
    assert _noalloc(lib, plan, rho, phi, None) == 5   # FSP_ERR_WORKSPACE
    assert lib.fsp_last_error() == 5
    assert _noalloc(lib, plan, rho, None, None) == 1   # FSP_ERR_INVALID: no output
    assert lib.fsp_last_error() == 1
