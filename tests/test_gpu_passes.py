"""Each FFT pass against the oracle's intermediate of the padded convolution.

The end-to-end parity tests check phi and E; these check every pass on its
own.  fsp_plan_run_passes stops a forward solve after pass k, and the two
intermediate buffers of the workspace are compared with the same stage of the
convolution of Sec. 1 (HE formula) taken one axis at a time with the oracle's
own FFT: zero padding and a forward transform along axis 0 (half spectrum),
along axis 1, along axis 2 with the product by the kernel spectrum (and
-i k_2 for E), the inverse along axis 2 with the crop, the inverse along axis
1 with the crop (and -i k_1).  Tolerance: relative L-inf <= 1e-5 per buffer,
as for phi and E.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fsp():
    from paper_2103_08531_gb300 import build
    build.build()
    import paper_2103_08531_gb300 as pkg
    pkg.load()
    return pkg


def rel(x, ref):
    x = np.asarray(x, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def _density(shape, h, seed):
    rng = np.random.default_rng(seed)
    side = [n * hh for n, hh in zip(shape, h)]
    gs = [(np.array([rng.uniform(-0.25, 0.25) * s for s in side]),
           np.array([rng.uniform(0.06, 0.12) * s for s in side]), rng.uniform(-1, 1)) for _ in range(3)]
    return W.Problem("mix", shape, h, gs).rho(np.float32)


def _fft_axis(oracle_mod, a, axis, sign):
    return np.apply_along_axis(lambda v: oracle_mod.fft(v, sign), axis, a)


def _wave(n, h):
    """-i k multipliers' k for indices 0 .. 2n-1: 2 pi m / (2 n h), m in [-n, n), 0 at m = -n."""
    k = np.arange(2 * n)
    m = np.where(k < n, k, np.where(k == n, 0, k - 2 * n))
    return 2 * np.pi * m / (2 * n * h)


def _fold(n):
    k = np.arange(2 * n)
    return np.where(k <= n, k, 2 * n - k)


def _stages_3d(oracle_mod, rho, h, Koct):
    """The convolution's intermediates after each of the first four passes (3D)."""
    n0, n1, n2 = rho.shape
    f = lambda a, ax, s: _fft_axis(oracle_mod, a, ax, s)
    P = np.zeros((2 * n0, n1, n2))
    P[:n0] = rho
    Z1 = f(P, 0, -1)[:n0 + 1]
    Q = np.zeros((n0 + 1, 2 * n1, n2), dtype=np.complex128)
    Q[:, :n1] = Z1
    Y1 = f(Q, 1, -1)
    R = np.zeros((n0 + 1, 2 * n1, 2 * n2), dtype=np.complex128)
    R[..., :n2] = Y1
    K = Koct[:, _fold(n1)][:, :, _fold(n2)]
    X = f(R, 2, -1) * K
    k2 = _wave(n2, h[2])[None, None, :]
    S_phi = f(X, 2, 1)[..., :n2]
    S_e2 = f(-1j * k2 * X, 2, 1)[..., :n2]
    k1 = _wave(n1, h[1])[None, :, None]
    T_phi = f(S_phi, 1, 1)[:, :n1]
    T_e1 = f(-1j * k1 * S_phi, 1, 1)[:, :n1]
    T_e2 = f(S_e2, 1, 1)[:, :n1]
    return Z1, Y1, (S_phi, S_e2), (T_phi, T_e1, T_e2)


def _stages_2d(oracle_mod, rho, h, Koct):
    n0, n2 = rho.shape
    f = lambda a, ax, s: _fft_axis(oracle_mod, a, ax, s)
    P = np.zeros((2 * n0, n2))
    P[:n0] = rho
    Z1 = f(P, 0, -1)[:n0 + 1]
    R = np.zeros((n0 + 1, 2 * n2), dtype=np.complex128)
    R[:, :n2] = Z1
    X = f(R, 1, -1) * Koct[:, _fold(n2)]
    k2 = _wave(n2, h[1])[None, :]
    return Z1, (f(X, 1, 1)[:, :n2], f(-1j * k2 * X, 1, 1)[:, :n2])


def _buffers(plan, rho, passes, with_E=True):
    b0, b1 = plan.intermediates(torch.from_numpy(rho).cuda(), passes, with_E)
    torch.cuda.synchronize()
    return b0.cpu().numpy(), b1.cpu().numpy()


@pytest.mark.parametrize("shape,h", [((32, 16, 32), (0.02, 0.03, 0.025)), ((48, 32, 96), (0.03, 0.02, 0.011))])
def test_each_3d_pass_matches_the_oracle_stage(fsp, oracle_mod, shape, h):
    rho = _density(shape, h, seed=91)
    plan = fsp.Plan(shape, h, "vgf")
    Koct = oracle_mod.scaled_spectrum_octant(oracle_mod.kernel_vgf(list(shape), h), h)
    Z1, Y1, (S_phi, S_e2), (T_phi, T_e1, T_e2) = _stages_3d(oracle_mod, rho.astype(np.float64), h, Koct)
    n1 = shape[1]
    b0, b1 = _buffers(plan, rho, 1)
    assert rel(b1[:, :n1], Z1) <= TOL                      # P1: axis-0 half spectrum in buf1
    b0, b1 = _buffers(plan, rho, 2)
    assert rel(b0, Y1) <= TOL                              # P2: axis-1 spectrum in buf0
    b0, b1 = _buffers(plan, rho, 3)
    assert rel(b0, S_phi) <= TOL and rel(b1, S_e2) <= TOL  # P3: phi and -i k2 streams
    b0, b1 = _buffers(plan, rho, 4)
    assert rel(b0[:, :n1], T_phi) <= TOL                   # P4: phi, -i k1 and -i k2 streams
    assert rel(b0[:, n1:], T_e1) <= TOL
    assert rel(b1[:, :n1], T_e2) <= TOL
    b0, _ = _buffers(plan, rho, 3, with_E=False)           # phi only: the same phi stream
    assert rel(b0, S_phi) <= TOL


@pytest.mark.parametrize("shape,h", [((64, 64), (0.02, 0.015)), ((64, 96), (0.015, 0.02))])
def test_each_2d_pass_matches_the_oracle_stage(fsp, oracle_mod, shape, h):
    rho = _density(shape, h, seed=92)
    plan = fsp.Plan(shape, h, "vgf")
    Koct = oracle_mod.scaled_spectrum_octant(oracle_mod.kernel_vgf(list(shape), h), h)
    Z1, (S_phi, S_e) = _stages_2d(oracle_mod, rho.astype(np.float64), h, Koct)
    b0, _ = _buffers(plan, rho, 1)
    assert rel(b0[:, 0], Z1) <= TOL
    b0, b1 = _buffers(plan, rho, 2)
    assert rel(b0[:, 0], S_phi) <= TOL and rel(b1[:, 0], S_e) <= TOL


def test_run_passes_rejects_bad_arguments(fsp):
    plan = fsp.Plan((32, 16, 32), (0.02, 0.03, 0.025), "vgf")
    rho = torch.zeros((32, 16, 32), device="cuda")
    for bad in (0, 5):
        with pytest.raises(fsp.FspError):
            plan.intermediates(rho, bad)
    direct = fsp.Plan((13, 17, 11), (0.05, 0.04, 0.06), "vgf", dtype="f64")
    with pytest.raises(fsp.FspError):
        direct.intermediates(torch.zeros((13, 17, 11), dtype=torch.float64, device="cuda"), 1)
