"""Python face of the solver: plans, solves, adjoints, batches, autograd.

Argument marshalling only: every step of a solve runs in libfsp.so's CUDA
kernels on the caller's current torch stream.  PyTorch provides device memory
(outputs and the plan workspace) and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import _lib

METHODS = {"he": _lib.FSP_HE, "vgf": _lib.FSP_VGF, "he_nearby": _lib.FSP_HE_NEARBY,
           "he_cellavg": _lib.FSP_HE_CELLAVG}


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


DTYPES = {"f32": (_lib.FSP_F32, torch.float32), "f64": (_lib.FSP_F64, torch.float64)}


class Plan:
    """One grid geometry: shape (nx, ny[, nz]) cells of spacing h, method 'vgf' or 'he'.

    Creating it runs the FP64 kernel precomputation on the current CUDA device
    and allocates the plan's workspace with torch.  dtype 'f32' or 'f64' sets
    the precision of the grids the plan takes and returns; direct=True runs
    the direct-sum path even where the FFT passes cover the size (sizes they
    do not cover, and every 'f64' plan, run it anyway).
    """

    def __init__(self, shape, h, method: str = "vgf", lam: float = 1.0, g0: float | None = None,
                 device=None, dtype: str = "f32", direct: bool = False):
        self.lib = _lib.load()
        shape = tuple(int(s) for s in shape)
        h = tuple(float(x) for x in (h if np.ndim(h) else [h] * len(shape)))
        if len(shape) not in (2, 3) or len(h) != len(shape):
            raise ValueError("shape/h must have 2 or 3 entries")
        if dtype not in DTYPES:
            raise ValueError("dtype must be 'f32' or 'f64'")
        self.shape, self.h, self.method, self.dim = shape, h, method, len(shape)
        self.dtype_name = dtype
        self.dtype = DTYPES[dtype][1]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        nz = shape[2] if self.dim == 3 else 0
        hz = h[2] if self.dim == 3 else 0.0
        with torch.cuda.device(self.device):
            handle = self.lib.fsp_plan_create_ex(shape[0], shape[1], nz, h[0], h[1], hz, METHODS[method],
                                                 DTYPES[dtype][0], float(lam), float("nan") if g0 is None else g0,
                                                 _lib.FSP_PLAN_DIRECT if direct else 0)
            if not handle:
                raise _lib.FspError(self.lib.fsp_last_error(), f"fsp_plan_create{shape}")
            self.handle = ctypes.c_void_p(handle)
            nbytes = self.lib.fsp_plan_workspace_bytes(self.handle, 1, 1)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            _lib.check(self.lib.fsp_plan_set_workspace(self.handle, _ptr(self.workspace), nbytes),
                       "fsp_plan_set_workspace")
            mode = os.environ.get("FSP_AUTOTUNE", "off")
            if mode in ("cached", "full", "retune"):
                cache = os.environ.get("FSP_TUNE_CACHE") or os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                                        "tune_cache.json")
                self.autotune(cache, {"cached": 0, "full": 1, "retune": 2}[mode])

    def autotune(self, cache_path=None, mode: int = 1):
        """Pick launch variants for this plan's passes (see fsp_autotune in include/fsp.h)."""
        path = None if cache_path is None else str(cache_path).encode()
        with torch.cuda.device(self.device):
            _lib.check(self.lib.fsp_autotune(self.handle, path, int(mode)), "fsp_autotune")

    # ----------------------------------------------------------------- info
    def geometry(self) -> dict:
        dim = ctypes.c_int()
        n = (ctypes.c_int * 3)()
        h = (ctypes.c_double * 3)()
        L = ctypes.c_double()
        M = (ctypes.c_int * 3)()
        _lib.check(self.lib.fsp_plan_geometry(self.handle, ctypes.byref(dim), n, h, ctypes.byref(L), M),
                   "fsp_plan_geometry")
        d = dim.value
        return {"dim": d, "n": list(n)[:d], "h": list(h)[:d], "L": L.value, "M": list(M)[:d]}

    def kernel_spectrum(self) -> np.ndarray:
        """FP32 kernel octant [nx+1][ny+1][(nz+1)] with prod(h)/prod(2n) folded in."""
        shp = tuple(s + 1 for s in self.shape)
        out = np.empty(shp, dtype=np.float32)
        _lib.check(self.lib.fsp_plan_kernel_spectrum(self.handle, out.ctypes.data_as(ctypes.c_void_p), out.nbytes),
                   "fsp_plan_kernel_spectrum")
        return out

    def intermediates(self, rho, passes: int, with_E: bool = True):
        """Test hook: run the first `passes` forward passes on rho and return the
        workspace's two intermediate buffers as complex64 tensors [nx+1][rows][nz]
        (views of the workspace; see fsp_plan_run_passes in include/fsp.h)."""
        off = ctypes.c_size_t(0)
        dims = (ctypes.c_int * 3)()
        _lib.check(self.lib.fsp_plan_workspace_layout(self.handle, ctypes.byref(off), dims), "fsp_plan_workspace_layout")
        with torch.cuda.device(self.device):
            _lib.check(self.lib.fsp_plan_run_passes(self.handle, _ptr(rho), int(passes), int(with_E), _stream()),
                       "fsp_plan_run_passes")
        n = dims[0] * dims[1] * dims[2]
        shape = (dims[0], dims[1], dims[2])
        b0 = self.workspace[:8 * n].view(torch.complex64).view(shape)
        b1 = self.workspace[off.value:off.value + 8 * n].view(torch.complex64).view(shape)
        return b0, b1

    def set_plane_group(self, planes: int):
        """Run the middle passes of single 3D solves in groups of `planes` k0 planes (0: off)."""
        _lib.check(self.lib.fsp_plan_set_plane_group(self.handle, int(planes)), "fsp_plan_set_plane_group")

    def device_status(self, clear: bool = True) -> int:
        """Device-side status of earlier solves (0, or 6 = FSP_ERR_TIMEOUT); synchronises."""
        return int(self.lib.fsp_plan_device_status(self.handle, int(clear)))

    def set_pass_events(self, events):
        """Record the given torch.cuda.Event objects at the pass boundaries of later solves (None: off)."""
        if not events:
            _lib.check(self.lib.fsp_plan_set_pass_events(self.handle, None, 0), "fsp_plan_set_pass_events")
            return
        handles = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
        _lib.check(self.lib.fsp_plan_set_pass_events(self.handle, handles, len(events)), "fsp_plan_set_pass_events")

    @property
    def passes(self) -> int:
        return 5 if self.dim == 3 else 3

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))

    # ---------------------------------------------------------------- solve
    def _check_grid(self, t, name, lead=()):
        want = tuple(lead) + self.shape
        if t.dtype != self.dtype or not t.is_cuda or tuple(t.shape) != want or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor of shape {want}")

    def solve(self, rho, with_phi: bool = True, with_E: bool = True, phi=None, E=None, stream=None):
        """phi, E for density rho (CUDA tensor of the plan's shape and dtype)."""
        self._check_grid(rho, "rho")
        if phi is not None:
            self._check_grid(phi, "phi")
        if E is not None:
            self._check_grid(E, "E", (self.dim,))
        if with_phi and phi is None:
            phi = torch.empty_like(rho)
        if with_E and E is None:
            E = torch.empty((self.dim,) + self.shape, dtype=self.dtype, device=rho.device)
        _lib.check(self.lib.fsp_solve(self.handle, _ptr(rho), _ptr(phi if with_phi else None),
                                      _ptr(E if with_E else None), _stream(stream)), "fsp_solve")
        return (phi if with_phi else None), (E if with_E else None)

    __call__ = solve

    def gradient_fd(self, phi, E=None, stream=None):
        """E = -grad(phi) by centred differences (second-order one-sided at the faces)."""
        self._check_grid(phi, "phi")
        if E is None:
            E = torch.empty((self.dim,) + self.shape, dtype=self.dtype, device=phi.device)
        _lib.check(self.lib.fsp_gradient_fd(self.handle, _ptr(phi), _ptr(E), _stream(stream)), "fsp_gradient_fd")
        return E

    def adjoint(self, g_phi=None, g_E=None, g_rho=None, stream=None):
        """g_rho = A^T g_phi + sum_a B_a^T g_E[a] (either input may be None)."""
        if g_phi is None and g_E is None:
            raise ValueError("need g_phi or g_E")
        if g_phi is not None:
            self._check_grid(g_phi, "g_phi")
        if g_E is not None:
            self._check_grid(g_E, "g_E", (self.dim,))
        ref = g_phi if g_phi is not None else g_E
        if g_rho is None:
            g_rho = torch.empty(self.shape, dtype=self.dtype, device=ref.device)
        _lib.check(self.lib.fsp_solve_adjoint(self.handle, _ptr(g_phi), _ptr(g_E), _ptr(g_rho), _stream(stream)),
                   "fsp_solve_adjoint")
        return g_rho

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fsp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PASS_KINDS = ["p1_fwd", "p1_adj", "p2_fwd", "p2_adj", "p3_fwd", "p3_adj", "p4_fwd", "p5_fwd"]


def tuned_variant(kind: str, N: int) -> int:
    """Current autotuner choice for a pass at padded length N."""
    return _lib.load().fsp_tuned_variant(PASS_KINDS.index(kind), int(N))


def _arr(ptrs):
    return (ctypes.c_void_p * len(ptrs))(*[p.value if p is not None else None for p in ptrs])


def solve_batched(plans, rhos, with_phi: bool = True, with_E: bool = True, stream=None):
    """Independent solves over several plans (distinct plans, one workspace each)."""
    lib = _lib.load()
    phis = [torch.empty_like(r) if with_phi else None for r in rhos]
    Es = [torch.empty((p.dim,) + p.shape, dtype=p.dtype, device=r.device) if with_E else None
          for p, r in zip(plans, rhos)]
    for p, r in zip(plans, rhos):
        p._check_grid(r, "rho")
    hp = _arr([p.handle for p in plans])
    _lib.check(lib.fsp_solve_batched(hp, len(plans), _arr([_ptr(r) for r in rhos]),
                                     _arr([_ptr(x) for x in phis]) if with_phi else None,
                                     _arr([_ptr(x) for x in Es]) if with_E else None, _stream(stream)),
               "fsp_solve_batched")
    return phis, Es


class Batch:
    """Prebuilt batch of independent solves with fixed input/output tensors (graph friendly)."""

    def __init__(self, plans, rhos, with_phi: bool = True, with_E: bool = True):
        self.lib = _lib.load()
        self.plans, self.rhos = list(plans), list(rhos)
        self.phis = [torch.empty_like(r) if with_phi else None for r in self.rhos]
        self.Es = [torch.empty((p.dim,) + p.shape, dtype=p.dtype, device=r.device) if with_E else None
                   for p, r in zip(self.plans, self.rhos)]
        h = self.lib.fsp_batch_create(_arr([p.handle for p in self.plans]), len(self.plans),
                                      _arr([_ptr(r) for r in self.rhos]),
                                      _arr([_ptr(x) for x in self.phis]) if with_phi else None,
                                      _arr([_ptr(x) for x in self.Es]) if with_E else None)
        if not h:
            raise _lib.FspError(self.lib.fsp_last_error(), "fsp_batch_create")
        self.handle = ctypes.c_void_p(h)

    def run(self, stream=None):
        _lib.check(self.lib.fsp_batch_solve(self.handle, _stream(stream)), "fsp_batch_solve")
        return self.phis, self.Es

    def kernel_count(self) -> int:
        """Kernels one run() launches (counted on a captured graph; nothing runs)."""
        n = ctypes.c_int(0)
        _lib.check(self.lib.fsp_batch_kernel_count(self.handle, ctypes.byref(n)), "fsp_batch_kernel_count")
        return n.value

    def capture(self, warmup: int = 1):
        """Record run() into a torch.cuda.CUDAGraph; replay with graph.replay()."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fsp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HostPipeline:
    """Solves host-resident densities through the C ABI's host pipe (fsp_host_pipe_*).

    The library owns `depth` device buffer sets and three streams (copy-in,
    compute, copy-out): slot i % depth is copied in, solved on the plan's
    workspace, and copied back, so the transfers of neighbouring solves run
    under each other's kernels.  Host tensors should be pinned
    (torch.Tensor.pin_memory()) for the copies to overlap.
    """

    def __init__(self, plan: Plan, depth: int = 2, with_phi: bool = True, with_E: bool = True):
        self.lib = _lib.load()
        self.plan, self.depth, self.with_phi, self.with_E = plan, depth, with_phi, with_E
        with torch.cuda.device(plan.device):
            h = self.lib.fsp_host_pipe_create(plan.handle, int(depth), int(with_phi), int(with_E))
        if not h:
            raise _lib.FspError(self.lib.fsp_last_error(), "fsp_host_pipe_create")
        self.handle = ctypes.c_void_p(h)

    def _check_host(self, t, name, lead=()):
        want = tuple(lead) + self.plan.shape
        if t.is_cuda or t.dtype != self.plan.dtype or tuple(t.shape) != want or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host {self.plan.dtype} tensor of shape {want}")

    def run(self, rho_host, phi_host=None, E_host=None, stream=None):
        """rho_host: list of host tensors; phi_host / E_host: lists of host outputs.

        Asynchronous: returns once queued; the given (default: current) stream
        waits for the last copy-out.  Returns that stream."""
        n = len(rho_host)
        for r in rho_host:
            self._check_host(r, "rho")
        if self.with_phi:
            if phi_host is None or len(phi_host) != n:
                raise ValueError("phi_host: one output per input")
            for t in phi_host:
                self._check_host(t, "phi")
        if self.with_E:
            if E_host is None or len(E_host) != n:
                raise ValueError("E_host: one output per input")
            for t in E_host:
                self._check_host(t, "E", (self.plan.dim,))
        s = torch.cuda.current_stream(self.plan.device) if stream is None else stream
        _lib.check(self.lib.fsp_host_pipe_solve(self.handle, n, _arr([_ptr(r) for r in rho_host]),
                                                _arr([_ptr(t) for t in phi_host]) if self.with_phi else None,
                                                _arr([_ptr(t) for t in E_host]) if self.with_E else None,
                                                _stream(s)), "fsp_host_pipe_solve")
        self._keep = (rho_host, phi_host, E_host)   # host buffers stay referenced while queued
        return s

    def close(self):
        if getattr(self, "handle", None):
            self.lib.fsp_host_pipe_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FspSolve(torch.autograd.Function):
    """rho -> (phi, E) with the hand-written adjoint as backward.

    The map is linear; its transpose is g_rho = A g_phi - sum_a B_a g_E[a]
    (A symmetric, B_a antisymmetric), computed by fsp_solve_adjoint.
    """

    @staticmethod
    def forward(ctx, rho, plan):
        ctx.plan = plan
        phi, E = plan.solve(rho.contiguous())
        return phi, E

    @staticmethod
    def backward(ctx, g_phi, g_E):
        plan = ctx.plan
        if g_phi is None and g_E is None:
            return None, None
        g = plan.adjoint(None if g_phi is None else g_phi.contiguous(), None if g_E is None else g_E.contiguous())
        return g, None


def solve(rho, h, method: str = "vgf", with_E: bool = True):
    """One-shot convenience: build a plan for rho's shape and solve."""
    plan = Plan(tuple(rho.shape), h, method)
    return plan.solve(rho, with_E=with_E)
