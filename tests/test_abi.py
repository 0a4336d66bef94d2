"""Host-side checks of the C ABI: the library loads, exports every symbol that
include/fsp.h declares, and rejects bad arguments with the documented status
codes before touching a GPU."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_08531_gb300 import build, _lib
    build.build()
    return _lib.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "fsp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fsp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ("fsp_plan_create", "fsp_solve", "fsp_solve_batched", "fsp_solve_adjoint", "fsp_plan_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2103_08531_gb300 import _lib
    for name in header_symbols():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"


def test_error_strings(lib):
    for code in range(7):
        assert lib.fsp_error_string(code)
    assert lib.fsp_error_string(0) == b"ok"


@pytest.mark.parametrize("args,code", [
    ((-1, 32, 32, 0.1, 0.1, 0.1, 1, 0), 1),          # negative size
    ((32, 32, 32, 0.0, 0.1, 0.1, 1, 0), 1),          # zero spacing
    ((32, 32, 32, 0.1, 0.1, 0.1, 9, 0), 1),          # unknown method
    ((32, 32, 32, 0.1, 0.1, 0.1, 1, 7), 1),          # unknown dtype
    ((513, 32, 32, 0.1, 0.1, 0.1, 1, 0), 2),         # 2n = 1026: no FFT pass, beyond the direct path
    ((32, 32, 600, 0.1, 0.1, 0.1, 0, 1), 2),         # FP64 (direct path) beyond 512 cells
    ((1024, 32, 32, 0.1, 0.1, 0.1, 0, 0), 2),        # 3D axis beyond 2n = 1024
    ((4096, 4097, 0, 0.1, 0.1, 0.0, 1, 0), 2),       # 2D odd contiguous axis beyond the direct path
])
def test_plan_create_rejects(lib, args, code):
    assert lib.fsp_plan_create(*args) is None
    assert lib.fsp_last_error() == code


def test_plan_create_ex_rejects_unknown_flags(lib):
    assert lib.fsp_plan_create_ex(32, 32, 32, 0.1, 0.1, 0.1, 1, 0, 1.0, float("nan"), 2) is None
    assert lib.fsp_last_error() == 1


def test_null_arguments(lib):
    assert lib.fsp_solve(None, None, None, None, None) == 1
    assert lib.fsp_solve_adjoint(None, None, None, None, None) == 1
    assert lib.fsp_plan_set_workspace(None, None, 0) == 1
    assert lib.fsp_plan_kernel_spectrum(None, None, 0) == 1
    assert lib.fsp_plan_geometry(None, None, None, None, None, None) == 1
    assert lib.fsp_plan_workspace_bytes(None, 1, 1) == 0
    assert lib.fsp_solve_batched(None, 0, None, None, None, None) == 1
    assert lib.fsp_batch_create(None, 0, None, None, None) is None
    assert lib.fsp_batch_solve(None, None) == 1
    assert lib.fsp_host_pipe_create(None, 2, 1, 1) is None
    assert lib.fsp_last_error() == 1
    assert lib.fsp_host_pipe_solve(None, 0, None, None, None, None) == 1
    assert lib.fsp_solve_noalloc(None, None, None, None, None) == 1
    assert lib.fsp_gradient_fd(None, None, None, None) == 1
    assert lib.fsp_autotune(None, None, 0) == 1
    assert lib.fsp_selftest_wait_timeout(-1.0) == 1
    # every entry point leaves its status in fsp_last_error()
    lib.fsp_plan_create_ex(32, 32, 32, 0.1, 0.1, 0.1, 1, 0, 1.0, float("nan"), 2)
    assert lib.fsp_last_error() == 1
    assert lib.fsp_error_string(0) == b"ok"
    for call in (lambda: lib.fsp_solve_noalloc(None, None, None, None, None),
                 lambda: lib.fsp_gradient_fd(None, None, None, None),
                 lambda: lib.fsp_autotune(None, None, 0),
                 lambda: lib.fsp_host_pipe_solve(None, 0, None, None, None, None)):
        lib.fsp_plan_create(-1, 1, 1, 0.1, 0.1, 0.1, 0, 0)   # sets 1
        assert lib.fsp_plan_create(513, 32, 32, 0.1, 0.1, 0.1, 1, 0) is None and lib.fsp_last_error() == 2
        assert call() == 1 and lib.fsp_last_error() == 1
    lib.fsp_plan_destroy(None)
    lib.fsp_batch_destroy(None)
    lib.fsp_host_pipe_destroy(None)


def test_python_package_has_no_cpu_fallback():
    """The package loads the CUDA library and nothing else; it never imports the oracle."""
    import paper_2103_08531_gb300 as pkg
    src_dir = os.path.dirname(pkg.__file__)
    for fn in os.listdir(src_dir):
        if fn.endswith(".py"):
            text = open(os.path.join(src_dir, fn)).read()
            assert "oracle" not in text.replace("oracle_", ""), fn
            assert "torch.fft" not in text, fn


def test_fault_injection_fails_creation_on_the_host(lib, monkeypatch):
    """FSP_FAULT_INJECT=alloc makes plan creation fail as an allocation failure (FSP_ERR_NOMEM),
    before any GPU call; unset, the same arguments reach the device step."""
    monkeypatch.setenv("FSP_FAULT_INJECT", "alloc")
    assert lib.fsp_plan_create(32, 32, 32, 0.1, 0.1, 0.1, 1, 0) is None
    assert lib.fsp_last_error() == 4
    assert lib.fsp_plan_create_ex(64, 64, 0, 0.1, 0.1, 0.0, 0, 0, 1.0, float("nan"), 0) is None
    assert lib.fsp_last_error() == 4
    monkeypatch.setenv("FSP_FAULT_INJECT", "other")
    lib.fsp_plan_create(-1, 1, 1, 0.1, 0.1, 0.1, 0, 0)
    assert lib.fsp_last_error() == 1   # argument checks still come first
