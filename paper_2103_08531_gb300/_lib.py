"""ctypes loader for libfsp.so: the C ABI of include/fsp.h, nothing else.

There is no fallback: if the library is missing or fails to load, every entry
point raises.  Call ``paper_2103_08531_gb300.build.build()`` (or
``__graft_entry__.build()``) to compile it.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfsp.so")

FSP_HE, FSP_VGF, FSP_HE_NEARBY, FSP_HE_CELLAVG = 0, 1, 2, 3
FSP_F32, FSP_F64 = 0, 1
FSP_PLAN_DIRECT = 1
STATUS = {0: "FSP_OK", 1: "FSP_ERR_INVALID", 2: "FSP_ERR_UNSUPPORTED_SIZE", 3: "FSP_ERR_CUDA",
          4: "FSP_ERR_NOMEM", 5: "FSP_ERR_WORKSPACE", 6: "FSP_ERR_TIMEOUT"}

# name -> (restype, argtypes); every symbol include/fsp.h declares
_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_ip, _dp, _vpp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "fsp_plan_create": (_vp, [_i, _i, _i, _d, _d, _d, _i, _i]),
    "fsp_plan_create_ex": (_vp, [_i, _i, _i, _d, _d, _d, _i, _i, _d, _d, _i]),
    "fsp_last_error": (_i, []),
    "fsp_error_string": (ctypes.c_char_p, [_i]),
    "fsp_plan_geometry": (_i, [_vp, _ip, _ip, _dp, _dp, _ip]),
    "fsp_plan_workspace_bytes": (_sz, [_vp, _i, _i]),
    "fsp_plan_set_workspace": (_i, [_vp, _vp, _sz]),
    "fsp_solve": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fsp_solve_adjoint": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fsp_solve_batched": (_i, [_vpp, _i, _vpp, _vpp, _vpp, _vp]),
    "fsp_batch_create": (_vp, [_vpp, _i, _vpp, _vpp, _vpp]),
    "fsp_batch_solve": (_i, [_vp, _vp]),
    "fsp_batch_destroy": (None, [_vp]),
    "fsp_batch_kernel_count": (_i, [_vp, _ip]),
    "fsp_plan_set_pass_events": (_i, [_vp, _vpp, _i]),
    "fsp_autotune": (_i, [_vp, ctypes.c_char_p, _i]),
    "fsp_gradient_fd": (_i, [_vp, _vp, _vp, _vp]),
    "fsp_tuned_variant": (_i, [_i, _i]),
    "fsp_plan_kernel_spectrum": (_i, [_vp, _vp, _sz]),
    "fsp_plan_run_passes": (_i, [_vp, _vp, _i, _i, _vp]),
    "fsp_plan_workspace_layout": (_i, [_vp, ctypes.POINTER(_sz), _ip]),
    "fsp_plan_destroy": (None, [_vp]),
    "fsp_solve_noalloc": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fsp_host_pipe_create": (_vp, [_vp, _i, _i, _i]),
    "fsp_host_pipe_solve": (_i, [_vp, _i, _vpp, _vpp, _vpp, _vp]),
    "fsp_host_pipe_destroy": (None, [_vp]),
    "fsp_plan_device_status": (_i, [_vp, _i]),
    "fsp_plan_set_plane_group": (_i, [_vp, _i]),
    "fsp_selftest_wait_timeout": (_i, [_d]),
}


class FspError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS.get(self.code, self.code)}" if what else STATUS.get(self.code, str(code)))


_lib = None


def load(path: str = LIB_PATH):
    """Load libfsp.so and attach the C signatures (raises if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise FspError(3, f"libfsp.so not built at {path}; run paper_2103_08531_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int, what: str):
    if code != 0:
        raise FspError(code, what)
