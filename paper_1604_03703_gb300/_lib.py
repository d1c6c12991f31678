"""ctypes binding of the sev C ABI (include/sev.h): argument marshalling only.

Every step of the computation runs in libsev.so's CUDA kernels.  Importing
this module raises if the library has not been built: there is no CPU or
PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsev.so")

SEV_FP64 = 0
SEV_MIXED = 1

STATUS = {
    0: "SEV_OK",
    1: "SEV_ERR_NONFINITE",
    2: "SEV_ERR_NOCONV",
    3: "SEV_ERR_TIMEOUT",
    4: "SEV_ERR_CUDA",
    5: "SEV_ERR_WORKSPACE",
    6: "SEV_ERR_UNSUPPORTED",
    7: "SEV_ERR_INTERNAL",
}

# name -> (restype, argtypes) for every function declared in include/sev.h
_vp, _i, _d, _sz, _l = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_long
SIGNATURES = {
    "sev_create": (_i, [ctypes.POINTER(_vp), _i]),
    "sev_destroy": (_i, [_vp]),
    "sev_set_stream": (_i, [_vp, _vp]),
    "sev_workspace_query": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_sz)]),
    "sev_set_workspace": (_i, [_vp, _vp, _sz]),
    "sev_eigvalsh": (_i, [_vp, _i, _vp, _i, _i, _i, _vp]),
    "sev_eigvalsh_host": (_i, [_vp, _i, _vp, _i, _i, _i, _vp]),
    "sev_full_to_band": (_i, [_vp, _i, _vp, _i, _i, _i, _vp, _i]),
    "sev_band_to_band": (_i, [_vp, _i, _vp, _i, _i, _i, _i]),
    "sev_tridiag_bisect": (_i, [_vp, _i, _vp, _vp, _d, _vp]),
    "sev_band_tridiag_extract": (_i, [_vp, _i, _vp, _i, _i, _vp, _vp]),
    "sev_tridiag_bisect_static": (_i, [_i, _vp, _vp, _d, _vp, _vp]),
    "sev_get_error": (_i, [_vp]),
    "sev_set_wait_limit": (_i, [_vp, ctypes.c_longlong]),
    "sev_status_string": (ctypes.c_char_p, [_i]),
    "sev_set_kernel_timing": (_i, [_vp, ctypes.c_ulonglong]),
    "sev_kernel_count": (_i, []),
    "sev_kernel_name": (ctypes.c_char_p, [_i]),
    "sev_kernel_time": (_i, [_vp, _i, ctypes.POINTER(_d), ctypes.POINTER(_l), _i]),
    "sev_batch_plan_create": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_vp), _i, _i, ctypes.POINTER(_vp)]),
    "sev_batch_run": (_i, [_vp, _vp]),
    "sev_batch_plan_destroy": (_i, [_vp]),
    "sev_batch_plan_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "sev_eigvalsh_batched": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_vp), _i, _i,
                                  ctypes.POINTER(_vp)]),
    "sev_batch_autotune": (_i, [_vp, _i, ctypes.POINTER(_i), _i, ctypes.POINTER(_i)]),
    "sev_diag_house_scalars": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sev_band_schedule": (_i, [_i, _i, _i, ctypes.POINTER(_i), _i]),
    "sev_autotune": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_i), _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "sev_eigvalsh_bands": (_i, [_vp, _i, _i, _i, ctypes.POINTER(_i), _i]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsev.so and declare every exported signature."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libsev.so is not built (%s); run `python -m paper_1604_03703_gb300.build` "
            "(there is no CPU fallback)" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SevError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        txt = STATUS.get(code, "invalid argument %d" % -code if code < 0 else "unknown")
        super().__init__("%s failed: %s (%d)" % (where, txt, code))


def check(code: int, where: str) -> None:
    if code != 0:
        raise SevError(code, where)
