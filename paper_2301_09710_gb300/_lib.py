"""ctypes binding of ``libspect.so`` (C ABI in ``include/spect.h``).

Argument marshalling only: every step of the projector, its adjoint and the
EM update runs in the library's CUDA kernels.  Device buffers are passed as
raw pointers taken from torch CUDA tensors; torch provides memory and
streams, nothing else.  If the library has not been built the import of
this module still succeeds, but every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libspect.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "spect.h")

STATUS = {0: "SPECT_OK", 1: "SPECT_EINVAL", 2: "SPECT_ENOMEM", 3: "SPECT_ECUDA", 4: "SPECT_ETIMEOUT",
          5: "SPECT_EUNSUPPORTED"}
SPECT_PLAN_PREFER_SEPARABLE = 1
SPECT_PLAN_LOW_MEMORY = 2
SPECT_PLAN_ROTATION_3PASS = 4
SPECT_PLAN_RECOMPUTE_ATTENUATION = 8
ROTATIONS = ("bilinear", "3pass")
KERNEL_CLASSES = ["rotate_atten", "conv_fwd", "conv_adj", "rotate_adj", "other"]


class SpectError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


_lock = threading.Lock()
_lib = None


def header_symbols() -> list[str]:
    """Names of the functions declared in include/spect.h."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(spect_\w+)\s*\(", text, flags=re.M)))


def load(path: str = LIB_PATH):
    """Load libspect.so and declare the C signatures; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2301_09710_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i = ctypes.c_int
        st = ctypes.c_int
        lib.spect_plan_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, vp, ctypes.c_float, vp, vp, vp, i, i, i,
                                          vp, ctypes.c_uint, vp]
        lib.spect_plan_create.restype = st
        lib.spect_forward.argtypes = [vp, vp, vp, vp]
        lib.spect_forward.restype = st
        lib.spect_back.argtypes = [vp, vp, vp, vp]
        lib.spect_back.restype = st
        lib.spect_em_step.argtypes = [vp, vp, vp, vp, i, vp]
        lib.spect_em_step.restype = st
        lib.spect_em_step_reg.argtypes = [vp, vp, vp, vp, vp, ctypes.c_float, i, vp]
        lib.spect_em_step_reg.restype = st
        sz = ctypes.c_size_t
        f32 = ctypes.c_float
        lib.spect_em_ratio.argtypes = [sz, vp, vp, vp, vp, vp]
        lib.spect_em_ratio.restype = st
        lib.spect_em_ratio_backward.argtypes = [sz, vp, vp, vp, vp, vp, vp]
        lib.spect_em_ratio_backward.restype = st
        lib.spect_em_update.argtypes = [sz, vp, vp, vp, vp, f32, vp, vp]
        lib.spect_em_update.restype = st
        lib.spect_em_update_backward.argtypes = [sz, vp, vp, vp, vp, f32, vp, vp, vp, vp, vp]
        lib.spect_em_update_backward.restype = st
        lib.spect_sensitivity.argtypes = [vp, vp, vp]
        lib.spect_sensitivity.restype = st
        lib.spect_plan_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                                        ctypes.POINTER(ctypes.c_size_t)]
        lib.spect_plan_info.restype = st
        lib.spect_profile_enable.argtypes = [vp, i]
        lib.spect_profile_enable.restype = st
        lib.spect_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double), i]
        lib.spect_profile_read.restype = st
        lib.spect_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
        lib.spect_fp32_peak.restype = st
        lib.spect_forward_static.argtypes = [i, i, i, i, vp, vp, ctypes.c_float, vp, vp, i, i, i, vp, vp, vp]
        lib.spect_forward_static.restype = st
        lib.spect_plan_check.argtypes = [vp]
        lib.spect_plan_check.restype = st
        ip = ctypes.POINTER(i)
        lib.spect_plan_set_tuning.argtypes = [vp, i, i, i, vp]
        lib.spect_plan_set_tuning.restype = st
        lib.spect_plan_get_tuning.argtypes = [vp, ip, ip, ip]
        lib.spect_plan_get_tuning.restype = st
        lib.spect_plan_autotune.argtypes = [vp, vp]
        lib.spect_plan_autotune.restype = st
        lib.spect_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), i]
        lib.spect_batch_create.restype = st
        lib.spect_batch_em_step.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp]
        lib.spect_batch_em_step.restype = st
        lib.spect_batch_set_grouped.argtypes = [vp, i]
        lib.spect_batch_set_grouped.restype = st
        lib.spect_batch_info.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_longlong)]
        lib.spect_batch_info.restype = st
        lib.spect_batch_destroy.argtypes = [vp]
        lib.spect_batch_destroy.restype = st
        lib.spect_plan_bytes.argtypes = [i, i, i, i, i, i, i, i, ctypes.c_uint, ctypes.POINTER(ctypes.c_size_t)]
        lib.spect_plan_bytes.restype = st
        lib.spect_plan_selftest_timeout.argtypes = [vp, ctypes.c_longlong, vp]
        lib.spect_plan_selftest_timeout.restype = st
        lib.spect_plan_check_stream.argtypes = [vp, vp]
        lib.spect_plan_check_stream.restype = st
        lib.spect_plan_destroy.argtypes = [vp]
        lib.spect_plan_destroy.restype = st
        lib.spect_plan_release.argtypes = [vp, vp]
        lib.spect_plan_release.restype = st
        lib.spect_last_error.argtypes = []
        lib.spect_last_error.restype = ctypes.c_char_p
        lib.spect_version.argtypes = []
        lib.spect_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def check(status: int) -> None:
    if status != 0:
        raise SpectError(status, load().spect_last_error().decode())


def last_error() -> str:
    return load().spect_last_error().decode()
