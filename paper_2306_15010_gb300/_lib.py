"""ctypes view of libvqnnf.so (the C ABI declared in include/vqnnf.h).

Loading fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvqnnf.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = range(6)
PREC = {"fp32": 0, "bf16": 1, "fp8": 2}
OP_FIT, OP_ASSIGN, OP_FILTER_RESPONSES, OP_SCORE = range(4)
NOALLOC_SCRATCH_BYTES = 16 << 20      # VQNNF_NOALLOC_SCRATCH_BYTES

# every entry point the header declares, with its ctypes signature
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
SIGNATURES = {
    "vqnnf_workspace_bytes": (_sz, [_i, _i, _i, _i, _i, _i, _i, _i, _i]),
    "vqnnf_fit_codebook": (_i, [_vp, _i, _i, _i, _i, _i, ctypes.c_uint64, _i, _vp, _vp, _sz, _vp]),
    "vqnnf_assign": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _vp, _vp, _vp, _sz, _vp]),
    "vqnnf_assign_noalloc": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _vp, _vp, _vp]),
    "vqnnf_filter_responses": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _vp, _sz, _vp]),
    "vqnnf_score": (_i, [_vp, _i, _i, _i, _i, _i, _vp, _i, _vp, _vp, _vp, _vp, _sz, _vp]),
    "vqnnf_status_str": (ctypes.c_char_p, [_i]),
    "vqnnf_last_device_error": (_i, [_vp]),
    "vqnnf_selftest_bounded_wait": (_i, [ctypes.c_longlong, _vp]),
    "vqnnf_set_kernel_events": (_i, [_i, _vp, _vp]),
    "vqnnf_soft_workspace_bytes": (ctypes.c_size_t, [_i, _i, _i, _i, _i, _i, _i, _i]),
    "vqnnf_soft_forward": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _i, _vp, _i, ctypes.c_float, _i, _vp, _vp,
                                _vp, ctypes.c_size_t, _vp]),
    "vqnnf_soft_backward": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _i, _vp, _i, ctypes.c_float, _i, _vp, _vp,
                                 _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "vqnnf_version": (_i, []),
    "vqnnf_match_host_workspace_bytes": (_sz, [_i, _i, _i, _i, _i, _i, _i, _i]),
    "vqnnf_match_host": (_i, [_vp, _i, _i, _i, _vp, _i, _i, _i, _i, ctypes.c_uint64, _i, _vp, _i, _vp, _vp, _vp,
                              _sz, _vp, _vp]),
    "vqnnf_batch_workspace_bytes": (_sz, [_vp, _i, _vp, _i, _i, _i]),
    "vqnnf_match_batch": (_i, [_vp, _i, _vp, _i, _i, _i, ctypes.c_uint64, _i, _vp, _vp, _vp, _vp, _sz, _vp]),
    "vqnnf_batch_tune": (_i, [_vp, _i, _vp, _i, _i, _i, ctypes.c_uint64, _i, _vp, _vp, _sz, _vp]),
}


class VqnnfRect(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_int32), ("y0", ctypes.c_int32), ("x1", ctypes.c_int32),
                ("y1", ctypes.c_int32), ("weight", ctypes.c_int32)]


class VqnnfFilter(ctypes.Structure):
    _fields_ = [("n_rects", ctypes.c_int32), ("rects", ctypes.POINTER(VqnnfRect)),
                ("w_f", ctypes.c_float), ("area", ctypes.c_float)]


class VqnnfImage(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("H", ctypes.c_int32), ("W", ctypes.c_int32)]


class VqnnfBatchTemplate(ctypes.Structure):
    _fields_ = [("T", ctypes.c_void_p), ("h", ctypes.c_int32), ("w", ctypes.c_int32), ("k", ctypes.c_int32)]


class VqnnfBatchPlan(ctypes.Structure):
    _fields_ = [("group_cols", ctypes.c_int32), ("sf", ctypes.c_int32), ("pf", ctypes.c_int32),
                ("stationary", ctypes.c_int32)]


class VqnnfError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__(f"{fn} failed: {msg} (status {status})")
        self.status = status


_lib = None


def load() -> ctypes.CDLL:
    """Load libvqnnf.so; raises if it has not been built (call __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                              "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(fn: str, status: int) -> None:
    if status != OK:
        msg = load().vqnnf_status_str(status).decode()
        raise VqnnfError(fn, status, msg)
