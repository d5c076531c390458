"""ctypes loader for libtsk.so (the C ABI declared in include/tsk.h).

The library is built in-tree by paper_1506_04448_gb300.build; there is no fallback: if it is
missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libtsk.so")

TSK_F32, TSK_F64, TSK_I32, TSK_C64, TSK_C128, TSK_CI64 = range(6)
STATUS = {0: "TSK_OK", -1: "TSK_EINVAL", -2: "TSK_ENOMEM", -3: "TSK_ECUDA", -4: "TSK_ETIMEOUT",
          -5: "TSK_ENONFINITE", -6: "TSK_EUNSUPPORTED"}

# exported symbol -> (restype, argtypes); must match include/tsk.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_D = ctypes.c_double
SIGNATURES = {
    "tsk_ctx_create": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "tsk_ctx_destroy": (_I, [_P]),
    "tsk_ctx_set_stream": (_I, [_P, _P]),
    "tsk_ctx_status": (_I, [_P]),
    "tsk_strerror": (ctypes.c_char_p, [_I]),
    "tsk_peak_launch": (_I, [_P, _I, _I, _P]),
    "tsk_peak_work": (_I, [_P, _I, _I, ctypes.POINTER(_D)]),
    "cs_hashes": (_I, [_P, _U64, _I, _I, _I, _P, _P, _P]),
    "sketch_tensor": (_I, [_P, _P, _I, _I, _P, _P, _P, _I, _I, _P, _I, _I]),
    "sketch_tensor_planes": (_I, [_P, _P, _I, _I, _I, _I, _P, _P, _I, _I, _P, _I, _I]),
    "sketch_fft": (_I, [_P, _P, _P, _I, _I, _I]),
    "sketch_rank1": (_I, [_P, _I64, _P, _P, _P, _P, _I, _P, _P, _P, _I, _I, _I, _P, _I]),
    "contract_iuu": (_I, [_P, _P, _P, _P, _P, _I, _I, _P, _I, _I64, _P, _P]),
    "contract_uuu": (_I, [_P, _P, _P, _P, _P, _I, _I, _P, _I, _I64, _P, _P]),
    "contract_iuu_static": (_I, [_P, _P, _P, _P, _I, _I, _P, _I, _I64, _P, _P]),
    "sketch_rfft": (_I, [_P, _P, _P, _I, _I]),
    "contract_ivw": (_I, [_P, _P, _P, _P, _I, _I, _P, _I, _P, _P, _I, _P, _P]),
    "cp_sketch_loss": (_I, [_P, _P, _P, _P, _I, _I, _P, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "cp_als_solve": (_I, [_P, _P, _P, _P, _I, _I64, _I64, _I64, _P, _P]),
    "tsk_batch_create": (_I, [_P, _P, _I, _I, _I, _I, _I, ctypes.POINTER(_P)]),
    "tsk_batch_run": (_I, [_P, _P]),
    "tsk_batch_destroy": (_I, [_P]),
    "tsk_batch_block_size": (_I, [_P, _I]),
    "robust_power_method_batched": (_I, [_P, _P, _I, _I, _I, _I]),
    "robust_power_method": (_I, [_P, _P, _P, _P, _I, _I, _I64, _I, _I, _I, _P, _P, _P, _P, _P,
                                 _P, _P]),
    "robust_power_method_launches": (_I64, [_P, _I, _I, _I64, _I, _I, _I]),
    "robust_power_method_asym": (_I, [_P, _P, _P, _P, _I, _I, _I64, _I, _I, _I, _P, _P, _P, _P,
                                      _P, _P]),
    "cs_hashes_p": (_I, [_P, _U64, _I, _I, _I, _I64, _P, _P]),
    "sketch_tensor_p": (_I, [_P, _P, _I, _I64, _P, _P, _I, _I, _I, _P]),
    "contract_p": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P, _I, _I64, _P, _P, _P, _P]),
    "robust_power_method_p": (_I, [_P, _P, _P, _P, _I, _I, _I, _I64, _I, _I, _I, _P, _P, _P, _P,
                                   _P, _P, _P]),
    "robust_power_method_p_launches": (_I64, [_P, _I, _I, _I]),
    "lda_m2_apply": (_I, [_P, _P, _P, _P, _I64, _I64, _D, _P, _I, _P]),
    "lda_whiten": (_I, [_P, _P, _P, _P, _I64, _I64, _I, _D, _P, _I, _I, _P, _P, _P]),
    "lda_whitened_m3": (_I, [_P, _P, _P, _P, _I64, _I64, _P, _I, _D, _P]),
    "lda_sketch_m3": (_I, [_P, _P, _P, _P, _I64, _I64, _P, _I, _D, _P, _P, _I, _I, _P, _P]),
    "lda_recover": (_I, [_P, _P, _I64, _I, _D, _P, _P, _P, _P]),
}


class TskError(RuntimeError):
    def __init__(self, fn: str, code: int, text: str):
        super().__init__(f"{fn}: {STATUS.get(code, code)} ({text})")
        self.code = code


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libtsk.so once; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_1506_04448_gb300.build` (needs nvcc)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(fn: str, code: int) -> None:
    if code != 0:
        raise TskError(fn, code, load().tsk_strerror(code).decode())
