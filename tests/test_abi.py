"""CPU-side checks of the C ABI: the library builds, loads, exports every function declared in
include/tsk.h with the binding's signatures, and rejects bad calls without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsk.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_04448_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("cs_hashes", "sketch_tensor", "sketch_rank1", "contract_uuu", "contract_iuu",
                     "robust_power_method", "sketch_fft", "tsk_ctx_create", "tsk_ctx_status"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1506_04448_gb300 import _lib
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks a signature for {name}"


def test_strerror_and_argument_errors_without_gpu(lib):
    assert lib.tsk_strerror(0) == b"ok"
    assert b"invalid" in lib.tsk_strerror(-1)
    # every entry point rejects a NULL context before touching the device
    assert lib.cs_hashes(None, 1, 1, 10, 1, None, None, None) == -1
    assert lib.contract_iuu(None, None, None, None, None, 1, 10, None, 1, 1, None, None) == -1
    assert lib.robust_power_method(None, None, None, None, 1, 10, 1, 1, 1, 1, None, None, None,
                                   None, None, None, None) == -1
    assert lib.tsk_ctx_status(None) == -1


def test_ctx_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.tsk_ctx_create(0, None, ctypes.byref(h)) == -3   # TSK_ECUDA, no device
    assert h.value is None


def test_binding_fails_loudly_when_library_missing(monkeypatch):
    from paper_1506_04448_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", os.path.join(ROOT, "does-not-exist", "libtsk.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_launch_count_query_rejects_a_null_context(lib):
    assert lib.robust_power_method_launches(None, 10, 14, 400, 20, 50, 30) == -1


def test_every_compute_entry_rejects_a_null_context(lib):
    """Each compute entry point of include/tsk.h returns TSK_EINVAL for a NULL context (or NULL
    buffers) before anything reaches a device."""
    from paper_1506_04448_gb300 import _lib
    skip = {"tsk_ctx_create", "tsk_ctx_destroy", "tsk_ctx_set_stream", "tsk_ctx_status",
            "tsk_strerror", "tsk_batch_destroy", "tsk_batch_block_size",
            "robust_power_method_launches", "contract_iuu_static"}
    checked = 0
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        if name in skip:
            continue
        args = [0 if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64) else
                (0.0 if t is ctypes.c_double else None) for t in argtypes]
        assert getattr(lib, name)(*args) == -1, name
        checked += 1
    assert checked >= 20


def test_static_contraction_rejects_null_buffers(lib):
    assert lib.contract_iuu_static(None, None, None, None, 1, 10, None, 1, 1, None, None) == -1


def test_batch_entry_points_reject_null_plans(lib):
    assert lib.tsk_batch_destroy(None) == -1
    assert lib.tsk_batch_block_size(None, 10) == -1
