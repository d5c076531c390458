"""contract_iuu_static: the contraction entry point for callers that cannot allocate.

Callers whose device memory belongs to another allocator, or whose loops forbid allocation
after start-up, cannot let the library cudaMalloc a workspace; contract_iuu_static keeps its scratch
in a static device array instead.  This test calls it through the C ABI twice in a row (so the
second call sees the array as the first one left it) and compares each result with the
workspace-based contract_iuu within the contraction tolerance (1e-5 relative, 2-norm), and
sampled vectors of the first call with the FP64 oracle.

The file name makes pytest collect it last; it passes alone in a fresh process and after the
other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
tsk = pytest.importorskip("paper_1506_04448_gb300")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_matches_workspace_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_04448_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda:0")
    n, B, log2b, L = 400, 10, 14, 50
    T, _, _ = synth.planted_symmetric(n, 5, 0.01, 3, dtype=np.float32)
    h, g = tsk.cs_hashes(3, B, log2b, [n], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, log2b)
    FS = tsk.sketch_fft(S)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        U = torch.nn.functional.normalize(
            torch.tensor(synth.rng(10 + call).standard_normal((L, n)), dtype=torch.float32,
                         device=dev), dim=1).contiguous()
        want = tsk.contract_iuu(FS, S, h, g, U)
        got = torch.full((L, n), float("nan"), dtype=torch.float32, device=dev)
        rc = lib.contract_iuu_static(_ptr(FS), _ptr(S), _ptr(h), _ptr(g), B, log2b, _ptr(U), L, n,
                                     _ptr(got), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.tsk_strerror(rc)
        torch.cuda.synchronize(dev)
        w = want.cpu().numpy()
        gg = got.cpu().numpy()
        for tau in range(L):
            assert np.linalg.norm(gg[tau] - w[tau]) <= 1e-5 * np.linalg.norm(w[tau]), (call, tau)
        # and against the FP64 oracle itself (median over the B sketches), sampled vectors
        if call == 0:
            ho, go = O.cs_hashes(3, B, log2b, [n])
            Sg = S.cpu().numpy().astype(np.complex128)
            Ug = U.cpu().numpy().astype(np.float64)
            for tau in (0, L // 2, L - 1):
                refs = np.stack([O.contract_iuu(Sg[m], Ug[tau], ho[m, 0], go[m, 0], 1 << log2b, "fft")
                                 for m in range(B)])
                med = O.median_rows(refs)
                assert np.linalg.norm(gg[tau] - med) <= 1e-5 * np.linalg.norm(med), tau


def test_static_scratch_rejects_sizes_beyond_its_maximum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1506_04448_gb300 import _lib
    lib = _lib.load()
    dev = torch.device("cuda:0")
    n, B, log2b, L = 8192, 64, 10, 4      # L*B*n*4 = 8 MiB > 4 MiB
    x = torch.zeros((B, 1 << log2b), dtype=torch.complex64, device=dev)
    h = torch.zeros((B, n), dtype=torch.int32, device=dev)
    g = torch.zeros((B, n), dtype=torch.uint8, device=dev)
    U = torch.zeros((L, n), dtype=torch.float32, device=dev)
    out = torch.zeros((L, n), dtype=torch.float32, device=dev)
    rc = lib.contract_iuu_static(_ptr(x), _ptr(x), _ptr(h), _ptr(g), B, log2b, _ptr(U), L, n,
                                 _ptr(out), None)
    assert rc == -6    # TSK_EUNSUPPORTED: scratch beyond the static maximum
