"""Calls on alternating torch streams share one context (its workspace and status word).

Re-binding the context to another stream makes the new stream wait for the work already queued
on the previous one, so back-to-back contractions on two streams, with no host synchronisation
between them, each match the FP64 oracle (1e-5 relative per vector and sketch)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
tsk = pytest.importorskip("paper_1506_04448_gb300")


def test_contractions_on_alternating_streams_match_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    n, B, log2b, L = 200, 6, 12, 64
    b = 1 << log2b
    T = synth.random_symmetric(n, 77).astype(np.float32)
    h, g = tsk.cs_hashes(21, B, log2b, [n], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, log2b)
    FS = tsk.sketch_fft(S)
    torch.cuda.synchronize(dev)
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    Us = [torch.nn.functional.normalize(
        torch.tensor(synth.rng(300 + r).standard_normal((L, n)), dtype=torch.float32,
                     device=dev), dim=1) for r in range(6)]
    outs = []
    for r, U in enumerate(Us):
        st = streams[r % 2]
        st.wait_stream(torch.cuda.current_stream(dev))   # U was made on the current stream
        with torch.cuda.stream(st):
            Vmed, Vall = tsk.contract_iuu(FS, S, h, g, U, return_all=True)
            Vall = Vall.clone()
        outs.append((U, Vall))
    torch.cuda.synchronize(dev)
    tsk.check_status(dev)
    ho, go = O.cs_hashes(21, B, log2b, [n])
    Sg = S.cpu().numpy().astype(np.complex128)
    for U, Vall in outs:
        Ug = U.cpu().numpy().astype(np.float64)
        Vg = Vall.cpu().numpy()
        for tau in (0, L // 2, L - 1):
            for m in (0, B - 1):
                ref = O.contract_iuu(Sg[m], Ug[tau], ho[m, 0], go[m, 0], b, "fft")
                assert np.linalg.norm(Vg[tau, m] - ref) <= 1e-5 * np.linalg.norm(ref)
