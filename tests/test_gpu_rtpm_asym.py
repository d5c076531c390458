"""GPU parity of Alg. 1 as printed (three hashes, asymmetric sketches) against the oracle,
step by step: every power update is compared with the oracle's update of the GPU's previous
iterate, every lambda_tau and selection with the oracle's, and the deflation through the next
round's updates (the oracle deflates its sketches with the GPU's lambda^ and u^)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle.contract import contract_ivw_asym
from oracle.sketch import sketch_rank1_asym

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k,L,T_it,B,log2b,noise", [(24, 3, 4, 5, 5, 10, 0.05),
                                                       (40, 2, 3, 4, 8, 12, 0.02),
                                                       (17, 2, 2, 3, 1, 9, 0.1)])
def test_asym_rtpm_stepwise(n, k, L, T_it, B, log2b, noise):
    import paper_1506_04448_gb300 as tsk
    dev = torch.device("cuda", 0)
    b = 1 << log2b
    T, _, _ = synth.planted_symmetric(n, k, noise, 7 + n)
    h, g = tsk.cs_hashes(9 + n, B, log2b, [n, n, n], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T.astype(np.float32)).to(dev), h, g, log2b)
    U0 = torch.from_numpy(synth.gaussian_inits(k, L, n, 11).astype(np.float32)).to(dev)
    res = tsk.robust_power_method_asym(S, h, g, U0, T_it, return_trace=True)
    tsk.check_status(dev)
    res = {key: val.cpu().numpy() for key, val in res.items()}
    ho, go = O.cs_hashes(9 + n, B, log2b, [n, n, n])
    Sg = np.real(S.cpu().numpy()).astype(np.float64)
    U0g = U0.cpu().numpy().astype(np.float64)

    def update(u):
        per = np.stack([contract_ivw_asym(Sg[m], u, u, ho[m], go[m], b, n, "fft") for m in range(B)])
        return per

    for r in range(k):
        prev = np.stack([O.rtpm.normalise(U0g[r, t]) for t in range(L)])
        for t in range(T_it):
            got = res["U_iters"][r, t].astype(np.float64)
            for tau in range(L):
                want = O.rtpm.normalise(O.median_rows(update(prev[tau])))
                assert np.linalg.norm(got[tau] - want) < 1e-4, (r, t, tau)
            prev = got
        lam_want = np.array([O.median(update(prev[tau]) @ prev[tau]) for tau in range(L)])
        scale = max(1.0, np.abs(lam_want).max())
        assert np.max(np.abs(res["lam_all"][r] - lam_want)) < 1e-4 * scale
        ts = int(res["tau"][r])
        assert res["lam_all"][r, ts] == res["lam_all"][r].max()
        assert res["lam_all"][r, ts] >= lam_want.max() - 2e-4 * scale
        assert abs(res["lam"][r] - res["lam_all"][r, ts]) < 1e-6 * scale
        np.testing.assert_array_equal(res["V"][r], res["U_iters"][r, T_it - 1, ts])
        u = res["V"][r].astype(np.float64)
        for m in range(B):
            Sg[m] = Sg[m] - res["lam"][r] * np.real(sketch_rank1_asym(u, u, u, ho[m], go[m], b))


def test_asym_rtpm_recovers_planted_components():
    import paper_1506_04448_gb300 as tsk
    dev = torch.device("cuda", 0)
    n, k, B, log2b = 60, 3, 10, 14
    T, lam, A = synth.planted_symmetric(n, k, 0.001, 3)
    h, g = tsk.cs_hashes(4, B, log2b, [n, n, n], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T.astype(np.float32)).to(dev), h, g, log2b)
    U0 = torch.from_numpy(synth.gaussian_inits(k, 10, n, 5).astype(np.float32)).to(dev)
    res = tsk.robust_power_method_asym(S, h, g, U0, 20)
    V = res["V"].cpu().numpy()
    for r in range(k):
        assert np.max(np.abs(A.T @ V[r])) > 0.99
    assert np.allclose(np.sort(res["lam"].cpu().numpy()), np.sort(lam), atol=0.05)
