"""Parity at the benchmarked size (dense symmetric n = 400, B = 10, b = 2^14, L = 50, T = 30,
k = 20) in the launch configuration bench.py times, on outputs the oracle computes one by one:
all ten sketches; and Alg. 1 step by step for sampled rounds, steps and initial vectors (64
iterates), with every round's selection and the whole deflation chain."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
tsk = pytest.importorskip("paper_1506_04448_gb300")

CFG = dict(n=400, k=20, noise=0.005, B=10, log2b=14, L=50, T=30, seed=1)


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    c = CFG
    T, _, _ = synth.planted_symmetric(c["n"], c["k"], c["noise"], c["seed"], dtype=np.float32)
    U0 = synth.gaussian_inits(c["k"], c["L"], c["n"], c["seed"] + 1).astype(np.float32)
    h, g = tsk.cs_hashes(c["seed"], c["B"], c["log2b"], [c["n"]], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, c["log2b"])
    res = tsk.robust_power_method(S, h, g, torch.from_numpy(U0).to(dev), c["T"],
                                  return_deflated=True, return_trace=True)
    tsk.check_status(dev)
    return dict(T=T, U0=U0, h=h.cpu().numpy()[:, 0], g=g.cpu().numpy()[:, 0],
                S=S.cpu().numpy().astype(np.complex128),
                res={key: val.cpu().numpy() for key, val in res.items()})


def test_fullsize_hashes_and_sampled_sketches(run):
    c = CFG
    b = 1 << c["log2b"]
    ho, go = O.cs_hashes(c["seed"], c["B"], c["log2b"], [c["n"]])
    np.testing.assert_array_equal(run["h"], ho[:, 0])
    np.testing.assert_array_equal(run["g"], go[:, 0])
    T64 = run["T"].astype(np.float64)
    for m in range(c["B"]):
        ref = O.sketch_tensor_sym(T64, ho[m, 0], go[m, 0], b)
        err = np.linalg.norm(run["S"][m] - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (m, err)


def test_fullsize_rtpm_stepwise_sampled(run):
    from rtpm_check import check_rtpm_stepwise
    c = CFG
    U0 = run["U0"].astype(np.float64)
    n_checked = check_rtpm_stepwise(run["res"], run["S"], run["h"], run["g"], 1 << c["log2b"], U0,
                                    c["T"], rounds=(0, 5, 10, c["k"] - 1),
                                    steps=(0, 1, 15, c["T"] - 1), taus=(0, 17, 33, c["L"] - 1))
    assert n_checked == 4 * 4 * 4
    V = run["res"]["V"]
    np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, rtol=1e-5)
    assert np.all(np.isfinite(run["res"]["lam"]))
