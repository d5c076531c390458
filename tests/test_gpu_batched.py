"""GPU parity for many independent decompositions in one plan (groups by sketch length, one
launch per power step and group, CUDA-graph capture): every problem's Alg. 1 is checked step by
step against the oracle from its own traces, for the default and the autotuned block sizes and
for a graph replay; the full configuration (256 problems, n ~ U{32..256}, k ~ U{4..16},
b = clamp(2^ceil(log2 nk), 2^10, 2^14), B = 8, L = 20, T = 20) on sampled problems."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
tsk = pytest.importorskip("paper_1506_04448_gb300")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def make_problems(dev, specs, B, L, noise=0.01):
    probs = []
    for s in specs:
        T, _, _ = synth.planted_symmetric(s["n"], s["k"], noise, s["seed"], dtype=np.float32)
        h, g = tsk.cs_hashes(s["seed"], B, s["log2b"], [s["n"]], dev)
        S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, s["log2b"])
        U0 = synth.gaussian_inits(s["k"], L, s["n"], s["seed"] + 1).astype(np.float32)
        probs.append({"S": S, "h": h, "g": g, "U0": torch.from_numpy(U0).to(dev), **s})
    return probs


def check_problem(p, res, B, T, rounds=None, steps=None, taus=None):
    from rtpm_check import check_rtpm_stepwise
    host = {key: val.cpu().numpy() for key, val in res.items()}
    ho, go = O.cs_hashes(p["seed"], B, p["log2b"], [p["n"]])
    # the deflated sketches are not an output of a batch: rebuild the chain in the oracle only
    Sd = np.array(p["S"].cpu().numpy(), dtype=np.complex128)
    for r in range(p["k"]):
        Sd = O.deflate_sketches(Sd, float(host["lam"][r]), host["V"][r].astype(np.float64),
                                ho[:, 0], go[:, 0], 1 << p["log2b"], "fft")
    host["S_deflated"] = Sd
    check_rtpm_stepwise(host, p["S"].cpu().numpy().astype(np.complex128), ho[:, 0], go[:, 0],
                        1 << p["log2b"], p["U0"].cpu().numpy().astype(np.float64), T,
                        rounds=rounds, steps=steps, taus=taus)


SMALL = [dict(n=30, k=3, log2b=10, seed=1), dict(n=77, k=2, log2b=11, seed=2),
         dict(n=45, k=4, log2b=10, seed=3), dict(n=120, k=1, log2b=13, seed=4),
         dict(n=200, k=2, log2b=14, seed=5), dict(n=64, k=3, log2b=12, seed=6),
         dict(n=33, k=0, log2b=10, seed=7)]


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_stepwise_parity(dev, autotune):
    B, L, T = 4, 5, 6
    probs = make_problems(dev, SMALL, B, L)
    plan = tsk.BatchPlan(probs, B, L, T, autotune=autotune, trace=True)
    plan.run()
    tsk.check_status(dev)
    for p, res in zip(probs, plan.results):
        if p["k"] > 0:
            check_problem(p, res, B, T)
    if autotune:
        assert plan.block_size(10) in (64, 32)
    plan.close()


def test_batch_graph_capture_and_replay(dev):
    B, L, T = 4, 5, 6
    probs = make_problems(dev, SMALL[:4], B, L)
    plan = tsk.BatchPlan(probs, B, L, T, autotune=False, trace=True)
    plan.run()                        # warm-up outside the capture (module loading)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        with torch.cuda.graph(graph, stream=stream):
            plan.run()
    for res in plan.results:
        for v in res.values():
            v.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize(dev)
    tsk.check_status(dev)
    for p, res in zip(probs, plan.results):
        check_problem(p, res, B, T)
    plan.close()


def test_batch_full_configuration_sampled(dev):
    B, L, T = 8, 20, 20
    specs = synth.batched_problem_specs(256, 3)
    probs = make_problems(dev, specs, B, L)
    plan = tsk.BatchPlan(probs, B, L, T, autotune=True, trace=True)
    plan.run()
    tsk.check_status(dev)
    for i in (0, 97, 255):
        p = probs[i]
        check_problem(p, plan.results[i], B, T, rounds=(0, p["k"] - 1), steps=(0, T - 1), taus=(0, L - 1))
    for p, res in zip(probs, plan.results):
        V = res["V"].cpu().numpy()
        assert np.all(np.isfinite(res["lam"].cpu().numpy()))
        np.testing.assert_allclose(np.linalg.norm(V, axis=1), 1.0, rtol=1e-5)
    plan.close()
