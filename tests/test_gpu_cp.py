"""GPU parity for the asymmetric path: half spectra, T^(I,v,w) (Prop. 1 / Alg. 2), the sketched
CP loss and its adjoint, the Eq. 15 solve, and the differentiable-fitting configuration
(500 x 400 x 300, rank 30, B = 8, b = 2^15).  Tolerances: 1e-5 relative (2-norm) for FP32 values
against the FP64 oracle on the same sketches; gradients also against central differences
(h = 1e-3) of the oracle's loss."""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu
tsk = pytest.importorskip("paper_1506_04448_gb300")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def t32(x, dev):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device=dev)


def _asym_setup(dev, dims, B, log2b, seed, R=3, noise=0.1):
    r = synth.rng(seed)
    A0, B0, C0 = (r.standard_normal((R, d)) for d in dims)
    T = np.einsum("ri,rj,rk->ijk", A0, B0, C0) + noise * r.standard_normal(dims)
    h, g = tsk.cs_hashes(seed, B, log2b, list(dims), dev)
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b)
    Xh = tsk.sketch_rfft(S)
    ho, go = O.cs_hashes(seed, B, log2b, list(dims))
    Sg = np.real(S.cpu().numpy()).astype(np.float64)
    return T, h, g, S, Xh, ho, go, Sg


@pytest.mark.parametrize("log2b", [9, 12, 15])
def test_sketch_rfft(dev, log2b):
    b = 1 << log2b
    r = synth.rng(log2b)
    X = r.standard_normal((3, b)) + 1j * r.standard_normal((3, b))
    Xd = torch.tensor(X, dtype=torch.complex64, device=dev)
    got = tsk.sketch_rfft(Xd).cpu().numpy()
    real = np.real(Xd.cpu().numpy()).astype(np.float64)
    for m in range(3):
        assert rel(got[m], np.fft.rfft(real[m])) < 2e-6


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("log2b,B", [(10, 3), (15, 2)])
def test_contract_ivw(dev, mode, log2b, B):
    dims = (37, 20, 45)
    b = 1 << log2b
    _, h, g, S, Xh, ho, go, Sg = _asym_setup(dev, dims, B, log2b, 11 + mode)
    others = [j for j in range(3) if j != mode]
    K = 4
    V = synth.rng(1).standard_normal((K, dims[others[0]]))
    W = synth.rng(2).standard_normal((K, dims[others[1]]))
    Vd, Wd = t32(V, dev), t32(W, dev)
    Vmed, Vall = tsk.contract_ivw(Xh, h, g, dims, mode, Vd, Wd, return_all=True)
    Vg, Wg = Vd.cpu().numpy().astype(np.float64), Wd.cpu().numpy().astype(np.float64)
    Vall = Vall.cpu().numpy()
    for r in range(K):
        refs = np.stack([O.contract_ivw_mode(Sg[m], ho[m], go[m], b, mode, Vg[r], Wg[r], dims[mode])
                         for m in range(B)])
        for m in range(B):
            assert rel(Vall[r, m], refs[m]) < 1e-5, (r, m)
        assert rel(Vmed[r].cpu().numpy(), O.median_rows(refs)) < 1e-5


def _cp_params(dev, dims, R, seed):
    r = synth.rng(seed)
    lam = r.uniform(0.5, 2.0, R)
    A, Bf, C = (r.standard_normal((R, d)) / np.sqrt(d) for d in dims)
    return [t32(x, dev) for x in (lam, A, Bf, C)]


@pytest.mark.parametrize("dims,R,B,log2b", [((30, 25, 20), 4, 3, 11), ((9, 7, 5), 2, 1, 9)])
def test_cp_loss_and_adjoint(dev, dims, R, B, log2b):
    b = 1 << log2b
    _, h, g, S, Xh, ho, go, Sg = _asym_setup(dev, dims, B, log2b, 21)
    params = _cp_params(dev, dims, R, 22)
    loss, *grads = tsk.cp_sketch_loss(Xh, h, g, dims, *params)
    pg = [p.cpu().numpy().astype(np.float64) for p in params]
    want_loss = O.cp_sketch_loss(Sg, ho, go, b, *pg)
    want = O.cp_sketch_grad(Sg, ho, go, b, *pg)
    assert abs(loss.item() - want_loss) <= 1e-5 * abs(want_loss)
    for got, ref in zip(grads, want):
        assert rel(got.cpu().numpy(), ref) < 1e-5


def test_cp_gradient_against_central_differences(dev):
    dims, R, B, log2b = (6, 5, 4), 2, 2, 9
    b = 1 << log2b
    _, h, g, S, Xh, ho, go, Sg = _asym_setup(dev, dims, B, log2b, 31)
    params = _cp_params(dev, dims, R, 32)
    _, *grads = tsk.cp_sketch_loss(Xh, h, g, dims, *params)
    pg = [p.cpu().numpy().astype(np.float64) for p in params]
    step = 1e-3
    for which in range(4):
        fd = np.zeros_like(pg[which])
        for idx in np.ndindex(pg[which].shape):
            up = [p.copy() for p in pg]
            dn = [p.copy() for p in pg]
            up[which][idx] += step
            dn[which][idx] -= step
            fd[idx] = (O.cp_sketch_loss(Sg, ho, go, b, *up) - O.cp_sketch_loss(Sg, ho, go, b, *dn)) / (2 * step)
        assert rel(grads[which].cpu().numpy(), fd) < 1e-4


def test_cp_autograd_function(dev):
    dims, R, B, log2b = (12, 10, 8), 3, 2, 10
    _, h, g, S, Xh, *_ = _asym_setup(dev, dims, B, log2b, 41)
    params = [p.clone().requires_grad_(True) for p in _cp_params(dev, dims, R, 42)]
    loss = tsk.cp_loss(*params, Xh, h, g, dims)
    (3.0 * loss).backward()
    _, *grads = tsk.cp_sketch_loss(Xh, h, g, dims, *[p.detach() for p in params])
    for p, gr in zip(params, grads):
        assert torch.allclose(p.grad, 3.0 * gr, rtol=1e-6, atol=1e-7)


def test_als_solve(dev):
    K, n, np_, nq = 5, 40, 30, 20
    r = synth.rng(7)
    M, P, Q = r.standard_normal((K, n)), r.standard_normal((K, np_)), r.standard_normal((K, nq))
    out, lam = tsk.cp_als_solve(t32(M, dev), t32(P, dev), t32(Q, dev))
    ro, rl = O.als_solve(*(t32(x, dev).cpu().numpy().astype(np.float64) for x in (M, P, Q)))
    assert rel(out.cpu().numpy(), ro) < 1e-5
    assert rel(lam.cpu().numpy(), rl) < 1e-5


# ------------------------------------------------------------------ the differentiable configuration
CFG4 = dict(dims=(500, 400, 300), R=30, B=8, log2b=15, noise=0.01, seed=4)


@pytest.fixture(scope="module")
def cfg4(dev):
    c = CFG4
    T, w, F0 = synth.planted_cp(c["dims"], c["R"], c["noise"], c["seed"])
    h, g = tsk.cs_hashes(c["seed"], c["B"], c["log2b"], list(c["dims"]), dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, c["log2b"])
    Xh = tsk.sketch_rfft(S)
    return dict(T=T, h=h, g=g, S=S, Xh=Xh, w=w, F0=F0)


def test_cfg4_sampled_sketch_and_loss_gradient_parity(dev, cfg4):
    c = CFG4
    b = 1 << c["log2b"]
    ho, go = O.cs_hashes(c["seed"], c["B"], c["log2b"], list(c["dims"]))
    Sg = np.real(cfg4["S"].cpu().numpy()).astype(np.float64)
    T64 = cfg4["T"].astype(np.float64)
    ref0 = np.real(O.sketch_tensor_asym(T64, ho[0], go[0], b))
    assert rel(Sg[0], ref0) < 1e-5
    params = _cp_params(dev, c["dims"], c["R"], 5)
    loss, *grads = tsk.cp_sketch_loss(cfg4["Xh"], cfg4["h"], cfg4["g"], c["dims"], *params)
    pg = [p.cpu().numpy().astype(np.float64) for p in params]
    assert abs(loss.item() - O.cp_sketch_loss(Sg, ho, go, b, *pg)) <= 1e-5 * loss.item()
    for got, ref in zip(grads, O.cp_sketch_grad(Sg, ho, go, b, *pg)):
        assert rel(got.cpu().numpy(), ref) < 1e-5


def test_cfg4_fitting_decreases_the_sketched_loss(dev, cfg4):
    """200 gradient steps through the autograd function, then ALS sweeps (Alg. 2 with Eq. 15)."""
    c = CFG4
    dims = c["dims"]
    params = [p.clone().requires_grad_(True) for p in _cp_params(dev, dims, c["R"], 6)]
    opt = torch.optim.Adam(params, lr=0.02)
    first = None
    for _ in range(200):
        opt.zero_grad()
        loss = tsk.cp_loss(*params, cfg4["Xh"], cfg4["h"], cfg4["g"], dims)
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    final = tsk.cp_loss(*params, cfg4["Xh"], cfg4["h"], cfg4["g"], dims).item()
    # with per-entry noise 0.01 over 6e7 entries the noise energy (~6e3) dwarfs the rank-30 signal
    # (~50), so the loss cannot fall far; it must fall
    assert np.isfinite(final) and final < 0.9 * first
    # ALS from the same random start (Eq. 15 fits the full tensor, not the sketch, so it is not
    # compared with the gradient-descent end point, which has partly fitted the sketch's noise)
    start = _cp_params(dev, dims, c["R"], 6)
    factors = [p.contiguous() for p in start[1:]]
    before = tsk.cp_sketch_loss(cfg4["Xh"], cfg4["h"], cfg4["g"], dims, start[0], *factors,
                                with_grad=False).item()
    for _ in range(3):
        lam, factors = tsk.cp_als_step(cfg4["Xh"], cfg4["h"], cfg4["g"], dims, factors)
    tsk.check_status(dev)
    after = tsk.cp_sketch_loss(cfg4["Xh"], cfg4["h"], cfg4["g"], dims, lam, *factors,
                               with_grad=False).item()
    assert np.isfinite(after) and after < before


def test_als_recovers_a_noise_free_low_rank_model(dev):
    """Alg. 2 with Eq. 15 on an exactly rank-4 tensor: the sketched loss drops by orders of
    magnitude from a random start."""
    dims, R, B, log2b = (60, 50, 40), 4, 4, 14
    r = synth.rng(8)
    F0 = [r.standard_normal((R, d)) for d in dims]
    T = np.einsum("ri,rj,rk->ijk", *F0)
    h, g = tsk.cs_hashes(8, B, log2b, list(dims), dev)
    Xh = tsk.sketch_rfft(tsk.sketch_tensor(t32(T, dev), h, g, log2b))
    factors = [t32(r.standard_normal((R, d)), dev) for d in dims]
    lam = torch.ones(R, device=dev)
    start = tsk.cp_sketch_loss(Xh, h, g, dims, lam, *factors, with_grad=False).item()
    for _ in range(25):
        lam, factors = tsk.cp_als_step(Xh, h, g, dims, factors)
    tsk.check_status(dev)
    end = tsk.cp_sketch_loss(Xh, h, g, dims, lam, *factors, with_grad=False).item()
    assert end < 1e-2 * start, (start, end)
