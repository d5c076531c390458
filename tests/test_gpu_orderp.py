"""GPU parity of the order-p symmetric sketches (p = 3..6) through the C ABI against the order-p
oracle (oracle/orderp.py): hashes bit-exact; sketches and per-sketch T^(I,u,...,u),
T^(u,...,u) within 1e-5 relative (2-norm per vector, or of the per-sketch eigenvalues); Alg. 1
for order p step by step (1e-4); planted recovery."""
import itertools

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

tsk = pytest.importorskip("paper_1506_04448_gb300")
P = O.orderp


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def t32(x, dev):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device=dev)


def random_sketches(B, log2b, seed, dev):
    r = synth.rng(seed)
    S = (r.standard_normal((B, 1 << log2b)) + 1j * r.standard_normal((B, 1 << log2b))).astype(np.complex64)
    Sd = torch.from_numpy(S).to(dev)
    return Sd, tsk.sketch_fft(Sd)


@pytest.mark.parametrize("p,n,B,log2b,seed", [(3, 37, 3, 10, 1), (4, 37, 5, 8, 2), (5, 100, 2, 12, 3),
                                              (6, 7, 64, 9, 4), (4, 1, 1, 8, 2**63 + 9)])
def test_hashes_bit_exact(dev, p, n, B, log2b, seed):
    h, g = tsk.cs_hashes_p(seed, B, log2b, p, n, dev)
    ho, go = P.cs_hashes_p(seed, B, log2b, p, n)
    np.testing.assert_array_equal(h.cpu().numpy(), ho)
    np.testing.assert_array_equal(g.cpu().numpy(), go)


def test_order3_hashes_equal_cs_hashes(dev):
    h, g = tsk.cs_hashes_p(9, 4, 11, 3, 50, dev)
    h3, g3 = tsk.cs_hashes(9, 4, 11, [50], dev)
    assert torch.equal(h, h3[:, 0]) and torch.equal(g, g3[:, 0])


@pytest.mark.parametrize("p,n,B,log2b", [(3, 11, 2, 9), (4, 9, 3, 10), (5, 6, 2, 8), (6, 5, 2, 12),
                                         (4, 33, 2, 12)])
def test_sketch_tensor_p(dev, p, n, B, log2b):
    T = synth.rng(20 + p).standard_normal((n,) * p)
    h, g = tsk.cs_hashes_p(5 + p, B, log2b, p, n, dev)
    S = tsk.sketch_tensor_p(t32(T, dev), h, g, log2b).cpu().numpy()
    ho, go = P.cs_hashes_p(5 + p, B, log2b, p, n)
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(S[m], P.sketch_sym_p(T32, ho[m], go[m], 1 << log2b, p)) < 1e-5, m


@pytest.mark.parametrize("p,n,B,log2b", [(3, 13, 2, 9), (4, 9, 3, 10), (5, 7, 2, 8), (6, 5, 2, 12),
                                         (4, 40, 2, 12), (3, 1, 1, 8)])
def test_sketch_tensor_p_symmetric_wedge(dev, p, n, B, log2b):
    """The wedge-only build of a symmetric tensor equals the definition (all ordered tuples) and
    the GPU's full-read build."""
    X = synth.rng(60 + p).standard_normal((n,) * p)
    T = sum(np.transpose(X, q) for q in itertools.permutations(range(p))) / np.prod(range(1, p + 1))
    h, g = tsk.cs_hashes_p(15 + p, B, log2b, p, n, dev)
    Td = t32(T, dev)
    Sw = tsk.sketch_tensor_p(Td, h, g, log2b, symmetric=True).cpu().numpy()
    Sf = tsk.sketch_tensor_p(Td, h, g, log2b).cpu().numpy()
    ho, go = P.cs_hashes_p(15 + p, B, log2b, p, n)
    T32 = Td.cpu().numpy().astype(np.float64)
    for m in range(B):
        ref = P.sketch_sym_p(T32, ho[m], go[m], 1 << log2b, p)
        assert rel(Sw[m], ref) < 1e-5, m
        assert rel(Sw[m], Sf[m]) < 1e-5, m


@pytest.mark.parametrize("p,n,B,L,log2b", [(3, 37, 3, 2, 10), (4, 37, 4, 3, 8), (4, 100, 5, 2, 12),
                                           (5, 33, 3, 2, 11), (6, 20, 2, 2, 12), (6, 5, 40, 1, 9)])
def test_contract_p(dev, p, n, B, L, log2b):
    b = 1 << log2b
    S, FS = random_sketches(B, log2b, 30 + p + n, dev)
    h, g = tsk.cs_hashes_p(40 + p, B, log2b, p, n, dev)
    ho, go = P.cs_hashes_p(40 + p, B, log2b, p, n)
    U = synth.rng(50 + n).standard_normal((L, n))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    Ud = t32(U, dev)
    out = tsk.contract_p(FS, S, h, g, Ud, p, per_sketch=True)
    Sg = S.cpu().numpy().astype(np.complex128)
    Ug = Ud.cpu().numpy().astype(np.float64)
    Vall, lam_all = out["Vall"].cpu().numpy(), out["lam_all"].cpu().numpy()
    Vmed, lam_med = out["Vmed"].cpu().numpy(), out["lam_med"].cpu().numpy()
    for tau in range(L):
        refs = np.stack([P.estimate_iuu_p(Sg[m], Ug[tau], ho[m], go[m], b, p) for m in range(B)])
        lrefs = np.array([P.estimate_uuu_p(Sg[m], Ug[tau], ho[m], go[m], b, p) for m in range(B)])
        for m in range(B):
            assert rel(Vall[tau, m], refs[m]) < 1e-5, (tau, m)
        assert rel(Vmed[tau], O.median_rows(refs)) < 1e-5
        scale = np.linalg.norm(lrefs) / np.sqrt(B) + np.linalg.norm(refs) / np.sqrt(B)
        assert np.max(np.abs(lam_all[tau] - lrefs)) < 1e-5 * scale
        assert abs(lam_med[tau] - O.median(lrefs)) < 1e-5 * scale
        # T^(u,...,u) = <u, T^(I,u,...,u)> per sketch (the gradient form is homogeneous of degree p)
        assert np.max(np.abs(Vall[tau] @ Ug[tau] - lam_all[tau])) < 1e-5 * scale


def test_order3_equals_the_app_b_kernels(dev):
    """At p = 3 the order-p kernel and the App. B contraction kernels compute the same values."""
    n, B, L, log2b = 45, 4, 3, 11
    S, FS = random_sketches(B, log2b, 77, dev)
    h, g = tsk.cs_hashes_p(8, B, log2b, 3, n, dev)
    U = synth.rng(78).standard_normal((L, n))
    Ud = t32(U / np.linalg.norm(U, axis=1, keepdims=True), dev)
    out = tsk.contract_p(FS, S, h, g, Ud, 3, per_sketch=True)
    _, Vall = tsk.contract_iuu(FS, S, h[:, None, :], g[:, None, :], Ud, return_all=True)
    _, lam_all = tsk.contract_uuu(FS, S, h[:, None, :], g[:, None, :], Ud, return_all=True)
    assert rel(out["Vall"].cpu().numpy(), Vall.cpu().numpy()) < 1e-5
    assert rel(out["lam_all"].cpu().numpy(), lam_all.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("p,n", [(4, 4), (5, 4)])
def test_collision_free_is_exact(dev, p, n):
    log2b = int(np.ceil(np.log2((p + 1) ** n)))
    T = synth.rng(90 + p).standard_normal((n,) * p)
    T = sum(np.transpose(T, q) for q in itertools.permutations(range(p)))
    hv = np.array([(p + 1) ** i for i in range(n)], dtype=np.int32)
    gv = synth.rng(91).integers(0, P.roots_order(p), n)
    h = torch.tensor(hv[None, :], dtype=torch.int32, device=dev)
    g = torch.tensor(gv[None, :], dtype=torch.uint8, device=dev)
    S = tsk.sketch_tensor_p(t32(T, dev), h, g, log2b)
    FS = tsk.sketch_fft(S)
    U = synth.rng(92).standard_normal((2, n))
    Ud = t32(U / np.linalg.norm(U, axis=1, keepdims=True), dev)
    out = tsk.contract_p(FS, S, h, g, Ud, p)
    T32 = T.astype(np.float32).astype(np.float64)
    Ug = Ud.cpu().numpy().astype(np.float64)
    for tau in range(2):
        assert rel(out["Vmed"][tau].cpu().numpy(), P.exact_iuu_p(T32, Ug[tau])) < 1e-5
        assert abs(out["lam_med"][tau].item() - P.exact_uuu_p(T32, Ug[tau])) < 1e-5 * np.linalg.norm(T32)


def planted_order_p(n, k, p, noise, seed):
    """sum_r lam_r a_r^{(x)p} (orthonormal a_r, lam ~ U[1, 2]) plus i.i.d. Gaussian noise."""
    A = synth.orthonormal_columns(n, k, seed)
    lam = synth.rng(seed + 1).uniform(1.0, 2.0, k)
    T = P.symmetric_rank1_sum(lam, A, p)
    if noise:
        T = T + noise * synth.rng(seed + 2).standard_normal((n,) * p)
    return T, lam, A


@pytest.mark.parametrize("p,n,k,L,T_it,B,log2b", [(4, 12, 2, 3, 4, 3, 10), (5, 8, 2, 2, 3, 2, 12),
                                                 (3, 20, 2, 3, 4, 4, 10)])
def test_rtpm_p_stepwise_parity(dev, p, n, k, L, T_it, B, log2b):
    from rtpm_check import check_rtpm_p_stepwise
    T, _, _ = planted_order_p(n, k, p, 0.01, 100 + p)
    h, g = tsk.cs_hashes_p(101 + p, B, log2b, p, n, dev)
    S = tsk.sketch_tensor_p(t32(T, dev), h, g, log2b)
    U0 = t32(synth.gaussian_inits(k, L, n, 102 + p), dev)
    res = tsk.robust_power_method_p(S, h, g, U0, T_it, p, return_deflated=True, return_trace=True)
    tsk.check_status(dev)
    host = {key: val.cpu().numpy() for key, val in res.items()}
    ho, go = P.cs_hashes_p(101 + p, B, log2b, p, n)
    assert check_rtpm_p_stepwise(host, S.cpu().numpy().astype(np.complex128), ho, go, 1 << log2b, p,
                                 U0.cpu().numpy().astype(np.float64), T_it) == k * T_it * L


def test_rtpm_order4_recovers_planted_components(dev):
    """Noise-free order-4 tensor with three orthonormal components: Alg. 1 on colliding order-4
    sketches finds them (even order: up to sign)."""
    p, n, k = 4, 30, 3
    T, lam, A = planted_order_p(n, k, p, 0.0, 7)
    h, g = tsk.cs_hashes_p(3, 10, 12, p, n, dev)
    S = tsk.sketch_tensor_p(t32(T, dev), h, g, 12)
    U0 = t32(synth.gaussian_inits(k, 12, n, 8), dev)
    res = tsk.robust_power_method_p(S, h, g, U0, 20, p)
    tsk.check_status(dev)
    V = res["V"].cpu().numpy()
    lam_hat = res["lam"].cpu().numpy()
    # planted eigenvalues closer than the sketch noise may come out in either order, so each
    # recovered component is matched to the planted one it is aligned with
    match = [int(np.argmax(np.abs(A.T @ V[r]))) for r in range(k)]
    assert sorted(match) == list(range(k))
    for r in range(k):
        assert abs(V[r] @ A[:, match[r]]) > 0.99
        assert lam_hat[r] == pytest.approx(lam[match[r]], rel=0.05)


def test_order_p_argument_errors(dev):
    with pytest.raises(tsk.TskError):
        tsk.cs_hashes_p(1, 2, 10, 7, 5, dev)          # p outside 3..6
    S, FS = random_sketches(2, 13, 1, dev)
    h, g = tsk.cs_hashes_p(1, 2, 13, 4, 5, dev)
    with pytest.raises(tsk.TskError):
        tsk.contract_p(FS, S, h, g, t32(np.ones((1, 5)), dev), 4)   # b = 2^13 above the limit
