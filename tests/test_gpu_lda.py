"""GPU parity of the spectral-LDA path (App. D, Alg. 3) against the FP64 oracle.

Tolerances (FP32 arithmetic on the device, FP64 in the oracle):
* M1^, M2^ X: float atomics over <= a few thousand documents per word -> 2e-5 of the largest
  entry;
* whitening: W^T M2^ W = I to 2e-4 (M2^ Q is accumulated in FP32, the Rayleigh-Ritz step and
  Jacobi in FP64), Ritz values to 1e-4 relative;
* M3^(W,W,W): FP32 running sums over <= 4096 documents, FP64 across them -> 2e-5 of the
  largest entry;
* sketches of the device's own M3: the sketch build's FP32 accumulation -> 1e-5;
* recovery: FP64 Cholesky, FP32 output -> 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from oracle import lda as L

pytestmark = pytest.mark.gpu

dev = torch.device("cuda", 0)


def corpus(V, k, D, seed, mean_len, extra_short=True, alpha=0.3, beta=0.1):
    c = synth.lda_corpus(V, k, D, seed, alpha=alpha, beta=beta, mean_len=mean_len)
    if extra_short:   # empty documents and documents of lengths 1 and 2 (the degenerate cases)
        ip = list(c["indptr"])
        idx = list(c["idx"])
        cnt = list(c["cnt"])
        for words, counts in [([], []), ([3], [1]), ([], []), ([5, 7], [1, 1]), ([2], [2])]:
            idx += words
            cnt += counts
            ip.append(ip[-1] + len(words))
        c = dict(c, indptr=np.array(ip, dtype=np.int64), idx=np.array(idx, dtype=np.int32),
                 cnt=np.array(cnt, dtype=np.int32))
    return c


def on_dev(c):
    return (torch.from_numpy(np.asarray(c["indptr"], dtype=np.int64)).to(dev),
            torch.from_numpy(np.asarray(c["idx"], dtype=np.int32)).to(dev),
            torch.from_numpy(np.asarray(c["cnt"], dtype=np.int32)).to(dev))


def tsk():
    import paper_1506_04448_gb300 as T
    return T


@pytest.mark.parametrize("c_cols", [7, 130])
def test_m2_apply(c_cols):
    T = tsk()
    V, k = 300, 5
    c = corpus(V, k, 3000, 1, mean_len=30)
    a0 = k * 0.3
    X = synth.gaussian_matrix(V, c_cols, 2).astype(np.float32)
    ref = L.moment2(c, V, a0) @ X.astype(np.float64)
    Y = T.lda_m2_apply(*on_dev(c), V, a0, torch.from_numpy(X).to(dev)).cpu().numpy()
    T.check_status(dev)
    np.testing.assert_allclose(Y, ref, rtol=0, atol=2e-5 * np.abs(ref).max())


def test_whiten():
    T = tsk()
    V, k, p = 400, 6, 10
    c = corpus(V, k, 6000, 3, mean_len=50)
    a0 = k * 0.3
    Om = synth.gaussian_matrix(V, k + p, 4).astype(np.float32)
    W, sig, M1 = T.lda_whiten(*on_dev(c), V, k, a0, torch.from_numpy(Om).to(dev), 2)
    T.check_status(dev)
    W = W.cpu().double().numpy()
    sig = sig.cpu().numpy()
    M2 = L.moment2(c, V, a0)
    M1o = L.moment1(c, V)
    np.testing.assert_allclose(M1.cpu().numpy(), M1o, rtol=0, atol=2e-6 * M1o.max())
    np.testing.assert_allclose(W.T @ M2 @ W, np.eye(k), atol=2e-4)
    Wo, sig_o = L.whiten(M2, k)
    np.testing.assert_allclose(sig, sig_o, rtol=1e-4)
    # same k-dimensional subspace: the projectors onto span(W) agree
    Pg = W @ np.linalg.pinv(W)
    Po = Wo @ np.linalg.pinv(Wo)
    vals = np.sort(np.linalg.eigvalsh(M2))[::-1]
    assert vals[k] < 0.5 * vals[k - 1]                 # a real spectral gap in this corpus
    assert np.abs(Pg - Po).max() < 1e-3


@pytest.mark.parametrize("V,k,D,mean_len", [(200, 3, 2500, 20), (300, 10, 2000, 30),
                                             (400, 13, 1500, 25), (500, 33, 600, 40)])
def test_whitened_m3(V, k, D, mean_len):
    T = tsk()
    c = corpus(V, k, D, 5 + k, mean_len=mean_len)
    a0 = k * 0.3
    W = (synth.gaussian_matrix(V, k, 6) / np.sqrt(V)).astype(np.float32)
    ref = L.whitened_m3(c, W.astype(np.float64), a0)
    M3 = T.lda_whitened_m3(*on_dev(c), V, torch.from_numpy(W).to(dev), a0).cpu().numpy()
    T.check_status(dev)
    np.testing.assert_allclose(M3, ref, rtol=0, atol=2e-5 * np.abs(ref).max())
    # exactly symmetric by construction
    assert np.array_equal(M3, M3.transpose(1, 0, 2)) and np.array_equal(M3, M3.transpose(2, 1, 0))


def test_whitened_m3_many_splits_streamed_check():
    """More documents than one FP32 split (4096): check contractions M3(x,x,x), M3(I,x,x)
    against the oracle's streamed evaluation at O(nnz k) cost."""
    T = tsk()
    V, k, D = 2000, 20, 30000
    c = corpus(V, k, D, 9, mean_len=60, alpha=0.1, beta=0.05)
    a0 = k * 0.1
    W = (synth.gaussian_matrix(V, k, 8) / np.sqrt(V)).astype(np.float32)
    M3 = T.lda_whitened_m3(*on_dev(c), V, torch.from_numpy(W).to(dev), a0).cpu().double().numpy()
    T.check_status(dev)
    for s in range(3):
        x = synth.rng(40 + s).standard_normal(k)
        xxx, ixx = L.whitened_m3_contract(c, W.astype(np.float64), a0, x)
        # |sum_bc d_abc x_b x_c| <= max|d| (sum|x|)^2 with max|d| <= 2e-5 max|M3|
        tol = 2e-5 * np.abs(M3).max() * np.abs(x).sum() ** 2
        np.testing.assert_allclose(np.einsum("abc,b,c->a", M3, x, x), ixx, rtol=0, atol=tol)
        assert abs(np.einsum("abc,a,b,c", M3, x, x, x) - xxx) <= tol * np.abs(x).sum()


def test_whitened_m3_tensor_core_groups_and_ragged_documents():
    """k = 100 (5050 pair rows over 40 tiles of the tensor-core document term) and 20001
    documents: many 1024-document compensated groups and several document splits, with a last
    step of a single document; checked by the oracle's streamed contractions."""
    T = tsk()
    V, k, D = 3000, 100, 20001
    c = synth.lda_corpus(V, k, D, 77, alpha=0.1, beta=0.02, mean_len=60)
    a0 = k * 0.1
    W = (synth.gaussian_matrix(V, k, 78) / np.sqrt(V)).astype(np.float32)
    M3 = T.lda_whitened_m3(*on_dev(c), V, torch.from_numpy(W).to(dev), a0).cpu().double().numpy()
    T.check_status(dev)
    assert np.array_equal(M3, M3.transpose(1, 0, 2)) and np.array_equal(M3, M3.transpose(0, 2, 1))
    for s in range(3):
        x = synth.rng(80 + s).standard_normal(k)
        xxx, ixx = L.whitened_m3_contract(c, W.astype(np.float64), a0, x)
        tol = 2e-5 * np.abs(M3).max() * np.abs(x).sum() ** 2
        np.testing.assert_allclose(np.einsum("abc,b,c->a", M3, x, x), ixx, rtol=0, atol=tol)
        assert abs(np.einsum("abc,a,b,c", M3, x, x, x) - xxx) <= tol * np.abs(x).sum()


def test_sketch_m3_and_paper_route():
    T = tsk()
    V, k, D = 300, 8, 1200
    c = corpus(V, k, D, 12, mean_len=30)
    a0 = 2.4
    W = (synth.gaussian_matrix(V, k, 13) / np.sqrt(V)).astype(np.float32)
    B, log2b = 3, 10
    h, g = T.cs_hashes(77, B, log2b, [k], dev)
    M3, S = T.lda_sketch_m3(*on_dev(c), V, torch.from_numpy(W).to(dev), a0, h, g, log2b)
    T.check_status(dev)
    M3 = M3.cpu().double().numpy()
    S = S.cpu().numpy()
    hn, gn = O.cs_hashes(77, B, log2b, [k])
    for m in range(B):
        own = O.sketch_tensor_sym(M3, hn[m, 0], gn[m, 0], 1 << log2b)
        np.testing.assert_allclose(S[m], own, rtol=0, atol=1e-5 * np.abs(own).max())
        paper = L.sketch_m3_per_doc(c, W.astype(np.float64), a0, hn[m, 0], gn[m, 0], 1 << log2b)
        np.testing.assert_allclose(S[m], paper, rtol=0, atol=5e-5 * np.abs(paper).max())


@pytest.mark.parametrize("V,k", [(50, 4), (3000, 37)])
def test_recover(V, k):
    T = tsk()
    r = synth.rng(k)
    W = r.standard_normal((V, k)).astype(np.float32)
    lam = r.uniform(0.5, 3.0, k)
    Vv = np.ascontiguousarray(np.linalg.qr(r.standard_normal((k, k)))[0].T, dtype=np.float32)
    a0 = 1.7
    a_ref, mu_ref = L.recover(lam, Vv.astype(np.float64), W.astype(np.float64), a0)
    a, mu = T.lda_recover(torch.from_numpy(W).to(dev), a0, torch.from_numpy(lam).to(dev),
                          torch.from_numpy(Vv).to(dev))
    T.check_status(dev)
    np.testing.assert_allclose(a.cpu().numpy(), a_ref, rtol=1e-12)
    np.testing.assert_allclose(mu.cpu().numpy(), mu_ref, rtol=0, atol=1e-5 * np.abs(mu_ref).max())


def test_bad_word_id_is_reported():
    T = tsk()
    V = 10
    ip = torch.tensor([0, 2, 3], dtype=torch.int64, device=dev)
    idx = torch.tensor([1, 12, 4], dtype=torch.int32, device=dev)     # 12 >= V
    cnt = torch.tensor([2, 1, 3], dtype=torch.int32, device=dev)
    X = torch.ones((V, 4), dtype=torch.float32, device=dev)
    T.lda_m2_apply(ip, idx, cnt, V, 1.0, X)
    assert T.ctx_status(dev) == -1          # TSK_EINVAL, skipped entry
    assert T.ctx_status(dev) == 0           # cleared


def test_spectral_lda_recovers_planted_topics():
    """Alg. 3 end to end on a planted corpus: topics and Dirichlet weights come back."""
    T = tsk()
    V, k, D = 500, 4, 40000
    alpha = 0.25
    c = synth.lda_corpus(V, k, D, 21, alpha=alpha, beta=0.05, mean_len=80)
    a0 = k * alpha
    Om = synth.gaussian_matrix(V, k + 8, 22).astype(np.float32)
    U0 = synth.gaussian_inits(k, 20, k, 23).astype(np.float32)
    res = T.spectral_lda(*on_dev(c), V, k, a0, torch.from_numpy(Om).to(dev),
                         torch.from_numpy(U0).to(dev), B=10, log2b=12, T=30, seed=24)
    T.check_status(dev)
    mu = res["mu"].cpu().numpy()
    al = res["alpha"].cpu().numpy()
    Phi = c["Phi"]
    for i in range(k):
        j = int(np.argmin(np.abs(mu - Phi[i]).sum(1)))
        assert np.abs(mu[j] - Phi[i]).sum() < 0.25, (i, np.abs(mu[j] - Phi[i]).sum())
        assert abs(al[j] - alpha) < 0.5 * alpha


def test_whitened_m3_at_benchmark_dimensions():
    """V = 50000 words and k = 100 topics as in the benchmarked corpus (13 blocks of 8 topics,
    3640 wedge units, 104-wide padded rows), with 4000 documents so that the oracle's streamed
    O(nnz k) contractions stay cheap; random whitening matrix (the dense M2 of V = 50000 is
    beyond the oracle)."""
    T = tsk()
    V, k, D = 50000, 100, 4000
    c = synth.lda_corpus(V, k, D, 31, alpha=0.1, beta=0.01, mean_len=200)
    a0 = k * 0.1
    W = (synth.gaussian_matrix(V, k, 32) / np.sqrt(V)).astype(np.float32)
    M3 = T.lda_whitened_m3(*on_dev(c), V, torch.from_numpy(W).to(dev), a0).cpu().double().numpy()
    T.check_status(dev)
    assert np.array_equal(M3, M3.transpose(1, 0, 2)) and np.array_equal(M3, M3.transpose(0, 2, 1))
    for s in range(3):
        x = synth.rng(50 + s).standard_normal(k)
        xxx, ixx = L.whitened_m3_contract(c, W.astype(np.float64), a0, x)
        tol = 2e-5 * np.abs(M3).max() * np.abs(x).sum() ** 2
        np.testing.assert_allclose(np.einsum("abc,b,c->a", M3, x, x), ixx, rtol=0, atol=tol)
        assert abs(np.einsum("abc,a,b,c", M3, x, x, x) - xxx) <= tol * np.abs(x).sum()
