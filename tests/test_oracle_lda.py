"""Pins for the spectral-LDA oracle (App. D, Alg. 3): facts fixed by the model, the paper's
closed forms and brute force, not by the oracle itself.

* N_d by enumeration of ordered distinct token-position triples (the definition of the
  empirical third moment) against the case formula;
* unbiasedness of the per-document estimators, by exact enumeration of all documents of a
  fixed length drawn from a fixed word distribution;
* Eq. td (whitened per-document moment from p = W^T n) against N_d(W, W, W) by einsum;
* Eq. moment2/moment3 applied to the exact LDA raw moments (Dirichlet moments) give the
  paper's closed forms sum_i alpha_i mu_i mu_i^T / (alpha0 (alpha0+1)) and
  2 sum_i alpha_i mu_i^(x)3 / (alpha0 (alpha0+1)(alpha0+2));
* whitening satisfies W^T M2 W = I and the eigen-equation; recovery (Alg. 3, line 6) returns
  the planted alpha and topics from the exact moments;
* the paper's per-document sketch route equals the sketch (Eq. 7) of the dense moment.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle import lda as L


def small_corpus(seed=3, V=30, k=3, D=200, alpha=0.5, beta=0.3, mean_len=8):
    return synth.lda_corpus(V, k, D, seed, alpha=alpha, beta=beta, mean_len=mean_len)


# ------------------------------------------------------------------ N_d, the per-document moment
@pytest.mark.parametrize("tokens", [[0, 0, 0, 1, 2, 2], [1, 1, 1, 1], [0, 1, 2], [2, 0, 2, 1, 0, 2, 2]])
def test_doc_moment3_matches_enumeration_of_distinct_positions(tokens):
    V = 3
    bf = L.doc_moment3_bruteforce(tokens)
    ids, n = np.unique(np.array(tokens), return_counts=True)
    N = L.doc_moment3(ids, n.astype(float), V)
    dense = np.zeros((V, V, V))
    for key, v in bf.items():
        dense[key] = v
    np.testing.assert_allclose(N, dense, rtol=0, atol=1e-15)
    assert abs(N.sum() - 1.0) < 1e-14             # a probability distribution over triples


def _multinomial_docs(pi, m):
    """Every word-count vector of length-m documents over len(pi) words, with its probability."""
    V = len(pi)
    for combo in itertools.combinations_with_replacement(range(V), m):
        n = np.bincount(combo, minlength=V)
        coef = math.factorial(m)                  # multinomial coefficient
        for c in n:
            coef //= math.factorial(int(c))
        yield n, coef * np.prod(np.asarray(pi) ** n)


@pytest.mark.parametrize("m", [3, 4, 5])
def test_per_document_estimators_are_unbiased(m):
    """E over documents of length m with i.i.d. words ~ pi: N_d -> pi^(x)3, E2_d -> pi pi^T."""
    pi = np.array([0.5, 0.3, 0.2])
    V = 3
    E3 = np.zeros((V, V, V))
    E2 = np.zeros((V, V))
    tot = 0.0
    for n, prob in _multinomial_docs(pi, m):
        ids = np.nonzero(n)[0]
        E3 += prob * L.doc_moment3(ids, n[ids].astype(float), V)
        c = {"indptr": np.array([0, len(ids)]), "idx": ids, "cnt": n[ids]}
        E2 += prob * L.raw_moment2(c, V)
        tot += prob
    assert abs(tot - 1) < 1e-14
    np.testing.assert_allclose(E3, np.einsum("a,b,c->abc", pi, pi, pi), atol=1e-15)
    np.testing.assert_allclose(E2, np.outer(pi, pi), atol=1e-15)


def test_eq_td_equals_whitened_case_formula():
    r = synth.rng(11)
    V, k = 7, 4
    W = r.standard_normal((V, k))
    ids = np.array([0, 2, 3, 6])
    n = np.array([3.0, 1.0, 4.0, 2.0])
    N = L.doc_moment3(ids, n, V)
    ref = np.einsum("ijl,ia,jb,lc->abc", N, W, W, W)
    np.testing.assert_allclose(L.whitened_doc_moment3(ids, n, W), ref, rtol=1e-12, atol=1e-14)


def test_whitened_raw_moments_match_dense_moments():
    c = small_corpus()
    V = 30
    W = synth.rng(4).standard_normal((V, 3))
    q, E2, E3 = L.whitened_raw_moments(c, W)
    np.testing.assert_allclose(q, W.T @ L.moment1(c, V), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(E2, W.T @ L.raw_moment2(c, V) @ W, rtol=1e-11, atol=1e-14)
    # E3 against the document-by-document dense N_d(W,W,W)
    m = L.doc_lengths(c)
    ref = np.zeros((3, 3, 3))
    cnt = 0
    for d in range(L.num_docs(c)):
        if m[d] < 3:
            continue
        ids, n = L.doc(c, d)
        ref += np.einsum("ijl,ia,jb,lc->abc", L.doc_moment3(ids, n, V)[np.ix_(ids, ids, ids)],
                         W[ids], W[ids], W[ids])
        cnt += 1
    np.testing.assert_allclose(E3, ref / cnt, rtol=1e-10, atol=1e-14)


# ------------------------------------------------------------------ Eq. moment2 / moment3
@pytest.mark.parametrize("alpha", [[0.1, 0.1, 0.1, 0.1], [0.3, 0.05, 0.7], [1.0, 2.0]])
def test_moment_combinations_give_lda_closed_forms(alpha):
    alpha = np.array(alpha)
    k, V = len(alpha), 6
    Phi = synth.rng(5).dirichlet(np.ones(V), size=k)
    a0 = alpha.sum()
    E1, E2, E3 = L.population_raw_moments(Phi, alpha)
    M2 = L.combine_m2(E1, E2, a0)
    M3 = L.combine_m3(E1, E2, E3, a0)
    M2_ref = sum(alpha[i] * np.outer(Phi[i], Phi[i]) for i in range(k)) / (a0 * (a0 + 1))
    M3_ref = 2 * sum(alpha[i] * np.einsum("a,b,c->abc", Phi[i], Phi[i], Phi[i])
                     for i in range(k)) / (a0 * (a0 + 1) * (a0 + 2))
    np.testing.assert_allclose(M2, M2_ref, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(M3, M3_ref, rtol=1e-11, atol=1e-16)


def test_population_raw_moments_against_monte_carlo():
    """The Dirichlet-moment formulas against sampled documents (statistical, generous)."""
    alpha = np.array([0.4, 0.2, 0.9])
    V = 4
    r = synth.rng(7)
    Phi = r.dirichlet(np.ones(V), size=3)
    E1, E2, _ = L.population_raw_moments(Phi, alpha)
    th = r.dirichlet(alpha, size=200000)
    pi = th @ Phi
    np.testing.assert_allclose(pi.mean(0), E1, atol=3e-3)
    np.testing.assert_allclose(np.einsum("da,db->ab", pi, pi) / len(pi), E2, atol=3e-3)


# ------------------------------------------------------------------ whitening and recovery
def test_whitening_identity_and_eigen_equation():
    c = small_corpus(D=400)
    V, k = 30, 3
    M2 = L.moment2(c, V, 1.5)
    W, sig = L.whiten(M2, k)
    np.testing.assert_allclose(W.T @ M2 @ W, np.eye(k), atol=1e-12)
    U = W * np.sqrt(sig)
    np.testing.assert_allclose(M2 @ U, U * sig, atol=1e-14)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    # top-k: no direction orthogonal to U has a larger Rayleigh quotient
    X = synth.rng(8).standard_normal((V, 200))
    X -= U @ (U.T @ X)
    rq = np.einsum("vi,vw,wi->i", X, M2, X) / np.einsum("vi,vi->i", X, X)
    assert rq.max() <= sig[-1] + 1e-12


@pytest.mark.parametrize("alpha", [[0.1] * 4, [0.5, 0.2, 0.3]])
def test_recovery_from_exact_moments_returns_planted_model(alpha):
    alpha = np.array(alpha)
    k, V = len(alpha), 9
    r = synth.rng(21)
    Phi = r.dirichlet(np.full(V, 0.5), size=k)
    a0 = alpha.sum()
    E1, E2, E3 = L.population_raw_moments(Phi, alpha)
    W, _ = L.whiten(L.combine_m2(E1, E2, a0), k)
    T = np.einsum("ijl,ia,jb,lc->abc", L.combine_m3(E1, E2, E3, a0), W, W, W)
    U0 = synth.gaussian_inits(k, 10, k, 3)
    res = O.rtpm_exact(T, U0, 60)
    a_hat, mu_hat = L.recover(res["lam"], res["V"], W, a0)
    for i in range(k):
        j = int(np.argmin(np.abs(mu_hat - Phi[i]).sum(1)))
        np.testing.assert_allclose(mu_hat[j], Phi[i], atol=1e-8)
        assert abs(a_hat[j] - alpha[i]) < 1e-8


# ------------------------------------------------------------------ the paper's sketch route
@pytest.mark.parametrize("b", [64, 256])
def test_per_document_sketch_route_equals_sketch_of_dense_moment(b):
    c = small_corpus(D=150)
    V, k = 30, 3
    W, _ = L.whiten(L.moment2(c, V, 1.5), k)
    log2b = int(np.log2(b))
    h, g = O.cs_hashes(5, 2, log2b, [k])
    for m in range(2):
        s_doc = L.sketch_m3_per_doc(c, W, 1.5, h[m, 0], g[m, 0], b)
        s_dense = O.sketch_tensor_sym(L.whitened_m3(c, W, 1.5), h[m, 0], g[m, 0], b)
        np.testing.assert_allclose(s_doc, s_dense, atol=1e-12 * np.abs(s_dense).max())


def test_streamed_contractions_match_dense_moment():
    c = small_corpus(D=300)
    V, k = 30, 3
    W = synth.rng(9).standard_normal((V, k))
    M3 = L.whitened_m3(c, W, 2.0)
    for s in range(3):
        x = synth.rng(100 + s).standard_normal(k)
        xxx, ixx = L.whitened_m3_contract(c, W, 2.0, x)
        assert abs(xxx - np.einsum("abc,a,b,c", M3, x, x, x)) < 1e-12 * max(1, abs(xxx))
        np.testing.assert_allclose(ixx, np.einsum("abc,b,c->a", M3, x, x), rtol=1e-11, atol=1e-13)
