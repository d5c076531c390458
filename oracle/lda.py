"""Oracle: spectral LDA moments, whitening, the whitened third moment and parameter recovery
(App. D, Alg. 3).

* Moments (App. D, Eq. moment1-3), with alpha0 = sum_k alpha_k:
      M1 = E[x1]
      M2 = E[x1 (x) x2] - alpha0/(alpha0+1) M1 (x) M1
      M3 = E[x1 (x) x2 (x) x3] - alpha0/(alpha0+2) (E[x1 (x) x2 (x) M1] + E[x1 (x) M1 (x) x2]
           + E[M1 (x) x1 (x) x2]) + 2 alpha0^2/((alpha0+1)(alpha0+2)) M1 (x) M1 (x) M1
  and, for the LDA model, M2 = sum_i alpha_i mu_i mu_i^T / (alpha0(alpha0+1)) and
  M3 = 2 sum_i alpha_i mu_i^(x)3 / (alpha0(alpha0+1)(alpha0+2)).
* Empirical moments from word counts n_d (length m_d = sum_i n_di).  Each document gives an
  unbiased estimate from DISTINCT token positions:
      E^[x1]              : n_d / m_d                                       (docs with m_d >= 1)
      E^[x1 (x) x2]       : (n_d n_d^T - diag(n_d)) / (m_d (m_d - 1))        (docs with m_d >= 2)
      E^[x1 (x) x2 (x) x3]: N_d, the count of ordered distinct position triples
                            / (m_d (m_d - 1)(m_d - 2))                      (docs with m_d >= 3)
  averaged over the documents that qualify (the 1/(m_d(m_d-1)(m_d-2)) weight and the average
  over documents are part of E^; Eq. td's sum over documents leaves them implicit).  N_d's
  case i = j = k is n_i(n_i - 1)(n_i - 2), and E^[x1 (x) x2 (x) M1^] is E^[x1 (x) x2] (x) M1^
  (Eq. applda_exxm's right-hand side, read per document as (p (x) p - sum_i n_i w_i (x) w_i)
  (x) q / (m_d (m_d - 1)) with q = W^T M1^).
* Whitened per-document third moment (App. D, Eq. td), with p = W^T n_d (printed "W n") and
  w_i the i-th row of W:
      T_d = p^(x)3 - sum_i n_i (w_i (x) w_i (x) p + w_i (x) p (x) w_i + p (x) w_i (x) w_i)
            + 2 sum_i n_i w_i^(x)3,   divided by m_d (m_d - 1)(m_d - 2).
* Whitening (Alg. 3, line 3): top-k eigenpairs (U, sigma) of M2^, W_ik = U_ik / sqrt(sigma_k),
  so that W^T M2^ W = I_k.
* Recovery (Alg. 3, line 6): alpha^_i = 4 alpha0 (alpha0+1) / ((alpha0+2)^2 lambda_i^2),
  mu^_i = (alpha0+2)/2 lambda_i (W^+)^T v_i.
* The paper's own sketch route (App. D): per document one count sketch of p, its cube in the
  frequency domain; the per-word sums r_i = sum_d a_d n_di p_d and c_i = sum_d a_d n_di are
  folded in once after the scan.  `sketch_m3_per_doc` follows that route literally so that
  it can be checked against the sketch of the dense whitened moment.

Corpora are CSR dicts {"indptr", "idx", "cnt", ...} as made by synth.lda_corpus.  Everything
is float64.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import itertools

import numpy as np

from .conv import fft as _fft, ifft as _ifft
from .sketch import count_sketch


def doc(corpus, d: int):
    """(word ids, counts) of document d."""
    a, e = int(corpus["indptr"][d]), int(corpus["indptr"][d + 1])
    return (np.asarray(corpus["idx"][a:e], dtype=np.int64),
            np.asarray(corpus["cnt"][a:e], dtype=np.float64))


def doc_lengths(corpus) -> np.ndarray:
    """m_d for every document."""
    cnt = np.asarray(corpus["cnt"], dtype=np.float64)
    ip = np.asarray(corpus["indptr"], dtype=np.int64)
    c = np.concatenate([[0.0], np.cumsum(cnt)])
    return c[ip[1:]] - c[ip[:-1]]


def num_docs(corpus) -> int:
    return int(len(corpus["indptr"]) - 1)


# ----------------------------------------------------------------------------- raw moments

def moment1(corpus, V: int) -> np.ndarray:
    """M1^ = E^[x1]: mean of n_d / m_d over the documents with m_d >= 1 (Eq. moment1)."""
    m = doc_lengths(corpus)
    M1 = np.zeros(V)
    cnt = 0
    for d in range(num_docs(corpus)):
        if m[d] < 1:
            continue
        i, n = doc(corpus, d)
        np.add.at(M1, i, n / m[d])
        cnt += 1
    return M1 / max(cnt, 1)


def raw_moment2(corpus, V: int) -> np.ndarray:
    """E^[x1 (x) x2] (dense V x V): mean over documents with m_d >= 2 of
    (n n^T - diag n) / (m (m - 1)) -- pairs of distinct token positions."""
    m = doc_lengths(corpus)
    E2 = np.zeros((V, V))
    cnt = 0
    for d in range(num_docs(corpus)):
        if m[d] < 2:
            continue
        i, n = doc(corpus, d)
        blk = np.outer(n, n)
        blk[np.arange(len(i)), np.arange(len(i))] -= n
        E2[np.ix_(i, i)] += blk / (m[d] * (m[d] - 1))
        cnt += 1
    return E2 / max(cnt, 1)


def moment2(corpus, V: int, alpha0: float) -> np.ndarray:
    """M2^ = E^[x1 (x) x2] - alpha0/(alpha0+1) M1^ M1^T (Eq. moment2), dense."""
    M1 = moment1(corpus, V)
    return raw_moment2(corpus, V) - alpha0 / (alpha0 + 1.0) * np.outer(M1, M1)


def m2_apply(corpus, V: int, alpha0: float, X: np.ndarray) -> np.ndarray:
    """M2^ X without forming M2^ (the operator the range finder uses)."""
    return moment2(corpus, V, alpha0) @ X


def doc_moment3_bruteforce(tokens) -> dict:
    """N_d of one document written as a token list, by enumerating every ordered triple of
    DISTINCT token positions (a, b, c): entry (w_a, w_b, w_c) gains 1 / (m (m-1) (m-2)).
    Returns {(i, j, k): value}; tiny documents only."""
    m = len(tokens)
    out: dict = {}
    for a, b_, c in itertools.permutations(range(m), 3):
        key = (tokens[a], tokens[b_], tokens[c])
        out[key] = out.get(key, 0.0) + 1.0
    den = m * (m - 1) * (m - 2)
    return {k: v / den for k, v in out.items()}


def doc_moment3(ids: np.ndarray, n: np.ndarray, V: int) -> np.ndarray:
    """N_d (dense V^3) from the case formula: n_i n_j n_k for distinct indices,
    n_i (n_i - 1) n_k when exactly two agree (in any of the three placements),
    n_i (n_i - 1)(n_i - 2) when i = j = k; divided by m (m-1)(m-2)."""
    cnt = np.zeros(V)
    cnt[ids] = n
    m = cnt.sum()
    N = np.zeros((V, V, V))
    for i in ids:
        for j in ids:
            for k in ids:
                if i == j == k:
                    v = cnt[i] * (cnt[i] - 1) * (cnt[i] - 2)
                elif i == j:
                    v = cnt[i] * (cnt[i] - 1) * cnt[k]
                elif j == k:
                    v = cnt[i] * cnt[j] * (cnt[j] - 1)
                elif i == k:
                    v = cnt[i] * (cnt[i] - 1) * cnt[j]
                else:
                    v = cnt[i] * cnt[j] * cnt[k]
                N[i, j, k] = v
    return N / (m * (m - 1) * (m - 2))


# ----------------------------------------------------------------------------- whitened moments

def whitened_doc_moment3(ids: np.ndarray, n: np.ndarray, W: np.ndarray) -> np.ndarray:
    """T_d = N_d(W, W, W) by Eq. td: p^(x)3 - sum_i n_i (w_i w_i p + w_i p w_i + p w_i w_i)
    + 2 sum_i n_i w_i^(x)3, divided by m (m-1)(m-2); p = W^T n."""
    Wd = np.asarray(W, dtype=np.float64)[ids]            # rows w_i of the words present
    p = Wd.T @ n
    m = n.sum()
    T = np.einsum("a,b,c->abc", p, p, p)
    for wi, ni in zip(Wd, n):
        T -= ni * (np.einsum("a,b,c->abc", wi, wi, p) + np.einsum("a,b,c->abc", wi, p, wi)
                   + np.einsum("a,b,c->abc", p, wi, wi))
        T += 2.0 * ni * np.einsum("a,b,c->abc", wi, wi, wi)
    return T / (m * (m - 1) * (m - 2))


def whitened_raw_moments(corpus, W: np.ndarray):
    """(q, E2w, E3w) = (W^T M1^, E^[x1 (x) x2](W, W), E^[x1 (x) x2 (x) x3](W, W, W)), each the
    average over the documents that qualify (m_d >= 1, 2, 3)."""
    W = np.asarray(W, dtype=np.float64)
    k = W.shape[1]
    m = doc_lengths(corpus)
    q = np.zeros(k)
    E2 = np.zeros((k, k))
    E3 = np.zeros((k, k, k))
    c1 = c2 = c3 = 0
    for d in range(num_docs(corpus)):
        ids, n = doc(corpus, d)
        md = m[d]
        if md >= 1:
            q += W[ids].T @ n / md
            c1 += 1
        if md >= 2:
            Wd = W[ids]
            p = Wd.T @ n
            E2 += (np.outer(p, p) - (Wd.T * n) @ Wd) / (md * (md - 1))
            c2 += 1
        if md >= 3:
            E3 += whitened_doc_moment3(ids, n, W)
            c3 += 1
    return q / max(c1, 1), E2 / max(c2, 1), E3 / max(c3, 1)


def combine_m3(q: np.ndarray, E2: np.ndarray, E3: np.ndarray, alpha0: float) -> np.ndarray:
    """Eq. moment3 from raw moments (any coordinates): E3 - alpha0/(alpha0+2) (E2 (x) q + the two
    other placements of q) + 2 alpha0^2/((alpha0+1)(alpha0+2)) q^(x)3."""
    a = alpha0 / (alpha0 + 2.0)
    c = 2.0 * alpha0 ** 2 / ((alpha0 + 1.0) * (alpha0 + 2.0))
    X = (np.einsum("ab,c->abc", E2, q) + np.einsum("ac,b->abc", E2, q)
         + np.einsum("bc,a->abc", E2, q))
    return E3 - a * X + c * np.einsum("a,b,c->abc", q, q, q)


def combine_m2(q: np.ndarray, E2: np.ndarray, alpha0: float) -> np.ndarray:
    """Eq. moment2 from raw moments: E2 - alpha0/(alpha0+1) q q^T."""
    return E2 - alpha0 / (alpha0 + 1.0) * np.outer(q, q)


def whitened_m3(corpus, W: np.ndarray, alpha0: float) -> np.ndarray:
    """M3^(W, W, W) (k x k x k), the tensor Alg. 3 sketches (line 4)."""
    q, E2, E3 = whitened_raw_moments(corpus, W)
    return combine_m3(q, E2, E3, alpha0)


def whitened_m3_contract(corpus, W: np.ndarray, alpha0: float, x: np.ndarray):
    """(M3^(W,W,W)(x,x,x), M3^(W,W,W)(I,x,x)) evaluated document by document at O(nnz k) cost,
    for corpora too large for the dense oracle.  Per document, with s = p.x, t_i = w_i.x:
      T_d(x,x,x) = s^3 - 3 sum_i n_i t_i^2 s + 2 sum_i n_i t_i^3,
      T_d(I,x,x) = p s^2 - sum_i n_i (2 w_i t_i s + p t_i^2) + 2 sum_i n_i w_i t_i^2."""
    W = np.asarray(W, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    k = W.shape[1]
    ip = np.asarray(corpus["indptr"], dtype=np.int64)
    ids = np.asarray(corpus["idx"], dtype=np.int64)
    n = np.asarray(corpus["cnt"], dtype=np.float64)
    D = len(ip) - 1
    docs = np.repeat(np.arange(D), np.diff(ip))
    m = np.bincount(docs, weights=n, minlength=D)
    t = W[ids] @ x                                          # w_i . x per nonzero
    P = np.zeros((D, k))
    np.add.at(P, docs, W[ids] * n[:, None])                 # p_d
    s = P @ x
    ok1, ok2, ok3 = m >= 1, m >= 2, m >= 3
    with np.errstate(divide="ignore", invalid="ignore"):
        a3 = np.where(ok3, 1.0 / (m * (m - 1) * (m - 2)), 0.0) / max(ok3.sum(), 1)
        a2 = np.where(ok2, 1.0 / (m * (m - 1)), 0.0) / max(ok2.sum(), 1)
        a1 = np.where(ok1, 1.0 / m, 0.0) / max(ok1.sum(), 1)
    q = P.T @ a1
    sq = q @ x
    nt2 = np.bincount(docs, weights=n * t * t, minlength=D)
    nt3 = np.bincount(docs, weights=n * t ** 3, minlength=D)
    e3_xxx = np.sum(a3 * (s ** 3 - 3 * nt2 * s + 2 * nt3))
    e2_xx = np.sum(a2 * (s * s - nt2))
    # vector parts
    e3_i = (P * (a3 * s * s)[:, None]).sum(0)
    wt = W[ids] * (n * t)[:, None]                           # n_i t_i w_i per nonzero
    wt2 = W[ids] * (n * t * t)[:, None]                      # n_i t_i^2 w_i per nonzero
    A = np.zeros((D, k))
    np.add.at(A, docs, wt)
    A2 = np.zeros((D, k))
    np.add.at(A2, docs, wt2)
    e3_i -= (2 * A * (a3 * s)[:, None]).sum(0) + (P * (a3 * nt2)[:, None]).sum(0)
    e3_i += 2 * (A2 * a3[:, None]).sum(0)
    e2_ix = (P * (a2 * s)[:, None]).sum(0) - (A * a2[:, None]).sum(0)     # E2(I, x)
    a = alpha0 / (alpha0 + 2.0)
    c = 2.0 * alpha0 ** 2 / ((alpha0 + 1.0) * (alpha0 + 2.0))
    xxx = e3_xxx - a * 3 * e2_xx * sq + c * sq ** 3
    ixx = e3_i - a * (2 * e2_ix * sq + q * e2_xx) + c * q * sq * sq
    return xxx, ixx


# ----------------------------------------------------------------------------- whitening

def whiten(M2: np.ndarray, k: int):
    """Alg. 3, line 3: the k eigenpairs of the symmetric M2^ with the largest eigenvalues,
    W = U diag(sigma)^(-1/2).  Returns (W [V x k], sigma [k], descending)."""
    M2 = 0.5 * (M2 + M2.T)
    vals, vecs = np.linalg.eigh(M2)
    order = np.argsort(vals)[::-1][:k]
    sig = vals[order]
    if np.any(sig <= 0):
        raise ValueError("M2 has fewer than k positive eigenvalues")
    return vecs[:, order] / np.sqrt(sig), sig


# ----------------------------------------------------------------------------- recovery

def recover(lam: np.ndarray, Vv: np.ndarray, W: np.ndarray, alpha0: float):
    """Alg. 3, line 6: alpha^_i = 4 alpha0 (alpha0+1) / ((alpha0+2)^2 lambda_i^2) and
    mu^_i = (alpha0+2)/2 lambda_i (W^+)^T v_i.  Vv is k x k with v_i in ROW i; returns
    (alpha^ [k], mu^ [k x V], row i = topic i)."""
    lam = np.asarray(lam, dtype=np.float64)
    Vv = np.asarray(Vv, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    alpha = 4.0 * alpha0 * (alpha0 + 1.0) / ((alpha0 + 2.0) ** 2 * lam ** 2)
    Wp = np.linalg.pinv(W)                                   # k x V
    mu = ((alpha0 + 2.0) / 2.0) * lam[:, None] * (Vv @ Wp)
    return alpha, mu


# ----------------------------------------------------------------------------- population moments

def population_raw_moments(Phi: np.ndarray, alpha: np.ndarray):
    """Exact E[x1], E[x1 (x) x2], E[x1 (x) x2 (x) x3] of the LDA model (words of one document
    are independent given theta ~ Dir(alpha)), from the Dirichlet moments
      E[theta_i] = alpha_i / alpha0,
      E[theta_i theta_j] = alpha_i (alpha_j + [i=j]) / (alpha0 (alpha0+1)),
      E[theta_i theta_j theta_l] = alpha_i (alpha_j + [i=j]) (alpha_l + [i=l] + [j=l])
                                   / (alpha0 (alpha0+1)(alpha0+2)).
    Phi is k x V (row t = mu_t)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    alpha = np.asarray(alpha, dtype=np.float64)
    k = len(alpha)
    a0 = alpha.sum()
    I = np.eye(k)
    E1t = alpha / a0
    E2t = alpha[:, None] * (alpha[None, :] + I) / (a0 * (a0 + 1))
    E3t = (alpha[:, None, None] * (alpha[None, :, None] + I[:, :, None])
           * (alpha[None, None, :] + I[:, None, :] + I[None, :, :]) / (a0 * (a0 + 1) * (a0 + 2)))
    E1 = Phi.T @ E1t
    E2 = Phi.T @ E2t @ Phi
    E3 = np.einsum("ijl,ia,jb,lc->abc", E3t, Phi, Phi, Phi)
    return E1, E2, E3


# ----------------------------------------------------------------------------- paper's sketch route

def sketch_m3_per_doc(corpus, W: np.ndarray, alpha0: float, h, g, b: int) -> np.ndarray:
    """Colliding sketch (Eq. 7) of M3^(W,W,W) built the way App. D describes: one count sketch
    of p_d per document, cubed in the frequency domain; the per-word sums
      r_i = sum_d a_d n_di p_d,  c_i = sum_d a_d n_di      (a_d = 1/(D3 m(m-1)(m-2)))
      e_i = sum_d b_d n_di                                  (b_d = 1/(D2 m(m-1)))
    are folded in after the scan with one sketch per word.  A rank-1 term x (x) y (x) z has
    sketch F^-1(F s_x F s_y F s_z), and the three placements of w w p share one sketch."""
    W = np.asarray(W, dtype=np.float64)
    k = W.shape[1]
    m = doc_lengths(corpus)
    D = num_docs(corpus)
    D1, D2, D3 = (m >= 1).sum(), (m >= 2).sum(), (m >= 3).sum()
    V = W.shape[0]

    def fs(x):
        return _fft(count_sketch(x, h, g, b))

    acc3 = np.zeros(b, dtype=complex)        # sum_d a_d (F s_p)^3
    acc2 = np.zeros(b, dtype=complex)        # sum_d b_d (F s_p)^2
    r = np.zeros((V, k))
    c = np.zeros(V)
    e = np.zeros(V)
    q = np.zeros(k)
    for d in range(D):
        ids, n = doc(corpus, d)
        md = m[d]
        p = W[ids].T @ n
        if md >= 1:
            q += p / md / D1
        if md >= 2:
            bd = 1.0 / (D2 * md * (md - 1))
            acc2 += bd * fs(p) ** 2
            e[ids] += bd * n
        if md >= 3:
            ad = 1.0 / (D3 * md * (md - 1) * (md - 2))
            acc3 += ad * fs(p) ** 3
            r[ids] += ad * n[:, None] * p[None, :]
            c[ids] += ad * n
    for i in range(V):
        if c[i] == 0.0 and e[i] == 0.0:
            continue
        Fw = fs(W[i])
        acc3 += -3.0 * Fw ** 2 * fs(r[i]) + 2.0 * c[i] * Fw ** 3
        acc2 += -e[i] * Fw ** 2
    Fq = fs(q)
    a = alpha0 / (alpha0 + 2.0)
    cc = 2.0 * alpha0 ** 2 / ((alpha0 + 1.0) * (alpha0 + 2.0))
    F = acc3 - a * 3.0 * acc2 * Fq + cc * Fq ** 3
    return _ifft(F)
