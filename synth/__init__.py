"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only draws random inputs (tensors, initial vectors); it holds none of the
sketching or power-method arithmetic.  Every generator takes an explicit integer seed
and uses numpy's PCG64 stream, so both sides of a parity test see identical bytes.

Workload shapes follow the paper's synthetic experiment (Sec. 5.1): a symmetric tensor
built from an orthonormal set of components plus a symmetric Gaussian noise tensor
whose independent entries are those with i <= j <= k.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "rng",
    "orthonormal_columns",
    "planted_symmetric",
    "symmetric_noise",
    "gaussian_inits",
    "random_symmetric",
    "random_symmetric_int",
    "random_vector",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def orthonormal_columns(n: int, k: int, seed: int) -> np.ndarray:
    """n x k matrix with orthonormal columns (QR of a Gaussian matrix, sign-fixed)."""
    g = rng(seed).standard_normal((n, k))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return q


def symmetric_noise(n: int, std: float, seed: int, dtype=np.float64) -> np.ndarray:
    """Symmetric n^3 tensor: entry (i,j,k) copies an N(0, std^2) draw made for the
    sorted triple (min, mid, max) -- one independent draw per i <= j <= k."""
    out = np.empty((n, n, n), dtype=dtype)
    if std == 0.0 or n == 0:
        out[...] = 0
        return out
    g = rng(seed).standard_normal((n, n, n)) * std
    jj, kk = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for i in range(n):
        ii = np.full_like(jj, i)
        lo = np.minimum(np.minimum(ii, jj), kk)
        hi = np.maximum(np.maximum(ii, jj), kk)
        mid = ii + jj + kk - lo - hi
        out[i] = g[lo, mid, hi]
    return out


def planted_symmetric(n: int, k: int, noise: float, seed: int,
                      lam_low: float = 1.0, lam_high: float = 2.0,
                      dtype=np.float64):
    """T = sum_r lam_r a_r (x) a_r (x) a_r + E with orthonormal a_r, lam_r ~ U[lam_low, lam_high]
    and E from :func:`symmetric_noise`.  Returns (T, lam, A) with A of shape n x k."""
    r = rng(seed)
    lam = r.uniform(lam_low, lam_high, size=k)
    A = orthonormal_columns(n, k, seed + 1)
    T = symmetric_noise(n, noise, seed + 2, dtype=np.float64)
    for i in range(n):
        T[i] += (A * (lam * A[i])[None, :]) @ A.T
    return T.astype(dtype, copy=False), lam, A


def paper_synthetic(n: int, sigma: float, seed: int):
    """The synthetic tensor of the paper's experiments (Sec. 5.1): T = S / ||S||_F + E with
    S = sum_{i<=n} lam_i v_i (x) v_i (x) v_i, lam_i = 1/i, v_i the orthonormal columns of V (full
    rank), and E symmetric with one N(0, (sigma / n^1.5)^2) draw per i <= j <= k.  Float32, built
    one slice T[i] at a time (n = 1000 is 4 GB).  Returns (T, lam_normalised, V)."""
    lam = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    lam /= np.linalg.norm(lam)                     # ||S||_F = ||lam||_2 for orthonormal v_i
    V = orthonormal_columns(n, n, seed + 1)
    std = sigma / n ** 1.5
    g = rng(seed + 2).standard_normal((n, n, n), dtype=np.float32)
    T = np.empty((n, n, n), dtype=np.float32)
    jj, kk = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for i in range(n):
        ii = np.full_like(jj, i)
        lo = np.minimum(np.minimum(ii, jj), kk)
        hi = np.maximum(np.maximum(ii, jj), kk)
        mid = ii + jj + kk - lo - hi
        sig_i = (V * (lam * V[i])[None, :]) @ V.T
        T[i] = (sig_i + std * g[lo, mid, hi].astype(np.float64)).astype(np.float32)
    return T, lam, V


def random_symmetric(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """Dense symmetric tensor with N(0,1) independent entries (i <= j <= k)."""
    return symmetric_noise(n, 1.0, seed, dtype=dtype)


def random_symmetric_int(n: int, seed: int, low: int = -1000, high: int = 1000) -> np.ndarray:
    """Dense symmetric int32 tensor with independent integer entries for i <= j <= k."""
    g = rng(seed).integers(low, high + 1, size=(n, n, n), dtype=np.int64)
    out = np.empty((n, n, n), dtype=np.int32)
    jj, kk = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for i in range(n):
        ii = np.full_like(jj, i)
        lo = np.minimum(np.minimum(ii, jj), kk)
        hi = np.maximum(np.maximum(ii, jj), kk)
        mid = ii + jj + kk - lo - hi
        out[i] = g[lo, mid, hi]
    return out


def gaussian_inits(k: int, L: int, n: int, seed: int) -> np.ndarray:
    """k x L x n standard Gaussian draws; normalising each row gives a uniform point on the
    unit sphere (the initial vectors of the robust tensor power method, Alg. 1)."""
    return rng(seed).standard_normal((k, L, n))


def random_vector(n: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal(n)


def batched_problem_specs(P: int, seed: int, n_low: int = 32, n_high: int = 256, k_low: int = 4,
                          k_high: int = 16, log2b_low: int = 10, log2b_high: int = 14):
    """Sizes of P independent planted problems: n ~ U{n_low..n_high}, k ~ U{k_low..k_high},
    sketch length b = 2^ceil(log2(n k)) clamped to [2^log2b_low, 2^log2b_high].  Returns a list of
    dicts (n, k, log2b, seed) with a per-problem seed for planted_symmetric / gaussian_inits."""
    r = rng(seed)
    specs = []
    for p in range(P):
        n = int(r.integers(n_low, n_high + 1))
        k = int(r.integers(k_low, k_high + 1))
        log2b = int(np.ceil(np.log2(n * k)))
        log2b = min(max(log2b, log2b_low), log2b_high)
        specs.append({"n": n, "k": k, "log2b": log2b, "seed": int(seed * 100003 + p)})
    return specs


def lda_corpus(V: int, k: int, D: int, seed: int, alpha: float = 0.1, beta: float = 0.01,
               mean_len: float = 200.0):
    """Synthetic LDA corpus (the generative model of App. D): topic-word distributions
    Phi[t] ~ Dir(beta 1_V), document mixtures theta_d ~ Dir(alpha 1_k), m_d ~ Poisson(mean_len)
    tokens with topics ~ Cat(theta_d) and words of topic t ~ Cat(Phi[t]).
    Sampled in an equivalent, vectorised form: the topic counts of a document are independent
    Poisson(mean_len theta_dt) (so m_d ~ Poisson(mean_len) and, given m_d, the counts are
    multinomial); the words of all tokens of topic t are one multinomial draw of their total,
    randomly permuted over those tokens.
    Returns dict(indptr int64 [D+1], idx int32 [nnz], cnt int32 [nnz], Phi [k][V], alpha [k],
    lengths [D], ...) with each document's distinct words sorted and counted (CSR)."""
    r = rng(seed)
    Phi = r.dirichlet(np.full(V, beta), size=k)
    alpha_vec = np.full(k, alpha)
    theta = r.dirichlet(alpha_vec, size=D)
    tc = r.poisson(mean_len * theta)                                 # D x k topic counts
    lengths = tc.sum(1).astype(np.int64)
    doc_ids = np.arange(D, dtype=np.int64)
    keys = []
    for t in range(k):
        ct = tc[:, t]
        tot = int(ct.sum())
        if tot == 0:
            continue
        w = np.repeat(np.arange(V, dtype=np.int64), r.multinomial(tot, Phi[t]))
        r.shuffle(w)
        keys.append(np.repeat(doc_ids, ct) * V + w)                # (document, word) of each token
    keys = np.sort(np.concatenate(keys)) if keys else np.zeros(0, dtype=np.int64)
    if keys.size:
        first = np.concatenate([[True], keys[1:] != keys[:-1]])
        uk = keys[first]
        cnt = np.diff(np.concatenate([np.nonzero(first)[0], [keys.size]]))
    else:
        uk = keys
        cnt = np.zeros(0, dtype=np.int64)
    indptr = np.zeros(D + 1, dtype=np.int64)
    indptr[1:] = np.cumsum(np.bincount(uk // V, minlength=D))
    return {"indptr": indptr, "idx": (uk % V).astype(np.int32), "cnt": cnt.astype(np.int32),
            "Phi": Phi, "alpha": alpha_vec, "lengths": lengths, "V": V, "k": k, "D": D}


def planted_cp(dims, R: int, noise: float, seed: int, dtype=np.float32):
    """Asymmetric rank-R tensor sum_r w_r a_r (x) b_r (x) c_r + noise: factor rows N(0, 1)
    normalised to unit length, weights U[0.5, 2], i.i.d. Gaussian noise of std `noise`.
    Returns (T [dims], w [R], [A [R][n1], B [R][n2], C [R][n3]])."""
    r = rng(seed)
    F0 = [r.standard_normal((R, d)) for d in dims]
    F0 = [f / np.linalg.norm(f, axis=1, keepdims=True) for f in F0]
    w = r.uniform(0.5, 2.0, R)
    T = np.einsum("r,ri,rj,rk->ijk", w, *F0).astype(dtype)
    T += (noise * r.standard_normal(tuple(dims))).astype(dtype)
    return T, w, F0


def gaussian_matrix(rows: int, cols: int, seed: int) -> np.ndarray:
    """Standard Gaussian test matrix (the random start of a randomized range finder)."""
    return rng(seed).standard_normal((rows, cols))


def planted_order4(n: int, k: int, noise: float, seed: int):
    """Symmetric order-4 tensor sum_r lam_r a_r^{(x)4} + E (orthonormal a_r from
    orthonormal_columns, lam_r ~ U[1, 2]), the signal built in FP32 as the n^2 x n^2 matrix
    Q diag(lam) Q^T with Q_r = vec(a_r a_r^T); E = noise times the average of an i.i.d. N(0, 1)
    tensor over the 24 permutations of its modes (symmetric; an entry with four distinct indices
    has std noise / sqrt(24)).  Returns (T [n][n][n][n] float32, lam, A)."""
    import itertools
    r = rng(seed)
    lam = r.uniform(1.0, 2.0, size=k)
    A = orthonormal_columns(n, k, seed + 1)
    Q = np.stack([np.outer(A[:, j], A[:, j]).ravel() for j in range(k)], axis=1).astype(np.float32)
    T = ((Q * lam.astype(np.float32)[None, :]) @ Q.T).reshape(n, n, n, n)
    if noise:
        G = rng(seed + 2).standard_normal((n, n, n, n), dtype=np.float32)
        E = np.zeros_like(G)
        for q in itertools.permutations(range(4)):
            E += G.transpose(q)
        T += np.float32(noise / 24.0) * E
    return T, lam, A
