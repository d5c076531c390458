"""Oracle: count sketches of vectors and tensor sketches, written from their definitions.

* Asymmetric tensor sketch, Eq. (1) (Sec. 2):
      s_T(t) = sum_{(h1(i)+h2(j)+h3(k)) mod b = t} xi1(i) xi2(j) xi3(k) T_ijk
* Colliding (symmetric) tensor sketch, Eq. (7) (Sec. 3.3):
      s~_T(t) = sum_{(h(i)+h(j)+h(k)) mod b = t} sigma(i) sigma(j) sigma(k) T_ijk
  over ALL ordered triples (i, j, k).
* "Upper-triangular" sketch of B~ (App. B, Eq. (12)): the same sum restricted to i <= j <= k;
  this is the query-side sketch of Eq. (11) and Lemma 1.
* Vector sketches of order p (App. B, below Eq. (13)):
      s~_{p, u^p}(t) = sum_{p h(i) mod b = t} sigma(i)^p u_i^p      (p = 1, 2, 3)
* Rank-1 sketches via convolution, Eq. (4): s_{u(x)v(x)w} = s_{1,u} * s_{2,v} * s_{3,w};
  for the colliding hash the full sketch of u^{(x)3} is s~_u * s~_u * s~_u (Sec. 3.3).

Every sum is taken literally (loops or bincount over index tuples), in float64 / complex128,
or exactly in int64 for integer tensors.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np

from .hashing import sigma_of, xi_of
from .conv import conv_direct


def _bincount_complex(idx: np.ndarray, w: np.ndarray, b: int) -> np.ndarray:
    re = np.bincount(idx, weights=w.real, minlength=b)
    im = np.bincount(idx, weights=w.imag, minlength=b)
    return re + 1j * im


def count_sketch(u: np.ndarray, h: np.ndarray, g: np.ndarray, b: int, p: int = 1) -> np.ndarray:
    """s~_{p,u^p}: bucket (p*h(i)) mod b receives sigma(i)^p u_i^p (App. B)."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[0]
    h = np.asarray(h[:n], dtype=np.int64)
    sig = sigma_of(g[:n])
    return _bincount_complex((p * h) % b, (sig ** p) * (u ** p), b)


def count_sketch_asym(u: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """Asymmetric count sketch s_{j,u}(t) = sum_{h_j(i)=t} xi_j(i) u_i (Sec. 3.1)."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[0]
    return np.bincount(np.asarray(h[:n], dtype=np.int64), weights=xi_of(g[:n]) * u,
                       minlength=b).astype(np.complex128)


def sketch_tensor_sym(T: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """Colliding sketch of a dense n^3 tensor over all ordered triples (Eq. 7).

    Float input -> complex128 result.  Integer input -> exact (re, im) int64 pair of shape [2, b].
    """
    n = T.shape[0]
    h = np.asarray(h[:n], dtype=np.int64)
    g = np.asarray(g[:n], dtype=np.int64)
    hjk = h[:, None] + h[None, :]
    gjk = g[:, None] + g[None, :]
    if np.issubdtype(T.dtype, np.integer):
        acc = np.zeros((2, b), dtype=np.int64)
        for i in range(n):
            t = ((h[i] + hjk) % b).ravel()
            e = ((g[i] + gjk) % 4).ravel()      # sigma(i) sigma(j) sigma(k) = sqrt(-1)^e
            v = T[i].astype(np.int64).ravel()
            for comp, sgn, ev in ((0, 1, 0), (1, 1, 1), (0, -1, 2), (1, -1, 3)):
                sel = e == ev
                np.add.at(acc[comp], t[sel], sgn * v[sel])
        return acc
    s = np.zeros(b, dtype=np.complex128)
    sig = sigma_of(g)
    sjk = sig[:, None] * sig[None, :]
    for i in range(n):
        t = ((h[i] + hjk) % b).ravel()
        w = (sig[i] * sjk * T[i].astype(np.float64)).ravel()
        s += _bincount_complex(t, w, b)
    return s


def sketch_tensor_sym_sorted(T: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """The same sketch read from i <= j <= k only, weighted by kappa in {1, 3, 6} (Sec. 3.3:
    all permutations of a symmetric entry collide).  Equal to sketch_tensor_sym for symmetric T."""
    n = T.shape[0]
    sig = sigma_of(g[:n])
    s = np.zeros(b, dtype=np.complex128)
    for i in range(n):
        for j in range(i, n):
            for k in range(j, n):
                kappa = 1 if (i == j == k) else (3 if (i == j or j == k) else 6)
                t = (h[i] + h[j] + h[k]) % b
                s[t] += kappa * sig[i] * sig[j] * sig[k] * float(T[i, j, k])
    return s


def sketch_truncated_sym(X: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """Sketch of the upper-triangular truncation X~ (App. B, Eq. (12)): only i <= j <= k."""
    n = X.shape[0]
    sig = sigma_of(g[:n])
    s = np.zeros(b, dtype=np.complex128)
    for i in range(n):
        for j in range(i, n):
            for k in range(j, n):
                t = (h[i] + h[j] + h[k]) % b
                s[t] += sig[i] * sig[j] * sig[k] * X[i, j, k]
    return s


def sketch_tensor_asym(T: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """Asymmetric tensor sketch, Eq. (1): h, g have shape [3][nmax]; result is real (complex128
    with zero imaginary part, or int64 [b] for integer input)."""
    n1, n2, n3 = T.shape
    h1, h2, h3 = (np.asarray(h[j], dtype=np.int64) for j in range(3))
    x1, x2, x3 = (xi_of(g[j]) for j in range(3))
    hjk = h2[:n2, None] + h3[None, :n3]
    xjk = x2[:n2, None] * x3[None, :n3]
    if np.issubdtype(T.dtype, np.integer):
        acc = np.zeros(b, dtype=np.int64)
        for i in range(n1):
            t = ((h1[i] + hjk) % b).ravel()
            v = (int(x1[i]) * xjk.astype(np.int64) * T[i].astype(np.int64)).ravel()
            np.add.at(acc, t, v)
        return acc
    s = np.zeros(b, dtype=np.float64)
    for i in range(n1):
        t = ((h1[i] + hjk) % b).ravel()
        s += np.bincount(t, weights=(x1[i] * xjk * T[i].astype(np.float64)).ravel(), minlength=b)
    return s.astype(np.complex128)


def sketch_rank1_sym(u: np.ndarray, h: np.ndarray, g: np.ndarray, b: int) -> np.ndarray:
    """Full colliding sketch of u (x) u (x) u = s~_u * s~_u * s~_u (Eq. 4 with h1 = h2 = h3)."""
    su = count_sketch(u, h, g, b, 1)
    return conv_direct(conv_direct(su, su), su)


def sketch_rank1_asym(u, v, w, h, g, b) -> np.ndarray:
    """s_{u(x)v(x)w} = s_{1,u} * s_{2,v} * s_{3,w} (Eq. 4)."""
    s1 = count_sketch_asym(u, h[0], g[0], b)
    s2 = count_sketch_asym(v, h[1], g[1], b)
    s3 = count_sketch_asym(w, h[2], g[2], b)
    return conv_direct(conv_direct(s1, s2), s3)


def recover_entry_sym(s: np.ndarray, h, g, b, i: int, j: int, k: int) -> complex:
    """Entry recovery rule below Eq. (7): T^_ijk = (1/kappa) conj(sigma_i sigma_j sigma_k) s(H)."""
    sig = sigma_of(np.asarray([g[i], g[j], g[k]]))
    ii, jj, kk = sorted((i, j, k))
    kappa = 1 if (ii == jj == kk) else (3 if (ii == jj or jj == kk) else 6)
    return np.conj(sig[0] * sig[1] * sig[2]) * s[(h[i] + h[j] + h[k]) % b] / kappa
